// Internal declarations of the MAPI CUDA library (not part of the ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <functional>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/mapi.h"

namespace mapi {

constexpr int kMaxVec = 8;  // start vectors sharing one read of A

// Per-vector state of one solve, resident on the device.
struct VecState {
  int done;     // 1 once converged, stopped or failed: later steps skip it
  int status;   // mapi_status of this vector
  int iters;    // products (Alg. 1 step 3) completed
  int pad_;
  float delta;  // last ||w_new - w_old||_1 (float storage)
  float norm;   // last ||y|| used for the normalisation
  long long idelta;  // last delta in units of 2^-q (integer storage)
};

// Control block of one solve: the last-CTA ticket, the early-exit flag and
// the per-vector states.  Lives in device memory, one per solve.
struct IterCtl {
  unsigned counter;   // CTAs of the current step that have finished
  int all_done;       // every vector done: later step kernels return at once
  int nvec;
  int pad_;
  float tol;          // float storage: stop when delta < tol
  float pad2_;
  long long itol;     // integer storage: stop when delta < itol
  VecState v[kMaxVec];
};

// Element type tags used as template arguments.
enum StTag { kF32 = 0, kBF16 = 1, kFP8 = 2, kI16 = 3, kI8 = 4 };

inline int elem_bytes(mapi_storage st) {
  switch (st) {
    case MAPI_ST_F32: return 4;
    case MAPI_ST_BF16: return 2;
    case MAPI_ST_FP8E4M3_ROWPOW2: return 1;
    case MAPI_ST_I16: return 2;
    case MAPI_ST_I8: return 1;
  }
  return 0;
}
inline bool is_int_storage(mapi_storage st) {
  return st == MAPI_ST_I16 || st == MAPI_ST_I8;
}

}  // namespace mapi

// Packed device matrix.
struct mapi_mat {
  int rows = 0, cols = 0;
  int rows_pad = 0;        // rows rounded up to a multiple of 64 (zero rows)
  int64_t ld = 0;          // padded row length in elements (16-byte rows)
  mapi_storage storage = MAPI_ST_F32;
  int q = 0;               // integer storage: A_q = RNE(A 2^q)
  void* data = nullptr;    // rows_pad x ld elements
  float* row_scale = nullptr;  // FP8: 2^(120 + k_i) per row, the decoder's factor
  int* row_exp = nullptr;      // FP8: k_i per row
  size_t bytes = 0;
  mapi_ctx* owner = nullptr;
  uint64_t id = 0;         // never reused: keys cached graphs (addresses are reused)
};

// Device scratch owned by a context; grown on demand.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

// One timed launch: events around it on its stream.
struct ProfMark {
  int cls;
  cudaEvent_t a, b;
  double bytes, terms;
  int count;  // launches (or persistent-kernel steps) the two events bracket
};

struct GraphEntry {
  cudaGraphExec_t exec = nullptr;
  uint64_t last_use = 0;
  uint64_t nodes = 0;              // kernel launches per replay
  std::vector<ProfMark> marks;     // event nodes inside the graph
};

namespace mapi {
struct Server;
}

namespace mapi {
// Time stamps of pair steps (%globaltimer, ns), filled while phase stamping
// is on: the earliest start of the current step's streaming CTAs (after the
// published iterate arrived), the first and last arrival of a streaming CTA
// at the end of its tiles, the previous step's publication, and per phase
// the nanoseconds summed over the steps: [0] previous publication -> start,
// [1] start -> first arrival, [2] start -> last arrival, [3] last arrival ->
// the epilogue cluster sees it, [4] reduction of the accumulated row sums,
// [5] deflation and its combination over the cluster, [6] norm,
// normalisation, stop test and publication, [7] steps stamped.
constexpr int kPairPhaseClusters = 128;  // streaming clusters the stamps cover at most
constexpr int kPairClusterCtas = 4;      // CTAs per cluster of the pair solve
struct PairPhases {
  unsigned long long start_min, loop_min, loop_max, prev_end;
  unsigned long long sum[8];
  // per streaming cluster: its CTAs' loop times (own start to arrival), summed
  unsigned long long cl_ns[kPairPhaseClusters];
};
}  // namespace mapi

constexpr int kMatPoolBlocks = 2;
struct mapi_ctx {
  int device = 0;
  int sm_count = 0;
  size_t l2_bytes = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  size_t hbm_budget = 0;
  int max_slots = 64;
  std::string tune_cache_path;
  std::string last_error;
  std::set<mapi_mat*> mats;

  // scratch for solves
  DevBuf ypart, wbuf0, wbuf1, ctl, aux, mcpart;
  DevBuf pca_c0, pca_c1, pca_q, pca_defl;  // PCA scratch (covariances, deflation)
  int* rec_host = nullptr;                 // pinned: per-component steps and statuses
  DevBuf batch;                            // batched solves: instance table and results
  DevBuf hyb;                              // MAPI -> RPI switch: the handed-over iterate
  DevBuf outer;                            // ranked components of an outer-product apply
  DevBuf img;                              // image reconstruction: centred images, mean
  mapi_mat* img_X = nullptr;               // image reconstruction: packed centred images
  int batch_rows_per_warp[2][2] = {{2, 2}, {2, 2}};  // [F32, BF16][1, 4 vectors], autotuned
  mapi::IterCtl* ctl_host = nullptr;  // pinned mirror of the control block

  // CUDA-graph cache: key -> executable graph
  std::map<std::vector<int64_t>, GraphEntry> graphs;
  uint64_t use_clock = 0;
  uint64_t next_mat_id = 1;
  cudaStream_t capture_stream = nullptr;

  // diagnostics
  bool prof_on = false;
  bool phases_on = false;      // stamp the phases of pair steps
  DevBuf pair_phases;          // one mapi::PairPhases
  // Host uploads are copied into this staging buffer (grown to the largest
  // upload, kept until mapi_destroy) before they are packed.
  DevBuf upload_staging;
  // Device storage of freed matrices kept for the next matrix of the same
  // size (at most kMatPoolBlocks blocks; off where memory is budgeted).
  std::vector<std::pair<void*, size_t>> mat_pool;
  bool pool_matrices = true;
  long long stall_ns = 0;      // > 0: fault-detection test of the bounded waits
  int pair_nstream = 0;        // streaming clusters of the last pair launch
  int pair_coop = -1;          // cooperative cluster launch accepted (-1: not asked)
  // K1 may run in 8-CTA clusters on large matrices; off for
  // the serving loop, whose solves share the GPU with a persistent batched
  // launch (a cluster waits for eight free CTA slots at once)
  bool gemv_clusters = true;
  bool capturing = false;
  uint64_t capture_count = 0;             // launches recorded into the graph being captured
  std::vector<ProfMark> pending;          // marks of direct launches
  std::vector<ProfMark>* mark_sink = nullptr;  // where new marks go
  std::vector<cudaEvent_t> ev_pool;
  mapi_stats stats = {};

  // serving loop (created by the first mapi_submit)
  std::mutex server_mu;
  mapi::Server* server = nullptr;
};

namespace mapi {

// ---------------------------------------------------------------- errors
mapi_status fail(mapi_ctx* ctx, mapi_status s, const std::string& msg);
mapi_status cuda_fail(mapi_ctx* ctx, cudaError_t e, const char* what);
#define MAPI_CUDA_TRY(ctx, call)                                  \
  do {                                                            \
    cudaError_t e_ = (call);                                      \
    if (e_ != cudaSuccess) return ::mapi::cuda_fail(ctx, e_, #call); \
  } while (0)

// ---------------------------------------------------------- diagnostics
// Count kernel launches (not while a graph is being captured).
inline void count_launch(mapi_ctx* ctx, uint64_t n = 1) {
  if (ctx->capturing) ctx->capture_count += n;
  else ctx->stats.launches += n;
}
// Start a timed launch: returns the start event (nullptr when profiling is off).
cudaEvent_t prof_begin(mapi_ctx* ctx, cudaStream_t s);
// End it: records the stop event and files the mark.
void prof_end(mapi_ctx* ctx, cudaStream_t s, cudaEvent_t a, int cls, double bytes,
              double terms, int count = 1);
// Fold completed marks into the counters (stream already synchronised).
void prof_collect(mapi_ctx* ctx, std::vector<ProfMark>& marks, bool recycle);
void destroy_graph(mapi_ctx* ctx, GraphEntry& g);

// Replay the CUDA graph cached under `key` on ctx->stream, capturing it from
// `enqueue` (stream work only, no allocation) the first time.  The caller
// synchronises and then calls finish_graph.
mapi_status launch_cached_graph(mapi_ctx* ctx, const std::vector<int64_t>& key,
                                const std::function<mapi_status(cudaStream_t)>& enqueue,
                                GraphEntry** out);
// After the stream has finished the replay: fold timings and launch counts.
void finish_graph(mapi_ctx* ctx, GraphEntry* g);

// Grow a scratch buffer (drops cached graphs when an address changes).
void release_matrix_pool(mapi_ctx* ctx);
mapi_status ensure(mapi_ctx* ctx, DevBuf& b, size_t bytes);

// Packed matrices owned by the context (api.cu): an uninitialised rows x cols
// matrix of storage st, and its release.
mapi_status alloc_matrix(mapi_ctx* ctx, int rows, int cols, mapi_storage st, mapi_mat** out);
mapi_status free_matrix(mapi_ctx* ctx, mapi_mat* m);

// --------------------------------------------------------- kernel launchers
// Iteration launch parameters chosen per shape (see tune.cu).
struct GemvPlan {
  int rows_per_warp;   // R
  int warps;           // warps per CTA
  int ksplit;          // column splits
  int grid_rows;       // CTAs along rows
};
GemvPlan plan_gemv(const mapi_ctx* ctx, const mapi_mat* A, int nvec);

// Grow the scratch a solve of A with nvec vectors needs (call before capture).
mapi_status prepare_solve(mapi_ctx* ctx, const mapi_mat* A, int nvec);

// Enqueue a full solve (start, max_iters steps, finish) on `stream`.
mapi_status enqueue_solve(mapi_ctx* ctx, cudaStream_t stream, const mapi_mat* A,
                          mapi_op op, int nvec, const float* w0, int64_t ldw,
                          int max_iters, double tol, unsigned flags,
                          float* w_out, int64_t ldo, const int* abort = nullptr);

// Pack kernels.
mapi_status launch_pack(mapi_ctx* ctx, const float* src_dev, int64_t ld_src,
                        mapi_mat* m);
mapi_status launch_unpack_f32(mapi_ctx* ctx, const mapi_mat* m, float* dst_dev);
mapi_status launch_fp8_rowexp(mapi_ctx* ctx, const float* src, int64_t ld_src,
                              mapi_mat* m, int* flag_dev);
mapi_status launch_google(mapi_ctx* ctx, const int* indptr, const int* indices,
                          int n, double alpha, float* dst, int64_t ld);
mapi_status launch_check_finite(mapi_ctx* ctx, const float* src, int rows,
                                int cols, int64_t ld, int* flag_dev);
mapi_status launch_absmax(mapi_ctx* ctx, const float* src, int rows, int cols,
                          int64_t ld, unsigned* out_bits_dev);

// Start-vector and finishing kernels of a float solve (solve.cu).
mapi_status launch_start_float(mapi_ctx* ctx, cudaStream_t s, const float* w0, int64_t ldw,
                               int n, int nvec, float* wb0, float* wb1, int64_t wst, int raw,
                               IterCtl* ctl, float tol, const int* abort = nullptr);
mapi_status launch_finish(mapi_ctx* ctx, cudaStream_t s, const float* wb0, const float* wb1,
                          int64_t wst, int n, int nvec, const IterCtl* ctl, int final_l2,
                          int is_int, int q, float* out, int64_t ldo);

// PCA kernels (pca.cu).
mapi_status launch_mincov_raw(mapi_ctx* ctx, const mapi_mat* X, mapi_op op, float denom,
                              float* C, int64_t ldc, cudaStream_t s);
size_t mincov_scratch_bytes(const mapi_ctx* ctx, const mapi_mat* X);

// Outer products w (+) w^T of Alg. 2 (outer.cu).  A component is ranked once
// into a slot: wt = the component at the unit norm of its iteration (l1 for
// MIN1 / MIN2, as kept for DOT), perm = the order of |wt|, wsort[p] =
// wt[perm[p]], ubi[i] = the last sorted position whose |wt| is <= |wt_i|.  A
// scratch of k slots holds 4 arrays of k x stride entries (wt, perm, wsort,
// ubi).
constexpr int kOuterMaxD = 16384;  // order of an applied outer product
constexpr int kOuterMaxK = 64;     // components in one apply
struct OuterSlot {
  float* wt;
  int* perm;
  float* wsort;
  int* ubi;
};
inline int64_t outer_stride(int D) { return ((int64_t)D + 3) / 4 * 4; }
OuterSlot outer_slot(void* base, int k, int64_t stride, int m);
size_t outer_scratch_bytes(int k, int D);
// Shared-memory limits of the outer-product kernels (call before capture).
mapi_status outer_prepare(mapi_ctx* ctx);
mapi_status launch_outer_prep(mapi_ctx* ctx, mapi_op op, const float* w, int D, OuterSlot slot,
                              cudaStream_t s);
// out_r = sum_{m<nprev} P_m in_r (+ add) for `rows` rows (slots first...).
mapi_status launch_outer_apply(mapi_ctx* ctx, mapi_op op, int D, int nprev, OuterSlot first,
                               int64_t stride, const float* in, int64_t ld_in, int rows,
                               const float* add, float* out, int64_t ld_out, cudaStream_t s);
// Alg. 2 step 6: C_c = C - sum_{m<c} P_m C for symmetric C (D x D, leading
// dimension ld).  Ranks component c - 1 (column c - 1 of P) into slot c - 1
// of `rank` (slots 0 .. c - 2 hold the earlier ones from the previous
// calls), forms T = rows of (sum_m P_m C)^T, then C_c = C - T^T.
mapi_status launch_deflate_mincov(mapi_ctx* ctx, mapi_op op, const float* P, int64_t ldp, int c,
                                  int D, const float* C, int64_t ld, float* T, void* rank,
                                  int kslots, int64_t stride, float* Cc, cudaStream_t s);

// Pair-mode PCA (pair.cu): every step of one component in one persistent
// launch.  The earlier components the iterate is deflated by, ranked by
// launch_outer_prep: perm[p] = index at sorted position p, wsort[p] = wt at
// that position, ubi[i] = the last sorted position whose |wt| is <= |wt_i|.
struct DeflArgs {
  int nprev;          // finished components to deflate (0: none)
  int op;             // MAPI_OP_MIN1 / MIN2 / DOT
  const float* P;     // outer-product vectors wt, column m at P + m * ldp
  int64_t ldp;
  const int* perm;    // [m][stride] per component
  const float* wsort;
  const int* ubi;
  int64_t stride;     // elements between components in perm / wsort / ubi
};
struct PairPlan {
  const void* fn = nullptr;
  const void* fn_stamp = nullptr;  // the variant with phase stamps (MIN1), or null
  int rw = 0;          // rows per warp (8, 16, 32)
  int clusters = 0;    // 4-CTA clusters of the launch, the epilogue's included
  int D_pad = 0;       // rows one cluster covers (4 x 8 x rw)
  size_t smem = 0;     // dynamic shared memory per CTA
  bool coop = false;   // cooperative launch accepted
  CUtensorMap map;     // X as [rows_pad][ld], one (columns x rows) box per tile
};
mapi_status plan_pair(mapi_ctx* ctx, const mapi_mat* X, mapi_op op, PairPlan* pl);
// Device scratch of a pair solve: the fixed-point accumulators and the
// launch's shared state.
size_t pair_scratch_bytes(const PairPlan& pl);
// Once per solve: clear the scratch and find max |X|.
mapi_status launch_pair_prepare(mapi_ctx* ctx, cudaStream_t s, const PairPlan& pl,
                                const mapi_mat* X, void* scratch);
// T steps of one component (start vector already in wb0, control block set).
mapi_status launch_pair_solve(mapi_ctx* ctx, cudaStream_t s, const PairPlan& pl,
                              const mapi_mat* X, void* scratch, float* wb0, float* wb1,
                              const DeflArgs& defl, IterCtl* ctl, int T, int norm_l2,
                              float denom, int dir0, float* raw_out = nullptr);
// y[r] = a_{row_begin + r}^T (+) w for r < rows, no normalisation (shard.cu).
mapi_status launch_rows_raw(mapi_ctx* ctx, const mapi_mat* A, int row_begin, int rows,
                            mapi_op op, const float* w, float* y, cudaStream_t s);
// One unnormalised pair product of X (y_d = sum_n X_dn (+) (x_n^T (+) w),
// no denominator, deflation or normalisation) into y (device, D floats).
mapi_status run_pair_partial(mapi_ctx* ctx, const mapi_mat* X, mapi_op op, const float* w,
                             float* y);

// Batched solves (batched.cu): one instance as the kernel sees it.
struct BatchDev {
  const uint8_t* A;   // packed rows (rows_pad x ld)
  int64_t row_bytes;
  int n;
  int chunks;         // 16-byte chunks per row
  const float* w0;    // n x nvec, column-major (ld = n)
  float* w_out;       // n x nvec, column-major (ld = n)
  int* res;           // per vector: iters, status (2 ints)
  float* delta;       // per vector: last delta
  int max_iters;      // steps of this launch
  float tol;          // stop rule (<= 0: none)
  int raw_start;      // 1: w0 as given; 0: w0 / ||w0||_2 first
  int final_l2;       // l2-normalise the result if the solve ends here
  int last;           // the solve ends after max_iters steps (else it resumes
                      // from w_out in a later launch)
};
// One persistent launch over the instances (all of storage st, nvec = V);
// res gets [iters, status] per vector and dl the last deltas.  Synchronous.
// With use_graph (and the context's stream) the launch is a cached CUDA graph.
mapi_status batched_run(mapi_ctx* ctx, cudaStream_t stream, std::vector<BatchDev>& host,
                        mapi_op op, mapi_storage st, int V, std::vector<int>& res,
                        std::vector<float>& dl, bool use_graph = false);
int batched_max_n(int nvec);

// Serving loop (serve.cu): stops the loop and releases what it holds.
void server_shutdown(mapi_ctx* ctx);
mapi_status run_pca(mapi_ctx* ctx, const mapi_mat* X, int k, int mode,
                    mapi_op op, int iters, double tol, double denom,
                    const float* w0, float* P_out, int* iters_done);

}  // namespace mapi
