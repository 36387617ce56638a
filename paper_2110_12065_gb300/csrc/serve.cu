// Serving loop: PCA (min-covariance route of Alg. 2) and PageRank (§3.3)
// requests admitted as they arrive, by a device-memory budget.  One host
// thread per context owns a private child context (its own stream and
// scratch).  Every admitted request gets its matrix built on the device (C
// by Eq. (5), or G by Eq. (11)) and its iterate kept resident; each round
// advances every resident solve by up to kRoundSteps steps of Alg. 1 (up to
// kLongRoundSteps, a whole component, when no request waits for admission)
// in one persistent batched launch per (storage, op), then deflates finished
// PCA components (Alg. 2 step 6) or copies finished results to the caller.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <thread>

#include "device_common.cuh"

namespace mapi {

using Clock = std::chrono::steady_clock;
constexpr int kRoundSteps = 25;
// a round with nobody waiting for admission: one PCA component, and a bound
// on how long a cancellation waits
constexpr int kLongRoundSteps = 100;
constexpr int kMaxComponents = 8;
// Solves this large iterate on the whole GPU (the split GEMV, one launch per
// step) instead of a share of the batched launch: one cluster per instance
// would leave most SMs idle while only a few large requests are resident.
constexpr int kWideN = 2048;

struct ServeReq {
  uint64_t ticket = 0;
  mapi_request r{};
  size_t need = 0;
  int state = 0;  // 0 queued, 1 running, 2 finished
  bool cancel = false;
  mapi_result res{};
  Clock::time_point t_submit, t_admit;
  // device state (loop thread only)
  mapi_mat* X = nullptr;
  mapi_mat* G = nullptr;
  float* C = nullptr;   // PCA: C, C_c and Q, D x ldc each
  float* Cc = nullptr;
  float* Q = nullptr;
  void* R = nullptr;    // PCA: ranked components of the deflation
  int64_t ldc = 0;
  float* P = nullptr;   // PCA components, D x k
  float* w0 = nullptr;  // start vectors
  float* wb[2] = {nullptr, nullptr};
  int n = 0;            // order of the iterated matrix
  const uint8_t* A = nullptr;
  int64_t row_bytes = 0;
  mapi_storage st = MAPI_ST_F32;
  mapi_mat view;        // the iterated matrix as the split GEMV reads it
  int comp = 0, it_comp = 0, cur = 0;
  bool resumed = false;
  Clock::time_point t_built;
};

struct Server {
  mapi_ctx* parent = nullptr;
  mapi_ctx* child = nullptr;    // the loop's context: rounds, deflation, copies out
  mapi_ctx* bchild = nullptr;   // the builder's context: uploads, Eq. (5) / (11)
  std::thread th, bth;
  std::mutex mu;
  std::condition_variable cv, bcv;
  bool stop = false, bstop = false;
  std::deque<ServeReq*> to_build;  // admitted, waiting for the builder
  std::deque<ServeReq*> built;     // built, waiting for the loop
  std::vector<mapi_mat*> to_free;  // matrices of finished requests (builder's)
  uint64_t next_ticket = 1;
  std::deque<ServeReq*> queue;
  std::map<uint64_t, ServeReq*> tickets;
  size_t budget = 0, used = 0;
  int resident = 0;
  std::vector<ServeReq*> live;  // loop thread only
  cudaStream_t batch_stream = nullptr;  // batched launches beside the wide solves
  cudaEvent_t round_start = nullptr;    // orders batch_stream after the loop stream
  IterCtl* wide_ctl = nullptr;          // pinned: control blocks of the wide solves
  int wide_cap = 0;
};

namespace {

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

int64_t packed_ld(int cols, mapi_storage st) {
  const int eb = elem_bytes(st);
  return ((int64_t)cols * eb + 15) / 16 * 16 / eb;
}

size_t packed_bytes(int rows, int cols, mapi_storage st) {
  return (size_t)((rows + 63) / 64 * 64) * packed_ld(cols, st) * elem_bytes(st);
}

// Device bytes a request holds at its peak (staging, packed matrix, C, C_c,
// Q, scratch, vectors).
size_t request_bytes(const mapi_ctx* ctx, const mapi_request& r) {
  if (r.kind == MAPI_REQ_PCA) {
    mapi_mat x;
    x.rows = r.D;
    x.cols = r.N;
    x.ld = packed_ld(r.N, r.storage);
    x.rows_pad = (r.D + 63) / 64 * 64;
    x.storage = r.storage;
    const size_t ldc = (size_t)(r.D + 3) / 4 * 4;
    return (size_t)r.D * r.N * 4 + packed_bytes(r.D, r.N, r.storage) +
           mincov_scratch_bytes(ctx, &x) + 3 * (size_t)((r.D + 63) / 64 * 64) * ldc * 4 +
           (size_t)r.D * (2 * r.k + 2) * 4 + outer_scratch_bytes(r.k, r.D);
  }
  const size_t nnz = (size_t)r.indptr[r.n];
  return (size_t)(r.n + 1 + nnz) * 4 + (size_t)r.n * ((r.n + 3) / 4 * 4) * 4 +
         packed_bytes(r.n, r.n, r.storage) + (size_t)r.n * 3 * 4;
}

mapi_status check_request(const mapi_request* q) {
  if (!q || !q->w0 || !q->out) return MAPI_EINVAL;
  if (q->op != MAPI_OP_MIN1 && q->op != MAPI_OP_MIN2 && q->op != MAPI_OP_DOT) return MAPI_EINVAL;
  if (q->storage != MAPI_ST_F32 && q->storage != MAPI_ST_BF16) return MAPI_EINVAL;
  if (q->max_iters < 1) return MAPI_EINVAL;
  if (q->kind == MAPI_REQ_PCA) {
    if (!q->X || q->D < 1 || q->N < 1 || q->k < 1 || q->k > kMaxComponents || q->k > q->D ||
        q->D > batched_max_n(1) || !(q->cov_denom > 0.0))
      return MAPI_EINVAL;
    return MAPI_OK;
  }
  if (q->kind == MAPI_REQ_PAGERANK) {
    if (!q->indptr || !q->indices || q->n < 1 || q->n > batched_max_n(1) ||
        !(q->alpha >= 0.0 && q->alpha <= 1.0) || q->indptr[0] != 0 || q->indptr[q->n] < 0)
      return MAPI_EINVAL;
    for (int j = 0; j < q->n; ++j)
      if (q->indptr[j + 1] < q->indptr[j]) return MAPI_EINVAL;
    for (int e = 0; e < q->indptr[q->n]; ++e)
      if (q->indices[e] < 0 || q->indices[e] >= q->n) return MAPI_EINVAL;
    return MAPI_OK;
  }
  return MAPI_EINVAL;
}

template <class T>
mapi_status dev_alloc(mapi_ctx* c, T** p, size_t bytes) {
  if (cudaMallocAsync((void**)p, bytes, c->stream) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return MAPI_ENOMEM;
  }
  return MAPI_OK;
}

void dev_free(mapi_ctx* c, void* p) {
  if (p) cudaFreeAsync(p, c->stream);
}

// Frees a request's device memory from the calling thread's context (the
// loop's or the builder's).  The packed matrices belong to the builder's
// context: the loop hands them to the builder to free.
void release(Server* sv, ServeReq* q, bool in_builder) {
  mapi_ctx* c = in_builder ? sv->bchild : sv->child;
  if (in_builder) {
    if (q->X) mapi_matrix_free(c, q->X);
    if (q->G) mapi_matrix_free(c, q->G);
  } else if (q->X || q->G) {
    std::lock_guard<std::mutex> lock(sv->mu);
    if (q->X) sv->to_free.push_back(q->X);
    if (q->G) sv->to_free.push_back(q->G);
    sv->bcv.notify_all();
  }
  for (void* p : {(void*)q->C, (void*)q->Cc, (void*)q->Q, q->R, (void*)q->P, (void*)q->w0,
                  (void*)q->wb[0], (void*)q->wb[1]})
    dev_free(c, p);
  q->X = q->G = nullptr;
  q->C = q->Cc = q->Q = q->P = q->w0 = q->wb[0] = q->wb[1] = nullptr;
  q->R = nullptr;
}

// Record the outcome and hand the request back to mapi_poll.
void finish(Server* sv, ServeReq* q, mapi_status s, bool in_builder = false) {
  release(sv, q, in_builder);
  cudaStreamSynchronize(in_builder ? sv->bchild->stream : sv->child->stream);
  const Clock::time_point t = Clock::now();
  std::lock_guard<std::mutex> lock(sv->mu);
  q->res.status = s;
  q->res.queue_ms = ms_between(q->t_submit, q->t_admit);
  q->res.run_ms = ms_between(q->t_admit, t);
  q->res.build_ms = q->t_built > q->t_admit ? ms_between(q->t_admit, q->t_built) : 0.0;
  q->res.latency_ms = ms_between(q->t_submit, t);
  q->res.user = q->r.user;
  q->state = 2;
  sv->used -= q->need;
  sv->resident -= 1;
  sv->cv.notify_all();
}

// Build the request's matrix and vectors on the device (builder thread).
mapi_status build(Server* sv, ServeReq* q) {
  mapi_ctx* c = sv->bchild;
  const mapi_request& r = q->r;
  mapi_status s;
  if (r.kind == MAPI_REQ_PCA) {
    const int D = r.D;
    q->ldc = (D + 3) / 4 * 4;
    const int rows_pad = (D + 63) / 64 * 64;
    const size_t cb = sizeof(float) * (size_t)rows_pad * q->ldc;
    if ((s = mapi_matrix_upload(c, r.X, 0, MAPI_SRC_F32, D, r.N, r.N, r.storage, MAPI_SCALE_AUTO,
                                &q->X)) != MAPI_OK)
      return s;
    if ((s = dev_alloc(c, &q->C, cb)) != MAPI_OK || (s = dev_alloc(c, &q->Cc, cb)) != MAPI_OK ||
        (s = dev_alloc(c, &q->Q, cb)) != MAPI_OK ||
        (s = dev_alloc(c, &q->R, outer_scratch_bytes(r.k, D))) != MAPI_OK ||
        (s = dev_alloc(c, &q->P, sizeof(float) * (size_t)D * r.k)) != MAPI_OK ||
        (s = dev_alloc(c, &q->w0, sizeof(float) * (size_t)D * r.k)) != MAPI_OK ||
        (s = dev_alloc(c, &q->wb[0], sizeof(float) * D)) != MAPI_OK ||
        (s = dev_alloc(c, &q->wb[1], sizeof(float) * D)) != MAPI_OK)
      return s;
    MAPI_CUDA_TRY(c, cudaMemsetAsync(q->C, 0, cb, c->stream));
    MAPI_CUDA_TRY(c, cudaMemsetAsync(q->Cc, 0, cb, c->stream));
    MAPI_CUDA_TRY(c, cudaMemcpyAsync(q->w0, r.w0, sizeof(float) * (size_t)D * r.k,
                                     cudaMemcpyHostToDevice, c->stream));
    if ((s = launch_mincov_raw(c, q->X, r.op, (float)r.cov_denom, q->C, q->ldc, c->stream)) !=
        MAPI_OK)
      return s;
    mapi_matrix_free(c, q->X);  // X is not needed after Eq. (5)
    q->X = nullptr;
    q->n = D;
    q->A = (const uint8_t*)q->C;
    q->row_bytes = q->ldc * 4;
    q->st = MAPI_ST_F32;
    q->view.rows = q->view.cols = D;
    q->view.rows_pad = rows_pad;
    q->view.ld = q->ldc;
    q->view.storage = MAPI_ST_F32;
    q->view.data = q->C;
    return MAPI_OK;
  }
  const int n = r.n;
  const size_t nnz = (size_t)r.indptr[n];
  int* csr = nullptr;
  if ((s = dev_alloc(c, &csr, sizeof(int) * (n + 1 + nnz + 1))) != MAPI_OK) return s;
  cudaMemcpyAsync(csr, r.indptr, sizeof(int) * (n + 1), cudaMemcpyHostToDevice, c->stream);
  if (nnz)
    cudaMemcpyAsync(csr + n + 1, r.indices, sizeof(int) * nnz, cudaMemcpyHostToDevice, c->stream);
  s = mapi_google_matrix(c, csr, csr + n + 1, n, r.alpha, r.storage, &q->G);
  dev_free(c, csr);
  if (s != MAPI_OK) return s;
  if ((s = dev_alloc(c, &q->w0, sizeof(float) * n)) != MAPI_OK ||
      (s = dev_alloc(c, &q->wb[0], sizeof(float) * n)) != MAPI_OK ||
      (s = dev_alloc(c, &q->wb[1], sizeof(float) * n)) != MAPI_OK)
    return s;
  MAPI_CUDA_TRY(c, cudaMemcpyAsync(q->w0, r.w0, sizeof(float) * n, cudaMemcpyHostToDevice,
                                   c->stream));
  q->n = n;
  q->A = (const uint8_t*)q->G->data;
  q->row_bytes = q->G->ld * elem_bytes(q->G->storage);
  q->st = q->G->storage;
  q->view = *q->G;
  q->view.owner = nullptr;
  return MAPI_OK;
}

// A component (or the PageRank solve) has ended with its result in wb[cur].
// Returns true when the whole request is done.
mapi_status component_done(Server* sv, ServeReq* q, bool* all_done) {
  mapi_ctx* c = sv->child;
  const mapi_request& r = q->r;
  *all_done = false;
  q->res.iters[q->comp] = q->it_comp;
  if (r.kind == MAPI_REQ_PAGERANK) {
    MAPI_CUDA_TRY(c, cudaMemcpyAsync(r.out, q->wb[q->cur], sizeof(float) * q->n,
                                     cudaMemcpyDeviceToHost, c->stream));
    MAPI_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    *all_done = true;
    return MAPI_OK;
  }
  const int D = r.D;
  MAPI_CUDA_TRY(c, cudaMemcpyAsync(q->P + (size_t)q->comp * D, q->wb[q->cur], sizeof(float) * D,
                                   cudaMemcpyDeviceToDevice, c->stream));
  q->comp += 1;
  if (q->comp == r.k) {
    MAPI_CUDA_TRY(c, cudaMemcpyAsync(r.out, q->P, sizeof(float) * (size_t)D * r.k,
                                     cudaMemcpyDeviceToHost, c->stream));
    MAPI_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    *all_done = true;
    return MAPI_OK;
  }
  // Alg. 2 step 6: C_c = C - sum_{m<c} P_m C
  mapi_status s = outer_prepare(c);
  if (s == MAPI_OK)
    s = launch_deflate_mincov(c, r.op, q->P, D, q->comp, D, q->C, q->ldc, q->Q, q->R, r.k,
                              outer_stride(D), q->Cc, c->stream);
  if (s != MAPI_OK) return s;
  q->A = (const uint8_t*)q->Cc;
  q->view.data = q->Cc;
  q->it_comp = 0;
  q->resumed = false;
  return MAPI_OK;
}

// w / ||w||_2 in place (Alg. 1's optional last step) for a wide solve that
// met its stop rule inside a round that was not its last.
__global__ void k_l2_normalize(float* w, int n) {
  __shared__ float sh[33];
  Kahan k;
  for (int i = threadIdx.x; i < n; i += blockDim.x) k.add(w[i] * w[i]);
  const float s = sqrtf(block_sum<1024>(k.value(), sh));
  if (!(s > 0.f)) return;
  for (int i = threadIdx.x; i < n; i += blockDim.x) w[i] = w[i] / s;
}

struct StepOutcome {
  int iters = 0, status = MAPI_OK;
  float delta = 0.f;
  bool converged_early = false;  // stop rule met in a round that was not the last
};

// Hands one round's outcome of a solve to its request; true if it ended.
bool absorb(Server* sv, ServeReq* q, const StepOutcome& o, bool last) {
  q->it_comp += o.iters;
  q->cur ^= 1;
  q->resumed = true;
  q->res.last_delta = o.delta;
  if (o.status != MAPI_OK) {
    q->res.iters[q->comp] = q->it_comp;
    finish(sv, q, (mapi_status)o.status);
    return true;
  }
  const bool converged = q->r.tol_l1 > 0 && o.delta < (float)q->r.tol_l1;
  if (!converged && q->it_comp < q->r.max_iters) return false;
  if (converged && !last && o.converged_early) {
    k_l2_normalize<<<1, 1024, 0, sv->child->stream>>>(q->wb[q->cur], q->n);
    if (cudaGetLastError() != cudaSuccess) {
      finish(sv, q, MAPI_ECUDA);
      return true;
    }
  }
  bool all = false;
  const mapi_status cs = component_done(sv, q, &all);
  if (cs != MAPI_OK || all) {
    finish(sv, q, cs);
    return true;
  }
  return false;
}

// One round over every resident solve: the wide ones on the loop's stream,
// one after another on the whole GPU; the rest in one batched launch per
// (storage, op) on a second stream at the same time.
void run_round(Server* sv) {
  mapi_ctx* c = sv->child;
  std::vector<ServeReq*> wide;
  std::map<std::pair<int, int>, std::vector<ServeReq*>> groups;
  for (ServeReq* q : sv->live) {
    if (q->n >= kWideN) wide.push_back(q);
    else groups[{(int)q->st, (int)q->r.op}].push_back(q);
  }
  // with nobody waiting to be admitted, a round takes every solve to the end
  // of its current component (fewer host round trips per request); otherwise
  // rounds stay short so that arrivals are admitted soon
  bool waiting;
  {
    std::lock_guard<std::mutex> lock(sv->mu);
    waiting = !sv->queue.empty() || !sv->built.empty() || !sv->to_build.empty();
  }
  auto steps_of = [waiting](const ServeReq* q) {
    const int rem = q->r.max_iters - q->it_comp;
    const int cap = waiting ? kRoundSteps : kLongRoundSteps;
    return rem < cap ? rem : cap;
  };
  // deflations and copies that ended the previous round ran on the loop's
  // stream: the batched launches of this round come after them
  if (cudaEventRecord(sv->round_start, c->stream) != cudaSuccess ||
      cudaStreamWaitEvent(sv->batch_stream, sv->round_start, 0) != cudaSuccess) {
    cudaGetLastError();
    cudaStreamSynchronize(c->stream);
  }
  std::vector<mapi_status> wide_err(wide.size(), MAPI_OK);
  if ((int)wide.size() > sv->wide_cap) {
    if (sv->wide_ctl) cudaFreeHost(sv->wide_ctl);
    sv->wide_cap = (int)wide.size() * 2;
    if (cudaMallocHost(&sv->wide_ctl, sizeof(IterCtl) * sv->wide_cap) != cudaSuccess) {
      cudaGetLastError();
      sv->wide_ctl = nullptr;
      sv->wide_cap = 0;
    }
  }
  for (size_t i = 0; i < wide.size(); ++i) {
    ServeReq* q = wide[i];
    if (!sv->wide_ctl) {
      wide_err[i] = MAPI_ENOMEM;
      continue;
    }
    const int steps = steps_of(q);
    const bool last = steps == q->r.max_iters - q->it_comp;
    const unsigned flags = (q->resumed ? MAPI_FLAG_RAW_START : 0u) | (last ? MAPI_FLAG_FINAL_L2 : 0u);
    const float* w0 = q->resumed ? q->wb[q->cur] : q->w0 + (size_t)q->comp * q->n;
    mapi_status s = prepare_solve(c, &q->view, 1);
    if (s == MAPI_OK)
      s = enqueue_solve(c, c->stream, &q->view, q->r.op, 1, w0, q->n, steps, q->r.tol_l1, flags,
                        q->wb[q->cur ^ 1], q->n);
    if (s == MAPI_OK && cudaMemcpyAsync(&sv->wide_ctl[i], c->ctl.p, sizeof(IterCtl),
                                        cudaMemcpyDeviceToHost, c->stream) != cudaSuccess) {
      cudaGetLastError();
      s = MAPI_ECUDA;
    }
    wide_err[i] = s;
  }
  std::vector<ServeReq*> ended;
  for (auto& kv : groups) {
    std::vector<ServeReq*>& qs = kv.second;
    std::vector<BatchDev> items(qs.size());
    for (size_t i = 0; i < qs.size(); ++i) {
      ServeReq* q = qs[i];
      const int steps = steps_of(q);
      BatchDev& b = items[i];
      b.A = q->A;
      b.row_bytes = q->row_bytes;
      b.n = q->n;
      b.chunks = (int)(q->row_bytes / 16);
      b.w0 = q->resumed ? q->wb[q->cur] : q->w0 + (size_t)q->comp * q->n;
      b.w_out = q->wb[q->cur ^ 1];
      b.max_iters = steps;
      b.tol = (float)q->r.tol_l1;
      b.raw_start = q->resumed ? 1 : 0;
      b.final_l2 = 1;
      b.last = steps == q->r.max_iters - q->it_comp ? 1 : 0;
    }
    std::vector<int> res;
    std::vector<float> dl;
    const mapi_status s = batched_run(c, sv->batch_stream, items, (mapi_op)kv.first.second,
                                      (mapi_storage)kv.first.first, 1, res, dl);
    for (size_t i = 0; i < qs.size(); ++i) {
      ServeReq* q = qs[i];
      if (s != MAPI_OK) {
        finish(sv, q, s);
        ended.push_back(q);
        continue;
      }
      StepOutcome o;
      o.iters = res[2 * i];
      o.status = res[2 * i + 1];
      o.delta = dl[i];
      // the batched kernel itself applies the l2 step when the stop rule ends a solve
      if (absorb(sv, q, o, true)) ended.push_back(q);
    }
  }
  if (!wide.empty() && cudaStreamSynchronize(c->stream) != cudaSuccess) {
    cudaGetLastError();
    for (auto& e : wide_err)
      if (e == MAPI_OK) e = MAPI_ECUDA;
  }
  for (size_t i = 0; i < wide.size(); ++i) {
    ServeReq* q = wide[i];
    if (wide_err[i] != MAPI_OK) {
      finish(sv, q, wide_err[i]);
      ended.push_back(q);
      continue;
    }
    const int steps = steps_of(q);
    const bool last = steps == q->r.max_iters - q->it_comp;
    const VecState& v = sv->wide_ctl[i].v[0];
    StepOutcome o;
    o.iters = v.iters;
    o.status = v.status;
    o.delta = v.delta;
    o.converged_early = v.iters < steps;
    if (absorb(sv, q, o, last)) ended.push_back(q);
  }
  if (!ended.empty()) {
    std::vector<ServeReq*> keep;
    for (ServeReq* q : sv->live)
      if (std::find(ended.begin(), ended.end(), q) == ended.end()) keep.push_back(q);
    sv->live.swap(keep);
  }
}

// A queued request fits now (resident bytes and slots).
bool admissible(const Server* sv) {
  return !sv->queue.empty() && sv->resident < sv->parent->max_slots &&
         sv->used + sv->queue.front()->need <= sv->budget;
}

void loop(Server* sv) {
  cudaSetDevice(sv->child->device);
  for (;;) {
    std::vector<ServeReq*> ready, dropped;
    {
      std::unique_lock<std::mutex> lock(sv->mu);
      sv->cv.wait(lock, [&] {
        return sv->stop || admissible(sv) || !sv->live.empty() || !sv->built.empty();
      });
      if (sv->stop) break;
      // admission: the builder takes it from here
      bool any = false;
      while (admissible(sv)) {
        ServeReq* q = sv->queue.front();
        sv->queue.pop_front();
        sv->used += q->need;
        sv->resident += 1;
        q->state = 1;
        q->t_admit = Clock::now();
        sv->to_build.push_back(q);
        any = true;
      }
      if (any) sv->bcv.notify_all();
      while (!sv->built.empty()) {
        ready.push_back(sv->built.front());
        sv->built.pop_front();
      }
    }
    for (ServeReq* q : ready) sv->live.push_back(q);
    {
      std::lock_guard<std::mutex> lock(sv->mu);
      for (ServeReq* q : sv->live)
        if (q->cancel) dropped.push_back(q);
    }
    for (ServeReq* q : dropped) {
      sv->live.erase(std::find(sv->live.begin(), sv->live.end(), q));
      finish(sv, q, MAPI_ECANCELLED);
    }
    if (!sv->live.empty()) run_round(sv);
  }
  // shutting down: everything still resident is dropped
  for (ServeReq* q : sv->live) {
    release(sv, q, false);
    q->state = 2;
  }
  sv->live.clear();
  cudaStreamSynchronize(sv->child->stream);
}

// Builder thread: uploads and builds admitted requests on its own context
// and stream while the loop runs rounds, and frees finished matrices.
void builder(Server* sv) {
  cudaSetDevice(sv->bchild->device);
  for (;;) {
    ServeReq* q = nullptr;
    std::vector<mapi_mat*> frees;
    {
      std::unique_lock<std::mutex> lock(sv->mu);
      sv->bcv.wait(lock, [&] {
        return sv->bstop || !sv->to_build.empty() || !sv->to_free.empty();
      });
      frees.swap(sv->to_free);
      if (!sv->bstop && !sv->to_build.empty()) {
        q = sv->to_build.front();
        sv->to_build.pop_front();
      }
    }
    for (mapi_mat* m : frees) mapi_matrix_free(sv->bchild, m);
    if (!q) {
      std::lock_guard<std::mutex> lock(sv->mu);
      if (sv->bstop && sv->to_free.empty()) break;
      continue;
    }
    bool cancelled;
    {
      std::lock_guard<std::mutex> lock(sv->mu);
      cancelled = q->cancel;
    }
    if (cancelled) {
      finish(sv, q, MAPI_ECANCELLED, true);
      continue;
    }
    mapi_status s = build(sv, q);
    if (s == MAPI_OK && cudaStreamSynchronize(sv->bchild->stream) != cudaSuccess) {
      cudaGetLastError();
      s = MAPI_ECUDA;
    }
    if (s != MAPI_OK) {
      finish(sv, q, s, true);
      continue;
    }
    q->t_built = Clock::now();
    {
      std::lock_guard<std::mutex> lock(sv->mu);
      sv->built.push_back(q);
    }
    sv->cv.notify_all();
  }
  // requests admitted but never built
  std::lock_guard<std::mutex> lock(sv->mu);
  for (ServeReq* q : sv->to_build) q->state = 2;
  sv->to_build.clear();
}

mapi_status ensure_server(mapi_ctx* ctx, Server** out) {
  std::lock_guard<std::mutex> lock(ctx->server_mu);
  if (!ctx->server) {
    auto* sv = new (std::nothrow) Server();
    if (!sv) return MAPI_ENOMEM;
    sv->parent = ctx;
    mapi_config cfg{};
    cfg.device = ctx->device;
    mapi_status s = mapi_create(&cfg, &sv->child);
    if (s != MAPI_OK) {
      delete sv;
      return s;
    }
    if ((s = mapi_create(&cfg, &sv->bchild)) != MAPI_OK) {
      mapi_destroy(sv->child);
      delete sv;
      return s;
    }
    sv->child->gemv_clusters = false;
    // the served matrices live within the admission budget: no kept blocks
    sv->child->pool_matrices = false;
    sv->bchild->pool_matrices = false;
    {
      int prev = 0;
      cudaGetDevice(&prev);
      cudaSetDevice(ctx->device);
      cudaError_t e = cudaStreamCreateWithFlags(&sv->batch_stream, cudaStreamNonBlocking);
      if (e == cudaSuccess)
        e = cudaEventCreateWithFlags(&sv->round_start, cudaEventDisableTiming);
      cudaSetDevice(prev);
      if (e != cudaSuccess) {
        cudaGetLastError();
        mapi_destroy(sv->child);
        delete sv;
        return MAPI_ECUDA;
      }
    }
    sv->child->batch_rows_per_warp[0][0] = ctx->batch_rows_per_warp[0][0];
    sv->child->batch_rows_per_warp[1][0] = ctx->batch_rows_per_warp[1][0];
    sv->budget = ctx->hbm_budget;
    if (!sv->budget) {
      int prev = 0;
      cudaGetDevice(&prev);
      cudaSetDevice(ctx->device);
      size_t fr = 0, tot = 0;
      if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) cudaGetLastError();
      cudaSetDevice(prev);
      sv->budget = fr / 10 * 8;
    }
    sv->th = std::thread(loop, sv);
    sv->bth = std::thread(builder, sv);
    ctx->server = sv;
  }
  *out = ctx->server;
  return MAPI_OK;
}

}  // namespace

void server_shutdown(mapi_ctx* ctx) {
  Server* sv = nullptr;
  {
    std::lock_guard<std::mutex> lock(ctx->server_mu);
    sv = ctx->server;
    ctx->server = nullptr;
  }
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lock(sv->mu);
    sv->stop = true;
  }
  sv->cv.notify_all();
  if (sv->th.joinable()) sv->th.join();
  {
    std::lock_guard<std::mutex> lock(sv->mu);
    sv->bstop = true;
  }
  sv->bcv.notify_all();
  if (sv->bth.joinable()) sv->bth.join();
  // requests the builder held or had built: their buffers go with the contexts
  for (ServeReq* q : sv->built) release(sv, q, true);
  sv->built.clear();
  for (auto& kv : sv->tickets) delete kv.second;
  if (sv->round_start) cudaEventDestroy(sv->round_start);
  if (sv->batch_stream) cudaStreamDestroy(sv->batch_stream);
  if (sv->wide_ctl) cudaFreeHost(sv->wide_ctl);
  mapi_destroy(sv->child);
  mapi_destroy(sv->bchild);
  delete sv;
}

}  // namespace mapi

using namespace mapi;

extern "C" mapi_status mapi_submit(mapi_ctx* ctx, const mapi_request* req, uint64_t* ticket) {
  if (!ctx) return MAPI_EINVAL;
  if (!ticket) return fail(ctx, MAPI_EINVAL, "null ticket");
  *ticket = 0;
  if (check_request(req) != MAPI_OK) return fail(ctx, MAPI_EINVAL, "bad request");
  Server* sv = nullptr;
  mapi_status s = ensure_server(ctx, &sv);
  if (s != MAPI_OK) return fail(ctx, s, "serving loop could not start");
  auto* q = new (std::nothrow) ServeReq();
  if (!q) return fail(ctx, MAPI_ENOMEM, "request record");
  q->r = *req;
  q->need = request_bytes(sv->child, *req);
  if (q->need > sv->budget) {
    delete q;
    return fail(ctx, MAPI_EBUDGET, "request needs more device memory than the budget");
  }
  q->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lock(sv->mu);
    q->ticket = sv->next_ticket++;
    sv->tickets[q->ticket] = q;
    sv->queue.push_back(q);
  }
  sv->cv.notify_all();
  *ticket = q->ticket;
  return MAPI_OK;
}

extern "C" mapi_status mapi_poll(mapi_ctx* ctx, uint64_t ticket, mapi_result* out) {
  if (!ctx) return MAPI_EINVAL;
  Server* sv = nullptr;
  {
    std::lock_guard<std::mutex> lock(ctx->server_mu);
    sv = ctx->server;
  }
  if (!sv) return fail(ctx, MAPI_EINVAL, "unknown ticket");
  ServeReq* q = nullptr;
  {
    std::lock_guard<std::mutex> lock(sv->mu);
    auto it = sv->tickets.find(ticket);
    if (it == sv->tickets.end()) return fail(ctx, MAPI_EINVAL, "unknown ticket");
    if (it->second->state != 2) return MAPI_EAGAIN;
    q = it->second;
    sv->tickets.erase(it);
  }
  if (out) *out = q->res;
  const mapi_status s = q->res.status;
  delete q;
  return s;
}

extern "C" mapi_status mapi_cancel(mapi_ctx* ctx, uint64_t ticket) {
  if (!ctx) return MAPI_EINVAL;
  Server* sv = nullptr;
  {
    std::lock_guard<std::mutex> lock(ctx->server_mu);
    sv = ctx->server;
  }
  if (!sv) return fail(ctx, MAPI_EINVAL, "unknown ticket");
  std::lock_guard<std::mutex> lock(sv->mu);
  auto it = sv->tickets.find(ticket);
  if (it == sv->tickets.end()) return fail(ctx, MAPI_EINVAL, "unknown ticket");
  ServeReq* q = it->second;
  if (q->state == 0) {
    sv->queue.erase(std::find(sv->queue.begin(), sv->queue.end(), q));
    q->t_admit = Clock::now();
    q->res.status = MAPI_ECANCELLED;
    q->res.queue_ms = ms_between(q->t_submit, q->t_admit);
    q->res.latency_ms = q->res.queue_ms;
    q->res.user = q->r.user;
    q->state = 2;
  } else if (q->state == 1) {
    q->cancel = true;
  }
  sv->cv.notify_all();
  return MAPI_OK;
}
