// C ABI entry points (include/mapi.h): context, matrices, solves.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "mapi_internal.cuh"

using namespace mapi;

namespace mapi {

mapi_status fail(mapi_ctx* ctx, mapi_status s, const std::string& msg) {
  if (ctx) ctx->last_error = msg;
  return s;
}

mapi_status cuda_fail(mapi_ctx* ctx, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  return fail(ctx, MAPI_ECUDA, m);
}

void destroy_graph(mapi_ctx* ctx, GraphEntry& g);

static void drop_graphs(mapi_ctx* ctx) {
  for (auto& kv : ctx->graphs) destroy_graph(ctx, kv.second);
  ctx->graphs.clear();
}

mapi_status ensure(mapi_ctx* ctx, DevBuf& b, size_t bytes) {
  if (b.bytes >= bytes && b.p) return MAPI_OK;
  // graphs captured earlier may point at the old buffer
  if (b.p) {
    cudaStreamSynchronize(ctx->stream);
    drop_graphs(ctx);
    cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
  }
  size_t want = bytes < 256 ? 256 : bytes;
  cudaError_t e = cudaMalloc(&b.p, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    return fail(ctx, MAPI_ENOMEM, "device allocation of " + std::to_string(want) + " bytes failed");
  }
  b.bytes = want;
  return MAPI_OK;
}

cudaEvent_t prof_begin(mapi_ctx* ctx, cudaStream_t s) {
  if (!ctx->prof_on) return nullptr;
  cudaEvent_t e = nullptr;
  if (!ctx->ev_pool.empty()) {
    e = ctx->ev_pool.back();
    ctx->ev_pool.pop_back();
  } else if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (ctx->capturing) cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
  else cudaEventRecord(e, s);
  return e;
}

void prof_end(mapi_ctx* ctx, cudaStream_t s, cudaEvent_t a, int cls, double bytes,
              double terms, int count) {
  if (!a) return;
  cudaEvent_t b = prof_begin(ctx, s);
  if (!b) {
    ctx->ev_pool.push_back(a);
    return;
  }
  std::vector<ProfMark>* sink = ctx->mark_sink ? ctx->mark_sink : &ctx->pending;
  sink->push_back(ProfMark{cls, a, b, bytes, terms, count});
}

void prof_collect(mapi_ctx* ctx, std::vector<ProfMark>& marks, bool recycle) {
  for (auto& m : marks) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, m.a, m.b) == cudaSuccess && m.cls >= 0 &&
        m.cls < MAPI_KC_COUNT) {
      ctx->stats.timed[m.cls] += (uint64_t)m.count;
      ctx->stats.ms[m.cls] += ms;
      ctx->stats.bytes[m.cls] += m.bytes;
      ctx->stats.terms[m.cls] += m.terms;
    } else {
      cudaGetLastError();
    }
    if (recycle) {
      ctx->ev_pool.push_back(m.a);
      ctx->ev_pool.push_back(m.b);
    }
  }
  if (recycle) marks.clear();
}

void destroy_graph(mapi_ctx* ctx, GraphEntry& g) {
  if (g.exec) cudaGraphExecDestroy(g.exec);
  g.exec = nullptr;
  for (auto& m : g.marks) {
    ctx->ev_pool.push_back(m.a);
    ctx->ev_pool.push_back(m.b);
  }
  g.marks.clear();
}

mapi_status launch_cached_graph(mapi_ctx* ctx, const std::vector<int64_t>& key,
                                const std::function<mapi_status(cudaStream_t)>& enqueue,
                                GraphEntry** out) {
  auto it = ctx->graphs.find(key);
  if (it == ctx->graphs.end()) {
    if (ctx->graphs.size() >= 32) {  // evict the least recently used graph
      auto victim = ctx->graphs.begin();
      for (auto j = ctx->graphs.begin(); j != ctx->graphs.end(); ++j)
        if (j->second.last_use < victim->second.last_use) victim = j;
      cudaStreamSynchronize(ctx->stream);
      destroy_graph(ctx, victim->second);
      ctx->graphs.erase(victim);
    }
    GraphEntry entry;
    cudaGraph_t graph = nullptr;
    MAPI_CUDA_TRY(ctx, cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal));
    ctx->capturing = true;
    ctx->capture_count = 0;
    ctx->mark_sink = &entry.marks;
    mapi_status s = enqueue(ctx->capture_stream);
    ctx->capturing = false;
    ctx->mark_sink = nullptr;
    entry.nodes = ctx->capture_count;
    cudaError_t e = cudaStreamEndCapture(ctx->capture_stream, &graph);
    if (s != MAPI_OK || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      destroy_graph(ctx, entry);
      cudaGetLastError();
      return s != MAPI_OK ? s : cuda_fail(ctx, e, "cudaStreamEndCapture");
    }
    e = cudaGraphInstantiate(&entry.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      destroy_graph(ctx, entry);
      return cuda_fail(ctx, e, "cudaGraphInstantiate");
    }
    it = ctx->graphs.emplace(key, std::move(entry)).first;
  }
  it->second.last_use = ++ctx->use_clock;
  MAPI_CUDA_TRY(ctx, cudaGraphLaunch(it->second.exec, ctx->stream));
  *out = &it->second;
  return MAPI_OK;
}

void finish_graph(mapi_ctx* ctx, GraphEntry* g) {
  ctx->stats.launches += g->nodes;
  prof_collect(ctx, g->marks, false);
  prof_collect(ctx, ctx->pending, true);
}

}  // namespace mapi

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace

namespace mapi {

void release_matrix_pool(mapi_ctx* ctx) {
  if (ctx->mat_pool.empty()) return;
  cudaStreamSynchronize(ctx->stream);
  for (auto& b : ctx->mat_pool) cudaFree(b.first);
  ctx->mat_pool.clear();
}

mapi_status free_matrix(mapi_ctx* ctx, mapi_mat* m) {
  // graphs captured for this matrix can never be replayed again
  for (auto it = ctx->graphs.begin(); it != ctx->graphs.end();) {
    if (it->first.size() > 1 && it->first[1] == (int64_t)m->id) {
      destroy_graph(ctx, it->second);
      it = ctx->graphs.erase(it);
    } else {
      ++it;
    }
  }
  if (m->data) {
    // kept for the next matrix of this size (a repeated upload of the same
    // shape then needs neither cudaMalloc nor the synchronising cudaFree)
    if (ctx->pool_matrices && (int)ctx->mat_pool.size() < kMatPoolBlocks) {
      ctx->mat_pool.emplace_back(m->data, m->bytes);
    } else {
      cudaFree(m->data);
    }
  }
  if (m->row_scale) cudaFree(m->row_scale);
  if (m->row_exp) cudaFree(m->row_exp);
  ctx->mats.erase(m);
  delete m;
  return MAPI_OK;
}

mapi_status alloc_matrix(mapi_ctx* ctx, int rows, int cols, mapi_storage st,
                         mapi_mat** out) {
  auto* m = new (std::nothrow) mapi_mat();
  if (!m) return fail(ctx, MAPI_ENOMEM, "host allocation failed");
  const int eb = elem_bytes(st);
  m->rows = rows;
  m->cols = cols;
  m->rows_pad = (rows + 63) / 64 * 64;
  m->ld = ((int64_t)cols * eb + 15) / 16 * 16 / eb;
  m->storage = st;
  m->bytes = (size_t)m->rows_pad * m->ld * eb;
  for (size_t i = 0; i < ctx->mat_pool.size(); ++i)
    if (ctx->mat_pool[i].second == m->bytes) {
      m->data = ctx->mat_pool[i].first;
      ctx->mat_pool.erase(ctx->mat_pool.begin() + i);
      break;
    }
  if (!m->data && cudaMalloc(&m->data, m->bytes) != cudaSuccess) {
    cudaGetLastError();
    // the kept blocks first go back to the device, then one more try
    release_matrix_pool(ctx);
    if (cudaMalloc(&m->data, m->bytes) != cudaSuccess) {
      cudaGetLastError();
      m->data = nullptr;
      delete m;
      return fail(ctx, MAPI_ENOMEM, "matrix allocation failed");
    }
  }
  if (st == MAPI_ST_FP8E4M3_ROWPOW2) {
    if (cudaMalloc(&m->row_scale, sizeof(float) * m->rows_pad) != cudaSuccess ||
        cudaMalloc(&m->row_exp, sizeof(int) * m->rows_pad) != cudaSuccess) {
      cudaGetLastError();
      m->owner = ctx;
      ctx->mats.insert(m);
      free_matrix(ctx, m);
      return fail(ctx, MAPI_ENOMEM, "row scale allocation failed");
    }
  }
  m->owner = ctx;
  m->id = ctx->next_mat_id++;
  ctx->mats.insert(m);
  *out = m;
  return MAPI_OK;
}

}  // namespace mapi

namespace {

bool valid_matrix(mapi_ctx* ctx, const mapi_mat* m) {
  return m && ctx && ctx->mats.count(const_cast<mapi_mat*>(m));
}

// Pack a device FP32 source (rows x cols, leading dimension ld) into `st`.
mapi_status pack_from_device(mapi_ctx* ctx, const float* src, int rows, int cols,
                             int64_t ld, mapi_storage st, int int_scale_log2,
                             mapi_mat** out) {
  mapi_status s;
  if ((s = ensure(ctx, ctx->aux, 64)) != MAPI_OK) return s;
  int* flag = (int*)ctx->aux.p;
  unsigned* mx = (unsigned*)((char*)ctx->aux.p + 16);
  MAPI_CUDA_TRY(ctx, cudaMemsetAsync(ctx->aux.p, 0, 64, ctx->stream));
  if ((s = launch_check_finite(ctx, src, rows, cols, ld, flag)) != MAPI_OK) return s;
  int q = 0;
  if (is_int_storage(st) && int_scale_log2 == MAPI_SCALE_AUTO) {
    if ((s = launch_absmax(ctx, src, rows, cols, ld, mx)) != MAPI_OK) return s;
  }
  int host[8] = {0};
  MAPI_CUDA_TRY(ctx, cudaMemcpyAsync(host, ctx->aux.p, 32, cudaMemcpyDeviceToHost, ctx->stream));
  MAPI_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  if (host[0]) return fail(ctx, MAPI_ENONFINITE, "matrix has a NaN or Inf entry");
  if (is_int_storage(st)) {
    const double qmax = (st == MAPI_ST_I16) ? 32767.0 : 127.0;
    if (int_scale_log2 == MAPI_SCALE_AUTO) {
      float fmx;
      unsigned bits = (unsigned)host[4];
      std::memcpy(&fmx, &bits, 4);
      q = 24;
      while (q >= 0 && (double)fmx * std::ldexp(1.0, q) > qmax) --q;
      if (q < 0) return fail(ctx, MAPI_EINVAL, "entries too large for integer storage");
    } else {
      q = int_scale_log2;
      if (q < 0 || q > 24) return fail(ctx, MAPI_EINVAL, "int_scale_log2 outside [0, 24]");
      // an explicit q must still keep every entry in range
      if ((s = launch_absmax(ctx, src, rows, cols, ld, mx)) != MAPI_OK) return s;
      MAPI_CUDA_TRY(ctx, cudaMemcpyAsync(host, ctx->aux.p, 32, cudaMemcpyDeviceToHost, ctx->stream));
      MAPI_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
      float fmx;
      unsigned bits = (unsigned)host[4];
      std::memcpy(&fmx, &bits, 4);
      if ((double)fmx * std::ldexp(1.0, q) > qmax)
        return fail(ctx, MAPI_EINVAL, "entries exceed the integer range at this scale");
    }
  }
  mapi_mat* m = nullptr;
  if ((s = alloc_matrix(ctx, rows, cols, st, &m)) != MAPI_OK) return s;
  m->q = q;
  if (st == MAPI_ST_FP8E4M3_ROWPOW2) {
    if ((s = launch_fp8_rowexp(ctx, src, ld, m, flag)) != MAPI_OK) { free_matrix(ctx, m); return s; }
    MAPI_CUDA_TRY(ctx, cudaMemcpyAsync(host, flag, 4, cudaMemcpyDeviceToHost, ctx->stream));
    MAPI_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    if (host[0] & 2) {
      free_matrix(ctx, m);
      return fail(ctx, MAPI_EINVAL, "FP8 row scale above 2^7 (row maximum > 57344)");
    }
  }
  if ((s = launch_pack(ctx, src, ld, m)) != MAPI_OK) { free_matrix(ctx, m); return s; }
  *out = m;
  return MAPI_OK;
}

uint64_t fbits(double d) {
  uint64_t u;
  std::memcpy(&u, &d, 8);
  return u;
}

}  // namespace

namespace {
// Keeps the first phase's state of a switched solve and stops the second
// phase when the first failed.
__global__ void k_keep_phase(const IterCtl* ctl, VecState* keep, int* abort) {
  const VecState st = ctl->v[0];
  *keep = st;
  *abort = st.status != MAPI_OK;
}
}  // namespace

extern "C" {

const char* mapi_status_str(mapi_status s) {
  switch (s) {
    case MAPI_OK: return "ok";
    case MAPI_EINVAL: return "invalid argument";
    case MAPI_ENOMEM: return "out of memory";
    case MAPI_EBUDGET: return "request exceeds the HBM budget";
    case MAPI_EZERONORM: return "zero norm";
    case MAPI_ENONFINITE: return "non-finite value";
    case MAPI_EAGAIN: return "pending";
    case MAPI_ETIMEOUT: return "device wait timed out";
    case MAPI_ECANCELLED: return "cancelled";
    case MAPI_ECUDA: return "CUDA error";
    case MAPI_ENOTSUP: return "not supported";
  }
  return "unknown status";
}

const char* mapi_last_error(const mapi_ctx* ctx) {
  return ctx ? ctx->last_error.c_str() : "";
}

mapi_status mapi_create(const mapi_config* cfg, mapi_ctx** out) {
  if (!cfg || !out) return MAPI_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev) {
    cudaGetLastError();
    return MAPI_EINVAL;
  }
  auto* ctx = new (std::nothrow) mapi_ctx();
  if (!ctx) return MAPI_ENOMEM;
  ctx->device = cfg->device;
  DeviceGuard g(ctx->device);
  cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, ctx->device);
  int l2 = 0;
  cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, ctx->device);
  ctx->l2_bytes = (size_t)l2;
  if (cfg->cuda_stream) {
    ctx->stream = (cudaStream_t)cfg->cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete ctx;
      return MAPI_ECUDA;
    }
    ctx->own_stream = true;
  }
  if (cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMallocHost(&ctx->ctl_host, sizeof(IterCtl)) != cudaSuccess ||
      cudaMallocHost(&ctx->rec_host, sizeof(int) * 256) != cudaSuccess) {
    cudaGetLastError();
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return MAPI_ECUDA;
  }
  ctx->hbm_budget = cfg->hbm_budget_bytes;
  ctx->max_slots = cfg->max_slots > 0 ? cfg->max_slots : 64;
  if (cfg->tune_cache_path) ctx->tune_cache_path = cfg->tune_cache_path;
  *out = ctx;
  return MAPI_OK;
}

mapi_status mapi_destroy(mapi_ctx* ctx) {
  if (!ctx) return MAPI_EINVAL;
  server_shutdown(ctx);  // served requests still open are dropped
  DeviceGuard g(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  for (auto& kv : ctx->graphs) destroy_graph(ctx, kv.second);
  ctx->graphs.clear();
  prof_collect(ctx, ctx->pending, true);
  std::set<mapi_mat*> ms = ctx->mats;
  for (auto* m : ms) free_matrix(ctx, m);
  release_matrix_pool(ctx);
  for (DevBuf* b : {&ctx->ypart, &ctx->wbuf0, &ctx->wbuf1, &ctx->ctl, &ctx->aux, &ctx->mcpart,
                    &ctx->pca_c0, &ctx->pca_c1, &ctx->pca_q, &ctx->pca_defl, &ctx->batch,
                    &ctx->hyb, &ctx->outer, &ctx->img, &ctx->pair_phases, &ctx->upload_staging})
    if (b->p) cudaFree(b->p);
  for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
  if (ctx->ctl_host) cudaFreeHost(ctx->ctl_host);
  if (ctx->rec_host) cudaFreeHost(ctx->rec_host);
  if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return MAPI_OK;
}

mapi_status mapi_matrix_upload(mapi_ctx* ctx, const void* src, int src_is_device,
                               int src_dtype, int rows, int cols, int64_t ld,
                               mapi_storage storage, int int_scale_log2,
                               mapi_mat** out) {
  if (!ctx || !src || !out) return fail(ctx, MAPI_EINVAL, "null argument");
  *out = nullptr;
  if (src_dtype != MAPI_SRC_F32) return fail(ctx, MAPI_EINVAL, "source must be FP32");
  if (rows <= 0 || cols <= 0 || ld < cols) return fail(ctx, MAPI_EINVAL, "bad shape or ld");
  if ((int)storage < 0 || (int)storage > MAPI_ST_I8) return fail(ctx, MAPI_EINVAL, "bad storage");
  DeviceGuard g(ctx->device);
  const float* dsrc = (const float*)src;
  int64_t dld = ld;
  if (!src_is_device) {
    // the context's staging buffer (grown here without touching the graphs,
    // which never refer to it)
    const size_t bytes = (size_t)rows * cols * sizeof(float);
    DevBuf& sb = ctx->upload_staging;
    if (sb.bytes < bytes) {
      cudaStreamSynchronize(ctx->stream);
      if (sb.p) cudaFree(sb.p);
      sb.p = nullptr;
      sb.bytes = 0;
      if (cudaMalloc(&sb.p, bytes) != cudaSuccess) {
        cudaGetLastError();
        sb.p = nullptr;
        return fail(ctx, MAPI_ENOMEM, "staging allocation failed");
      }
      sb.bytes = bytes;
    }
    // one flat copy when the rows are contiguous, else a pitched one
    cudaError_t e =
        ld == cols
            ? cudaMemcpyAsync(sb.p, src, bytes, cudaMemcpyHostToDevice, ctx->stream)
            : cudaMemcpy2DAsync(sb.p, cols * sizeof(float), src, ld * sizeof(float),
                                cols * sizeof(float), rows, cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "host to device copy");
    dsrc = (const float*)sb.p;
    dld = cols;
  }
  mapi_status s = pack_from_device(ctx, dsrc, rows, cols, dld, storage, int_scale_log2, out);
  // the caller may reuse its host buffer once this returns
  if (!src_is_device) cudaStreamSynchronize(ctx->stream);
  return s;
}

mapi_status mapi_matrix_free(mapi_ctx* ctx, mapi_mat* m) {
  if (!valid_matrix(ctx, m)) return fail(ctx, MAPI_EINVAL, "unknown matrix");
  DeviceGuard g(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  return free_matrix(ctx, m);
}

mapi_status mapi_matrix_info(const mapi_mat* m, int* rows, int* cols, int64_t* ld_elems,
                             int* storage, int* int_scale_log2) {
  if (!m) return MAPI_EINVAL;
  if (rows) *rows = m->rows;
  if (cols) *cols = m->cols;
  if (ld_elems) *ld_elems = m->ld;
  if (storage) *storage = (int)m->storage;
  if (int_scale_log2) *int_scale_log2 = m->q;
  return MAPI_OK;
}

mapi_status mapi_matrix_download(mapi_ctx* ctx, const mapi_mat* m, double* host_out,
                                 int* row_exp) {
  if (!valid_matrix(ctx, m) || !host_out) return fail(ctx, MAPI_EINVAL, "bad argument");
  DeviceGuard g(ctx->device);
  const size_t count = (size_t)m->rows * m->cols;
  float* dtmp = nullptr;
  if (cudaMalloc(&dtmp, count * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, MAPI_ENOMEM, "download buffer");
  }
  mapi_status s = launch_unpack_f32(ctx, m, dtmp);
  std::vector<float> h(count);
  if (s == MAPI_OK) {
    cudaError_t e = cudaMemcpyAsync(h.data(), dtmp, count * sizeof(float),
                                    cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) s = cuda_fail(ctx, e, "download copy");
  }
  if (s == MAPI_OK && row_exp && m->row_exp) {
    cudaError_t e = cudaMemcpy(row_exp, m->row_exp, sizeof(int) * m->rows, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) s = cuda_fail(ctx, e, "row exponents");
  }
  cudaFree(dtmp);
  if (s != MAPI_OK) return s;
  for (size_t i = 0; i < count; ++i) host_out[i] = (double)h[i];
  return MAPI_OK;
}

mapi_status mapi_iterate(mapi_ctx* ctx, const mapi_mat* A, mapi_op op, int nvec,
                         const float* w0, int64_t ldw, int max_iters, double tol_l1,
                         unsigned flags, float* w_out, int* iters_done,
                         double* last_delta) {
  if (!ctx) return MAPI_EINVAL;
  if (!valid_matrix(ctx, A)) return fail(ctx, MAPI_EINVAL, "unknown matrix");
  if (A->rows != A->cols) return fail(ctx, MAPI_EINVAL, "MAPI needs a square matrix");
  if (nvec < 1 || nvec > kMaxVec) return fail(ctx, MAPI_EINVAL, "nvec must be 1..8");
  if (!w0 || !w_out || ldw < A->rows || max_iters < 0)
    return fail(ctx, MAPI_EINVAL, "bad vector arguments");
  if ((int)op < 0 || (int)op > MAPI_OP_DOT) return fail(ctx, MAPI_EINVAL, "bad op");
  if (is_int_storage(A->storage) && op != MAPI_OP_MIN1 && op != MAPI_OP_MIN2)
    return fail(ctx, MAPI_EINVAL, "integer storage supports MIN1 and MIN2 only");
  if (op == MAPI_OP_DIAMOND && (A->storage != MAPI_ST_F32 || nvec != 1))
    return fail(ctx, MAPI_EINVAL, "DIAMOND needs F32 storage and one vector");
  if (is_int_storage(A->storage) && (int64_t)A->cols * 32767 >= 2147483647LL)
    return fail(ctx, MAPI_EINVAL, "integer storage needs n * 32767 < 2^31");
  DeviceGuard g(ctx->device);
  mapi_status s = prepare_solve(ctx, A, nvec);
  if (s != MAPI_OK) return s;

  std::vector<int64_t> key = {1,
                              (int64_t)A->id,
                              (int64_t)op,
                              nvec,
                              (int64_t)(uintptr_t)w0,
                              ldw,
                              max_iters,
                              (int64_t)fbits(tol_l1),
                              (int64_t)flags,
                              (int64_t)(uintptr_t)w_out,
                              (int64_t)(uintptr_t)ctx->wbuf0.p,
                              (int64_t)(uintptr_t)ctx->ypart.p,
                              (int64_t)ctx->prof_on};
  GraphEntry* ge = nullptr;
  s = launch_cached_graph(
      ctx, key,
      [&](cudaStream_t cs) {
        return enqueue_solve(ctx, cs, A, op, nvec, w0, ldw, max_iters, tol_l1, flags, w_out, ldw);
      },
      &ge);
  if (s != MAPI_OK) return s;
  MAPI_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->ctl_host, ctx->ctl.p, sizeof(IterCtl),
                                     cudaMemcpyDeviceToHost, ctx->stream));
  MAPI_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  finish_graph(ctx, ge);
  mapi_status result = MAPI_OK;
  for (int v = 0; v < nvec; ++v) {
    const VecState& st = ctx->ctl_host->v[v];
    if (iters_done) iters_done[v] = st.iters;
    if (last_delta)
      last_delta[v] = is_int_storage(A->storage)
                          ? (st.idelta < 0 ? NAN : std::ldexp((double)st.idelta, -A->q))
                          : (double)st.delta;
    if (result == MAPI_OK && st.status != MAPI_OK) result = (mapi_status)st.status;
  }
  if (result != MAPI_OK) fail(ctx, result, "a vector stopped early with this status");
  return result;
}


mapi_status mapi_iterate_switch(mapi_ctx* ctx, const mapi_mat* A, mapi_op op, const float* w0,
                                int mapi_iters, double mapi_tol, int rpi_iters, double rpi_tol,
                                unsigned flags, float* w_out, int* iters_done,
                                double* last_delta) {
  if (!ctx) return MAPI_EINVAL;
  if (!valid_matrix(ctx, A)) return fail(ctx, MAPI_EINVAL, "unknown matrix");
  if (A->rows != A->cols) return fail(ctx, MAPI_EINVAL, "MAPI needs a square matrix");
  if (!w0 || !w_out || mapi_iters < 0 || rpi_iters < 0)
    return fail(ctx, MAPI_EINVAL, "bad vector arguments");
  if (op != MAPI_OP_MIN1 && op != MAPI_OP_MIN2 && op != MAPI_OP_DIAMOND)
    return fail(ctx, MAPI_EINVAL, "the first phase takes MIN1, MIN2 or DIAMOND");
  if (is_int_storage(A->storage)) return fail(ctx, MAPI_EINVAL, "float storage only");
  if (op == MAPI_OP_DIAMOND && A->storage != MAPI_ST_F32)
    return fail(ctx, MAPI_EINVAL, "DIAMOND needs F32 storage");
  DeviceGuard g(ctx->device);
  mapi_status s = prepare_solve(ctx, A, 1);
  if (s != MAPI_OK) return s;
  const int64_t n = A->rows;
  if ((s = ensure(ctx, ctx->hyb, 256 + sizeof(float) * n)) != MAPI_OK) return s;
  VecState* keep = (VecState*)ctx->hyb.p;
  int* abort = (int*)((char*)ctx->hyb.p + 128);
  float* mid = (float*)((char*)ctx->hyb.p + 256);
  std::vector<int64_t> key = {3,
                              (int64_t)A->id,
                              (int64_t)op,
                              (int64_t)(uintptr_t)w0,
                              mapi_iters,
                              (int64_t)fbits(mapi_tol),
                              rpi_iters,
                              (int64_t)fbits(rpi_tol),
                              (int64_t)flags,
                              (int64_t)(uintptr_t)w_out,
                              (int64_t)(uintptr_t)ctx->wbuf0.p,
                              (int64_t)(uintptr_t)ctx->ypart.p,
                              (int64_t)(uintptr_t)ctx->hyb.p,
                              (int64_t)ctx->prof_on};
  GraphEntry* ge = nullptr;
  s = launch_cached_graph(
      ctx, key,
      [&](cudaStream_t cs) -> mapi_status {
        // MAPI first (Alg. 1), its last iterate handed to regular power
        // iteration (Eq. (1)) for the final convergence
        mapi_status r = enqueue_solve(ctx, cs, A, op, 1, w0, n, mapi_iters, mapi_tol,
                                      flags & MAPI_FLAG_RAW_START, mid, n);
        if (r != MAPI_OK) return r;
        k_keep_phase<<<1, 1, 0, cs>>>((const IterCtl*)ctx->ctl.p, keep, abort);
        MAPI_CUDA_TRY(ctx, cudaGetLastError());
        count_launch(ctx);
        return enqueue_solve(ctx, cs, A, MAPI_OP_DOT, 1, mid, n, rpi_iters, rpi_tol,
                             flags & MAPI_FLAG_FINAL_L2, w_out, n, abort);
      },
      &ge);
  if (s != MAPI_OK) return s;
  VecState first;
  MAPI_CUDA_TRY(ctx, cudaMemcpyAsync(&first, keep, sizeof(VecState), cudaMemcpyDeviceToHost,
                                     ctx->stream));
  MAPI_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->ctl_host, ctx->ctl.p, sizeof(IterCtl),
                                     cudaMemcpyDeviceToHost, ctx->stream));
  MAPI_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  finish_graph(ctx, ge);
  const VecState& second = ctx->ctl_host->v[0];
  if (iters_done) {
    iters_done[0] = first.iters;
    iters_done[1] = first.status == MAPI_OK ? second.iters : 0;
  }
  if (last_delta) {
    last_delta[0] = (double)first.delta;
    last_delta[1] = first.status == MAPI_OK ? (double)second.delta : NAN;
  }
  if (first.status != MAPI_OK) {
    // the MAPI phase failed: its last good iterate is the result
    MAPI_CUDA_TRY(ctx, cudaMemcpyAsync(w_out, mid, sizeof(float) * n, cudaMemcpyDeviceToDevice,
                                       ctx->stream));
    MAPI_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return fail(ctx, (mapi_status)first.status, "the MAPI phase stopped early");
  }
  if (second.status != MAPI_OK) return fail(ctx, (mapi_status)second.status, "the RPI phase failed");
  return MAPI_OK;
}

mapi_status mapi_mincov(mapi_ctx* ctx, const mapi_mat* X, mapi_op op, double denom,
                        float* C_out) {
  if (!ctx) return MAPI_EINVAL;
  if (!valid_matrix(ctx, X) || !C_out) return fail(ctx, MAPI_EINVAL, "bad argument");
  if (op != MAPI_OP_MIN1 && op != MAPI_OP_MIN2 && op != MAPI_OP_DOT)
    return fail(ctx, MAPI_EINVAL, "min-covariance needs MIN1, MIN2 or DOT");
  if (!(denom > 0.0) || !std::isfinite(denom)) return fail(ctx, MAPI_EINVAL, "denom must be > 0");
  DeviceGuard g(ctx->device);
  return launch_mincov_raw(ctx, X, op, (float)denom, C_out, X->rows, ctx->stream);
}

mapi_status mapi_rows_product(mapi_ctx* ctx, const mapi_mat* A, int row_begin, int row_end,
                              mapi_op op, const float* w, float* y_out) {
  if (!ctx) return MAPI_EINVAL;
  if (!valid_matrix(ctx, A) || !w || !y_out) return fail(ctx, MAPI_EINVAL, "bad argument");
  if (row_begin < 0 || row_end < row_begin || row_end > A->rows)
    return fail(ctx, MAPI_EINVAL, "rows outside the matrix");
  DeviceGuard g(ctx->device);
  mapi_status st = launch_rows_raw(ctx, A, row_begin, row_end - row_begin, op, w, y_out,
                                   ctx->stream);
  if (st != MAPI_OK) return st;
  MAPI_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  return MAPI_OK;
}

mapi_status mapi_pair_partial(mapi_ctx* ctx, const mapi_mat* X, mapi_op op, const float* w,
                              float* y_out) {
  if (!ctx) return MAPI_EINVAL;
  if (!valid_matrix(ctx, X) || !w || !y_out) return fail(ctx, MAPI_EINVAL, "bad argument");
  if (op != MAPI_OP_MIN1 && op != MAPI_OP_MIN2 && op != MAPI_OP_DOT)
    return fail(ctx, MAPI_EINVAL, "pair step needs MIN1, MIN2 or DOT");
  DeviceGuard g(ctx->device);
  return run_pair_partial(ctx, X, op, w, y_out);
}

mapi_status mapi_pca_topk(mapi_ctx* ctx, const mapi_mat* X, int k, int mode, mapi_op op,
                          int iters_per_vec, double tol_l1, double cov_denom, const float* w0,
                          float* P_out, int* iters_done) {
  if (!ctx) return MAPI_EINVAL;
  if (!valid_matrix(ctx, X) || !w0 || !P_out) return fail(ctx, MAPI_EINVAL, "bad argument");
  if (k < 1 || k > 64 || k > X->rows) return fail(ctx, MAPI_EINVAL, "k must be 1..min(D, 64)");
  if (op != MAPI_OP_MIN1 && op != MAPI_OP_MIN2 && op != MAPI_OP_DOT)
    return fail(ctx, MAPI_EINVAL, "PCA needs MIN1, MIN2 or DOT");
  if (iters_per_vec < 0) return fail(ctx, MAPI_EINVAL, "iters_per_vec < 0");
  if (!(cov_denom > 0.0) || !std::isfinite(cov_denom))
    return fail(ctx, MAPI_EINVAL, "cov_denom must be > 0");
  DeviceGuard g(ctx->device);
  return run_pca(ctx, X, k, mode, op, iters_per_vec, tol_l1, cov_denom, w0, P_out, iters_done);
}

mapi_status mapi_google_matrix(mapi_ctx* ctx, const int* indptr, const int* indices, int n,
                               double alpha, mapi_storage storage, mapi_mat** out) {
  if (!ctx) return MAPI_EINVAL;
  if (!indptr || !indices || !out || n <= 0) return fail(ctx, MAPI_EINVAL, "bad argument");
  if (!(alpha >= 0.0 && alpha <= 1.0)) return fail(ctx, MAPI_EINVAL, "alpha outside [0, 1]");
  if ((int)storage < 0 || (int)storage > MAPI_ST_I8) return fail(ctx, MAPI_EINVAL, "bad storage");
  *out = nullptr;
  DeviceGuard g(ctx->device);
  const int64_t ld = ((int64_t)n + 3) / 4 * 4;
  float* G = nullptr;
  if (cudaMalloc(&G, sizeof(float) * (size_t)n * ld) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, MAPI_ENOMEM, "Google matrix staging");
  }
  mapi_status s = launch_google(ctx, indptr, indices, n, alpha, G, ld);
  if (s == MAPI_OK) s = pack_from_device(ctx, G, n, n, ld, storage, MAPI_SCALE_AUTO, out);
  cudaStreamSynchronize(ctx->stream);
  cudaFree(G);
  return s;
}

mapi_status mapi_pagerank(mapi_ctx* ctx, const int* indptr, const int* indices, int n,
                          double alpha, mapi_storage storage, mapi_op op, const float* w0,
                          int max_iters, double tol_l1, float* rank_out, int* iters_done,
                          double* last_delta) {
  if (!ctx) return MAPI_EINVAL;
  mapi_mat* G = nullptr;
  mapi_status s = mapi_google_matrix(ctx, indptr, indices, n, alpha, storage, &G);
  if (s != MAPI_OK) return s;
  s = mapi_iterate(ctx, G, op, 1, w0, n, max_iters, tol_l1, MAPI_FLAG_FINAL_L2, rank_out,
                   iters_done, last_delta);
  mapi_matrix_free(ctx, G);
  return s;
}


mapi_status mapi_profile(mapi_ctx* ctx, int enable) {
  if (!ctx) return MAPI_EINVAL;
  ctx->prof_on = enable != 0;
  return MAPI_OK;
}

mapi_status mapi_pair_phases(mapi_ctx* ctx, int enable, double* out_us) {
  if (!ctx) return MAPI_EINVAL;
  DeviceGuard g(ctx->device);
  MAPI_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  if (out_us) {
    for (int i = 0; i < 8; ++i) out_us[i] = 0.0;
    if (ctx->pair_phases.p) {
      PairPhases h;
      MAPI_CUDA_TRY(ctx, cudaMemcpy(&h, ctx->pair_phases.p, sizeof(h), cudaMemcpyDeviceToHost));
      const double n = (double)h.sum[7];
      out_us[0] = n;
      if (n > 0)
        for (int i = 0; i < 7; ++i) out_us[1 + i] = (double)h.sum[i] / n / 1e3;
    }
  }
  if (enable) {
    mapi_status st = ensure(ctx, ctx->pair_phases, sizeof(PairPhases));
    if (st != MAPI_OK) return st;
    PairPhases h{};
    h.start_min = ~0ull;
    h.loop_min = ~0ull;
    MAPI_CUDA_TRY(ctx, cudaMemcpy(ctx->pair_phases.p, &h, sizeof(h), cudaMemcpyHostToDevice));
  }
  ctx->phases_on = enable != 0;
  return MAPI_OK;
}

mapi_status mapi_pair_cluster_times(mapi_ctx* ctx, double* us, int capacity, int* n) {
  if (!ctx || !n || capacity < 0 || (capacity > 0 && !us)) return MAPI_EINVAL;
  DeviceGuard g(ctx->device);
  MAPI_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  const int ns = std::min(ctx->pair_nstream, kPairPhaseClusters);
  *n = ctx->pair_phases.p ? ns : 0;
  if (!ctx->pair_phases.p) return MAPI_OK;
  if (capacity < ns) return fail(ctx, MAPI_EINVAL, "capacity below the streaming clusters");
  PairPhases h;
  MAPI_CUDA_TRY(ctx, cudaMemcpy(&h, ctx->pair_phases.p, sizeof(h), cudaMemcpyDeviceToHost));
  const double steps = (double)h.sum[7];
  for (int c = 0; c < ns; ++c)
    us[c] = steps > 0 ? (double)h.cl_ns[c] / (kPairClusterCtas * steps) / 1e3 : 0.0;
  return MAPI_OK;
}

mapi_status mapi_debug_stall(mapi_ctx* ctx, int64_t limit_ns) {
  if (!ctx || limit_ns < 0 || limit_ns > 2000000000LL) return MAPI_EINVAL;
  ctx->stall_ns = (long long)limit_ns;
  return MAPI_OK;
}

mapi_status mapi_get_stats(mapi_ctx* ctx, mapi_stats* out, int reset) {
  if (!ctx) return MAPI_EINVAL;
  DeviceGuard g(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  prof_collect(ctx, ctx->pending, true);
  if (out) *out = ctx->stats;
  if (reset) ctx->stats = mapi_stats{};
  return MAPI_OK;
}

}  // extern "C"
