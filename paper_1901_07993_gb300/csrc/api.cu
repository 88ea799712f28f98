// api.cu -- the extern "C" boundary declared in include/ifac.h: contexts,
// allocation, host<->device transfer, argument checks, and translation of
// internal errors into status codes.
#include <cstdio>
#include <cstring>

#include "internal.cuh"

namespace ifac {

void fail(int code, const std::string& msg) { throw Error{code, msg}; }

void check_cuda(cudaError_t e, const char* what, const char* file, int line) {
  if (e == cudaSuccess) return;
  char buf[512];
  snprintf(buf, sizeof buf, "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
  if (e == cudaErrorMemoryAllocation) fail(IFAC_ERR_OOM, buf);
  fail(IFAC_ERR_CUDA, buf);
}

namespace {
// larger blocks go to the pool directly; a pool allocation of a large block
// costs about 40 us of host time (105 of them, 4.3 ms, per factorization of
// the 262,144-row chain), so blocks up to 4 GB are kept
constexpr size_t kCacheMaxBlock = (size_t)4 << 30;
constexpr size_t kCacheMaxBytes = (size_t)24 << 30;  // held in the lists at most

// size classes: multiples of 256 bytes up to 4 KB, then 2^k and 3 2^(k-1)
size_t size_class(size_t b) {
  if (b <= 4096) return b < 256 ? 256 : (b + 255) & ~(size_t)255;
  size_t p = 4096;
  while (p < b) {
    if (p + p / 2 >= b) return p + p / 2;
    p <<= 1;
  }
  return p;
}

void cache_flush(ifac_ctx* ctx) {
  for (auto& kv : ctx->cache)
    for (void* q : kv.second) cudaFreeAsync(q, ctx->stream);
  ctx->cache.clear();
  ctx->cached_bytes = 0;
}

void* pool_alloc(ifac_ctx* ctx, size_t bytes) {
  void* p = nullptr;
  cudaError_t e = cudaMallocAsync(&p, bytes, ctx->stream);
  if (e != cudaSuccess || !p) {  // give the cached blocks back to the pool and try once more
    cudaGetLastError();
    cache_flush(ctx);
    p = nullptr;
    e = cudaMallocAsync(&p, bytes, ctx->stream);
  }
  if (e != cudaSuccess || !p) {
    cudaGetLastError();
    fail(IFAC_ERR_OOM, "cudaMallocAsync of " + std::to_string(bytes) + " bytes failed");
  }
  return p;
}
}  // namespace

void* dalloc(ifac_ctx* ctx, size_t bytes) {
  void* p = nullptr;
  if (ctx->custom_alloc) {
    p = ctx->alloc.alloc(ctx->alloc.user, bytes, ctx->stream);
    if (!p) fail(IFAC_ERR_OOM, "allocator returned NULL for " + std::to_string(bytes) + " bytes");
    return p;
  }
  if (bytes > kCacheMaxBlock) return pool_alloc(ctx, bytes);
  const size_t c = size_class(bytes);
  auto it = ctx->cache.find(c);
  if (it != ctx->cache.end() && !it->second.empty()) {
    p = it->second.back();
    it->second.pop_back();
    ctx->cached_bytes -= c;
  } else {
    p = pool_alloc(ctx, c);
  }
  ctx->cache_live.emplace(p, c);
  return p;
}

void dfree(ifac_ctx* ctx, void* p) {
  if (!p) return;
  if (ctx->custom_alloc) {
    ctx->alloc.free(ctx->alloc.user, p, ctx->stream);
    return;
  }
  auto it = ctx->cache_live.find(p);
  if (it != ctx->cache_live.end()) {
    const size_t c = it->second;
    ctx->cache_live.erase(it);
    if (ctx->cached_bytes + c <= kCacheMaxBytes) {
      ctx->cache[c].push_back(p);
      ctx->cached_bytes += c;
      return;
    }
  }
  cudaFreeAsync(p, ctx->stream);
}

void Mat::reset() {
  if (!ctx) return;
  dfree(ctx, m.row_ptr);
  dfree(ctx, m.col_idx);
  dfree(ctx, m.val);
  dfree(ctx, m.norms);
  m = ifac_bsr{};
  f32 = false;
}

Mat mat_alloc(ifac_ctx* ctx, int64_t n, int bs, int nb, int64_t nnzb) {
  Mat M(ctx);
  M.m.n = n;
  M.m.bs = bs;
  M.m.nb = nb;
  M.m.nnzb = nnzb;
  M.m.row_ptr = static_cast<int32_t*>(dalloc(ctx, sizeof(int32_t) * (nb + 1)));
  M.m.col_idx = static_cast<int32_t*>(dalloc(ctx, sizeof(int32_t) * (nnzb ? nnzb : 1)));
  M.m.val = static_cast<double*>(dalloc(ctx, sizeof(double) * (size_t)(nnzb ? nnzb : 1) * bs * bs));
  M.m.norms = static_cast<double*>(dalloc(ctx, sizeof(double) * (nnzb ? nnzb : 1)));
  return M;
}

void to_host(ifac_ctx* ctx, void* host, const void* dev, size_t bytes) {
  if (bytes <= 4096) {
    IFAC_CK(cudaMemcpyAsync(ctx->pinned, dev, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    IFAC_CK(cudaStreamSynchronize(ctx->stream));
    memcpy(host, ctx->pinned, bytes);
  } else {
    IFAC_CK(cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    IFAC_CK(cudaStreamSynchronize(ctx->stream));
  }
}

void to_host_many(ifac_ctx* ctx, std::initializer_list<HostRead> reads) {
  size_t off = 0;
  for (const HostRead& r : reads) {
    if (off + r.bytes > 4096) fail(IFAC_ERR_INVALID, "to_host_many: more than 4096 bytes");
    IFAC_CK(cudaMemcpyAsync(static_cast<char*>(ctx->pinned) + off, r.dev, r.bytes, cudaMemcpyDeviceToHost,
                            ctx->stream));
    off += (r.bytes + 15) & ~(size_t)15;
  }
  IFAC_CK(cudaStreamSynchronize(ctx->stream));
  off = 0;
  for (const HostRead& r : reads) {
    memcpy(r.host, static_cast<char*>(ctx->pinned) + off, r.bytes);
    off += (r.bytes + 15) & ~(size_t)15;
  }
}

void validate(const ifac_bsr* A, const char* name) {
  std::string nm(name);
  if (!A) fail(IFAC_ERR_INVALID, nm + " is NULL");
  if (A->bs <= 0 || A->nb <= 0 || A->n <= 0) fail(IFAC_ERR_INVALID, nm + ": non-positive n, bs or nb");
  if ((int64_t)A->nb != (A->n + A->bs - 1) / A->bs) fail(IFAC_ERR_INVALID, nm + ": nb != ceil(n/bs)");
  if (A->nnzb < 0 || A->nnzb > (int64_t)A->nb * A->nb) fail(IFAC_ERR_INVALID, nm + ": bad nnzb");
  if (A->nnzb > 0x7fffffffLL) fail(IFAC_ERR_UNSUPPORTED, nm + ": more than 2^31-1 blocks");
  if (!A->row_ptr || !A->col_idx || (!A->val && A->nnzb > 0)) fail(IFAC_ERR_INVALID, nm + ": NULL array");
}

static cudaEvent_t next_event(ifac_ctx* ctx) {
  if (ctx->events_used == ctx->events.size()) {
    cudaEvent_t e;
    IFAC_CK(cudaEventCreate(&e));
    ctx->events.push_back(e);
  }
  return ctx->events[ctx->events_used++];
}

void prof_begin(ifac_ctx* ctx, int kind) {
  if (!ctx->profile) return;
  const size_t pair = ctx->events_used / 2;
  if (ctx->event_kind.size() <= pair) ctx->event_kind.resize(pair + 1);
  ctx->event_kind[pair] = (char)kind;
  IFAC_CK(cudaEventRecord(next_event(ctx), ctx->stream));
}

void prof_end(ifac_ctx* ctx) {
  if (ctx->profile) IFAC_CK(cudaEventRecord(next_event(ctx), ctx->stream));
}

void prof_collect(ifac_ctx* ctx, double* ms_fp64, double* ms_tc, double* ms_split) {
  *ms_fp64 = 0.0;
  *ms_tc = 0.0;
  if (ms_split) *ms_split = 0.0;
  if (ctx->events_used) {
    IFAC_CK(cudaStreamSynchronize(ctx->stream));
    for (size_t i = 0; i + 1 < ctx->events_used; i += 2) {
      float t = 0.f;
      IFAC_CK(cudaEventElapsedTime(&t, ctx->events[i], ctx->events[i + 1]));
      const int k = ctx->event_kind[i / 2];
      if (k == 0) *ms_fp64 += t;
      else if (k == 1 || !ms_split) *ms_tc += t;
      else *ms_split += t;
    }
  }
  ctx->events_used = 0;
}

void reset_device_counters(ifac_ctx* ctx) {
  IFAC_CK(cudaMemsetAsync(ctx->dev_pairs, 0, 4 * sizeof(unsigned long long), ctx->stream));
}

void read_device_counters(ifac_ctx* ctx, int64_t* pairs_fp64, int64_t* pairs_tc, int64_t* pairs_split,
                          int64_t* slice_pairs) {
  unsigned long long h[4] = {0, 0, 0, 0};
  to_host(ctx, h, ctx->dev_pairs, sizeof(h));
  *pairs_fp64 = (int64_t)h[0];
  *pairs_tc = (int64_t)h[1];
  if (pairs_split) *pairs_split = (int64_t)h[2];
  else *pairs_tc += (int64_t)h[2];
  if (slice_pairs) *slice_pairs = (int64_t)h[3];
}

void check_device_error(ifac_ctx* ctx) {
  int e = 0;
  to_host(ctx, &e, ctx->dev_err, sizeof(int));
  if (e) {
    IFAC_CK(cudaMemsetAsync(ctx->dev_err, 0, sizeof(int), ctx->stream));
    if (e == 2) fail(IFAC_ERR_CUDA, "split product: fixed-point overflow (scale bound violated)");
    fail(IFAC_ERR_TIMEOUT, "a bounded device-side wait expired (tensor-core pipeline)");
  }
}

}  // namespace ifac

using namespace ifac;

template <typename F>
static int guarded(ifac_ctx* ctx, F&& f) {
  if (!ctx) return IFAC_ERR_INVALID;
  // run on the context's device; the caller's current device is restored on return
  struct DeviceScope {
    int prev = -1;
    explicit DeviceScope(int dev) {
      if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
      else prev = -1;
    }
    ~DeviceScope() {
      if (prev >= 0) cudaSetDevice(prev);
    }
  } scope(ctx->device);
  try {
    int rc = f();
    if (rc != 0) {
      if (ctx->err.empty()) ctx->err = "status " + std::to_string(rc);
    } else {
      ctx->err.clear();
    }
    return rc;
  } catch (const Error& e) {
    ctx->err = e.msg;
    return e.code;
  } catch (const std::bad_alloc&) {
    ctx->err = "host allocation failed";
    return IFAC_ERR_OOM;
  } catch (...) {
    ctx->err = "unexpected internal error";
    return IFAC_ERR_CUDA;
  }
}

extern "C" {

void ifac_opts_default(ifac_opts* o) {
  if (!o) return;
  o->m = 2;
  o->max_iter = 50;
  o->fixed_iters = 0;
  o->c_rule = 0;
  o->leaf_size = 512;
  o->prec = IFAC_FP64;
  o->profile = 0;
  o->delta_prec = IFAC_FP64_SPLIT;
  o->rinch_rows = 0;
  o->local_delta = 0;
}

int ifac_create(ifac_ctx** out, void* stream, const ifac_allocator* alloc) {
  if (!out) return IFAC_ERR_INVALID;
  *out = nullptr;
  ifac_ctx* c = new (std::nothrow) ifac_ctx();
  if (!c) return IFAC_ERR_OOM;
  if (cudaGetDevice(&c->device) != cudaSuccess) { delete c; return IFAC_ERR_CUDA; }
  c->stream = static_cast<cudaStream_t>(stream);
  if (alloc) {
    if (!alloc->alloc || !alloc->free) { delete c; return IFAC_ERR_INVALID; }
    c->custom_alloc = true;
    c->alloc = *alloc;
  } else {
    // keep freed blocks in the device pool between calls
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, c->device) == cudaSuccess) {
      uint64_t thr = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
  }
  if (cudaMallocHost(&c->pinned, 4096) != cudaSuccess) { delete c; return IFAC_ERR_CUDA; }
  void* words = nullptr;
  if (cudaMalloc(&words, 64) != cudaSuccess) { cudaFreeHost(c->pinned); delete c; return IFAC_ERR_CUDA; }
  cudaMemset(words, 0, 64);
  c->dev_err = static_cast<int*>(words);
  c->dev_pairs = reinterpret_cast<unsigned long long*>(static_cast<char*>(words) + 16);  // 4 counters
  *out = c;
  return IFAC_OK;
}

void ifac_destroy(ifac_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  ifac::cache_flush(ctx);
  cudaStreamSynchronize(ctx->stream);
  for (cudaEvent_t e : ctx->events) cudaEventDestroy(e);
  if (ctx->pinned) cudaFreeHost(ctx->pinned);
  if (ctx->dev_err) cudaFree(ctx->dev_err);
  delete ctx;
}

int ifac_set_stream(ifac_ctx* ctx, void* stream) {
  if (!ctx) return IFAC_ERR_INVALID;
  // the cached blocks were last used on the old stream: let it drain first
  if (stream != static_cast<void*>(ctx->stream)) cudaStreamSynchronize(ctx->stream);
  ctx->stream = static_cast<cudaStream_t>(stream);
  return IFAC_OK;
}

int ifac_set_split_slices(ifac_ctx* ctx, int slices) {
  if (!ctx || slices < 3 || slices > 8) return IFAC_ERR_INVALID;
  ctx->split_slices = slices;
  return IFAC_OK;
}

int ifac_set_fp32_intermediates(ifac_ctx* ctx, int on) {
  if (!ctx) return IFAC_ERR_INVALID;
  ctx->fp32_mid = on != 0;
  return IFAC_OK;
}

const char* ifac_last_error(const ifac_ctx* ctx) { return ctx ? ctx->err.c_str() : "NULL context"; }

int ifac_bsr_upload(ifac_ctx* ctx, int64_t n, int32_t bs, int32_t nb, int64_t nnzb, const int32_t* row_ptr,
                    const int32_t* col_idx, const double* val, ifac_bsr* out) {
  if (out) *out = ifac_bsr{};
  return guarded(ctx, [&]() -> int {
    if (!out || !row_ptr || (nnzb > 0 && (!col_idx || !val))) fail(IFAC_ERR_INVALID, "upload: NULL argument");
    if (bs <= 0 || nb <= 0 || n <= 0 || (int64_t)nb != (n + bs - 1) / bs) fail(IFAC_ERR_INVALID, "upload: bad n/bs/nb");
    if (row_ptr[0] != 0 || row_ptr[nb] != nnzb) fail(IFAC_ERR_INVALID, "upload: row_ptr[0] != 0 or row_ptr[nb] != nnzb");
    for (int i = 0; i < nb; ++i) {
      if (row_ptr[i + 1] < row_ptr[i]) fail(IFAC_ERR_INVALID, "upload: row_ptr not monotone");
      for (int p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
        if (col_idx[p] < 0 || col_idx[p] >= nb) fail(IFAC_ERR_INVALID, "upload: column index out of range");
        if (p > row_ptr[i] && col_idx[p] <= col_idx[p - 1]) fail(IFAC_ERR_INVALID, "upload: columns not strictly increasing");
      }
    }
    Mat M = mat_alloc(ctx, n, bs, nb, nnzb);
    IFAC_CK(cudaMemcpyAsync(M.m.row_ptr, row_ptr, sizeof(int32_t) * (nb + 1), cudaMemcpyHostToDevice, ctx->stream));
    if (nnzb) {
      IFAC_CK(cudaMemcpyAsync(M.m.col_idx, col_idx, sizeof(int32_t) * nnzb, cudaMemcpyHostToDevice, ctx->stream));
      IFAC_CK(cudaMemcpyAsync(M.m.val, val, sizeof(double) * (size_t)nnzb * bs * bs, cudaMemcpyHostToDevice, ctx->stream));
      block_norms(ctx, M.m, M.m.norms);
    }
    IFAC_CK(cudaStreamSynchronize(ctx->stream));
    *out = M.release();
    return IFAC_OK;
  });
}

int ifac_bsr_download(ifac_ctx* ctx, const ifac_bsr* a, int32_t* row_ptr, int32_t* col_idx, double* val) {
  return guarded(ctx, [&]() -> int {
    validate(a, "A");
    if (row_ptr) IFAC_CK(cudaMemcpyAsync(row_ptr, a->row_ptr, sizeof(int32_t) * (a->nb + 1), cudaMemcpyDeviceToHost, ctx->stream));
    if (col_idx && a->nnzb) IFAC_CK(cudaMemcpyAsync(col_idx, a->col_idx, sizeof(int32_t) * a->nnzb, cudaMemcpyDeviceToHost, ctx->stream));
    if (val && a->nnzb) IFAC_CK(cudaMemcpyAsync(val, a->val, sizeof(double) * (size_t)a->nnzb * a->bs * a->bs, cudaMemcpyDeviceToHost, ctx->stream));
    IFAC_CK(cudaStreamSynchronize(ctx->stream));
    return IFAC_OK;
  });
}

void ifac_bsr_free(ifac_ctx* ctx, ifac_bsr* a) {
  if (!ctx || !a) return;
  Mat M(ctx);
  M.m = *a;
  M.reset();
  *a = ifac_bsr{};
}

static void check_pair(const ifac_bsr* A, const ifac_bsr* B) {
  if (A->n != B->n || A->bs != B->bs || A->nb != B->nb) fail(IFAC_ERR_INVALID, "operands differ in n or block size");
}

int bsr_gemm_trunc(ifac_ctx* ctx, const ifac_bsr* A, int transA, const ifac_bsr* B, int transB, double alpha,
                   double tau, int prec, ifac_bsr* C) {
  if (C) *C = ifac_bsr{};
  return guarded(ctx, [&]() -> int {
    validate(A, "A");
    validate(B, "B");
    check_pair(A, B);
    if (!C) fail(IFAC_ERR_INVALID, "C is NULL");
    if (prec != IFAC_FP64 && prec != IFAC_TF32 && prec != IFAC_BF16 && prec != IFAC_FP64_SPLIT)
      fail(IFAC_ERR_INVALID, "unknown precision");
    if (!(tau >= 0)) fail(IFAC_ERR_INVALID, "tau must be >= 0");
    Mat R = ifac::gemm(ctx, *A, transA != 0, *B, transB != 0, alpha, tau, prec);
    check_device_error(ctx);
    *C = R.release();
    return IFAC_OK;
  });
}

int bsr_gemm_sym_trunc(ifac_ctx* ctx, const ifac_bsr* A, int transA, const ifac_bsr* B, int transB, double alpha,
                       double tau, int prec, ifac_bsr* C) {
  if (C) *C = ifac_bsr{};
  return guarded(ctx, [&]() -> int {
    validate(A, "A");
    validate(B, "B");
    check_pair(A, B);
    if (!C) fail(IFAC_ERR_INVALID, "C is NULL");
    if (prec != IFAC_FP64 && prec != IFAC_TF32 && prec != IFAC_BF16 && prec != IFAC_FP64_SPLIT)
      fail(IFAC_ERR_INVALID, "unknown precision");
    if (!(tau >= 0)) fail(IFAC_ERR_INVALID, "tau must be >= 0");
    if (A->bs != 64) fail(IFAC_ERR_UNSUPPORTED, "symmetric product built for bs = 64");
    Mat U = ifac::gemm(ctx, *A, transA != 0, *B, transB != 0, alpha, tau, prec, true);
    Mat R = ifac::sym_sum(ctx, 1.0, U.m, 0.0, nullptr, 0.0);
    check_device_error(ctx);
    *C = R.release();
    return IFAC_OK;
  });
}

int bsr_add(ifac_ctx* ctx, double alpha, const ifac_bsr* A, double beta, const ifac_bsr* B, double gamma, ifac_bsr* C) {
  if (C) *C = ifac_bsr{};
  return guarded(ctx, [&]() -> int {
    validate(A, "A");
    if (B) { validate(B, "B"); check_pair(A, B); }
    if (!C) fail(IFAC_ERR_INVALID, "C is NULL");
    Mat R = ifac::add(ctx, alpha, *A, beta, B, gamma);
    IFAC_CK(cudaStreamSynchronize(ctx->stream));
    *C = R.release();
    return IFAC_OK;
  });
}

int bsr_truncate(ifac_ctx* ctx, const ifac_bsr* A, double tau, ifac_bsr* C) {
  if (C) *C = ifac_bsr{};
  return guarded(ctx, [&]() -> int {
    validate(A, "A");
    if (!C) fail(IFAC_ERR_INVALID, "C is NULL");
    Mat R = ifac::truncate(ctx, *A, tau);
    IFAC_CK(cudaStreamSynchronize(ctx->stream));
    *C = R.release();
    return IFAC_OK;
  });
}

int bsr_fro(ifac_ctx* ctx, const ifac_bsr* A, double* out) {
  return guarded(ctx, [&]() -> int {
    validate(A, "A");
    if (!out) fail(IFAC_ERR_INVALID, "out is NULL");
    *out = fro_host(ctx, *A);
    return IFAC_OK;
  });
}

int bsr_gershgorin(ifac_ctx* ctx, const ifac_bsr* A, double* out) {
  return guarded(ctx, [&]() -> int {
    validate(A, "A");
    if (!out) fail(IFAC_ERR_INVALID, "out is NULL");
    *out = gershgorin_host(ctx, *A);
    return IFAC_OK;
  });
}

int leaf_invchol_batched(ifac_ctx* ctx, int count, int nl, const double* S, double* Z, int* info) {
  return guarded(ctx, [&]() -> int {
    if (count < 0 || nl <= 0 || nl > 1024 || !S || !Z || !info) fail(IFAC_ERR_INVALID, "leaf: bad arguments");
    if (count == 0) return IFAC_OK;
    if (S != Z)
      IFAC_CK(cudaMemcpyAsync(Z, S, sizeof(double) * (size_t)count * nl * nl, cudaMemcpyDeviceToDevice, ctx->stream));
    leaf_invchol(ctx, count, nl, Z, info);
    std::vector<int> h(count);
    to_host(ctx, h.data(), info, sizeof(int) * count);
    for (int k = 0; k < count; ++k)
      if (h[k]) fail(IFAC_ERR_NOT_SPD, "leaf " + std::to_string(k) + ": pivot " + std::to_string(h[k] - 1) + " not positive");
    return IFAC_OK;
  });
}

static void check_opts(const ifac_opts* o, bool mixed_ok) {
  if (!o) fail(IFAC_ERR_INVALID, "opts is NULL");
  if (o->m < 1 || o->m > 8) fail(IFAC_ERR_INVALID, "m must be in 1..8");
  if (o->max_iter < 0 || o->fixed_iters < 0) fail(IFAC_ERR_INVALID, "negative iteration count");
  if (o->prec != IFAC_FP64 && o->prec != IFAC_FP64_SPLIT &&
      !(mixed_ok && (o->prec == IFAC_TF32 || o->prec == IFAC_BF16)))
    fail(IFAC_ERR_UNSUPPORTED, "precision not available for this call");
  if (o->rinch_rows < 0) fail(IFAC_ERR_INVALID, "rinch_rows must be >= 0");
  if (o->delta_prec != IFAC_FP64 && o->delta_prec != IFAC_FP64_SPLIT)
    fail(IFAC_ERR_INVALID, "delta_prec must be IFAC_FP64 or IFAC_FP64_SPLIT");
}

// opts->prec == IFAC_FP64_SPLIT: the driver runs its FP64 schedule while
// gemm() routes every FP64 product through the split tensor-core kernel
struct SplitScope {
  ifac_ctx* c;
  int old;
  SplitScope(ifac_ctx* c_, bool on) : c(c_), old(c_->fp64_prec) {
    if (on) c->fp64_prec = IFAC_FP64_SPLIT;
  }
  ~SplitScope() { c->fp64_prec = old; }
};

static ifac_opts split_opts(const ifac_opts* in, int bs, bool* split) {
  ifac_opts o = *in;
  *split = o.prec == IFAC_FP64_SPLIT;
  if (*split) {
    if (bs != 32 && bs != 64 && bs != 128) fail(IFAC_ERR_UNSUPPORTED, "split tensor-core products: bs 32, 64 or 128");
    o.prec = IFAC_FP64;
  }
  return o;
}

int inv_factor_refine(ifac_ctx* ctx, const ifac_bsr* S, double tau, double target, const ifac_opts* opts,
                      ifac_bsr* Z, ifac_report* rep) {
  if (Z) *Z = ifac_bsr{};
  return guarded(ctx, [&]() -> int {
    validate(S, "S");
    check_opts(opts, true);
    if (!Z) fail(IFAC_ERR_INVALID, "Z is NULL");
    if (!(tau >= 0) || !(target >= 0)) fail(IFAC_ERR_INVALID, "tau and target must be >= 0");
    bool split = false;
    const ifac_opts o = split_opts(opts, S->bs, &split);
    SplitScope scope(ctx, split);
    if (o.prec != IFAC_FP64) return refine_irsi_mixed(ctx, *S, tau, target, o, Z, rep);
    return refine_irsi(ctx, *S, tau, target, o, Z, rep);
  });
}

int inv_factor_localized(ifac_ctx* ctx, const ifac_bsr* S, double tau, double target, const ifac_opts* opts,
                         ifac_bsr* Z, ifac_report* rep) {
  if (Z) *Z = ifac_bsr{};
  return guarded(ctx, [&]() -> int {
    validate(S, "S");
    check_opts(opts, false);
    if (!Z) fail(IFAC_ERR_INVALID, "Z is NULL");
    if (opts->leaf_size < 1) fail(IFAC_ERR_INVALID, "leaf_size must be >= 1");
    if (!(tau >= 0) || !(target >= 0)) fail(IFAC_ERR_INVALID, "tau and target must be >= 0");
    bool split = false;
    const ifac_opts o = split_opts(opts, S->bs, &split);
    SplitScope scope(ctx, split);
    return lif(ctx, *S, tau, target, o, Z, rep);
  });
}

int inv_factor_rinch(ifac_ctx* ctx, const ifac_bsr* S, double tau, const ifac_opts* opts, ifac_bsr* Z,
                     ifac_report* rep) {
  if (Z) *Z = ifac_bsr{};
  return guarded(ctx, [&]() -> int {
    validate(S, "S");
    check_opts(opts, false);
    if (!Z) fail(IFAC_ERR_INVALID, "Z is NULL");
    if (opts->leaf_size < 1) fail(IFAC_ERR_INVALID, "leaf_size must be >= 1");
    if (!(tau >= 0)) fail(IFAC_ERR_INVALID, "tau must be >= 0");
    bool split = false;
    const ifac_opts o = split_opts(opts, S->bs, &split);
    SplitScope scope(ctx, split);
    return rinch(ctx, *S, tau, o, Z, rep);
  });
}

int inv_factor_refine_batched(ifac_ctx* ctx, int count, const ifac_bsr* const* S, double tau, double target,
                              const ifac_opts* opts, ifac_bsr* Z, ifac_report* rep) {
  if (Z && count > 0)
    for (int k = 0; k < count; ++k) Z[k] = ifac_bsr{};
  return guarded(ctx, [&]() -> int {
    if (count <= 0 || !S || !Z) fail(IFAC_ERR_INVALID, "batched: empty batch or NULL arrays");
    check_opts(opts, true);
    for (int k = 0; k < count; ++k) {
      validate(S[k], "S[k]");
      if (S[k]->bs != S[0]->bs) fail(IFAC_ERR_INVALID, "batched: members differ in block size");
    }
    if (opts->prec != IFAC_FP64 && S[0]->bs != 32 && S[0]->bs != 64 && S[0]->bs != 128)
      fail(IFAC_ERR_UNSUPPORTED, "batched mixed precision: bs 32, 64 or 128");
    if (!(tau >= 0) || !(target >= 0)) fail(IFAC_ERR_INVALID, "tau and target must be >= 0");
    bool split = false;
    const ifac_opts o = split_opts(opts, S[0]->bs, &split);
    SplitScope scope(ctx, split);
    return refine_batched(ctx, count, S, tau, target, o, Z, rep);
  });
}

int inv_factor_refine_adjoint(ifac_ctx* ctx, const ifac_bsr* S, const ifac_bsr* F, int K, double tau, double* L,
                              ifac_bsr* Sbar) {
  if (Sbar) *Sbar = ifac_bsr{};
  return guarded(ctx, [&]() -> int {
    validate(S, "S");
    validate(F, "F");
    check_pair(S, F);
    if (!L || !Sbar) fail(IFAC_ERR_INVALID, "L or Sbar is NULL");
    if (K < 0 || K > 64) fail(IFAC_ERR_INVALID, "K must be in 0..64");
    if (!(tau >= 0)) fail(IFAC_ERR_INVALID, "tau must be >= 0");
    return refine_adjoint(ctx, *S, *F, K, tau, L, Sbar);
  });
}

int inv_factor_resid(ifac_ctx* ctx, const ifac_bsr* S, const ifac_bsr* Z, double* out) {
  return guarded(ctx, [&]() -> int {
    validate(S, "S");
    validate(Z, "Z");
    check_pair(S, Z);
    if (!out) fail(IFAC_ERR_INVALID, "out is NULL");
    *out = resid(ctx, *S, *Z);
    return IFAC_OK;
  });
}

int bsr_reblock(ifac_ctx* ctx, const ifac_bsr* A, int32_t bs, ifac_bsr* out) {
  if (out) *out = ifac_bsr{};
  return guarded(ctx, [&]() -> int {
    validate(A, "A");
    if (!out) fail(IFAC_ERR_INVALID, "out is NULL");
    if (bs != 32 && bs != 64 && bs != 128) fail(IFAC_ERR_UNSUPPORTED, "reblock: bs 32, 64 or 128");
    if (A->bs % 32 != 0) fail(IFAC_ERR_UNSUPPORTED, "reblock: input bs must be a multiple of 32");
    Mat R = reblock(ctx, *A, bs);
    IFAC_CK(cudaStreamSynchronize(ctx->stream));
    *out = R.release();
    return IFAC_OK;
  });
}

int ifac_set_schedule(ifac_ctx* ctx, int32_t narrow_kmax, int32_t narrow_kmax_split) {
  if (!ctx) return IFAC_ERR_INVALID;
  if (narrow_kmax < -1 || narrow_kmax_split < -1) return IFAC_ERR_INVALID;
  ctx->narrow_kmax = narrow_kmax;
  ctx->narrow_kmax_split = narrow_kmax_split;
  return IFAC_OK;
}

int ifac_autotune_batched(ifac_ctx* ctx, int count, const ifac_bsr* const* S, double tau, const ifac_opts* opts,
                          ifac_tune_result* out) {
  return guarded(ctx, [&]() -> int {
    if (count <= 0 || !S || !out) fail(IFAC_ERR_INVALID, "autotune: empty batch or NULL arrays");
    check_opts(opts, true);
    for (int k = 0; k < count; ++k) {
      validate(S[k], "S[k]");
      if (S[k]->bs != S[0]->bs) fail(IFAC_ERR_INVALID, "autotune: members differ in block size");
      if (S[k]->bs % 32 != 0) fail(IFAC_ERR_UNSUPPORTED, "autotune: block size must be a multiple of 32");
    }
    if (!(tau >= 0)) fail(IFAC_ERR_INVALID, "tau must be >= 0");
    autotune(ctx, count, S, tau, *opts, out);
    ctx->narrow_kmax = out->narrow_kmax;
    ctx->narrow_kmax_split = out->narrow_kmax_split;
    return IFAC_OK;
  });
}

int ifac_selftest_wait_timeout(ifac_ctx* ctx, int64_t wait_limit) {
  return guarded(ctx, [&]() -> int {
    if (wait_limit < 1 || wait_limit > ((int64_t)1 << 30)) fail(IFAC_ERR_INVALID, "wait_limit must be in 1..2^30");
    tc_wait_timeout_selftest(ctx, (long long)wait_limit);
    check_device_error(ctx);  // IFAC_ERR_TIMEOUT, flag cleared
    return IFAC_OK;
  });
}

}  // extern "C"
