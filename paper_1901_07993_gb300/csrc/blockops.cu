// blockops.cu -- memory-bound block operations: sums on a union pattern,
// block Frobenius norms, ||A||_F, the Gershgorin bound and Z_0 = c I.
//
// Sums follow the definition alpha*a + beta*b + gamma*[diag] with explicit
// round-to-nearest multiplies and adds (no fused multiply-add), in that
// order, so each element is rounded exactly as the plain definition is.
// Reductions run in a fixed order (per row, then over rows), so results are
// deterministic from run to run.
#include "internal.cuh"

namespace ifac {

__device__ __forceinline__ int find_col(const int32_t* __restrict__ ci, int lo, int hi, int c) {
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (ci[mid] < c) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ double block_reduce_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < nw; ++w) t += red[w];
  __syncthreads();
  return t;  // valid in thread 0
}

// one CTA per output block (grid-stride)
__global__ void k_add(const int32_t* __restrict__ crow, const int32_t* __restrict__ cci, int64_t cnnz, int bs,
                      double alpha, const int32_t* __restrict__ arp, const int32_t* __restrict__ aci,
                      const double* __restrict__ aval, double beta, const int32_t* __restrict__ brp,
                      const int32_t* __restrict__ bci, const double* __restrict__ bval, double gamma,
                      double* __restrict__ cval, double* __restrict__ cnorm) {
  __shared__ double red[32];
  __shared__ int sa, sb;
  const int bsz = bs * bs;
  for (int64_t p = blockIdx.x; p < cnnz; p += gridDim.x) {
    const int I = crow[p], J = cci[p];
    if (threadIdx.x == 0) {
      int q = find_col(aci, arp[I], arp[I + 1], J);
      sa = (q < arp[I + 1] && aci[q] == J) ? q : -1;
      sb = -1;
      if (bval) {
        int r = find_col(bci, brp[I], brp[I + 1], J);
        sb = (r < brp[I + 1] && bci[r] == J) ? r : -1;
      }
    }
    __syncthreads();
    const int qa = sa, qb = sb;
    const double* a = qa >= 0 ? aval + (size_t)qa * bsz : nullptr;
    const double* b = qb >= 0 ? bval + (size_t)qb * bsz : nullptr;
    double* c = cval + (size_t)p * bsz;
    double ss = 0.0;
    for (int e = threadIdx.x; e < bsz; e += blockDim.x) {
      double v = 0.0;
      if (a) v = __dadd_rn(v, __dmul_rn(alpha, a[e]));
      if (b) v = __dadd_rn(v, __dmul_rn(beta, b[e]));
      if (I == J && (e / bs) == (e % bs)) v = __dadd_rn(v, gamma);
      c[e] = v;
      ss = fma(v, v, ss);
    }
    double t = block_reduce_sum(ss, red);
    if (threadIdx.x == 0) cnorm[p] = sqrt(t);
  }
}

void add_numeric(ifac_ctx* ctx, double alpha, const ifac_bsr& A, double beta, const ifac_bsr* B, double gamma,
                 ifac_bsr& C, const int32_t* crow) {
  if (C.nnzb == 0) return;
  int grid = (int)std::min<int64_t>(C.nnzb, 152 * 16);
  k_add<<<grid, 256, 0, ctx->stream>>>(crow, C.col_idx, C.nnzb, C.bs, alpha, A.row_ptr, A.col_idx, A.val, beta,
                                       B ? B->row_ptr : nullptr, B ? B->col_idx : nullptr, B ? B->val : nullptr,
                                       gamma, C.val, C.norms);
  IFAC_CK_LAUNCH();
}

__global__ void k_block_norms(const double* __restrict__ val, int64_t nnzb, int bsz, double* __restrict__ norms) {
  __shared__ double red[32];
  for (int64_t p = blockIdx.x; p < nnzb; p += gridDim.x) {
    const double* v = val + (size_t)p * bsz;
    double ss = 0.0;
    for (int e = threadIdx.x; e < bsz; e += blockDim.x) ss = fma(v[e], v[e], ss);
    double t = block_reduce_sum(ss, red);
    if (threadIdx.x == 0) norms[p] = sqrt(t);
  }
}

void block_norms(ifac_ctx* ctx, const ifac_bsr& A, double* norms) {
  if (A.nnzb == 0) return;
  int grid = (int)std::min<int64_t>(A.nnzb, 152 * 16);
  k_block_norms<<<grid, 256, 0, ctx->stream>>>(A.val, A.nnzb, A.bs * A.bs, norms);
  IFAC_CK_LAUNCH();
}

// rowsq[I] = sum over the blocks of block row I of norm^2 (warp per row)
__global__ void k_row_sq(const int32_t* __restrict__ rp, int nb, const double* __restrict__ norms,
                         double* __restrict__ rowsq) {
  int row = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (row >= nb) return;
  double s = 0.0;
  for (int p = rp[row] + lane; p < rp[row + 1]; p += 32) s = fma(norms[p], norms[p], s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) rowsq[row] = s;
}

void row_sq_norms(ifac_ctx* ctx, const ifac_bsr& A, double* rowsq) {
  Buf<double> tmp;
  const double* norms = A.norms;
  if (!norms) {
    tmp = Buf<double>(ctx, A.nnzb);
    block_norms(ctx, A, tmp.p);
    norms = tmp.p;
  }
  k_row_sq<<<cdiv((int64_t)A.nb * 32, 256), 256, 0, ctx->stream>>>(A.row_ptr, A.nb, norms, rowsq);
  IFAC_CK_LAUNCH();
}

// out = sum of x[0..n) in a fixed order (single CTA)
__global__ void k_sum(const double* __restrict__ x, int n, double* __restrict__ out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += x[i];
  double t = block_reduce_sum(s, red);
  if (threadIdx.x == 0) *out = t;
}

double fro_host(ifac_ctx* ctx, const ifac_bsr& A) {
  Buf<double> rowsq(ctx, A.nb), out(ctx, 1);
  row_sq_norms(ctx, A, rowsq.p);
  k_sum<<<1, 1024, 0, ctx->stream>>>(rowsq.p, A.nb, out.p);
  IFAC_CK_LAUNCH();
  double h = 0.0;
  to_host(ctx, &h, out.p, sizeof(double));
  return sqrt(h);
}

// row sums of |a_ij| for every scalar row (warp per scalar row), then max
__global__ void k_abs_rowsum(const int32_t* __restrict__ rp, int nb, int bs, const double* __restrict__ val,
                             double* __restrict__ rs) {
  int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (w >= (int64_t)nb * bs) return;
  int I = (int)(w / bs), r = (int)(w % bs);
  double s = 0.0;
  for (int p = rp[I]; p < rp[I + 1]; ++p) {
    const double* row = val + (size_t)p * bs * bs + (size_t)r * bs;
    for (int c = lane; c < bs; c += 32) s += fabs(row[c]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) rs[w] = s;
}

__global__ void k_max(const double* __restrict__ x, int64_t n, double* __restrict__ out) {
  __shared__ double red[32];
  double m = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, x[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t = fmax(t, red[i]);
    *out = t;
  }
}

void gershgorin_rows(ifac_ctx* ctx, const ifac_bsr& A, double* rs) {
  const int64_t rows = (int64_t)A.nb * A.bs;
  k_abs_rowsum<<<cdiv(rows * 32, 256), 256, 0, ctx->stream>>>(A.row_ptr, A.nb, A.bs, A.val, rs);
  IFAC_CK_LAUNCH();
}

double gershgorin_host(ifac_ctx* ctx, const ifac_bsr& A) {
  int64_t rows = (int64_t)A.nb * A.bs;
  Buf<double> rs(ctx, rows), out(ctx, 1);
  k_abs_rowsum<<<cdiv(rows * 32, 256), 256, 0, ctx->stream>>>(A.row_ptr, A.nb, A.bs, A.val, rs.p);
  IFAC_CK_LAUNCH();
  k_max<<<1, 1024, 0, ctx->stream>>>(rs.p, rows, out.p);
  IFAC_CK_LAUNCH();
  double h = 0.0;
  to_host(ctx, &h, out.p, sizeof(double));
  return h;
}

__global__ void k_scaled_identity(int nb, int bs, double c, int32_t* __restrict__ rp, int32_t* __restrict__ ci,
                                  double* __restrict__ val) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t bsz = (int64_t)bs * bs;
  if (e < (int64_t)nb * bsz) {
    int64_t k = e % bsz;
    val[e] = ((k / bs) == (k % bs)) ? c : 0.0;
  }
  if (e < nb) ci[e] = (int32_t)e;
  if (e <= nb) rp[e] = (int32_t)e;
}

Mat scaled_identity(ifac_ctx* ctx, int64_t n, int bs, int nb, double c) {
  Mat M = mat_alloc(ctx, n, bs, nb, nb);
  int64_t tot = std::max<int64_t>((int64_t)nb * bs * bs, nb + 1);
  k_scaled_identity<<<cdiv(tot, 256), 256, 0, ctx->stream>>>(nb, bs, c, M.m.row_ptr, M.m.col_idx, M.m.val);
  IFAC_CK_LAUNCH();
  block_norms(ctx, M.m, M.m.norms);
  return M;
}

}  // namespace ifac
