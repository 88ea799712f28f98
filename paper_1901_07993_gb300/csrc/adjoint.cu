// adjoint.cu -- reverse-mode derivative of K refinement sweeps (Eq. 2.1,
// m = 2, from Z_0 = c I with c held constant) on a frozen block pattern, for
// L = tr(Z_K^T F Z_K).
//
// Frozen pattern: a recording run with truncation at tau fixes the block
// pattern of every intermediate; the differentiated function restricts each
// product to that pattern (Pi_X = projection onto the pattern of X), which
// makes L a polynomial in the stored entries of S.  One sweep:
//   X = Pi_X(S Z), Y = Pi_Y(Z^T X), delta = I - Y, D = Pi_D(delta delta),
//   P = delta/2 + 3D/8, M = Pi_M(Z P), Z' = Z + M.
// Reverse sweep (all products FP64, restricted to the named pattern):
//   Mh = Pi_M(Zh'), Zh = Pi_Z(Zh') + Pi_Z(Mh P^T), Ph = Pi_P(Z^T Mh),
//   Dh = 3/8 Pi_D(Ph), deltah = 1/2 Pi_delta(Ph) + Pi_delta(Dh delta^T + delta^T Dh),
//   Yh = -Pi_Y(deltah), Zh += Pi_Z(X Yh^T), Xh = Pi_X(Z Yh), Zh += Pi_Z(S^T Xh),
//   Sh += Pi_S(Xh Z^T),
// from Zh_K = Pi_{Z_K}((F + F^T) Z_K).  The recording run keeps every
// intermediate of every sweep (checkpoints), so nothing is recomputed.
#include <cmath>
#include <vector>

#include "internal.cuh"

namespace ifac {

// alpha op(A) op(B) computed on exactly the block pattern of P
static Mat gemm_masked(ifac_ctx* ctx, const ifac_bsr& A, bool tA, const ifac_bsr& B, bool tB, double alpha,
                       const ifac_bsr& P) {
  Mat C = mat_alloc(ctx, A.n, A.bs, A.nb, P.nnzb);
  IFAC_CK(cudaMemcpyAsync(C.m.row_ptr, P.row_ptr, sizeof(int32_t) * (P.nb + 1), cudaMemcpyDeviceToDevice,
                          ctx->stream));
  if (P.nnzb == 0) return C;
  IFAC_CK(cudaMemcpyAsync(C.m.col_idx, P.col_idx, sizeof(int32_t) * P.nnzb, cudaMemcpyDeviceToDevice, ctx->stream));
  Buf<int32_t> row(ctx, P.nnzb);
  expand_rows(ctx, C.m.row_ptr, C.m.nb, row.p);
  View arows = view_rows(ctx, A, tA);
  View bcols = view_rows(ctx, B, !tB);
  Buf<unsigned long long> pairs(ctx, 1);
  IFAC_CK(cudaMemsetAsync(pairs.p, 0, sizeof(unsigned long long), ctx->stream));
  gemm_numeric_fp64(ctx, arows, tA, A, bcols, tB, B, alpha, C.m, row.p, pairs.p);
  ctx->products += 1;
  return C;
}

// Pi_P(A): A's blocks on the pattern of P, zero blocks where A has none
static Mat project(ifac_ctx* ctx, const ifac_bsr& A, const ifac_bsr& P) {
  Mat C = mat_alloc(ctx, A.n, A.bs, A.nb, P.nnzb);
  IFAC_CK(cudaMemcpyAsync(C.m.row_ptr, P.row_ptr, sizeof(int32_t) * (P.nb + 1), cudaMemcpyDeviceToDevice,
                          ctx->stream));
  if (P.nnzb == 0) return C;
  IFAC_CK(cudaMemcpyAsync(C.m.col_idx, P.col_idx, sizeof(int32_t) * P.nnzb, cudaMemcpyDeviceToDevice, ctx->stream));
  Buf<int32_t> row(ctx, P.nnzb);
  expand_rows(ctx, C.m.row_ptr, C.m.nb, row.p);
  add_numeric(ctx, 1.0, A, 0.0, nullptr, 0.0, C.m, row.p);
  return C;
}

// per-CTA partial sums of a[i] * b[i], then a fixed-order total
__global__ void k_dot_partial(const double* __restrict__ a, const double* __restrict__ b, int64_t n,
                              double* __restrict__ part) {
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s = fma(a[i], b[i], s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}

__global__ void k_sum_parts(const double* __restrict__ part, int n, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < n; ++i) t += part[i];
    *out = t;
  }
}

// <A, B> over the pattern of A (B restricted to it)
static double dot_on(ifac_ctx* ctx, const ifac_bsr& A, const ifac_bsr& B) {
  Mat Bp = project(ctx, B, A);
  const int64_t n = A.nnzb * (int64_t)A.bs * A.bs;
  const int grid = 152 * 4;
  Buf<double> part(ctx, grid), out(ctx, 1);
  k_dot_partial<<<grid, 256, 0, ctx->stream>>>(A.val, Bp.m.val, n, part.p);
  IFAC_CK_LAUNCH();
  k_sum_parts<<<1, 32, 0, ctx->stream>>>(part.p, grid, out.p);
  IFAC_CK_LAUNCH();
  double h = 0.0;
  to_host(ctx, &h, out.p, sizeof(double));
  return h;
}

static void zero_values(ifac_ctx* ctx, ifac_bsr& A) {
  if (A.nnzb) {
    IFAC_CK(cudaMemsetAsync(A.val, 0, sizeof(double) * (size_t)A.nnzb * A.bs * A.bs, ctx->stream));
    IFAC_CK(cudaMemsetAsync(A.norms, 0, sizeof(double) * A.nnzb, ctx->stream));
  }
}

int refine_adjoint(ifac_ctx* ctx, const ifac_bsr& S_in, const ifac_bsr& F, int K, double tau, double* L_out,
                   ifac_bsr* Sbar_out) {
  ctx->products = 0;
  ctx->pairs = 0;
  Mat S = truncate(ctx, S_in, tau);
  const double beta = gershgorin_host(ctx, S.m);
  const double c = 1.0 / std::sqrt(beta);
  std::vector<Mat> X(K), Y(K), D(K), M(K), Z(K + 1);
  Z[0] = scaled_identity(ctx, S.m.n, S.m.bs, S.m.nb, c);
  for (int k = 0; k < K; ++k) {  // recording run: truncation fixes the patterns
    X[k] = gemm(ctx, S.m, false, Z[k].m, false, 1.0, tau);
    Y[k] = gemm(ctx, Z[k].m, true, X[k].m, false, 1.0, tau);
    Mat delta = add(ctx, -1.0, Y[k].m, 0.0, nullptr, 1.0);
    D[k] = gemm(ctx, delta.m, false, delta.m, false, 1.0, tau);
    Mat P = add(ctx, 0.5, delta.m, 0.375, &D[k].m, 0.0);
    M[k] = gemm(ctx, Z[k].m, false, P.m, false, 1.0, tau);
    Z[k + 1] = add(ctx, 1.0, Z[k].m, 1.0, &M[k].m, 0.0);
  }
  const ifac_bsr& ZK = Z[K].m;
  {
    Mat FZ = gemm_masked(ctx, F, false, ZK, false, 1.0, ZK);
    *L_out = dot_on(ctx, ZK, FZ.m);
  }
  Mat Zh;
  {
    Mat FZ = gemm_masked(ctx, F, false, ZK, false, 1.0, ZK);
    Mat FtZ = gemm_masked(ctx, F, true, ZK, false, 1.0, ZK);
    Zh = add(ctx, 1.0, FZ.m, 1.0, &FtZ.m, 0.0);
  }
  Mat Sh = project(ctx, S.m, S.m);
  zero_values(ctx, Sh.m);
  for (int k = K - 1; k >= 0; --k) {
    const ifac_bsr& Zk = Z[k].m;
    const ifac_bsr& Xk = X[k].m;
    Mat delta = add(ctx, -1.0, Y[k].m, 0.0, nullptr, 1.0);
    Mat P = add(ctx, 0.5, delta.m, 0.375, &D[k].m, 0.0);
    Mat Mh = project(ctx, Zh.m, M[k].m);
    Mat Zn = project(ctx, Zh.m, Zk);
    Mat t1 = gemm_masked(ctx, Mh.m, false, P.m, true, 1.0, Zk);       // Pi_Z(Mh P^T)
    Mat Zacc = add(ctx, 1.0, Zn.m, 1.0, &t1.m, 0.0);
    Mat Ph = gemm_masked(ctx, Zk, true, Mh.m, false, 1.0, P.m);       // Pi_P(Z^T Mh)
    Mat Dh = project(ctx, Ph.m, D[k].m);
    Mat Dh38 = add(ctx, 0.375, Dh.m, 0.0, nullptr, 0.0);
    Mat a1 = gemm_masked(ctx, Dh38.m, false, delta.m, true, 1.0, delta.m);  // Pi_delta(Dh delta^T)
    Mat a2 = gemm_masked(ctx, delta.m, true, Dh38.m, false, 1.0, delta.m);  // Pi_delta(delta^T Dh)
    Mat Phd = project(ctx, Ph.m, delta.m);
    Mat s1 = add(ctx, 0.5, Phd.m, 1.0, &a1.m, 0.0);
    Mat deltah = add(ctx, 1.0, s1.m, 1.0, &a2.m, 0.0);
    Mat Yh0 = project(ctx, deltah.m, Y[k].m);
    Mat Yh = add(ctx, -1.0, Yh0.m, 0.0, nullptr, 0.0);
    Mat t2 = gemm_masked(ctx, Xk, false, Yh.m, true, 1.0, Zk);         // Pi_Z(X Yh^T)
    Mat Zacc2 = add(ctx, 1.0, Zacc.m, 1.0, &t2.m, 0.0);
    Mat Xh = gemm_masked(ctx, Zk, false, Yh.m, false, 1.0, Xk);        // Pi_X(Z Yh)
    Mat t3 = gemm_masked(ctx, S.m, true, Xh.m, false, 1.0, Zk);        // Pi_Z(S^T Xh)
    Mat t4 = gemm_masked(ctx, Xh.m, false, Zk, true, 1.0, S.m);        // Pi_S(Xh Z^T)
    Sh = add(ctx, 1.0, Sh.m, 1.0, &t4.m, 0.0);
    Zh = add(ctx, 1.0, Zacc2.m, 1.0, &t3.m, 0.0);
  }
  // the gradient on the pattern of the caller's S (zero on truncated blocks)
  Mat G = project(ctx, Sh.m, S_in);
  IFAC_CK(cudaStreamSynchronize(ctx->stream));
  *Sbar_out = G.release();
  return IFAC_OK;
}

}  // namespace ifac
