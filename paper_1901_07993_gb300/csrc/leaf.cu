// leaf.cu -- batched leaf routine of Algorithms 1-2 ("factorize S^-1 = Z Z*"):
// for each nl x nl SPD matrix, the Cholesky factor S = L L^T and Z = L^-T.
//
// One CTA per matrix, FP64, 32 x 32 tiles staged in shared memory, the matrix
// itself kept in global memory (it is L2-resident while its CTA works on it):
//   1. right-looking tiled Cholesky: factor tile (k,k), solve the panel
//      A_ik <- A_ik L_kk^-T, update the trailing tiles A_ij -= A_ik A_jk^T;
//   2. W_kk = L_kk^-1 for every diagonal tile (into scratch);
//   3. W = L^-1 by tile columns, W_ik = -W_ii sum_{l=k}^{i-1} L_il W_lk, and
//      Z = W^T is written into the upper triangle (which step 1 never reads);
//   4. diagonal tiles Z_kk = W_kk^T, strictly lower part cleared.
// A non-positive pivot j sets info = j + 1 (the pivot is replaced by 1 so the
// arithmetic stays finite; that matrix's Z is then meaningless).
#include "internal.cuh"

namespace ifac {

namespace {
constexpr int TB = 32;
constexpr int LD = TB + 1;  // padded shared-memory row
constexpr int NT = 256;
}  // namespace

__global__ void __launch_bounds__(NT) k_leaf_invchol(double* __restrict__ Abase, int nl, int* __restrict__ info,
                                                     double* __restrict__ Wdiag_base) {
  __shared__ double t0[TB * LD], t1[TB * LD], t2[TB * LD];
  __shared__ int bad;
  const int tid = threadIdx.x;
  const int T = nl / TB;
  double* A = Abase + (size_t)blockIdx.x * nl * nl;
  double* Wd = Wdiag_base + (size_t)blockIdx.x * T * TB * TB;
  auto at = [&](int r, int c) -> double& { return A[(size_t)r * nl + c]; };
  if (tid == 0) bad = 0;
  __syncthreads();
  // thread's 2x2 output in a 32x32 tile
  const int orow = (tid >> 4) * 2, ocol = (tid & 15) * 2;

  // ---------------- 1. Cholesky ----------------
  for (int k = 0; k < T; ++k) {
    const int k0 = k * TB;
    for (int e = tid; e < TB * TB; e += NT) t0[(e / TB) * LD + e % TB] = at(k0 + e / TB, k0 + e % TB);
    __syncthreads();
    for (int j = 0; j < TB; ++j) {
      if (tid == 0) {
        double d = t0[j * LD + j];
        if (!(d > 0.0)) {
          if (!bad) bad = k0 + j + 1;
          d = 1.0;
        }
        t0[j * LD + j] = sqrt(d);
      }
      __syncthreads();
      if (tid > j && tid < TB) t0[tid * LD + j] /= t0[j * LD + j];
      __syncthreads();
      for (int e = tid; e < TB * TB; e += NT) {
        int i = e / TB, l = e % TB;
        if (l > j && i >= l) t0[i * LD + l] -= t0[i * LD + j] * t0[l * LD + j];
      }
      __syncthreads();
    }
    for (int e = tid; e < TB * TB; e += NT) {
      int i = e / TB, l = e % TB;
      if (i >= l) at(k0 + i, k0 + l) = t0[i * LD + l];
    }
    // panel: each thread solves one row x of A_ik in place: x L_kk^T = a
    for (int rr = tid; rr < (T - k - 1) * TB; rr += NT) {
      const int gr = k0 + TB + rr;
      for (int j = 0; j < TB; ++j) {
        double s = at(gr, k0 + j);
        for (int l = 0; l < j; ++l) s -= at(gr, k0 + l) * t0[j * LD + l];
        at(gr, k0 + j) = s / t0[j * LD + j];
      }
    }
    __syncthreads();
    // trailing update A_ij -= A_ik A_jk^T for k < j <= i
    for (int j = k + 1; j < T; ++j) {
      for (int e = tid; e < TB * TB; e += NT) t1[(e / TB) * LD + e % TB] = at(j * TB + e / TB, k0 + e % TB);
      for (int i = j; i < T; ++i) {
        for (int e = tid; e < TB * TB; e += NT) t2[(e / TB) * LD + e % TB] = at(i * TB + e / TB, k0 + e % TB);
        __syncthreads();
        double c00 = 0, c01 = 0, c10 = 0, c11 = 0;
#pragma unroll 8
        for (int l = 0; l < TB; ++l) {
          double a0 = t2[orow * LD + l], a1 = t2[(orow + 1) * LD + l];
          double b0 = t1[ocol * LD + l], b1 = t1[(ocol + 1) * LD + l];
          c00 = fma(a0, b0, c00);
          c01 = fma(a0, b1, c01);
          c10 = fma(a1, b0, c10);
          c11 = fma(a1, b1, c11);
        }
        const int gi = i * TB + orow, gj = j * TB + ocol;
        at(gi, gj) -= c00;
        at(gi, gj + 1) -= c01;
        at(gi + 1, gj) -= c10;
        at(gi + 1, gj + 1) -= c11;
        __syncthreads();
      }
    }
  }
  __syncthreads();

  // ---------------- 2. W_kk = L_kk^-1 (one warp per tile, one lane per column) ----------------
  {
    const int lane = tid & 31, wid = tid >> 5;
    for (int k = wid; k < T; k += NT / 32) {
      const int k0 = k * TB;
      double* W = Wd + (size_t)k * TB * TB;  // row-major 32x32, lower triangular
      const int c = lane;
      for (int i = 0; i < TB; ++i) {
        double v;
        if (i < c) v = 0.0;
        else if (i == c) v = 1.0 / at(k0 + c, k0 + c);
        else {
          double s = 0.0;
          for (int l = c; l < i; ++l) s += at(k0 + i, k0 + l) * W[l * TB + c];
          v = -s / at(k0 + i, k0 + i);
        }
        W[i * TB + c] = v;
        __syncwarp();
      }
    }
  }
  __syncthreads();

  // ---------------- 3. off-diagonal tiles of W, stored as Z_ki = W_ik^T ----------------
  for (int k = 0; k < T; ++k) {
    for (int i = k + 1; i < T; ++i) {
      double c00 = 0, c01 = 0, c10 = 0, c11 = 0;  // (sum_l L_il W_lk) at (orow.., ocol..)
      for (int l = k; l < i; ++l) {
        // t1 <- L_il, t2 <- W_lk (W_kk from scratch, else the transpose of Z tile (k,l))
        for (int e = tid; e < TB * TB; e += NT) {
          int r = e / TB, c = e % TB;
          t1[r * LD + c] = at(i * TB + r, l * TB + c);
          t2[r * LD + c] = (l == k) ? Wd[(size_t)k * TB * TB + r * TB + c] : at(k * TB + c, l * TB + r);
        }
        __syncthreads();
#pragma unroll 8
        for (int q = 0; q < TB; ++q) {
          double a0 = t1[orow * LD + q], a1 = t1[(orow + 1) * LD + q];
          double b0 = t2[q * LD + ocol], b1 = t2[q * LD + ocol + 1];
          c00 = fma(a0, b0, c00);
          c01 = fma(a0, b1, c01);
          c10 = fma(a1, b0, c10);
          c11 = fma(a1, b1, c11);
        }
        __syncthreads();
      }
      // t1 <- the sum, t2 <- W_ii; W_ik = -W_ii * sum
      t1[orow * LD + ocol] = c00;
      t1[orow * LD + ocol + 1] = c01;
      t1[(orow + 1) * LD + ocol] = c10;
      t1[(orow + 1) * LD + ocol + 1] = c11;
      for (int e = tid; e < TB * TB; e += NT) t2[(e / TB) * LD + e % TB] = Wd[(size_t)i * TB * TB + e];
      __syncthreads();
      double d00 = 0, d01 = 0, d10 = 0, d11 = 0;
#pragma unroll 8
      for (int q = 0; q < TB; ++q) {
        double a0 = t2[orow * LD + q], a1 = t2[(orow + 1) * LD + q];
        double b0 = t1[q * LD + ocol], b1 = t1[q * LD + ocol + 1];
        d00 = fma(a0, b0, d00);
        d01 = fma(a0, b1, d01);
        d10 = fma(a1, b0, d10);
        d11 = fma(a1, b1, d11);
      }
      // Z tile (k, i) = W_ik^T: element (r, c) of W_ik goes to Z(k*TB + c, i*TB + r)
      at(k * TB + ocol, i * TB + orow) = -d00;
      at(k * TB + ocol + 1, i * TB + orow) = -d01;
      at(k * TB + ocol, i * TB + orow + 1) = -d10;
      at(k * TB + ocol + 1, i * TB + orow + 1) = -d11;
      __syncthreads();
    }
  }
  __syncthreads();

  // ---------------- 4. diagonal tiles, clear the strictly lower part ----------------
  for (int k = 0; k < T; ++k)
    for (int e = tid; e < TB * TB; e += NT) {
      int r = e / TB, c = e % TB;
      at(k * TB + r, k * TB + c) = (c >= r) ? Wd[(size_t)k * TB * TB + c * TB + r] : 0.0;
    }
  for (int i = 1; i < T; ++i)
    for (int j = 0; j < i; ++j)
      for (int e = tid; e < TB * TB; e += NT) at(i * TB + e / TB, j * TB + e % TB) = 0.0;
  if (tid == 0) info[blockIdx.x] = bad;
}

__global__ void k_pad_identity(const double* __restrict__ src, int nl, double* __restrict__ dst, int np, int count) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t per = (int64_t)np * np;
  if (e >= per * count) return;
  int64_t k = e / per, q = e % per;
  int r = (int)(q / np), c = (int)(q % np);
  dst[e] = (r < nl && c < nl) ? src[k * nl * nl + (int64_t)r * nl + c] : (r == c ? 1.0 : 0.0);
}

__global__ void k_unpad(const double* __restrict__ src, int np, double* __restrict__ dst, int nl, int count) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t per = (int64_t)nl * nl;
  if (e >= per * count) return;
  int64_t k = e / per, q = e % per;
  int r = (int)(q / nl), c = (int)(q % nl);
  dst[e] = src[k * np * np + (int64_t)r * np + c];
}

// A: count matrices of nl x nl (in place).  Pads to a multiple of 32 with an
// identity block when needed (the padded part factors to the identity).
void leaf_invchol(ifac_ctx* ctx, int count, int nl, double* A, int* info) {
  if (count == 0) return;
  const int np = ((nl + TB - 1) / TB) * TB;
  const int T = np / TB;
  Buf<double> wd(ctx, (size_t)count * T * TB * TB);
  if (np == nl) {
    k_leaf_invchol<<<count, NT, 0, ctx->stream>>>(A, nl, info, wd.p);
    IFAC_CK_LAUNCH();
    return;
  }
  Buf<double> pad(ctx, (size_t)count * np * np);
  int64_t tot = (int64_t)count * np * np;
  k_pad_identity<<<cdiv(tot, 256), 256, 0, ctx->stream>>>(A, nl, pad.p, np, count);
  IFAC_CK_LAUNCH();
  k_leaf_invchol<<<count, NT, 0, ctx->stream>>>(pad.p, np, info, wd.p);
  IFAC_CK_LAUNCH();
  int64_t tot2 = (int64_t)count * nl * nl;
  k_unpad<<<cdiv(tot2, 256), 256, 0, ctx->stream>>>(pad.p, np, A, nl, count);
  IFAC_CK_LAUNCH();
}

}  // namespace ifac

namespace ifac {

// Same computation as leaf_invchol, with the scratch supplied by the caller
// instead of allocated: wd holds count * ceil(nl/32) * 32 * 32 doubles and,
// when nl is not a multiple of 32, pad holds count * np * np doubles
// (np = nl rounded up to 32).  Returns the launch status.
cudaError_t leaf_invchol_launch_scratch(cudaStream_t stream, int count, int nl, double* A, int* info, double* wd,
                                        double* pad) {
  if (count == 0) return cudaSuccess;
  const int np = ((nl + TB - 1) / TB) * TB;
  if (np == nl) {
    k_leaf_invchol<<<count, NT, 0, stream>>>(A, nl, info, wd);
    return cudaGetLastError();
  }
  int64_t tot = (int64_t)count * np * np;
  k_pad_identity<<<cdiv(tot, 256), 256, 0, stream>>>(A, nl, pad, np, count);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_leaf_invchol<<<count, NT, 0, stream>>>(pad, np, info, wd);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int64_t tot2 = (int64_t)count * nl * nl;
  k_unpad<<<cdiv(tot2, 256), 256, 0, stream>>>(pad, np, A, nl, count);
  return cudaGetLastError();
}

}  // namespace ifac
