// blockops.cu -- memory-bound block operations: sums on a union pattern,
// block Frobenius norms, ||A||_F, the Gershgorin bound and Z_0 = c I.
//
// Sums follow the definition alpha*a + beta*b + gamma*[diag] with explicit
// round-to-nearest multiplies and adds (no fused multiply-add), in that
// order, so each element is rounded exactly as the plain definition is.
// Reductions run in a fixed order (per row, then over rows), so results are
// deterministic from run to run.  The block norms of sums are summed through
// FP32 (SqAcc: about 2^-44 relative) so that these kernels spend the FP64
// pipe -- GB300 runs about two FP64 operations per clock per SM -- on the
// sums alone.
#include <cmath>

#include "internal.cuh"
#include "tc_common.cuh"

using ifac::tc::SqAcc;

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

// alpha x, rounded to nearest.  GB300's FP64 pipe is narrow, so the common
// scales avoid it: alpha = +-1 is a sign change and alpha = 2^k an exponent
// change on the bit pattern (same result), other alphas one multiply.
struct Scale {
  int mode;  // 0 multiply, 1 identity, 2 negate, 3 power of two
  int k;     // mode 3: alpha = 2^k
  double alpha;
};

static Scale make_scale(double alpha) {
  Scale s{0, 0, alpha};
  if (alpha == 1.0) s.mode = 1;
  else if (alpha == -1.0) s.mode = 2;
  else if (alpha > 0.0 && std::isfinite(alpha)) {
    int e = 0;
    if (std::frexp(alpha, &e) == 0.5) {
      s.mode = 3;
      s.k = e - 1;
    }
  }
  return s;
}

__device__ __forceinline__ double scaled(const Scale& s, double x) {
  if (s.mode == 1) return x;
  const int hi = __double2hiint(x), lo = __double2loint(x);
  if (s.mode == 2) return __hiloint2double(hi ^ (int)0x80000000, lo);
  if (s.mode == 3) {
    const int ex = (hi >> 20) & 0x7ff, en = ex + s.k;
    if (ex > 0 && ex < 0x7ff && en > 0 && en < 0x7ff) return __hiloint2double(hi + (s.k << 20), lo);
  }
  return __dmul_rn(s.alpha, x);
}

// an operand value as FP64: FP32 values (the exact results of a TF32/BF16
// product) are widened on the bit pattern, off the FP64 pipe
__device__ __forceinline__ double as_f64(double x) { return x; }
__device__ __forceinline__ double as_f64(float x) { return ifac::tc::f32_to_f64(x); }

// two consecutive operand values (8- or 16-byte aligned) as FP64
__device__ __forceinline__ void load2(const double* p, double& x, double& y) {
  const double2 t = *reinterpret_cast<const double2*>(p);
  x = t.x;
  y = t.y;
}
__device__ __forceinline__ void load2(const float* p, double& x, double& y) {
  const float2 t = *reinterpret_cast<const float2*>(p);
  x = as_f64(t.x);
  y = as_f64(t.y);
}

// add_elem on loaded values: ha / hb say whether a / b exist
__device__ __forceinline__ double add_vals(const Scale& sa, bool ha, double a, const Scale& sb, bool hb, double b,
                                           bool diag, double gamma) {
  double v = 0.0;
  if (ha) v = scaled(sa, a);
  if (hb) {
    const double t = scaled(sb, b);
    v = ha ? __dadd_rn(v, t) : t;
  }
  if (diag) v = (ha || hb) ? __dadd_rn(v, gamma) : gamma;
  return v;
}

template <typename TA, typename TB>
__device__ __forceinline__ double add_elem(const Scale& sa, const TA* a, const Scale& sb, const TB* b, bool diag,
                                           double gamma, int e, int ea = -1) {
  double v = 0.0;
  if (a) v = scaled(sa, as_f64(a[ea < 0 ? e : ea]));
  if (b) {
    const double t = scaled(sb, as_f64(b[e]));
    v = a ? __dadd_rn(v, t) : t;
  }
  if (diag) v = (a || b) ? __dadd_rn(v, gamma) : gamma;
  return v;
}

// the K-major low-precision copy that the tensor-core products read (TF32:
// FP32 round-to-nearest-even then TF32 round-half-away; BF16 round-to-
// nearest-even, as their operand conversion rounds), written beside the
// FP64 result: lp_elt 4 TF32, 2 BF16, 0 none
__device__ __forceinline__ void lp_store2(void* lp, int lp_elt, size_t i, double x, double y) {
  if (lp_elt == 4) {
    uint2 w;
    w.x = ifac::tc::f32_to_tf32(__uint_as_float(ifac::tc::f64_to_f32_bits_rne(x)));
    w.y = ifac::tc::f32_to_tf32(__uint_as_float(ifac::tc::f64_to_f32_bits_rne(y)));
    *reinterpret_cast<uint2*>(static_cast<uint32_t*>(lp) + i) = w;
  } else if (lp_elt == 2) {
    const uint32_t w = (uint32_t)ifac::tc::f64_to_bf16_bits_rne(x) | ((uint32_t)ifac::tc::f64_to_bf16_bits_rne(y) << 16);
    *reinterpret_cast<uint32_t*>(static_cast<uint16_t*>(lp) + i) = w;
  }
}

// one warp per output block (grid-stride over blocks).  Element by element
// v = 0 + alpha a + beta b + gamma [diagonal], left to right, each step
// rounded; the leading 0 + x is x.  The FP64 Frobenius norm of the block.
// Lanes take consecutive elements (VEC of them: two for even bs * bs).  B's
// values are FP64 or FP32 (TB).
template <int VEC, typename TB>
__global__ void k_add(const int32_t* __restrict__ crow, const int32_t* __restrict__ cci, int64_t cnnz, int bs,
                      Scale sa, const int32_t* __restrict__ arp, const int32_t* __restrict__ aci,
                      const double* __restrict__ aval, Scale sb, const int32_t* __restrict__ brp,
                      const int32_t* __restrict__ bci, const TB* __restrict__ bval,
                      const int32_t* __restrict__ bmap, double gamma, double* __restrict__ cval,
                      double* __restrict__ cnorm, void* __restrict__ lp, int lp_elt) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int bsz = bs * bs;
  for (int64_t p = w0; p < cnnz; p += nw) {
    const int I = crow[p], J = cci[p];
    int qa = -1, qb = -1;
    if (lane == 0) {
      int q = find_col(aci, arp[I], arp[I + 1], J);
      qa = (q < arp[I + 1] && aci[q] == J) ? q : -1;
      if (bval) {
        int r = find_col(bci, brp[I], brp[I + 1], J);
        qb = (r < brp[I + 1] && bci[r] == J) ? r : -1;
      }
    }
    qa = __shfl_sync(0xffffffffu, qa, 0);
    qb = __shfl_sync(0xffffffffu, qb, 0);
    const double* a = qa >= 0 ? aval + (size_t)qa * bsz : nullptr;
    const TB* b = qb >= 0 ? bval + (size_t)(bmap ? bmap[qb] : qb) * bsz : nullptr;
    double* c = cval + (size_t)p * bsz;
    const bool dblk = I == J && gamma != 0.0;
    SqAcc sq;
#pragma unroll 4
    for (int e = lane * VEC; e < bsz; e += 32 * VEC) {
      if constexpr (VEC == 2) {
        // one vector load per operand (pairs never straddle two blocks)
        double ax = 0.0, ay = 0.0, bx = 0.0, by = 0.0;
        if (a) load2(a + e, ax, ay);
        if (b) load2(b + e, bx, by);
        double2 v;
        v.x = add_vals(sa, a != nullptr, ax, sb, b != nullptr, bx, dblk && e / bs == e % bs, gamma);
        v.y = add_vals(sa, a != nullptr, ay, sb, b != nullptr, by, dblk && (e + 1) / bs == (e + 1) % bs, gamma);
        *reinterpret_cast<double2*>(c + e) = v;
        if (lp_elt) lp_store2(lp, lp_elt, (size_t)p * bsz + e, v.x, v.y);
        sq.add_f64(v.x);
        sq.add_f64(v.y);
      } else {
        const double v = add_elem(sa, a, sb, b, dblk && e / bs == e % bs, gamma, e);
        c[e] = v;
        sq.add_f64(v);
      }
    }
    const double ss = sq.warp_total();
    if (lane == 0) cnorm[p] = sqrt(ss);
  }
}

void add_numeric(ifac_ctx* ctx, double alpha, const ifac_bsr& A, double beta, const ifac_bsr* B, double gamma,
                 ifac_bsr& C, const int32_t* crow, const int32_t* bmap, void* lp, int lp_elt, bool b32) {
  if (lp_elt && (C.bs * C.bs) % 2 != 0) fail(IFAC_ERR_UNSUPPORTED, "low-precision copy: even bs * bs");
  if (C.nnzb == 0) return;
  const int64_t warps = std::min<int64_t>(C.nnzb, 152 * 64);
  const Scale sa = make_scale(alpha), sb = make_scale(beta);
  const int32_t* brp = B ? B->row_ptr : nullptr;
  const int32_t* bci = B ? B->col_idx : nullptr;
  const double* bv = B ? B->val : nullptr;
  const int grid = cdiv(warps * 32, 256);
  if (b32 && B) {
    if ((C.bs * C.bs) % 2 != 0) fail(IFAC_ERR_UNSUPPORTED, "FP32 operand values: even bs * bs");
    k_add<2, float><<<grid, 256, 0, ctx->stream>>>(crow, C.col_idx, C.nnzb, C.bs, sa, A.row_ptr, A.col_idx, A.val, sb,
                                                   brp, bci, reinterpret_cast<const float*>(bv), bmap, gamma, C.val,
                                                   C.norms, lp, lp_elt);
  } else if ((C.bs * C.bs) % 2 == 0) {  // pairs never straddle two blocks
    k_add<2, double><<<grid, 256, 0, ctx->stream>>>(crow, C.col_idx, C.nnzb, C.bs, sa, A.row_ptr, A.col_idx, A.val,
                                                    sb, brp, bci, bv, bmap, gamma, C.val, C.norms, lp, lp_elt);
  } else {
    k_add<1, double><<<grid, 256, 0, ctx->stream>>>(crow, C.col_idx, C.nnzb, C.bs, sa, A.row_ptr, A.col_idx, A.val,
                                                    sb, brp, bci, bv, bmap, gamma, C.val, C.norms, nullptr, 0);
  }
  IFAC_CK_LAUNCH();
}

// C = alpha (U + strict_upper(U)^T) + beta B + gamma I, one warp per output
// block.  Block (I, J), J >= I, is add_elem of alpha U_IJ and beta B_IJ;
// block (I, J), J < I, takes alpha U_JI^T in place of alpha U_IJ, moved
// through shared memory in stripes of four output rows (four-value column
// segments of U_JI per source row: whole 32-byte sectors for FP64 values, half
// sectors for FP32 values, whose other half the next stripe reads from cache;
// eight-row stripes for FP32 measured slower: the doubled shared memory cuts
// the resident warps).  bs = 64.  U's values are FP64 or FP32 (TU).
constexpr int SYM_WARPS = 8;

template <typename TU>
__global__ void __launch_bounds__(32 * SYM_WARPS)
    k_sym(const int32_t* __restrict__ crow, const int32_t* __restrict__ cci, int64_t cnnz, Scale sa,
          const int32_t* __restrict__ urp, const int32_t* __restrict__ uci, const TU* __restrict__ uval,
          const int32_t* __restrict__ umap, Scale sb,
          const int32_t* __restrict__ brp, const int32_t* __restrict__ bci, const double* __restrict__ bval,
          double gamma, double* __restrict__ cval, double* __restrict__ cnorm, int mirror, void* __restrict__ lp,
          int lp_elt) {
  constexpr int BS = 64, BSZ = BS * BS;
  constexpr int RW = 4;  // output rows per stripe
  __shared__ double stripe[SYM_WARPS][RW][BS + 1];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double(*st)[BS + 1] = stripe[wid];  // RW rows
  for (int64_t p = w0; p < cnnz; p += nw) {
    const int I = crow[p], J = cci[p];
    const bool lower = J < I;
    const int r = lower ? J : I, c = lower ? I : J;
    int qu = -1, qb = -1;
    if (lane == 0) {
      const int k = find_col(uci, urp[r], urp[r + 1], c);
      qu = (k < urp[r + 1] && uci[k] == c) ? k : -1;
      if (bval) {
        const int m = find_col(bci, brp[I], brp[I + 1], J);
        qb = (m < brp[I + 1] && bci[m] == J) ? m : -1;
      }
    }
    qu = __shfl_sync(0xffffffffu, qu, 0);
    qb = __shfl_sync(0xffffffffu, qb, 0);
    const TU* u = qu >= 0 ? uval + (size_t)(umap ? umap[qu] : qu) * BSZ : nullptr;
    const double* b = qb >= 0 ? bval + (size_t)qb * BSZ : nullptr;
    double* out = cval + (size_t)p * BSZ;
    const bool dblk = I == J && gamma != 0.0;
    // mirror: a diagonal block takes its strictly lower triangle from its
    // upper one as well, so the result is exactly symmetric
    const bool mir = mirror && I == J;
    SqAcc sq;
    if (!lower || !u) {
#pragma unroll 4
      for (int e = lane * 2; e < BSZ; e += 64) {
        const int rr = e / BS, c0 = e % BS;
        double2 v;
        if (!mir) {  // one vector load per operand
          const TU* uu = lower ? nullptr : u;
          double ux = 0.0, uy = 0.0, bx = 0.0, by = 0.0;
          if (uu) load2(uu + e, ux, uy);
          if (b) load2(b + e, bx, by);
          v.x = add_vals(sa, uu != nullptr, ux, sb, b != nullptr, bx, dblk && rr == c0, gamma);
          v.y = add_vals(sa, uu != nullptr, uy, sb, b != nullptr, by, dblk && rr == c0 + 1, gamma);
        } else {
          const int e0 = c0 < rr ? c0 * BS + rr : -1, e1 = c0 + 1 < rr ? (c0 + 1) * BS + rr : -1;
          v.x = add_elem(sa, lower ? nullptr : u, sb, b, dblk && rr == c0, gamma, e, e0);
          v.y = add_elem(sa, lower ? nullptr : u, sb, b, dblk && rr == c0 + 1, gamma, e + 1, e1);
        }
        *reinterpret_cast<double2*>(out + e) = v;
        if (lp_elt) lp_store2(lp, lp_elt, (size_t)p * BSZ + e, v.x, v.y);
        sq.add_f64(v.x);
        sq.add_f64(v.y);
      }
    } else {
      for (int r0 = 0; r0 < BS; r0 += RW) {
        // alpha U_JI, source rows s = 0..63, columns r0..r0+RW-1
#pragma unroll 8
        for (int k = 0; k < 2 * RW; ++k) {
          const int idx = k * 32 + lane, s = idx / RW, j = idx % RW;
          st[j][s] = scaled(sa, as_f64(u[s * BS + r0 + j]));
        }
        __syncwarp();
        // output rows r0..r0+RW-1: alpha U_JI^T (+ beta B_IJ), columns 0..63
#pragma unroll
        for (int k = 0; k < RW; ++k) {
          const int idx = k * 64 + lane * 2, j = idx >> 6, col = idx & 63, e = (r0 + j) * BS + col;
          double2 v;
          v.x = st[j][col];
          v.y = st[j][col + 1];
          if (b) {
            v.x = __dadd_rn(v.x, scaled(sb, b[e]));
            v.y = __dadd_rn(v.y, scaled(sb, b[e + 1]));
          }
          *reinterpret_cast<double2*>(out + e) = v;
          if (lp_elt) lp_store2(lp, lp_elt, (size_t)p * BSZ + e, v.x, v.y);
          sq.add_f64(v.x);
          sq.add_f64(v.y);
        }
        __syncwarp();
      }
    }
    const double ss = sq.warp_total();
    if (lane == 0) cnorm[p] = sqrt(ss);
  }
}

void sym_numeric(ifac_ctx* ctx, double alpha, const ifac_bsr& U, double beta, const ifac_bsr* B, double gamma,
                 ifac_bsr& C, const int32_t* crow, const int32_t* umap, bool mirror, void* lp, int lp_elt, bool u32) {
  if (C.nnzb == 0) return;
  if (U.bs != 64) fail(IFAC_ERR_UNSUPPORTED, "symmetric completion needs bs = 64");
  const int64_t ctas = std::min<int64_t>(cdiv(C.nnzb, SYM_WARPS), 152 * 8);
  if (u32)
    k_sym<float><<<(int)ctas, 32 * SYM_WARPS, 0, ctx->stream>>>(
        crow, C.col_idx, C.nnzb, make_scale(alpha), U.row_ptr, U.col_idx, reinterpret_cast<const float*>(U.val), umap,
        make_scale(beta), B ? B->row_ptr : nullptr, B ? B->col_idx : nullptr, B ? B->val : nullptr, gamma, C.val,
        C.norms, mirror ? 1 : 0, lp, lp_elt);
  else
    k_sym<double><<<(int)ctas, 32 * SYM_WARPS, 0, ctx->stream>>>(
        crow, C.col_idx, C.nnzb, make_scale(alpha), U.row_ptr, U.col_idx, U.val, umap, make_scale(beta),
        B ? B->row_ptr : nullptr, B ? B->col_idx : nullptr, B ? B->val : nullptr, gamma, C.val, C.norms,
        mirror ? 1 : 0, lp, lp_elt);
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
