// pattern.cu -- block-pattern (symbolic) work on the device.
//
// Patterns are handled as bitmaps: one bit per (block row, block column),
// W = ceil(nb/32) 32-bit words per block row.  The pattern of a product
// op(A) op(B) is, row by row, the OR of the op(B)-row bitmaps selected by the
// stored blocks of the op(A) row (every (I, J) with some K such that both
// blocks are stored); the pattern of a sum is the OR of the operands' bitmaps.
// Enumerating set bits in word order yields sorted column lists directly, so
// no sort is needed.  Row pointers come from an exclusive scan of popcounts.
#include "internal.cuh"

namespace ifac {

int words_per_row(int nb) { return (nb + 31) / 32; }

// ---------------------------------------------------------------------------
// exclusive scan of n int32 (single CTA): each thread takes 16 consecutive
// entries (loads issued together), the CTA scans the thread totals, carries
// between chunks of 16 blockDim entries; out[n] = the total
// ---------------------------------------------------------------------------
__global__ void k_scan_excl(const int32_t* __restrict__ in, int32_t* __restrict__ out, int n) {
  constexpr int K = 16;
  __shared__ int32_t wsum[32];
  __shared__ int32_t carry;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < n; base += blockDim.x * K) {
    const int i0 = base + threadIdx.x * K;
    int v[K];
    int t = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      v[k] = (i0 + k < n) ? in[i0 + k] : 0;
      t += v[k];
    }
    int x = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
      int sw = (lane < nw) ? wsum[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, sw, o);
        if (lane >= o) sw += y;
      }
      wsum[lane] = sw;
    }
    __syncthreads();
    int run = carry + (wid > 0 ? wsum[wid - 1] : 0) + x - t;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (i0 + k < n) out[i0 + k] = run;
      run += v[k];
    }
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = run;
    __syncthreads();
  }
  if (threadIdx.x == 0) out[n] = carry;
}

int64_t scan_counts(ifac_ctx* ctx, const int32_t* in, int32_t* out, int n, bool want_total) {
  k_scan_excl<<<1, 1024, 0, ctx->stream>>>(in, out, n);
  IFAC_CK_LAUNCH();
  if (!want_total) return -1;
  int32_t tot = 0;
  to_host(ctx, &tot, out + n, sizeof(int32_t));
  return tot;
}

// ---------------------------------------------------------------------------
// bitmaps
// ---------------------------------------------------------------------------
// one warp per block row of A; sets bit (r, c) of op(A)
__global__ void k_bitmap(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, int nb, int W,
                         int trans, uint32_t* __restrict__ bm) {
  int row = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (row >= nb) return;
  for (int p = rp[row] + lane; p < rp[row + 1]; p += 32) {
    int c = ci[p];
    int r = trans ? c : row, col = trans ? row : c;
    atomicOr(&bm[(size_t)r * W + (col >> 5)], 1u << (col & 31));
  }
}

__global__ void k_bitmap_diag(int nb, int W, uint32_t* __restrict__ bm) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nb) bm[(size_t)i * W + (i >> 5)] |= 1u << (i & 31);
}

Buf<uint32_t> pattern_bitmap(ifac_ctx* ctx, const ifac_bsr& A, bool trans) {
  int W = words_per_row(A.nb);
  Buf<uint32_t> bm(ctx, (size_t)A.nb * W);
  IFAC_CK(cudaMemsetAsync(bm.p, 0, sizeof(uint32_t) * (size_t)A.nb * W, ctx->stream));
  if (A.nnzb > 0) {
    k_bitmap<<<cdiv((int64_t)A.nb * 32, 256), 256, 0, ctx->stream>>>(A.row_ptr, A.col_idx, A.nb, W, trans ? 1 : 0, bm.p);
    IFAC_CK_LAUNCH();
  }
  return bm;
}

// per-row popcount (warp per row)
__global__ void k_row_popc(const uint32_t* __restrict__ bm, int nb, int W, int32_t* __restrict__ cnt) {
  int row = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (row >= nb) return;
  int c = 0;
  for (int w = lane; w < W; w += 32) c += __popc(bm[(size_t)row * W + w]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if (lane == 0) cnt[row] = c;
}

// enumerate set bits of each row in increasing column (warp per row)
__global__ void k_row_fill(const uint32_t* __restrict__ bm, int nb, int W, const int32_t* __restrict__ rp,
                           int32_t* __restrict__ ci, int32_t* __restrict__ row_of) {
  int row = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (row >= nb) return;
  int pos = rp[row];
  for (int base = 0; base < W; base += 32) {
    int w = base + lane;
    uint32_t word = (w < W) ? bm[(size_t)row * W + w] : 0u;
    int c = __popc(word);
    int x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    int off = pos + x - c;
    while (word) {
      int b = __ffs(word) - 1;
      ci[off] = w * 32 + b;
      if (row_of) row_of[off] = row;
      ++off;
      word &= word - 1;
    }
    pos += __shfl_sync(0xffffffffu, x, 31);
  }
}

Pattern pattern_from_bitmap(ifac_ctx* ctx, const uint32_t* bm, int nb, int64_t known_nnzb) {
  int W = words_per_row(nb);
  Pattern P;
  P.rp = Buf<int32_t>(ctx, nb + 1);
  Buf<int32_t> cnt(ctx, nb);
  int grid = cdiv((int64_t)nb * 32, 256);
  k_row_popc<<<grid, 256, 0, ctx->stream>>>(bm, nb, W, cnt.p);
  IFAC_CK_LAUNCH();
  P.nnzb = scan_counts(ctx, cnt.p, P.rp.p, nb, known_nnzb < 0);
  if (known_nnzb >= 0) P.nnzb = known_nnzb;
  P.ci = Buf<int32_t>(ctx, P.nnzb);
  P.row = Buf<int32_t>(ctx, P.nnzb);
  if (P.nnzb > 0) {
    k_row_fill<<<grid, 256, 0, ctx->stream>>>(bm, nb, W, P.rp.p, P.ci.p, P.row.p);
    IFAC_CK_LAUNCH();
  }
  return P;
}

// ---------------------------------------------------------------------------
// transposed views
// ---------------------------------------------------------------------------
// entry q of A^T (row c = row_t[q], column r = ci_t[q]) comes from block (r, c)
// of A, found by binary search in A's sorted row r.
__global__ void k_find_src(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, int64_t nnz,
                           const int32_t* __restrict__ row_t, const int32_t* __restrict__ ci_t,
                           int32_t* __restrict__ src) {
  int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= nnz) return;
  int r = ci_t[q], c = row_t[q];
  int lo = rp[r], hi = rp[r + 1];
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (ci[mid] < c) lo = mid + 1;
    else hi = mid;
  }
  src[q] = lo;
}

void transposed_positions(ifac_ctx* ctx, const ifac_bsr& A, const int32_t* row, int32_t* out) {
  if (A.nnzb == 0) return;
  k_find_src<<<cdiv(A.nnzb, 256), 256, 0, ctx->stream>>>(A.row_ptr, A.col_idx, A.nnzb, row, A.col_idx, out);
  IFAC_CK_LAUNCH();
}

View view_rows(ifac_ctx* ctx, const ifac_bsr& A, bool trans) {
  View v;
  if (!trans) {
    v.rp = A.row_ptr;
    v.ci = A.col_idx;
    v.src = nullptr;
    return v;
  }
  Buf<uint32_t> bm = pattern_bitmap(ctx, A, true);
  Pattern P = pattern_from_bitmap(ctx, bm.p, A.nb, A.nnzb);  // A^T has A's blocks
  v.own_src = Buf<int32_t>(ctx, P.nnzb);
  if (P.nnzb > 0) {
    k_find_src<<<cdiv(P.nnzb, 256), 256, 0, ctx->stream>>>(A.row_ptr, A.col_idx, P.nnzb, P.row.p, P.ci.p, v.own_src.p);
    IFAC_CK_LAUNCH();
  }
  v.own_rp = std::move(P.rp);
  v.own_ci = std::move(P.ci);
  v.rp = v.own_rp.p;
  v.ci = v.own_ci.p;
  v.src = v.own_src.p;
  return v;
}

// ---------------------------------------------------------------------------
// product and union patterns
// ---------------------------------------------------------------------------
// bmC[I] = OR over K in row I of op(A) of bmB[K]   (warp per row)
__global__ void k_product_rows(const int32_t* __restrict__ arp, const int32_t* __restrict__ aci, int nb, int W,
                               const uint32_t* __restrict__ bmB, uint32_t* __restrict__ bmC) {
  int row = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (row >= nb) return;
  int p0 = arp[row], p1 = arp[row + 1];
  for (int w = lane; w < W; w += 32) {
    uint32_t acc = 0;
    for (int p = p0; p < p1; ++p) acc |= bmB[(size_t)aci[p] * W + w];
    bmC[(size_t)row * W + w] = acc;
  }
}

// keep the bits of row i at columns j >= i (the upper block triangle)
__global__ void k_bitmap_upper(int nb, int W, uint32_t* __restrict__ bm) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)nb * W) return;
  const int i = (int)(e / W), w = (int)(e % W);
  if (w < (i >> 5)) bm[e] = 0u;
  else if (w == (i >> 5)) bm[e] &= ~((1u << (i & 31)) - 1u);
}

Pattern product_pattern(ifac_ctx* ctx, const View& arows, const ifac_bsr& B, bool transB, int nb, bool upper) {
  int W = words_per_row(nb);
  Buf<uint32_t> bmB = pattern_bitmap(ctx, B, transB);
  Buf<uint32_t> bmC(ctx, (size_t)nb * W);
  k_product_rows<<<cdiv((int64_t)nb * 32, 256), 256, 0, ctx->stream>>>(arows.rp, arows.ci, nb, W, bmB.p, bmC.p);
  IFAC_CK_LAUNCH();
  if (upper) {
    k_bitmap_upper<<<cdiv((int64_t)nb * W, 256), 256, 0, ctx->stream>>>(nb, W, bmC.p);
    IFAC_CK_LAUNCH();
  }
  return pattern_from_bitmap(ctx, bmC.p, nb);
}

__global__ void k_or_into(uint32_t* __restrict__ dst, const uint32_t* __restrict__ src, size_t n) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) dst[i] |= src[i];
}

Pattern union_pattern(ifac_ctx* ctx, const ifac_bsr& A, const ifac_bsr* B, bool diag) {
  int nb = A.nb, W = words_per_row(nb);
  Buf<uint32_t> bm = pattern_bitmap(ctx, A, false);
  if (B) {
    Buf<uint32_t> bb = pattern_bitmap(ctx, *B, false);
    size_t n = (size_t)nb * W;
    k_or_into<<<cdiv(n, 256), 256, 0, ctx->stream>>>(bm.p, bb.p, n);
    IFAC_CK_LAUNCH();
  }
  if (diag) {
    k_bitmap_diag<<<cdiv(nb, 256), 256, 0, ctx->stream>>>(nb, W, bm.p);
    IFAC_CK_LAUNCH();
  }
  return pattern_from_bitmap(ctx, bm.p, nb);
}

Pattern sym_pattern(ifac_ctx* ctx, const ifac_bsr& U, const ifac_bsr* B, bool diag) {
  int nb = U.nb, W = words_per_row(nb);
  Buf<uint32_t> bm = pattern_bitmap(ctx, U, false);
  if (U.nnzb > 0) {
    k_bitmap<<<cdiv((int64_t)nb * 32, 256), 256, 0, ctx->stream>>>(U.row_ptr, U.col_idx, nb, W, 1, bm.p);
    IFAC_CK_LAUNCH();
  }
  if (B && B->nnzb > 0) {
    k_bitmap<<<cdiv((int64_t)nb * 32, 256), 256, 0, ctx->stream>>>(B->row_ptr, B->col_idx, nb, W, 0, bm.p);
    IFAC_CK_LAUNCH();
  }
  if (diag) {
    k_bitmap_diag<<<cdiv(nb, 256), 256, 0, ctx->stream>>>(nb, W, bm.p);
    IFAC_CK_LAUNCH();
  }
  return pattern_from_bitmap(ctx, bm.p, nb);
}

__global__ void k_expand_rows(const int32_t* __restrict__ rp, int nb, int32_t* __restrict__ row) {
  int r = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (r >= nb) return;
  for (int p = rp[r] + lane; p < rp[r + 1]; p += 32) row[p] = r;
}

void expand_rows(ifac_ctx* ctx, const int32_t* rp, int nb, int32_t* row) {
  k_expand_rows<<<cdiv((int64_t)nb * 32, 256), 256, 0, ctx->stream>>>(rp, nb, row);
  IFAC_CK_LAUNCH();
}

// ---------------------------------------------------------------------------
// block selection / truncation with order-preserving compaction
// ---------------------------------------------------------------------------
__global__ void k_keep_from_norms(const double* __restrict__ norms, int64_t n, double tau, uint8_t* __restrict__ keep) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p < n) keep[p] = (norms[p] < tau) ? 0 : 1;  // NaN norms are kept, as in the oracle
}

__global__ void k_row_keep_count(const int32_t* __restrict__ rp, int nb, const uint8_t* __restrict__ keep,
                                 int32_t* __restrict__ cnt) {
  int row = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (row >= nb) return;
  int c = 0;
  for (int p = rp[row] + lane; p < rp[row + 1]; p += 32) c += keep[p];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if (lane == 0) cnt[row] = c;
}

// dest[p]: the new position of block p (-1: dropped); vmap (optional):
// vmap[new position] = p
__global__ void k_row_keep_dest(const int32_t* __restrict__ rp, int nb, const uint8_t* __restrict__ keep,
                                const int32_t* __restrict__ rp_new, const int32_t* __restrict__ ci,
                                const double* __restrict__ norms, int32_t* __restrict__ ci_new,
                                double* __restrict__ norms_new, int32_t* __restrict__ dest,
                                int32_t* __restrict__ vmap = nullptr) {
  int row = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (row >= nb) return;
  int pos = rp_new[row];
  for (int base = rp[row]; base < rp[row + 1]; base += 32) {
    int p = base + lane;
    bool k = (p < rp[row + 1]) && keep[p];
    unsigned m = __ballot_sync(0xffffffffu, k);
    if (p < rp[row + 1]) {
      int d = k ? pos + __popc(m & ((1u << lane) - 1u)) : -1;
      if (dest) dest[p] = d;
      if (k) {
        ci_new[d] = ci[p];
        norms_new[d] = norms[p];
        if (vmap) vmap[d] = p;
      }
    }
    pos += __popc(m);
  }
}

__global__ void k_copy_blocks(const double* __restrict__ src, const int32_t* __restrict__ dest, int64_t nblk,
                              int bsz, double* __restrict__ dst) {
  for (int64_t p = blockIdx.x; p < nblk; p += gridDim.x) {
    int d = dest[p];
    if (d < 0) continue;
    if ((bsz & 1) == 0) {  // even block size: every block starts 16-byte aligned
      const double2* s = reinterpret_cast<const double2*>(src + (size_t)p * bsz);
      double2* t = reinterpret_cast<double2*>(dst + (size_t)d * bsz);
      for (int e = threadIdx.x; e < bsz / 2; e += blockDim.x) t[e] = s[e];
    } else {
      for (int e = threadIdx.x; e < bsz; e += blockDim.x) dst[(size_t)d * bsz + e] = src[(size_t)p * bsz + e];
    }
  }
}

// row pointers of the kept blocks (keep[p] = 1), returns their number
static int64_t count_kept(ifac_ctx* ctx, const ifac_bsr& A, const uint8_t* keep, Buf<int32_t>& rp_new) {
  const int nb = A.nb;
  Buf<int32_t> cnt(ctx, nb);
  if (A.nnzb > 0) {
    k_row_keep_count<<<cdiv((int64_t)nb * 32, 256), 256, 0, ctx->stream>>>(A.row_ptr, nb, keep, cnt.p);
    IFAC_CK_LAUNCH();
  } else {
    IFAC_CK(cudaMemsetAsync(cnt.p, 0, sizeof(int32_t) * nb, ctx->stream));
  }
  rp_new = Buf<int32_t>(ctx, nb + 1);
  return scan_counts(ctx, cnt.p, rp_new.p, nb, true);
}

// a new matrix of the kept blocks of A, in order
static Mat gather_kept(ifac_ctx* ctx, const ifac_bsr& A, const uint8_t* keep, Buf<int32_t>&& rp_new, int64_t tot) {
  const int nb = A.nb;
  Mat R(ctx);
  R.m.n = A.n;
  R.m.bs = A.bs;
  R.m.nb = nb;
  R.m.nnzb = tot;
  R.m.row_ptr = rp_new.release();
  R.m.col_idx = static_cast<int32_t*>(dalloc(ctx, sizeof(int32_t) * (tot ? tot : 1)));
  R.m.norms = static_cast<double*>(dalloc(ctx, sizeof(double) * (tot ? tot : 1)));
  R.m.val = static_cast<double*>(dalloc(ctx, sizeof(double) * (size_t)(tot ? tot : 1) * A.bs * A.bs));
  if (A.nnzb > 0 && tot > 0) {
    const int grid = cdiv((int64_t)nb * 32, 256);
    Buf<int32_t> dest(ctx, A.nnzb);
    k_row_keep_dest<<<grid, 256, 0, ctx->stream>>>(A.row_ptr, nb, keep, R.m.row_ptr, A.col_idx, A.norms,
                                                   R.m.col_idx, R.m.norms, dest.p);
    IFAC_CK_LAUNCH();
    int blocks = (int)std::min<int64_t>(A.nnzb, 152 * 16);
    k_copy_blocks<<<blocks, 256, 0, ctx->stream>>>(A.val, dest.p, A.nnzb, A.bs * A.bs, R.m.val);
    IFAC_CK_LAUNCH();
  }
  return R;
}

Mat select_blocks(ifac_ctx* ctx, const ifac_bsr& A, const int32_t* row, const uint8_t* keep) {
  (void)row;
  Buf<int32_t> rp_new;
  const int64_t tot = count_kept(ctx, A, keep, rp_new);
  return gather_kept(ctx, A, keep, std::move(rp_new), tot);
}

Mat compact(ifac_ctx* ctx, Mat&& full, const int32_t* row, double tau, bool nocopy) {
  (void)row;
  if (full.m.nnzb == 0 || !(tau > 0)) return std::move(full);
  Buf<uint8_t> keep(ctx, full.m.nnzb);
  k_keep_from_norms<<<cdiv(full.m.nnzb, 256), 256, 0, ctx->stream>>>(full.m.norms, full.m.nnzb, tau, keep.p);
  IFAC_CK_LAUNCH();
  Buf<int32_t> rp_new;
  const int64_t tot = count_kept(ctx, full.m, keep.p, rp_new);
  if (tot == full.m.nnzb) return std::move(full);  // nothing dropped: no copy
  if (!nocopy) return gather_kept(ctx, full.m, keep.p, std::move(rp_new), tot);
  // the kept blocks stay in full's value array, which the result takes over
  const int nb = full.m.nb;
  Mat R(ctx);
  R.m.n = full.m.n;
  R.m.bs = full.m.bs;
  R.m.nb = nb;
  R.m.nnzb = tot;
  R.m.row_ptr = rp_new.release();
  R.m.col_idx = static_cast<int32_t*>(dalloc(ctx, sizeof(int32_t) * (tot ? tot : 1)));
  R.m.norms = static_cast<double*>(dalloc(ctx, sizeof(double) * (tot ? tot : 1)));
  R.vmap = Buf<int32_t>(ctx, (size_t)(tot ? tot : 1));
  if (tot > 0) {
    k_row_keep_dest<<<cdiv((int64_t)nb * 32, 256), 256, 0, ctx->stream>>>(
        full.m.row_ptr, nb, keep.p, R.m.row_ptr, full.m.col_idx, full.m.norms, R.m.col_idx, R.m.norms, nullptr,
        R.vmap.p);
    IFAC_CK_LAUNCH();
  }
  R.m.val = full.m.val;
  full.m.val = nullptr;
  return R;
}

}  // namespace ifac
