// reblock.cu -- the same matrix stored with another block size, and the
// autotuner that picks the block size and tile schedule of a batch.
//
// Re-blocking is exact: block (I', J') of the result holds the entries of
// rows [I' bs', (I' + 1) bs') and columns [J' bs', (J' + 1) bs') of the
// padded input, gathered from every input block that overlaps it.  A result
// block exists where some stored input block overlaps it; blocks that come
// out all zero are dropped, except diagonal blocks.  Rows past the input's
// padded size that the new padding adds get a unit diagonal, as the storage
// convention asks of every padding row.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.cuh"

namespace ifac {

// bit (I', J') for every result block overlapped by a stored input block
__global__ void k_reblock_bits(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, int nb_a, int bs_a,
                               int nb_b, int bs_b, int W, uint32_t* __restrict__ bm) {
  const int I = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (I >= nb_a) return;
  const int r0 = (I * bs_a) / bs_b, r1 = min(nb_b - 1, ((I + 1) * bs_a - 1) / bs_b);
  for (int p = rp[I] + lane; p < rp[I + 1]; p += 32) {
    const int J = ci[p];
    const int c0 = (J * bs_a) / bs_b, c1 = min(nb_b - 1, ((J + 1) * bs_a - 1) / bs_b);
    for (int r = r0; r <= r1; ++r)
      for (int c = c0; c <= c1; ++c) atomicOr(&bm[(size_t)r * W + (c >> 5)], 1u << (c & 31));
  }
}

__global__ void k_set_bit(uint32_t* __restrict__ bm, int W, int r, int c) {
  if (threadIdx.x == 0 && blockIdx.x == 0) bm[(size_t)r * W + (c >> 5)] |= 1u << (c & 31);
}

// one CTA per result block: zero it, copy the overlapping parts of the input
// blocks, unit diagonal on the rows past the input's padded size (pad_from),
// Frobenius norm; keep[q] = 1 when the block is non-zero or diagonal
__global__ void k_reblock_fill(const int32_t* __restrict__ arp, const int32_t* __restrict__ aci,
                               const double* __restrict__ aval, int nb_a, int bs_a, const int32_t* __restrict__ row,
                               const int32_t* __restrict__ bci, int64_t nnzb_b, int bs_b, int64_t pad_from,
                               double* __restrict__ bval, double* __restrict__ bnorm, uint8_t* __restrict__ keep) {
  __shared__ double red[8];
  for (int64_t q = blockIdx.x; q < nnzb_b; q += gridDim.x) {
    const int Ib = row[q], Jb = bci[q];
    double* dst = bval + (size_t)q * bs_b * bs_b;
    for (int e = threadIdx.x; e < bs_b * bs_b; e += blockDim.x) dst[e] = 0.0;
    __syncthreads();
    const int64_t rlo = (int64_t)Ib * bs_b, clo = (int64_t)Jb * bs_b;
    // input block rows and columns that overlap (none past the input's last)
    const int I0 = (int)(rlo / bs_a), I1 = min(nb_a - 1, (int)((rlo + bs_b - 1) / bs_a));
    const int J0 = (int)(clo / bs_a), J1 = min(nb_a - 1, (int)((clo + bs_b - 1) / bs_a));
    for (int I = I0; I <= I1; ++I) {
      // the input blocks of row I with columns J0..J1 (sorted columns)
      int lo = arp[I], hi = arp[I + 1];
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (aci[mid] < J0) lo = mid + 1;
        else hi = mid;
      }
      for (int p = lo; p < arp[I + 1] && aci[p] <= J1; ++p) {
        const int J = aci[p];
        const double* src = aval + (size_t)p * bs_a * bs_a;
        // overlap of input block (I, J) with the result block, in scalar rows/columns
        const int64_t r0 = max(rlo, (int64_t)I * bs_a), r1 = min(rlo + bs_b, (int64_t)(I + 1) * bs_a);
        const int64_t c0 = max(clo, (int64_t)J * bs_a), c1 = min(clo + bs_b, (int64_t)(J + 1) * bs_a);
        const int w = (int)(c1 - c0), h = (int)(r1 - r0);
        for (int e = threadIdx.x; e < w * h; e += blockDim.x) {
          const int64_t r = r0 + e / w, c = c0 + e % w;
          dst[(size_t)(r - rlo) * bs_b + (c - clo)] = src[(size_t)(r - (int64_t)I * bs_a) * bs_a + (c - (int64_t)J * bs_a)];
        }
      }
    }
    __syncthreads();
    if (Ib == Jb)
      for (int e = threadIdx.x; e < bs_b; e += blockDim.x)
        if (rlo + e >= pad_from) dst[(size_t)e * bs_b + e] = 1.0;
    __syncthreads();
    double ss = 0.0;
    int nz = 0;  // a non-zero entry (its square may underflow)
    for (int e = threadIdx.x; e < bs_b * bs_b; e += blockDim.x) {
      ss = fma(dst[e], dst[e], ss);
      nz |= dst[e] != 0.0;
    }
    nz = __syncthreads_or(nz);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
      bnorm[q] = sqrt(t);
      keep[q] = (nz || Ib == Jb) ? 1 : 0;
    }
    __syncthreads();
  }
}

Mat reblock(ifac_ctx* ctx, const ifac_bsr& A, int bs_b) {
  const int bs_a = A.bs, nb_a = A.nb;
  const int nb_b = (int)((A.n + bs_b - 1) / bs_b);
  const int W = words_per_row(nb_b);
  Buf<uint32_t> bm(ctx, (size_t)nb_b * W);
  IFAC_CK(cudaMemsetAsync(bm.p, 0, sizeof(uint32_t) * (size_t)nb_b * W, ctx->stream));
  if (A.nnzb) {
    k_reblock_bits<<<cdiv((int64_t)nb_a * 32, 256), 256, 0, ctx->stream>>>(A.row_ptr, A.col_idx, nb_a, bs_a, nb_b,
                                                                           bs_b, W, bm.p);
    IFAC_CK_LAUNCH();
  }
  // padding rows the new block size adds need their (diagonal) block
  const int64_t pad_from = (int64_t)nb_a * bs_a;
  if ((int64_t)nb_b * bs_b > pad_from) {
    k_set_bit<<<1, 32, 0, ctx->stream>>>(bm.p, W, nb_b - 1, nb_b - 1);
    IFAC_CK_LAUNCH();
  }
  Pattern P = pattern_from_bitmap(ctx, bm.p, nb_b);
  Mat F(ctx);
  F.m.n = A.n;
  F.m.bs = bs_b;
  F.m.nb = nb_b;
  F.m.nnzb = P.nnzb;
  F.m.row_ptr = P.rp.release();
  F.m.col_idx = P.ci.release();
  F.m.val = static_cast<double*>(dalloc(ctx, sizeof(double) * (size_t)std::max<int64_t>(P.nnzb, 1) * bs_b * bs_b));
  F.m.norms = static_cast<double*>(dalloc(ctx, sizeof(double) * (size_t)std::max<int64_t>(P.nnzb, 1)));
  Buf<uint8_t> keep(ctx, (size_t)std::max<int64_t>(P.nnzb, 1));
  if (P.nnzb) {
    k_reblock_fill<<<(int)std::min<int64_t>(P.nnzb, 152 * 16), 256, 0, ctx->stream>>>(
        A.row_ptr, A.col_idx, A.val, nb_a, bs_a, P.row.p, F.m.col_idx, P.nnzb, bs_b, pad_from, F.m.val, F.m.norms,
        keep.p);
    IFAC_CK_LAUNCH();
  }
  return select_blocks(ctx, F.m, nullptr, keep.p);
}

// ---------------------------------------------------------------------------
// autotuner
// ---------------------------------------------------------------------------

// block-diagonal matrix of the members (all at one block size)
Mat block_diag(ifac_ctx* ctx, int count, const ifac_bsr* const* S);

namespace {

double time_ms(ifac_ctx* ctx, cudaEvent_t a, cudaEvent_t b) {
  IFAC_CK(cudaEventSynchronize(b));
  float ms = 0.f;
  IFAC_CK(cudaEventElapsedTime(&ms, a, b));
  return ms;
}

}  // namespace

// The probe of one configuration: X = S S and Y = X X in the schedule's
// precision (X, with about the pattern of the later iterates Z, stands in for
// them), and the FP64-accurate split product X X; the best of `reps` runs
// each.
static void probe(ifac_ctx* ctx, const ifac_bsr& S, double tau, int prec, int reps, double* lp_ms, double* split_ms) {
  cudaEvent_t e0, e1;
  IFAC_CK(cudaEventCreate(&e0));
  IFAC_CK(cudaEventCreate(&e1));
  *lp_ms = INFINITY;
  *split_ms = INFINITY;
  try {
    Mat X = gemm(ctx, S, false, S, false, 1.0, tau, prec);
    for (int r = 0; r < reps; ++r) {
      IFAC_CK(cudaEventRecord(e0, ctx->stream));
      {
        Mat X2 = gemm(ctx, S, false, S, false, 1.0, tau, prec);
        Mat Y = gemm(ctx, X2.m, false, X2.m, false, 1.0, tau, prec);
      }
      IFAC_CK(cudaEventRecord(e1, ctx->stream));
      *lp_ms = std::min(*lp_ms, time_ms(ctx, e0, e1));
      IFAC_CK(cudaEventRecord(e0, ctx->stream));
      { Mat Y = gemm(ctx, X.m, false, X.m, false, 1.0, tau, IFAC_FP64_SPLIT); }
      IFAC_CK(cudaEventRecord(e1, ctx->stream));
      *split_ms = std::min(*split_ms, time_ms(ctx, e0, e1));
    }
  } catch (...) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    throw;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
}

void autotune(ifac_ctx* ctx, int count, const ifac_bsr* const* S, double tau, const ifac_opts& o,
              ifac_tune_result* out) {
  *out = ifac_tune_result{};
  const int prec = (o.prec == IFAC_TF32 || o.prec == IFAC_BF16) ? o.prec : IFAC_TF32;
  // predicted products of a batch refinement: low-precision sweeps of four
  // products (X, Y, delta^2, the correction) and FP64-accurate delta
  // evaluations of two; the probe runs two and one of them
  out->low_sweeps_est = 6;
  out->split_evals_est = 4;
  const double w_lp = 4.0 * out->low_sweeps_est / 2.0;
  const double w_split = 2.0 * out->split_evals_est;
  const int bss[3] = {32, 64, 128};
  const int old_lp = ctx->narrow_kmax, old_sp = ctx->narrow_kmax_split;
  double best = INFINITY;
  for (int i = 0; i < 3; ++i) {
    const int bs = bss[i];
    std::vector<Mat> held;
    held.reserve(count);  // no reallocation: the pointers below stay valid
    std::vector<const ifac_bsr*> ptrs(count);
    for (int k = 0; k < count; ++k) {
      if (S[k]->bs == bs) {
        ptrs[k] = S[k];
      } else {
        held.push_back(reblock(ctx, *S[k], bs));
        ptrs[k] = &held.back().m;
      }
    }
    Mat D = block_diag(ctx, count, ptrs.data());
    Mat St = truncate(ctx, D.m, tau);
    D.reset();
    held.clear();
    // tile schedules: at bs 64 the narrow tiles for tiles of at most KW K
    // blocks (default), for none, or for all, chosen separately for the
    // low-precision and the split products; the other sizes have one
    const int sched[3] = {-1, 0, 1 << 30};
    const int nsched = bs == 64 ? 3 : 1;
    double best_lp = INFINITY, best_sp = INFINITY;
    int sched_lp = -1, sched_sp = -1;
    for (int si = 0; si < nsched; ++si) {
      ctx->narrow_kmax = ctx->narrow_kmax_split = bs == 64 ? sched[si] : -1;
      double lp = 0, sp = 0;
      probe(ctx, St.m, tau, prec, 2, &lp, &sp);
      if (bs == 64) {
        out->probe64_lp_ms[si] = w_lp * lp;
        out->probe64_split_ms[si] = w_split * sp;
      }
      if (lp < best_lp) {
        best_lp = lp;
        sched_lp = ctx->narrow_kmax;
      }
      if (sp < best_sp) {
        best_sp = sp;
        sched_sp = ctx->narrow_kmax_split;
      }
    }
    const double pred = w_lp * best_lp + w_split * best_sp;
    out->probe_ms[i] = pred;
    if (pred < best) {
      best = pred;
      out->bs = bs;
      out->narrow_kmax = sched_lp;
      out->narrow_kmax_split = sched_sp;
    }
  }
  ctx->narrow_kmax = old_lp;
  ctx->narrow_kmax_split = old_sp;
}

}  // namespace ifac
