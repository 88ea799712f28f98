// rinch.cu -- recursive inverse Cholesky (Algorithm 1, left-looking, two
// blocks per dimension) on block-sparse matrices.
//
// With S = [S00 S01; S01^T S11] split at the block-aligned midpoint:
//   Z00 = rinch(S00),  R = Z00^T S01,  Q = -R^T R + S11,  Z11 = rinch(Q),
//   Z01 = -(Z00 R) Z11,  Z10 = 0,
// every product truncated at tau (Section 5), sums not truncated, and at the
// lowest level the dense leaf routine Z = L^-T (truncated).  Every matrix
// stays in the full n x n index space: S00, S01, S11 are S restricted to the
// quadrants of the range, so each product is an ordinary square block-sparse
// product whose pattern is confined to the right quadrant.
//
// Several disjoint ranges can be factorized together (the ranges of one
// recursion position move through the same launches, a product never
// coupling two ranges): a range at leaf size goes to the batched leaf
// launch, the others split.  A single matrix is one range.
#include <vector>

#include "internal.cuh"

namespace ifac {

namespace {

// keep block (I, J) when both lie in range s = seg[I] = seg[J], I on side qr
// and J on side qc of the range's midpoint (0: below mid, 1: at or above)
__global__ void k_quadrant_mask(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, int nb,
                                const int32_t* __restrict__ seg, const int32_t* __restrict__ mid, int qr, int qc,
                                uint8_t* __restrict__ keep) {
  const int row = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (row >= nb) return;
  const int s = seg[row];
  for (int p = rp[row] + lane; p < rp[row + 1]; p += 32) {
    const int J = ci[p];
    bool k = s >= 0 && seg[J] == s;
    if (k) k = ((row >= mid[s]) == (qr != 0)) && ((J >= mid[s]) == (qc != 0));
    keep[p] = k ? 1 : 0;
  }
}

struct Ranges {
  std::vector<std::pair<int, int>> r;  // [b0, b1) block ranges, disjoint
};

Mat quadrant(ifac_ctx* ctx, const ifac_bsr& A, const int32_t* seg, const int32_t* mid, int qr, int qc) {
  Buf<uint8_t> keep(ctx, A.nnzb);
  if (A.nnzb) {
    k_quadrant_mask<<<cdiv((int64_t)A.nb * 32, 256), 256, 0, ctx->stream>>>(A.row_ptr, A.col_idx, A.nb, seg, mid,
                                                                            qr, qc, keep.p);
    IFAC_CK_LAUNCH();
  }
  return select_blocks(ctx, A, nullptr, keep.p);
}

// Z for the ranges of S (S holds blocks inside those ranges only)
Mat rinch_rec(ifac_ctx* ctx, const ifac_bsr& S, const Ranges& ranges, double tau, int leaf_size, int depth,
              int* levels) {
  const int bs = S.bs, nb = S.nb;
  *levels = std::max(*levels, depth);
  std::vector<std::pair<int, int>> leaves, inner;
  for (const auto& r : ranges.r) {
    const int nbs = r.second - r.first;
    if ((int64_t)nbs * bs <= leaf_size || nbs == 1) leaves.push_back(r);
    else inner.push_back(r);
  }
  Mat Zl;
  if (!leaves.empty()) Zl = leaf_factors_ranges(ctx, S, leaves, tau);
  if (inner.empty()) return Zl;
  std::vector<int32_t> seg(nb, -1), mid(inner.size());
  Ranges ra, rc;
  for (size_t s = 0; s < inner.size(); ++s) {
    const int b0 = inner[s].first, b1 = inner[s].second, bm = b0 + (b1 - b0) / 2;
    for (int I = b0; I < b1; ++I) seg[I] = (int32_t)s;
    mid[s] = bm;
    ra.r.push_back({b0, bm});
    rc.r.push_back({bm, b1});
  }
  Buf<int32_t> dseg(ctx, nb), dmid(ctx, mid.size());
  IFAC_CK(cudaMemcpyAsync(dseg.p, seg.data(), sizeof(int32_t) * nb, cudaMemcpyHostToDevice, ctx->stream));
  IFAC_CK(cudaMemcpyAsync(dmid.p, mid.data(), sizeof(int32_t) * mid.size(), cudaMemcpyHostToDevice, ctx->stream));
  Mat S00 = quadrant(ctx, S, dseg.p, dmid.p, 0, 0);
  Mat S01 = quadrant(ctx, S, dseg.p, dmid.p, 0, 1);
  Mat S11 = quadrant(ctx, S, dseg.p, dmid.p, 1, 1);
  IFAC_CK(cudaStreamSynchronize(ctx->stream));  // seg / mid host vectors leave scope
  Mat Z00 = rinch_rec(ctx, S00.m, ra, tau, leaf_size, depth + 1, levels);
  S00.reset();
  Mat R = gemm(ctx, Z00.m, true, S01.m, false, 1.0, tau);     // R = Z00^T S01
  S01.reset();
  Mat RtR = gemm(ctx, R.m, true, R.m, false, 1.0, tau);       // R^T R
  Mat Q = add(ctx, -1.0, RtR.m, 1.0, &S11.m, 0.0);            // Q = -R^T R + S11
  RtR.reset();
  S11.reset();
  Mat Z11 = rinch_rec(ctx, Q.m, rc, tau, leaf_size, depth + 1, levels);
  Q.reset();
  Mat T = gemm(ctx, Z00.m, false, R.m, false, 1.0, tau);      // Z00 R
  R.reset();
  Mat Z01 = gemm(ctx, T.m, false, Z11.m, false, -1.0, tau);   // Z01 = -(Z00 R) Z11
  T.reset();
  Mat Z = add(ctx, 1.0, Z00.m, 1.0, &Z01.m, 0.0);
  Z = add(ctx, 1.0, Z.m, 1.0, &Z11.m, 0.0);
  if (!leaves.empty()) Z = add(ctx, 1.0, Z.m, 1.0, &Zl.m, 0.0);
  return Z;
}

}  // namespace

Mat rinch_ranges(ifac_ctx* ctx, const ifac_bsr& S, const std::vector<std::pair<int, int>>& ranges, double tau,
                 int leaf_size, int* levels) {
  Ranges r;
  r.r = ranges;
  return rinch_rec(ctx, S, r, tau, leaf_size, 0, levels);
}

int rinch(ifac_ctx* ctx, const ifac_bsr& S_in, double tau, const ifac_opts& o, ifac_bsr* Zout, ifac_report* rep) {
  report_init(ctx, rep, o);
  Mat S = truncate(ctx, S_in, tau);
  Ranges all;
  all.r.push_back({0, S.m.nb});
  int levels = 0;
  Mat Z = rinch_rec(ctx, S.m, all, tau, o.leaf_size, 0, &levels);
  Z.m.n = S_in.n;
  if (rep) {
    rep->levels = levels;
    rep->stop_reason = 0;
  }
  report_finish(ctx, rep, Z.m);
  if (rep) rep->levels = levels;
  IFAC_CK(cudaStreamSynchronize(ctx->stream));
  *Zout = Z.release();
  return IFAC_OK;
}

}  // namespace ifac
