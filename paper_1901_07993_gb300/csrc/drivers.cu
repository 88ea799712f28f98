// drivers.cu -- the factorization drivers: refinement from a scaled identity
// (Section 2.2, Eq. 2.1) and localized inverse factorization (Algorithm 2
// with the localized update of Eq. 2.2 and the stop rule of Algorithm 4),
// plus the direct factorization error ||I - Z^T S Z||_F.
//
// Localized inverse factorization is run level by level: the bisection tree
// is built on the host, every leaf is factorized in one batched launch, and
// then, from the deepest internal level up, all sub-problems of one depth are
// refined together.  Their matrices are the block-diagonal restrictions of S
// and Z to the sub-problems, so one block-sparse product serves every
// sub-problem of the level (the products never couple two sub-problems); the
// stop rule is applied per sub-problem, and a stopped sub-problem's rows are
// removed from delta so its Z stays at the iterate the rule returned.
#include <cmath>
#include <vector>

#include "internal.cuh"

namespace ifac {

static double coef_b(int k) {
  double b = 1.0;
  for (int j = 1; j <= k; ++j) b = b * (double)(2 * j - 1) / (double)(2 * j);
  return b;
}

// P = sum_{k=1}^{m} b_k delta^k, powers by truncated products.  The first two
// terms are summed in one call, b_1 delta + b_2 delta^2, which rounds exactly
// as (0 + b_1 delta) + b_2 delta^2 (b_1 = 1/2 scales exactly).  sym: delta is
// symmetric, and each power (a polynomial in delta, so symmetric too) is formed
// on its upper block triangle only and completed by symmetry.  pc (sym, m =
// 2, TF32/BF16): P is returned as its pattern with its low-precision op(B)
// copy in *pc, all M = Z P needs (poly2_operand).
static Mat poly_P(ifac_ctx* ctx, const ifac_bsr& delta, int m, double tau, int prec = IFAC_FP64,
                  bool sym = false, OperandCache* pc = nullptr, OperandCache* dc = nullptr) {
  if (m < 2) return add(ctx, coef_b(1), delta, 0.0, nullptr, 0.0);
  const bool fused = sym && m == 2 && pc && (prec == IFAC_TF32 || prec == IFAC_BF16);
  // (fused: delta^2's kept blocks stay in place, in FP32, for the P kernel;
  // dc: delta's low-precision copy from its producer, serving both operands)
  Mat D = gemm(ctx, delta, false, delta, false, 1.0, tau, prec, sym, dc, nullptr, dc, fused, nullptr, nullptr,
               fused && ctx->fp32_mid);
  if (fused) return poly2_operand(ctx, D.m, delta, coef_b(1), coef_b(2), prec, pc, D.map(), D.f32);
  if (sym && m == 2) return sym_sum(ctx, coef_b(2), D.m, coef_b(1), &delta, 0.0);
  if (sym) D = sym_sum(ctx, 1.0, D.m, 0.0, nullptr, 0.0);
  Mat P = add(ctx, coef_b(1), delta, coef_b(2), &D.m, 0.0);
  for (int k = 3; k <= m; ++k) {
    Mat Dn = gemm(ctx, D.m, false, delta, false, 1.0, tau, prec, sym);
    if (sym) Dn = sym_sum(ctx, 1.0, Dn.m, 0.0, nullptr, 0.0);
    D = std::move(Dn);
    P = add(ctx, 1.0, P.m, coef_b(k), &D.m, 0.0);
  }
  return P;
}

void report_init(ifac_ctx* ctx, ifac_report* r, const ifac_opts& o) {
  ctx->products = 0;
  ctx->pairs = 0;
  ctx->launches = 0;
  ctx->gemm_launches = 0;
  ctx->tc_launches = 0;
  ctx->split_launches = 0;
  ctx->pairs_fp64 = 0;
  ctx->pairs_tc = 0;
  ctx->pairs_split = 0;
  ctx->slice_pairs = 0;
  ctx->bytes_fp64 = ctx->bytes_tc = ctx->bytes_split = 0;
  ctx->events_used = 0;
  ctx->profile = o.profile != 0;
  reset_device_counters(ctx);
  if (r) *r = ifac_report{};
}

// precision of FP64-accurate delta products: the split tensor-core product
// where the options ask for it and it is built (bs 32, 64, 128), else the
// FP64 pipe
int delta_prec_of(const ifac_opts& o, int bs) {
  return (o.delta_prec == IFAC_FP64_SPLIT && (bs == 32 || bs == 64 || bs == 128)) ? IFAC_FP64_SPLIT : IFAC_FP64;
}

// A split product with s slices per operand errs by about 2^-(7 s - 3)
// relative to the row and column maxima of its operands; for Z^T (S Z) near
// convergence that puts the error of ||delta||_F at about 2^-(7 s - 3)
// ||I||_F = 2^-(7 s - 3) sqrt(n) (seven slices: 7e-12 at n = 262,144, as
// measured).
double split_delta_error(int slices, int64_t n) {
  return std::ldexp(std::sqrt((double)n), -(7 * slices - 3));
}

double unit_roundoff(int prec) { return prec == IFAC_BF16 ? std::ldexp(1.0, -8) : std::ldexp(1.0, -11); }

// Once the low-precision floor is reached, a sweep whose delta is exact
// leaves ||delta'||_F of about u ||delta||_F (the correction M carries the
// low format's rounding; measured: 0.7 u to 1.4 u with TF32), and an error
// in delta passes into delta' about one to one.  An evaluation error below a
// tenth of u e therefore costs no convergence; below the target, no false
// stop.
double delta_need(double e, double target, double u) { return 0.1 * std::max(target, u * e); }

// the fewest slices (at least 3, at most the context's count) whose error
// meets delta_need for the predicted ||delta||_F
int delta_slices(const ifac_ctx* ctx, double e_pred, double target, double u, int64_t n) {
  const int full = ctx->split_slices;
  if (!(e_pred < 1.0e300)) return full;
  const double need = delta_need(e_pred, target, u);
  int s = 3;
  while (s < full && split_delta_error(s, n) > need) ++s;
  return std::min(full, s);
}

void report_finish(ifac_ctx* ctx, ifac_report* r, const ifac_bsr& Z) {
  check_device_error(ctx);
  read_device_counters(ctx, &ctx->pairs_fp64, &ctx->pairs_tc, &ctx->pairs_split, &ctx->slice_pairs);
  ctx->pairs = ctx->pairs_fp64 + ctx->pairs_tc + ctx->pairs_split;
  if (!r) {
    double a, b;
    prof_collect(ctx, &a, &b);
    ctx->profile = false;
    return;
  }
  r->products = ctx->products;
  r->block_pairs = ctx->pairs;
  r->nnzb_Z = Z.nnzb;
  r->flops = 2.0 * (double)Z.bs * Z.bs * Z.bs * (double)ctx->pairs;
  prof_collect(ctx, &r->gemm_ms, &r->tc_ms, &r->split_ms);
  r->launches = ctx->launches;
  r->gemm_launches = ctx->gemm_launches;
  r->tc_launches = ctx->tc_launches;
  r->split_launches = ctx->split_launches;
  r->split_pairs = ctx->pairs_split;
  r->split_slice_pairs = ctx->slice_pairs;
  r->fp64_bytes = ctx->bytes_fp64;
  r->tc_bytes = ctx->bytes_tc;
  r->split_bytes = ctx->bytes_split;
  r->fp64_pairs = ctx->pairs_fp64;
  r->tc_pairs = ctx->pairs_tc;
  ctx->profile = false;
}

// ---------------------------------------------------------------------------
// refinement from a scaled identity
// ---------------------------------------------------------------------------
int refine_irsi(ifac_ctx* ctx, const ifac_bsr& S_in, double tau, double target, const ifac_opts& o, ifac_bsr* Zout,
                ifac_report* rep) {
  report_init(ctx, rep, o);
  Mat S = truncate(ctx, S_in, tau);
  const double beta = gershgorin_host(ctx, S.m);
  const double c = (o.c_rule == 1) ? std::sqrt(2.0 / beta) : 1.0 / std::sqrt(beta);
  Mat Z = scaled_identity(ctx, S.m.n, S.m.bs, S.m.nb, c);
  if (rep) rep->beta = beta;
  double e_prev = INFINITY;
  int stop = 0, it = 0;
  double e = 0.0;
  auto direct_delta = [&](const ifac_bsr& Zc) {
    OperandCache zcache;  // split products: Z's slices (op(B) of S Z) serve op(A) = Z^T
    Mat X = gemm(ctx, S.m, false, Zc, false, 1.0, tau, IFAC_FP64, false, nullptr, &zcache);  // S Z
    Mat Y = gemm(ctx, Zc, true, X.m, false, 1.0, tau, IFAC_FP64, false, &zcache);            // Z^T (S Z)
    X.reset();
    return add(ctx, -1.0, Y.m, 0.0, nullptr, 1.0);         // I - Z^T S Z
  };
  Mat D = direct_delta(Z.m);
  for (it = 0;; ++it) {
    e = fro_host(ctx, D.m);
    if (rep && rep->n_delta < 64) rep->delta_fro[rep->n_delta++] = e;
    if (o.fixed_iters > 0) {
      if (it == o.fixed_iters) stop = IFAC_STOP_FIXED;
    } else if (e <= target) {
      stop = IFAC_STOP_TARGET;
    } else if (e > std::pow(e_prev, (double)(o.m + 1))) {
      stop = IFAC_STOP_RULE;
    } else if (it == o.max_iter) {
      stop = IFAC_STOP_MAXITER;
    }
    if (stop) break;
    Mat P = poly_P(ctx, D.m, o.m, tau);
    Mat M = gemm(ctx, Z.m, false, P.m, false, 1.0, tau);   // M = Z sum b_k delta^k
    P.reset();
    Mat Zn = add(ctx, 1.0, Z.m, 1.0, &M.m, 0.0);           // Z + M
    if (o.local_delta) {
      // Eq. (2.2): delta' = delta - Z_{i+1}^T (S M) - (M^T S) Z_i, M^T S = (S M)^T
      Mat T = gemm(ctx, S.m, false, M.m, false, 1.0, tau);
      Mat U = gemm(ctx, Zn.m, true, T.m, false, 1.0, tau);
      Mat V = gemm(ctx, T.m, true, Z.m, false, 1.0, tau);
      T.reset();
      Mat D1 = add(ctx, 1.0, D.m, -1.0, &U.m, 0.0);
      D = add(ctx, 1.0, D1.m, -1.0, &V.m, 0.0);
    }
    M.reset();
    Z = std::move(Zn);
    if (!o.local_delta) D = direct_delta(Z.m);
    e_prev = e;
  }
  if (rep) {
    rep->sweeps = it;
    rep->stop_reason = stop;
  }
  if (stop == IFAC_STOP_MAXITER) {
    IFAC_CK(cudaStreamSynchronize(ctx->stream));
    fail(IFAC_ERR_NO_CONVERGENCE, "no convergence in max_iter sweeps; ||delta||_F = " + std::to_string(e));
  }
  report_finish(ctx, rep, Z.m);
  IFAC_CK(cudaStreamSynchronize(ctx->stream));
  *Zout = Z.release();
  return (stop == IFAC_STOP_RULE && e > target) ? IFAC_WARN_TARGET_NOT_MET : IFAC_OK;
}

// ---------------------------------------------------------------------------
// mixed-precision refinement from a scaled identity
// ---------------------------------------------------------------------------
int refine_irsi_mixed(ifac_ctx* ctx, const ifac_bsr& S_in, double tau, double target, const ifac_opts& o,
                      ifac_bsr* Zout, ifac_report* rep) {
  if (S_in.bs != 32 && S_in.bs != 64 && S_in.bs != 128)
    fail(IFAC_ERR_UNSUPPORTED, "mixed precision: bs 32, 64 or 128");
  if (S_in.bs == 128 && delta_prec_of(o, 128) != IFAC_FP64_SPLIT)
    fail(IFAC_ERR_UNSUPPORTED, "mixed precision at bs 128 needs split delta products (the FP64 pipe kernel stops at 64)");
  // upper-triangle symmetric products (and their completion kernel) at bs 64
  const bool sym = S_in.bs == 64;
  report_init(ctx, rep, o);
  const int low = o.prec;
  Mat S = truncate(ctx, S_in, tau);
  const double beta = gershgorin_host(ctx, S.m);
  const double c = (o.c_rule == 1) ? std::sqrt(2.0 / beta) : 1.0 / std::sqrt(beta);
  Mat Z = scaled_identity(ctx, S.m.n, S.m.bs, S.m.nb, c);
  if (rep) rep->beta = beta;
  bool fp64_phase = false, all_slices = false, slices_fixed = false;
  double e_prev = INFINITY, e = 0.0, e_pred = INFINITY;
  const double u = unit_roundoff(low);
  // S's converted copies serve every X = S Z of the refinement
  OperandCache scache;
  scache.want_ns = ctx->split_slices;
  // low-precision copies written by the sums that produce delta (for
  // delta^2) and Z (for M = Z P), so neither is converted in a separate pass
  OperandCache dcache, znat;
  int stop = 0, sweeps = 0, fp64_evals = 0, low_sweeps = 0;
  for (int it = 0;; ++it) {
    const int dprec = fp64_phase ? delta_prec_of(o, S.m.bs) : low;
    // split evaluations take as many slices as this delta needs (predicted
    // from the last one)
    const int ns = (dprec == IFAC_FP64_SPLIT && !all_slices && !slices_fixed)
                       ? delta_slices(ctx, e_pred, target, u, S.m.n)
                       : ctx->split_slices;
    Mat D;
    {
      SlicesScope scope(ctx, ns);
      // Z^T S Z is symmetric: its upper block triangle is formed and the
      // lower one taken from it, halving the second product
      // Z's converted copy (op(B) of S Z) serves again as op(A) = Z^T
      // truncated products keep their kept blocks in place where the next
      // step reads them through a value map (no compaction copies)
      // low-precision sweeps keep X and the upper triangle of Y in FP32, as
      // their products accumulated them (the next step reads them exactly)
      OperandCache zcache;
      const bool inplace = dprec != IFAC_FP64;
      const bool lp = (dprec == IFAC_TF32 || dprec == IFAC_BF16) && ctx->fp32_mid;
      Mat X = gemm(ctx, S.m, false, Z.m, false, 1.0, tau, dprec, false, &scache, &zcache, nullptr, inplace, nullptr,
                   nullptr, lp);  // S Z
      Mat Y = gemm(ctx, Z.m, true, X.m, false, 1.0, tau, dprec, sym, &zcache, nullptr, nullptr, sym, nullptr,
                   X.map(), lp && sym, X.f32);  // Z^T (S Z), J >= I
      X.reset();
      // I - Z^T S Z, exactly symmetric, with its low-precision copy for delta^2
      D = sym ? sym_sum(ctx, -1.0, Y.m, 0.0, nullptr, 1.0, Y.map(), true, low, &dcache, Y.f32)
              : add(ctx, -1.0, Y.m, 0.0, nullptr, 1.0);
    }
    e = fro_host(ctx, D.m);
    const bool stall = fp64_phase && e > kStallRatio * e_prev;
    if (dprec == IFAC_FP64_SPLIT && ns < ctx->split_slices &&
        (split_delta_error(ns, S.m.n) > delta_need(e, target, u) || e <= target || stall)) {
      // delta came out below its predicted size, past what this many slices
      // resolve, or at the target, where the stop must not rest on fewer
      // slices (on dense operands the error of an s-slice evaluation is far
      // above the chain-derived estimate), or it stalls: evaluate it again
      // with all of them; after a stall the comparison restarts
      if (stall) {
        slices_fixed = true;
        e_prev = INFINITY;
      }
      all_slices = true;
      --it;
      continue;
    }
    all_slices = false;
    e_pred = u * e;
    if (rep && rep->n_delta < 64) rep->delta_fro[rep->n_delta++] = e;
    if (fp64_phase) {
      ++fp64_evals;
      if (e <= target) stop = IFAC_STOP_TARGET;
      else if (!(e < e_prev)) stop = IFAC_STOP_RULE;   // no longer decreasing: the FP64 floor
      else if (it >= o.max_iter) stop = IFAC_STOP_MAXITER;
      if (stop) break;
    } else if (e > std::pow(e_prev, (double)(o.m + 1)) || !(e < e_prev) || it >= o.max_iter) {
      // rounding of the low-precision products dominates: the automatic rule
      // of Section 2.2 fires, or -- when that floor of ||delta||_F lies above
      // 1, where the rule cannot fire -- delta stops decreasing.  Evaluate
      // delta with FP64 products for this Z.
      fp64_phase = true;
      e_prev = INFINITY;
      e_pred = 0.1 * e;  // the same Z; its low-precision ||delta||_F may sit on that format's floor
      // a block-dense factor: the slice rule's error estimate (from banded
      // factors, where each product sums a few blocks) is far too small, and
      // the first evaluations it allows would stall (kStallRatio); every
      // evaluation takes all slices
      if (2 * Z.m.nnzb > (int64_t)Z.m.nb * Z.m.nb) slices_fixed = true;
      if (rep && rep->n_delta > 0) --rep->n_delta;
      --it;
      continue;
    }
    OperandCache pcache;  // P's low-precision op(B) copy, written with P
    Mat P = poly_P(ctx, D.m, o.m, tau, low, sym, &pcache, sym ? &dcache : nullptr);
    D.reset();
    dcache.reset();
    Mat M = gemm(ctx, Z.m, false, P.m, false, 1.0, tau, low, false, &znat, nullptr, &pcache, true, nullptr, nullptr,
                 ctx->fp32_mid);  // M = Z P, kept in FP32
    P.reset();
    Z = add(ctx, 1.0, Z.m, 1.0, &M.m, 0.0, M.map(), low, &znat, M.f32);  // with Z's copy for the next M
    ++sweeps;
    e_prev = e;
    if (!fp64_phase) {
      ++low_sweeps;
      // cubic convergence from e predicts e^(m+1) for the new Z; below
      // u sqrt(n) -- about where the low-precision corrections stop the
      // sweeps on every input measured (262,144-row chain: TF32 floor 0.33,
      // u sqrt(n) = 0.25) -- the next low-precision delta would only find
      // that floor, so the new Z's delta is evaluated FP64-accurately at once
      const double pred = std::pow(e, (double)(o.m + 1)), floor_est = u * std::sqrt((double)S.m.n);
      if (e < 1.0 && pred < floor_est) {
        fp64_phase = true;
        e_prev = INFINITY;
        e_pred = 0.1 * std::max(pred, floor_est);
        if (2 * Z.m.nnzb > (int64_t)Z.m.nb * Z.m.nb) slices_fixed = true;  // block-dense: all slices
      }
    }
  }
  if (rep) {
    rep->sweeps = sweeps;
    rep->stop_reason = stop;
    rep->fp64_delta_evals = fp64_evals;
    rep->low_sweeps = low_sweeps;
  }
  if (stop == IFAC_STOP_MAXITER) {
    IFAC_CK(cudaStreamSynchronize(ctx->stream));
    fail(IFAC_ERR_NO_CONVERGENCE, "no convergence in max_iter sweeps; ||delta||_F = " + std::to_string(e));
  }
  report_finish(ctx, rep, Z.m);
  IFAC_CK(cudaStreamSynchronize(ctx->stream));
  *Zout = Z.release();
  return (e > target) ? IFAC_WARN_TARGET_NOT_MET : IFAC_OK;
}

// ---------------------------------------------------------------------------
// localized inverse factorization helpers
// ---------------------------------------------------------------------------
enum FilterMode { F_ROWS_IN = 0, F_ROWS_OUT = 1, F_SAME = 2, F_COUPLE = 3 };

__global__ void k_filter_mask(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, int nb,
                              const int32_t* __restrict__ seg, const int32_t* __restrict__ mid,
                              const uint8_t* __restrict__ active, int mode, uint8_t* __restrict__ keep) {
  int row = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (row >= nb) return;
  const int s = seg[row];
  for (int p = rp[row] + lane; p < rp[row + 1]; p += 32) {
    const int J = ci[p];
    bool k;
    switch (mode) {
      case F_ROWS_IN: k = s >= 0 && (!active || active[s]); break;
      case F_ROWS_OUT: k = s < 0; break;
      case F_SAME: k = s >= 0 && seg[J] == s; break;
      default: k = s >= 0 && seg[J] == s && row < mid[s] && J >= mid[s]; break;
    }
    keep[p] = k ? 1 : 0;
  }
}

static Mat filter(ifac_ctx* ctx, const ifac_bsr& A, const int32_t* seg, const int32_t* mid, const uint8_t* active,
                  int mode) {
  Buf<uint8_t> keep(ctx, A.nnzb);
  if (A.nnzb) {
    k_filter_mask<<<cdiv((int64_t)A.nb * 32, 256), 256, 0, ctx->stream>>>(A.row_ptr, A.col_idx, A.nb, seg, mid,
                                                                          active, mode, keep.p);
    IFAC_CK_LAUNCH();
  }
  return select_blocks(ctx, A, nullptr, keep.p);
}

// explicit transpose: block q of A^T = (block src[q] of A)^T
__global__ void k_transpose_blocks(const double* __restrict__ val, const double* __restrict__ norms,
                                   const int32_t* __restrict__ src, int64_t nnzb, int bs, double* __restrict__ out,
                                   double* __restrict__ onorms) {
  const int bsz = bs * bs;
  for (int64_t q = blockIdx.x; q < nnzb; q += gridDim.x) {
    const double* s = val + (size_t)src[q] * bsz;
    double* t = out + (size_t)q * bsz;
    for (int e = threadIdx.x; e < bsz; e += blockDim.x) {
      int r = e / bs, c = e % bs;
      t[e] = s[c * bs + r];
    }
    if (threadIdx.x == 0) onorms[q] = norms[src[q]];
  }
}

static Mat transpose_mat(ifac_ctx* ctx, const ifac_bsr& A) {
  View v = view_rows(ctx, A, true);
  Mat T(ctx);
  T.m.n = A.n;
  T.m.bs = A.bs;
  T.m.nb = A.nb;
  T.m.nnzb = A.nnzb;
  T.m.row_ptr = v.own_rp.release();
  T.m.col_idx = v.own_ci.release();
  T.m.val = static_cast<double*>(dalloc(ctx, sizeof(double) * (size_t)(A.nnzb ? A.nnzb : 1) * A.bs * A.bs));
  T.m.norms = static_cast<double*>(dalloc(ctx, sizeof(double) * (A.nnzb ? A.nnzb : 1)));
  if (A.nnzb) {
    int grid = (int)std::min<int64_t>(A.nnzb, 152 * 16);
    k_transpose_blocks<<<grid, 256, 0, ctx->stream>>>(A.val, A.norms, v.src, A.nnzb, A.bs, T.m.val, T.m.norms);
    IFAC_CK_LAUNCH();
  }
  return T;
}

// dense leaf buffers: identity everywhere, then the diagonal range of S of
// each leaf copied in (block (I, J) of S with both rows in leaf k)
__global__ void k_identity_fill(double* __restrict__ buf, int np, int count) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t per = (int64_t)np * np;
  if (e >= per * count) return;
  int64_t q = e % per;
  buf[e] = ((q / np) == (q % np)) ? 1.0 : 0.0;
}

__global__ void k_leaf_gather(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                              const double* __restrict__ val, int nb, int bs, const int32_t* __restrict__ leaf_of,
                              const int32_t* __restrict__ leaf_b0, int np, double* __restrict__ buf) {
  // one CTA per block row; rows outside every leaf (leaf_of < 0) are skipped
  const int I = blockIdx.x;
  if (I >= nb || leaf_of[I] < 0) return;
  const int k = leaf_of[I], b0 = leaf_b0[k];
  double* dst = buf + (size_t)k * np * np;
  for (int p = rp[I]; p < rp[I + 1]; ++p) {
    const int J = ci[p];
    if (leaf_of[J] != k) continue;
    const double* s = val + (size_t)p * bs * bs;
    for (int e = threadIdx.x; e < bs * bs; e += blockDim.x) {
      int r = e / bs, c = e % bs;
      dst[(size_t)((I - b0) * bs + r) * np + (J - b0) * bs + c] = s[e];
    }
  }
}

// blocks (I, J), I <= J inside each leaf, copied out of the dense factors
__global__ void k_leaf_scatter(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, int nb, int bs,
                               const int32_t* __restrict__ leaf_of, const int32_t* __restrict__ leaf_b0, int np,
                               const double* __restrict__ buf, double* __restrict__ val, double* __restrict__ norms) {
  __shared__ double red[8];
  const int I = blockIdx.x;
  if (I >= nb || leaf_of[I] < 0) return;
  const int k = leaf_of[I], b0 = leaf_b0[k];
  const double* src = buf + (size_t)k * np * np;
  for (int p = rp[I]; p < rp[I + 1]; ++p) {
    const int J = ci[p];
    double ss = 0.0;
    for (int e = threadIdx.x; e < bs * bs; e += blockDim.x) {
      int r = e / bs, c = e % bs;
      double v = src[(size_t)((I - b0) * bs + r) * np + (J - b0) * bs + c];
      val[(size_t)p * bs * bs + e] = v;
      ss = fma(v, v, ss);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
      norms[p] = sqrt(t);
    }
    __syncthreads();
  }
}

struct Node {
  int b0, bm, b1, depth;
  bool leaf;
};

static void build_tree(int b0, int b1, int depth, int bs, int leaf_size, std::vector<Node>& out) {
  const int nbs = b1 - b0;
  if ((int64_t)nbs * bs <= leaf_size || nbs == 1) {
    out.push_back({b0, b1, b1, depth, true});
    return;
  }
  const int bm = b0 + nbs / 2;
  out.push_back({b0, bm, b1, depth, false});
  build_tree(b0, bm, depth + 1, bs, leaf_size, out);
  build_tree(bm, b1, depth + 1, bs, leaf_size, out);
}

template <typename T>
static Buf<T> upload_vec(ifac_ctx* ctx, const std::vector<T>& h) {
  Buf<T> d(ctx, h.size());
  if (!h.empty())
    IFAC_CK(cudaMemcpyAsync(d.p, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, ctx->stream));
  return d;
}

// all leaves: Z_leaf = L^-T from the batched leaf routine, then truncation;
// block rows outside every leaf get no blocks
static Mat leaf_factors(ifac_ctx* ctx, const ifac_bsr& S, const std::vector<Node>& leaves, double tau) {
  const int nb = S.nb, bs = S.bs, count = (int)leaves.size();
  int nl_max = 0;
  std::vector<int32_t> leaf_of(nb, -1), leaf_b0(count);
  for (int k = 0; k < count; ++k) {
    nl_max = std::max(nl_max, (leaves[k].b1 - leaves[k].b0) * bs);
    leaf_b0[k] = leaves[k].b0;
    for (int I = leaves[k].b0; I < leaves[k].b1; ++I) leaf_of[I] = k;
  }
  const int np = ((nl_max + 31) / 32) * 32;
  Buf<int32_t> d_leaf_of = upload_vec(ctx, leaf_of), d_leaf_b0 = upload_vec(ctx, leaf_b0);
  Buf<double> buf(ctx, (size_t)count * np * np);
  int64_t tot = (int64_t)count * np * np;
  k_identity_fill<<<cdiv(tot, 256), 256, 0, ctx->stream>>>(buf.p, np, count);
  IFAC_CK_LAUNCH();
  k_leaf_gather<<<nb, 256, 0, ctx->stream>>>(S.row_ptr, S.col_idx, S.val, nb, bs, d_leaf_of.p, d_leaf_b0.p, np, buf.p);
  IFAC_CK_LAUNCH();
  Buf<int> info(ctx, count);
  leaf_invchol(ctx, count, np, buf.p, info.p);
  std::vector<int> hinfo(count);
  to_host(ctx, hinfo.data(), info.p, sizeof(int) * count);
  for (int k = 0; k < count; ++k)
    if (hinfo[k])
      fail(IFAC_ERR_NOT_SPD, "leaf " + std::to_string(k) + " (block rows " + std::to_string(leaves[k].b0) + ".." +
                                 std::to_string(leaves[k].b1 - 1) + "): pivot " + std::to_string(hinfo[k] - 1) +
                                 " not positive");
  // upper-triangular block pattern of every leaf
  std::vector<int32_t> rp(nb + 1, 0), ci;
  for (int I = 0; I < nb; ++I) {
    if (leaf_of[I] >= 0) {
      const Node& L = leaves[leaf_of[I]];
      for (int J = I; J < L.b1; ++J) ci.push_back(J);
    }
    rp[I + 1] = (int32_t)ci.size();
  }
  Mat Z = mat_alloc(ctx, S.n, bs, nb, (int64_t)ci.size());
  IFAC_CK(cudaMemcpyAsync(Z.m.row_ptr, rp.data(), sizeof(int32_t) * (nb + 1), cudaMemcpyHostToDevice, ctx->stream));
  IFAC_CK(cudaMemcpyAsync(Z.m.col_idx, ci.data(), sizeof(int32_t) * ci.size(), cudaMemcpyHostToDevice, ctx->stream));
  k_leaf_scatter<<<nb, 256, 0, ctx->stream>>>(Z.m.row_ptr, Z.m.col_idx, nb, bs, d_leaf_of.p, d_leaf_b0.p, np, buf.p,
                                              Z.m.val, Z.m.norms);
  IFAC_CK_LAUNCH();
  IFAC_CK(cudaStreamSynchronize(ctx->stream));  // host vectors rp/ci go out of scope
  return compact(ctx, std::move(Z), nullptr, tau);
}

Mat leaf_factors_ranges(ifac_ctx* ctx, const ifac_bsr& S, const std::vector<std::pair<int, int>>& ranges,
                        double tau) {
  std::vector<Node> leaves;
  for (const auto& r : ranges) leaves.push_back({r.first, r.second, r.second, 0, true});
  return leaf_factors(ctx, S, leaves, tau);
}

Mat filter_rows_active(ifac_ctx* ctx, const ifac_bsr& A, const int32_t* seg, const uint8_t* active) {
  return filter(ctx, A, seg, nullptr, active, F_ROWS_IN);
}

// per-sub-problem ||delta||_F: rows of sub-problem s are [b0_s, b1_s)
__global__ void k_node_fro(const double* __restrict__ rowsq, const int32_t* __restrict__ nb0,
                           const int32_t* __restrict__ nb1, int nnodes, double* __restrict__ out) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nnodes) return;
  double t = 0.0;
  for (int r = nb0[s]; r < nb1[s]; ++r) t += rowsq[r];
  out[s] = sqrt(t);
}

void node_fro(ifac_ctx* ctx, const ifac_bsr& A, const int32_t* nb0, const int32_t* nb1, int nn, double* out_dev) {
  Buf<double> rowsq(ctx, A.nb);
  row_sq_norms(ctx, A, rowsq.p);
  k_node_fro<<<cdiv(nn, 128), 128, 0, ctx->stream>>>(rowsq.p, nb0, nb1, nn, out_dev);
  IFAC_CK_LAUNCH();
}

// ---------------------------------------------------------------------------
// localized inverse factorization
// ---------------------------------------------------------------------------
int lif(ifac_ctx* ctx, const ifac_bsr& S_in, double tau, double target, const ifac_opts& o, ifac_bsr* Zout,
        ifac_report* rep) {
  report_init(ctx, rep, o);
  Mat S = truncate(ctx, S_in, tau);
  const int nb = S.m.nb, bs = S.m.bs;
  std::vector<Node> tree;
  // sub-problems up to rinch_rows rows (when above leaf_size) are the tree's
  // leaves and are factorized by recursive inverse Cholesky (Algorithm 1)
  const bool to_rinch = o.rinch_rows > o.leaf_size;
  build_tree(0, nb, 0, bs, to_rinch ? o.rinch_rows : o.leaf_size, tree);
  int max_depth = 0;
  std::vector<Node> leaves;
  for (const Node& n : tree) {
    max_depth = std::max(max_depth, n.depth);
    if (n.leaf) leaves.push_back(n);
  }
  Mat Z;
  if (to_rinch) {
    std::vector<std::pair<int, int>> ranges;
    for (const Node& n : leaves) ranges.push_back({n.b0, n.b1});
    int rl = 0;
    Z = rinch_ranges(ctx, S.m, ranges, tau, o.leaf_size, &rl);
  } else {
    Z = leaf_factors(ctx, S.m, leaves, tau);
  }
  int total_sweeps = 0, top_stop = 0;
  bool any_maxiter = false;
  double top_e = 0.0;

  for (int d = max_depth - 1; d >= 0; --d) {
    std::vector<Node> nodes;
    for (const Node& n : tree)
      if (!n.leaf && n.depth == d) nodes.push_back(n);
    if (nodes.empty()) continue;
    const int nn = (int)nodes.size();
    std::vector<int32_t> seg(nb, -1), mid(nn), nb0(nn), nb1(nn);
    for (int s = 0; s < nn; ++s) {
      mid[s] = nodes[s].bm;
      nb0[s] = nodes[s].b0;
      nb1[s] = nodes[s].b1;
      for (int I = nodes[s].b0; I < nodes[s].b1; ++I) seg[I] = s;
    }
    Buf<int32_t> dseg = upload_vec(ctx, seg), dmid = upload_vec(ctx, mid), dnb0 = upload_vec(ctx, nb0),
                 dnb1 = upload_vec(ctx, nb1);
    Mat Sd = filter(ctx, S.m, dseg.p, dmid.p, nullptr, F_SAME);
    Mat Bh = filter(ctx, S.m, dseg.p, dmid.p, nullptr, F_COUPLE);
    Mat Zd = filter(ctx, Z.m, dseg.p, dmid.p, nullptr, F_ROWS_IN);
    Mat Zrest = filter(ctx, Z.m, dseg.p, dmid.p, nullptr, F_ROWS_OUT);
    Z.reset();
    // delta_0 = [0 X; X^T 0], X = -Z_A^T (B Z_C)
    Mat T = gemm(ctx, Bh.m, false, Zd.m, false, 1.0, tau);
    Bh.reset();
    Mat X = gemm(ctx, Zd.m, true, T.m, false, -1.0, tau);
    T.reset();
    Mat Xt = transpose_mat(ctx, X.m);
    Mat delta = add(ctx, 1.0, X.m, 1.0, &Xt.m, 0.0);
    X.reset();
    Xt.reset();

    std::vector<double> e_prev(nn, INFINITY), e(nn, 0.0);
    std::vector<uint8_t> active(nn, 1);
    std::vector<int> sweeps(nn, 0), stop(nn, 0);
    Buf<uint8_t> dactive(ctx, nn);
    Buf<double> rowsq(ctx, nb), node_e(ctx, nn);
    for (int it = 0;; ++it) {
      Mat P = poly_P(ctx, delta.m, o.m, tau);
      Mat M = gemm(ctx, Zd.m, false, P.m, false, 1.0, tau);      // M = Z sum_{k>=1} b_k delta^k
      P.reset();
      Mat Zn = add(ctx, 1.0, Zd.m, 1.0, &M.m, 0.0);              // Z_{i+1} = Z_i + M
      Mat TS = gemm(ctx, Sd.m, false, M.m, false, 1.0, tau);     // S M
      M.reset();
      Mat U = gemm(ctx, Zn.m, true, TS.m, false, 1.0, tau);      // Z_{i+1}^T (S M)
      Mat V = gemm(ctx, TS.m, true, Zd.m, false, 1.0, tau);      // (M^T S) Z_i = (S M)^T Z_i
      TS.reset();
      Mat d1 = add(ctx, 1.0, delta.m, -1.0, &U.m, 0.0);
      U.reset();
      delta = add(ctx, 1.0, d1.m, -1.0, &V.m, 0.0);
      d1.reset();
      V.reset();
      Zd = std::move(Zn);
      // per-sub-problem norms
      row_sq_norms(ctx, delta.m, rowsq.p);
      k_node_fro<<<cdiv(nn, 128), 128, 0, ctx->stream>>>(rowsq.p, dnb0.p, dnb1.p, nn, node_e.p);
      IFAC_CK_LAUNCH();
      to_host(ctx, e.data(), node_e.p, sizeof(double) * nn);
      bool any_active = false;
      for (int s = 0; s < nn; ++s) {
        if (!active[s]) continue;
        sweeps[s]++;
        int st = 0;
        if (e[s] <= target) st = IFAC_STOP_TARGET;
        else if (e[s] > std::pow(e_prev[s], (double)(o.m + 1))) st = IFAC_STOP_RULE;
        else if (sweeps[s] >= o.max_iter) st = IFAC_STOP_MAXITER;
        if (st) {
          active[s] = 0;
          stop[s] = st;
          if (st == IFAC_STOP_MAXITER) any_maxiter = true;
        } else {
          any_active = true;
        }
        e_prev[s] = e[s];
        if (d == 0 && rep && rep->n_delta < 64) rep->delta_fro[rep->n_delta++] = e[s];
      }
      if (!any_active) break;
      // drop the rows of stopped sub-problems from delta
      IFAC_CK(cudaMemcpyAsync(dactive.p, active.data(), nn, cudaMemcpyHostToDevice, ctx->stream));
      delta = filter(ctx, delta.m, dseg.p, dmid.p, dactive.p, F_ROWS_IN);
      IFAC_CK(cudaStreamSynchronize(ctx->stream));  // `active` is reused on the host
    }
    for (int s = 0; s < nn; ++s) total_sweeps += sweeps[s];
    if (d == 0) {
      top_stop = stop[0];
      top_e = e[0];
    }
    delta.reset();
    Sd.reset();
    Z = add(ctx, 1.0, Zrest.m, 1.0, &Zd.m, 0.0);
    IFAC_CK(cudaStreamSynchronize(ctx->stream));  // host vectors of this level go out of scope
  }
  if (rep) {
    rep->sweeps = total_sweeps;
    rep->stop_reason = top_stop;
    rep->levels = max_depth;
  }
  if (any_maxiter) fail(IFAC_ERR_NO_CONVERGENCE, "a sub-problem reached max_iter sweeps");
  report_finish(ctx, rep, Z.m);
  IFAC_CK(cudaStreamSynchronize(ctx->stream));
  *Zout = Z.release();
  if (max_depth == 0) return IFAC_OK;  // a single leaf: exact up to rounding
  return (top_stop == IFAC_STOP_RULE && top_e > target) ? IFAC_WARN_TARGET_NOT_MET : IFAC_OK;
}

double resid(ifac_ctx* ctx, const ifac_bsr& S, const ifac_bsr& Z) {
  int64_t p0 = ctx->products, q0 = ctx->pairs;
  OperandCache zcache;
  Mat X = gemm(ctx, S, false, Z, false, 1.0, 0.0, IFAC_FP64, false, nullptr, &zcache);
  Mat Y = gemm(ctx, Z, true, X.m, false, 1.0, 0.0, IFAC_FP64, false, &zcache);
  X.reset();
  Mat D = add(ctx, -1.0, Y.m, 0.0, nullptr, 1.0);
  double e = fro_host(ctx, D.m);
  ctx->products = p0;
  ctx->pairs = q0;
  return e;
}

}  // namespace ifac
