// batched.cu -- refinement from a scaled identity (Section 2.2, Eq. 2.1) of
// many independent matrices together.
//
// The members are placed on the diagonal of one block-diagonal matrix; every
// block-sparse product of a sweep then serves all members at once (a product
// of block-diagonal matrices never couples two members), so one launch
// sequence refines the whole batch.  Each member keeps its own Gershgorin
// bound, start Z_0 = c_i I, delta norm and stop test; a member that stopped
// is removed from S and delta, so it costs nothing further and its Z stays at
// the iterate its stop test returned.  With TF32/BF16 products the members
// follow the mixed-precision schedule (low-precision sweeps, then delta with
// FP64-accurate products); the final residual ||I - Z_i^T S_i Z_i||_F of
// every member is evaluated with FP64-accurate products.
#include <cmath>
#include <vector>

#include "internal.cuh"

namespace ifac {

// block-diagonal concatenation: member k occupies block rows [boff[k], boff[k+1])
__global__ void k_concat_rows(const int32_t* __restrict__ rp, int nb, int32_t boff, int32_t poff,
                              int32_t* __restrict__ rp_out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nb) rp_out[boff + i] = rp[i] + poff;
}

__global__ void k_offset_cols(const int32_t* __restrict__ ci, int64_t nnz, int32_t boff, int32_t* __restrict__ out) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p < nnz) out[p] = ci[p] + boff;
}

__global__ void k_set_last(int32_t* __restrict__ rp, int idx, int32_t v) {
  if (threadIdx.x == 0 && blockIdx.x == 0) rp[idx] = v;
}

// split member k back out: rows [b0, b1), blocks [p0, p1)
__global__ void k_slice_rows(const int32_t* __restrict__ rp, int b0, int nb, int32_t p0, int32_t* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i <= nb) out[i] = rp[b0 + i] - p0;
}

// Gershgorin bound per member: max over the member's scalar rows of the row sums
__global__ void k_seg_max(const double* __restrict__ rs, const int32_t* __restrict__ boff, int bs,
                          double* __restrict__ out) {
  __shared__ double red[32];
  const int k = blockIdx.x;
  const int64_t r0 = (int64_t)boff[k] * bs, r1 = (int64_t)boff[k + 1] * bs;
  double m = 0.0;
  for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) m = fmax(m, rs[r]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmax(t, red[w]);
    out[k] = t;
  }
}

// Z_0: diagonal blocks c_k I on the rows of member k
__global__ void k_seg_identity(const int32_t* __restrict__ seg, const double* __restrict__ c, int nb, int bs,
                               int32_t* __restrict__ rp, int32_t* __restrict__ ci, double* __restrict__ val) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t bsz = (int64_t)bs * bs;
  if (e < (int64_t)nb * bsz) {
    const int64_t b = e / bsz, k = e % bsz;
    val[e] = ((k / bs) == (k % bs)) ? c[seg[b]] : 0.0;
  }
  if (e < nb) ci[e] = (int32_t)e;
  if (e <= nb) rp[e] = (int32_t)e;
}

// Defined in drivers.cu / pattern helpers used here.
Mat filter_rows_active(ifac_ctx* ctx, const ifac_bsr& A, const int32_t* seg, const uint8_t* active);
void node_fro(ifac_ctx* ctx, const ifac_bsr& A, const int32_t* nb0, const int32_t* nb1, int nn, double* out_dev);

// the members on the diagonal of one matrix (block rows in member order)
Mat block_diag(ifac_ctx* ctx, int count, const ifac_bsr* const* Sv) {
  const int bs = Sv[0]->bs;
  std::vector<int32_t> boff(count + 1, 0);
  std::vector<int64_t> poff(count + 1, 0);
  for (int k = 0; k < count; ++k) {
    boff[k + 1] = boff[k] + Sv[k]->nb;
    poff[k + 1] = poff[k] + Sv[k]->nnzb;
  }
  const int nb = boff[count];
  if (poff[count] > 0x7fffffffLL) fail(IFAC_ERR_UNSUPPORTED, "batch holds more than 2^31-1 blocks");
  Mat Sbd = mat_alloc(ctx, (int64_t)nb * bs, bs, nb, poff[count]);
  for (int k = 0; k < count; ++k) {
    const ifac_bsr& A = *Sv[k];
    k_concat_rows<<<cdiv(A.nb, 256), 256, 0, ctx->stream>>>(A.row_ptr, A.nb, boff[k], (int32_t)poff[k],
                                                            Sbd.m.row_ptr);
    IFAC_CK_LAUNCH();
    if (A.nnzb) {
      k_offset_cols<<<cdiv(A.nnzb, 256), 256, 0, ctx->stream>>>(A.col_idx, A.nnzb, boff[k],
                                                                 Sbd.m.col_idx + poff[k]);
      IFAC_CK_LAUNCH();
      IFAC_CK(cudaMemcpyAsync(Sbd.m.val + (size_t)poff[k] * bs * bs, A.val, sizeof(double) * (size_t)A.nnzb * bs * bs,
                              cudaMemcpyDeviceToDevice, ctx->stream));
    }
  }
  k_set_last<<<1, 32, 0, ctx->stream>>>(Sbd.m.row_ptr, nb, (int32_t)poff[count]);
  IFAC_CK_LAUNCH();
  if (poff[count]) block_norms(ctx, Sbd.m, Sbd.m.norms);
  return Sbd;
}

int refine_batched(ifac_ctx* ctx, int count, const ifac_bsr* const* Sv, double tau, double target,
                   const ifac_opts& o, ifac_bsr* Zout, ifac_report* reps) {
  const int bs = Sv[0]->bs;
  std::vector<int32_t> boff(count + 1, 0);
  std::vector<int64_t> poff(count + 1, 0);
  for (int k = 0; k < count; ++k) {
    boff[k + 1] = boff[k] + Sv[k]->nb;
    poff[k + 1] = poff[k] + Sv[k]->nnzb;
  }
  const int nb = boff[count];
  if (poff[count] > 0x7fffffffLL) fail(IFAC_ERR_UNSUPPORTED, "batch holds more than 2^31-1 blocks");
  ctx->products = 0;
  ctx->launches = 0;
  ctx->gemm_launches = 0;
  ctx->tc_launches = 0;
  ctx->split_launches = 0;
  ctx->bytes_fp64 = ctx->bytes_tc = ctx->bytes_split = 0;
  ctx->events_used = 0;
  ctx->profile = o.profile != 0;
  reset_device_counters(ctx);
  // block-diagonal S
  Mat Sbd = block_diag(ctx, count, Sv);
  Mat S = truncate(ctx, Sbd.m, tau);
  Sbd.reset();
  // segments and per-member Gershgorin bounds
  std::vector<int32_t> seg(nb), nb0(count), nb1(count);
  for (int k = 0; k < count; ++k) {
    nb0[k] = boff[k];
    nb1[k] = boff[k + 1];
    for (int I = boff[k]; I < boff[k + 1]; ++I) seg[I] = k;
  }
  Buf<int32_t> dseg(ctx, nb), dnb0(ctx, count), dnb1(ctx, count), dboff(ctx, count + 1);
  IFAC_CK(cudaMemcpyAsync(dseg.p, seg.data(), sizeof(int32_t) * nb, cudaMemcpyHostToDevice, ctx->stream));
  IFAC_CK(cudaMemcpyAsync(dnb0.p, nb0.data(), sizeof(int32_t) * count, cudaMemcpyHostToDevice, ctx->stream));
  IFAC_CK(cudaMemcpyAsync(dnb1.p, nb1.data(), sizeof(int32_t) * count, cudaMemcpyHostToDevice, ctx->stream));
  IFAC_CK(cudaMemcpyAsync(dboff.p, boff.data(), sizeof(int32_t) * (count + 1), cudaMemcpyHostToDevice, ctx->stream));
  std::vector<double> beta(count), c(count);
  {
    const int64_t rows = (int64_t)nb * bs;
    Buf<double> rs(ctx, rows), db(ctx, count);
    gershgorin_rows(ctx, S.m, rs.p);
    k_seg_max<<<count, 256, 0, ctx->stream>>>(rs.p, dboff.p, bs, db.p);
    IFAC_CK_LAUNCH();
    to_host(ctx, beta.data(), db.p, sizeof(double) * count);
  }
  for (int k = 0; k < count; ++k) c[k] = (o.c_rule == 1) ? std::sqrt(2.0 / beta[k]) : 1.0 / std::sqrt(beta[k]);
  Buf<double> dc(ctx, count);
  IFAC_CK(cudaMemcpyAsync(dc.p, c.data(), sizeof(double) * count, cudaMemcpyHostToDevice, ctx->stream));
  Mat Z = mat_alloc(ctx, (int64_t)nb * bs, bs, nb, nb);
  {
    const int64_t tot = std::max<int64_t>((int64_t)nb * bs * bs, nb + 1);
    k_seg_identity<<<cdiv(tot, 256), 256, 0, ctx->stream>>>(dseg.p, dc.p, nb, bs, Z.m.row_ptr, Z.m.col_idx, Z.m.val);
    IFAC_CK_LAUNCH();
    block_norms(ctx, Z.m, Z.m.norms);
  }
  // sweeps.  Stage 0 runs every product in opts.prec.  With TF32/BF16 a
  // member whose low-precision floor is reached (the rule of Section 2.2
  // fires, or ||delta||_F stops falling) is parked at its current Z; stage 1
  // then evaluates delta of the parked members with FP64-accurate products
  // (opts.delta_prec), M staying in opts.prec, until the target or until
  // ||delta||_F stops falling -- the schedule of the single-matrix refinement.
  const bool low = o.prec != IFAC_FP64;
  const int dprec = delta_prec_of(o, bs);
  std::vector<double> e(count, 0.0), e_prev(count, INFINITY), e_pred(count, INFINITY);
  const double u = unit_roundoff(o.prec);
  std::vector<uint8_t> active(count, 1), parked(count, 0);
  std::vector<int> sweeps(count, 0), stop(count, 0), fp64_evals(count, 0), low_sweeps(count, 0);
  std::vector<std::vector<double>> hist(count);
  Buf<uint8_t> dactive(ctx, count);
  Buf<double> ne(ctx, count);
  Mat Sa = copy_mat(ctx, S.m);
  OperandCache znat;  // Z's low-precision op(A) copy for M = Z P, written with Z
  for (int stage = 0; stage < (low ? 2 : 1); ++stage) {
    if (stage == 1) {
      bool any_parked = false;
      for (int k = 0; k < count; ++k)
        if (parked[k]) {
          active[k] = 1;
          e_prev[k] = INFINITY;
          any_parked = true;
        }
      if (!any_parked) break;
      IFAC_CK(cudaMemcpyAsync(dactive.p, active.data(), count, cudaMemcpyHostToDevice, ctx->stream));
      Sa = filter_rows_active(ctx, S.m, dseg.p, dactive.p);
      IFAC_CK(cudaStreamSynchronize(ctx->stream));  // the host flags are reused below
    }
    const int pd = stage == 0 ? o.prec : dprec;
    bool all_slices = false, slices_fixed = false;
    if (stage == 1 && pd == IFAC_FP64_SPLIT) {
      // a parked member whose factor is block-dense: every evaluation of the
      // stage takes all slices (the slice rule's error estimate holds for
      // banded factors only; reading of the refinement's driver)
      std::vector<int32_t> zrp(nb + 1);
      to_host(ctx, zrp.data(), Z.m.row_ptr, sizeof(int32_t) * (nb + 1));
      for (int k = 0; k < count; ++k) {
        const int64_t m = nb1[k] - nb0[k];
        if (parked[k] && 2 * (int64_t)(zrp[nb1[k]] - zrp[nb0[k]]) > m * m) slices_fixed = true;
      }
    }
    for (int it = 0;; ++it) {
      // split evaluations take as many slices as the active member that needs
      // the most (from its last ||delta||_F)
      int ns = ctx->split_slices;
      if (pd == IFAC_FP64_SPLIT && !all_slices && !slices_fixed) {
        ns = 3;
        for (int k = 0; k < count; ++k)
          if (active[k])
            ns = std::max(ns, delta_slices(ctx, e_pred[k], target, u, (int64_t)(nb1[k] - nb0[k]) * bs));
      }
      Mat Dall;
      {
        SlicesScope scope(ctx, ns);
        // with low-precision sweeps, the upper block triangle of the
        // symmetric Z^T S Z is formed and the lower one taken from it
        const bool sym = low && bs == 64;
        OperandCache zcache;  // Z's copy (op(B) of S Z) serves again as op(A) = Z^T
        // truncated products keep their kept blocks in place where the next
        // step reads them through a value map (no compaction copies)
        // (low-precision sweeps keep X and Y's upper triangle in FP32, as
        // their products accumulated them)
        const bool inplace = pd != IFAC_FP64;
        const bool lp = (pd == IFAC_TF32 || pd == IFAC_BF16) && ctx->fp32_mid;
        Mat X = gemm(ctx, Sa.m, false, Z.m, false, 1.0, tau, pd, false, nullptr, &zcache, nullptr, inplace, nullptr,
                     nullptr, lp);  // S Z
        Mat Y = gemm(ctx, Z.m, true, X.m, false, 1.0, tau, pd, sym, &zcache, nullptr, nullptr, sym, nullptr,
                     X.map(), lp && sym, X.f32);  // Z^T (S Z)
        X.reset();
        Dall = sym ? sym_sum(ctx, -1.0, Y.m, 0.0, nullptr, 1.0, Y.map(), false, 0, nullptr, Y.f32)  // I - Z^T S Z
                   : add(ctx, -1.0, Y.m, 0.0, nullptr, 1.0);
      }
      IFAC_CK(cudaMemcpyAsync(dactive.p, active.data(), count, cudaMemcpyHostToDevice, ctx->stream));
      Mat D = filter_rows_active(ctx, Dall.m, dseg.p, dactive.p);
      Dall.reset();
      node_fro(ctx, D.m, dnb0.p, dnb1.p, count, ne.p);
      to_host(ctx, e.data(), ne.p, sizeof(double) * count);
      if (ns < ctx->split_slices) {
        // a member's delta far below its predicted size, at the target (a
        // stop must not rest on fewer slices), or stalling (the sweeps then
        // converge toward the s-slice evaluation's own error, kStallRatio):
        // evaluate again with all slices; after a stall every evaluation of
        // the stage takes all of them and the comparison restarts
        bool redo = false, stall = false;
        for (int k = 0; k < count; ++k) {
          if (!active[k]) continue;
          const bool st = stage == 1 && e[k] > kStallRatio * e_prev[k];
          stall = stall || st;
          if (split_delta_error(ns, (int64_t)(nb1[k] - nb0[k]) * bs) > delta_need(e[k], target, u) ||
              e[k] <= target || st)
            redo = true;
        }
        if (stall) {
          slices_fixed = true;
          for (int k = 0; k < count; ++k)
            if (active[k]) e_prev[k] = INFINITY;
        }
        if (redo) {
          all_slices = true;
          --it;
          continue;
        }
      }
      all_slices = false;
      for (int k = 0; k < count; ++k)  // parked members: the same Z in stage 1
        if (active[k]) e_pred[k] = stage == 0 ? 0.1 * e[k] : u * e[k];
      bool any = false;
      for (int k = 0; k < count; ++k) {
        if (!active[k]) continue;
        int st = 0;
        bool park = false;
        if (stage == 1) ++fp64_evals[k];
        if (e[k] <= target) {
          st = IFAC_STOP_TARGET;
        } else if (stage == 0) {
          if (e[k] > std::pow(e_prev[k], (double)(o.m + 1)) || (low && !(e[k] < e_prev[k]))) {
            if (low) park = true;
            else st = IFAC_STOP_RULE;
          } else if (sweeps[k] >= o.max_iter) {
            st = IFAC_STOP_MAXITER;
          }
        } else if (!(e[k] < e_prev[k])) {
          st = IFAC_STOP_RULE;  // the FP64 floor
        } else if (sweeps[k] >= o.max_iter) {
          st = IFAC_STOP_MAXITER;
        }
        if (park) {  // delta is evaluated again, with FP64-accurate products, in stage 1
          active[k] = 0;
          parked[k] = 1;
          continue;
        }
        hist[k].push_back(e[k]);
        if (st) {
          active[k] = 0;
          parked[k] = 0;
          stop[k] = st;
        } else {
          any = true;
        }
        e_prev[k] = e[k];
      }
      if (!any) break;
      IFAC_CK(cudaMemcpyAsync(dactive.p, active.data(), count, cudaMemcpyHostToDevice, ctx->stream));
      D = filter_rows_active(ctx, D.m, dseg.p, dactive.p);
      Sa = filter_rows_active(ctx, Sa.m, dseg.p, dactive.p);
      IFAC_CK(cudaStreamSynchronize(ctx->stream));  // the host flags are reused next sweep
      Mat P;
      OperandCache pcache;
      {  // P = sum_{k=1}^{m} b_k delta^k (first two terms in one sum)
        Mat Dk;
        double b = 0.5;
        if (o.m < 2) P = add(ctx, 0.5, D.m, 0.0, nullptr, 0.0);
        for (int k = 2; k <= o.m; ++k) {
          b = b * (double)(2 * k - 1) / (double)(2 * k);
          const bool sym = low && bs == 64;
          const bool fused = sym && k == 2 && o.m == 2;
          Mat Dn = gemm(ctx, k == 2 ? D.m : Dk.m, false, D.m, false, 1.0, tau, o.prec, sym, nullptr, nullptr, nullptr,
                        fused, nullptr, nullptr, fused && ctx->fp32_mid);
          if (fused) {  // delta^2 (in FP32) completed by symmetry inside the sum
            // P only as the low-precision op(B) copy that M = Z P reads
            P = poly2_operand(ctx, Dn.m, D.m, 0.5, b, o.prec, &pcache, Dn.map(), Dn.f32);
            break;
          }
          if (sym) Dn = sym_sum(ctx, 1.0, Dn.m, 0.0, nullptr, 0.0);
          Dk = std::move(Dn);
          P = (k == 2) ? add(ctx, 0.5, D.m, b, &Dk.m, 0.0) : add(ctx, 1.0, P.m, b, &Dk.m, 0.0);
        }
      }
      D.reset();
      Mat M = gemm(ctx, Z.m, false, P.m, false, 1.0, tau, o.prec, false, &znat, nullptr, &pcache, true, nullptr,
                   nullptr, ctx->fp32_mid);  // M = Z P (FP32 when low precision)
      P.reset();
      Z = add(ctx, 1.0, Z.m, 1.0, &M.m, 0.0, M.map(), o.prec, &znat, M.f32);  // with Z's copy for the next M
      for (int k = 0; k < count; ++k)
        if (active[k]) {
          ++sweeps[k];
          if (stage == 0 && low) ++low_sweeps[k];
        }
    }
  }
  // FP64 residual of every member
  std::vector<double> resid(count, 0.0);
  {
    const int rprec = delta_prec_of(o, bs);
    OperandCache zcache;
    Mat X = gemm(ctx, S.m, false, Z.m, false, 1.0, 0.0, rprec, false, nullptr, &zcache);
    Mat Y = gemm(ctx, Z.m, true, X.m, false, 1.0, 0.0, rprec, false, &zcache);
    X.reset();
    Mat D = add(ctx, -1.0, Y.m, 0.0, nullptr, 1.0);
    node_fro(ctx, D.m, dnb0.p, dnb1.p, count, ne.p);
    to_host(ctx, resid.data(), ne.p, sizeof(double) * count);
  }
  check_device_error(ctx);
  int64_t pf = 0, pt = 0;
  int64_t ps = 0, pss = 0;
  read_device_counters(ctx, &pf, &pt, &ps, &pss);
  double ms_fp64 = 0.0, ms_tc = 0.0;
  double ms_split = 0.0;
  prof_collect(ctx, &ms_fp64, &ms_tc, &ms_split);
  ctx->profile = false;
  // split Z into the members
  std::vector<int32_t> zrp(nb + 1);
  to_host(ctx, zrp.data(), Z.m.row_ptr, sizeof(int32_t) * (nb + 1));
  bool any_maxiter = false;
  std::vector<Mat> outs;
  for (int k = 0; k < count; ++k) {
    const int b0 = boff[k], nbk = boff[k + 1] - boff[k];
    const int32_t p0 = zrp[b0], p1 = zrp[boff[k + 1]];
    Mat Zk = mat_alloc(ctx, Sv[k]->n, bs, nbk, p1 - p0);
    k_slice_rows<<<cdiv(nbk + 1, 256), 256, 0, ctx->stream>>>(Z.m.row_ptr, b0, nbk, p0, Zk.m.row_ptr);
    IFAC_CK_LAUNCH();
    if (p1 > p0) {
      k_offset_cols<<<cdiv(p1 - p0, 256), 256, 0, ctx->stream>>>(Z.m.col_idx + p0, p1 - p0, -b0, Zk.m.col_idx);
      IFAC_CK_LAUNCH();
      IFAC_CK(cudaMemcpyAsync(Zk.m.val, Z.m.val + (size_t)p0 * bs * bs, sizeof(double) * (size_t)(p1 - p0) * bs * bs,
                              cudaMemcpyDeviceToDevice, ctx->stream));
      IFAC_CK(cudaMemcpyAsync(Zk.m.norms, Z.m.norms + p0, sizeof(double) * (size_t)(p1 - p0), cudaMemcpyDeviceToDevice,
                              ctx->stream));
    }
    if (stop[k] == IFAC_STOP_MAXITER) any_maxiter = true;
    if (reps) {
      ifac_report& r = reps[k];
      r = ifac_report{};
      r.sweeps = sweeps[k];
      r.stop_reason = stop[k];
      r.beta = beta[k];
      r.n_delta = (int)std::min<size_t>(hist[k].size(), 64);
      for (int i = 0; i < r.n_delta; ++i) r.delta_fro[i] = hist[k][i];
      r.nnzb_Z = p1 - p0;
      r.resid_fro = resid[k];
      r.fp64_delta_evals = fp64_evals[k];
      r.low_sweeps = low_sweeps[k];
      // batch-wide counters are reported on every member
      r.products = ctx->products;
      r.block_pairs = pf + pt + ps;
      r.fp64_pairs = pf;
      r.tc_pairs = pt;
      r.split_pairs = ps;
      r.split_slice_pairs = pss;
      r.flops = 2.0 * (double)bs * bs * bs * (double)(pf + pt + ps);
      r.launches = ctx->launches;
      r.gemm_launches = ctx->gemm_launches;
      r.tc_launches = ctx->tc_launches;
      r.gemm_ms = ms_fp64;
      r.tc_ms = ms_tc;
      r.split_launches = ctx->split_launches;
      r.split_ms = ms_split;
      r.fp64_bytes = ctx->bytes_fp64;
      r.tc_bytes = ctx->bytes_tc;
      r.split_bytes = ctx->bytes_split;
    }
    outs.push_back(std::move(Zk));
  }
  if (any_maxiter) fail(IFAC_ERR_NO_CONVERGENCE, "a batch member reached max_iter sweeps");
  IFAC_CK(cudaStreamSynchronize(ctx->stream));
  for (int k = 0; k < count; ++k) Zout[k] = outs[k].release();
  bool target_met = true;
  for (int k = 0; k < count; ++k) target_met = target_met && stop[k] == IFAC_STOP_TARGET;
  return target_met ? IFAC_OK : IFAC_WARN_TARGET_NOT_MET;
}

}  // namespace ifac
