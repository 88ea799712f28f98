// ops.cu -- block-sparse operations composed from the pattern and numeric
// kernels: the truncated product of Section 5, pattern-union sums,
// truncation, copies and transposes.
#include "internal.cuh"

namespace ifac {

// C = alpha op(A) op(B), then removal of blocks with norm < tau.
//   rows of op(A): A's own rows, or the rows of A^T (blocks then used transposed)
//   columns of op(B): rows of B^T when B is used as is, or B's rows when B^T
//   upper: only the blocks (I, J) with J >= I are formed (a product known to
//   be symmetric, completed by sym_sum)
//   acache: converted copies of op(A) kept across calls (tensor-core products)
//   bcache: receives op(B)'s converted copies when op(B) = B (tensor-core
//   products), for a following product with op(A) = B^T
//   bpre: op(B)'s low-precision copy written by B's producer (poly2_operand);
//   B then needs no values
//   nocopy: truncation leaves the kept blocks in place (the result's vmap)
//   avmap / bvmap: value maps of A / B (tensor-core and split products)
//   out32: a TF32/BF16 product truncated with nocopy keeps its values in FP32
//   (the accumulators exactly; Mat::f32); b32: B's values are FP32
Mat gemm(ifac_ctx* ctx, const ifac_bsr& A, bool tA, const ifac_bsr& B, bool tB, double alpha, double tau,
         int prec, bool upper, OperandCache* acache, OperandCache* bcache, const OperandCache* bpre, bool nocopy,
         const int32_t* avmap, const int32_t* bvmap, bool out32, bool b32) {
  const int nb = A.nb;
  if (prec == IFAC_FP64 && ctx->fp64_prec == IFAC_FP64_SPLIT && (A.bs == 32 || A.bs == 64 || A.bs == 128))
    prec = IFAC_FP64_SPLIT;
  if ((avmap || bvmap) && prec == IFAC_FP64) fail(IFAC_ERR_INVALID, "FP64 products take no value maps");
  const bool lowp = prec == IFAC_TF32 || prec == IFAC_BF16;
  if (b32 && !lowp) fail(IFAC_ERR_INVALID, "FP32 operand values: TF32/BF16 products only");
  out32 = out32 && lowp && nocopy;  // compaction copies would move FP64 values
  View arows = view_rows(ctx, A, tA);
  Pattern P = product_pattern(ctx, arows, B, tB, nb, upper);
  Mat C(ctx);
  C.m.n = A.n;
  C.m.bs = A.bs;
  C.m.nb = nb;
  C.m.nnzb = P.nnzb;
  C.m.row_ptr = P.rp.release();
  C.m.col_idx = P.ci.release();
  const size_t vbytes = out32 ? sizeof(float) : sizeof(double);
  C.m.val = static_cast<double*>(dalloc(ctx, vbytes * (size_t)(P.nnzb ? P.nnzb : 1) * A.bs * A.bs));
  C.m.norms = static_cast<double*>(dalloc(ctx, sizeof(double) * (P.nnzb ? P.nnzb : 1)));
  C.f32 = out32;
  // algorithmic bytes of the product launch: each operand block read once at
  // the width the kernel reads it, each result block written once
  {
    const double blk = (double)A.bs * A.bs;
    const double ab = (double)(A.nnzb + B.nnzb) * blk, cb = (double)P.nnzb * blk * (double)vbytes;
    if (prec == IFAC_FP64) ctx->bytes_fp64 += ab * 8.0 + cb;
    else if (prec == IFAC_FP64_SPLIT) ctx->bytes_split += ab * 2.0 * ctx->split_slices + cb;
    else ctx->bytes_tc += ab * (prec == IFAC_BF16 ? 2.0 : 4.0) + cb;
  }
  // multiplied block pairs accumulate in the context's device counters
  if (prec == IFAC_FP64) {
    View bcols = view_rows(ctx, B, !tB);
    gemm_numeric_fp64(ctx, arows, tA, A, bcols, tB, B, alpha, C.m, P.row.p, ctx->dev_pairs);
  } else {
    View brows = view_rows(ctx, B, tB);
    gemm_numeric_tc(ctx, prec, arows, tA, A, brows, tB, B, alpha, C.m, P.row.p, upper,
                    ctx->dev_pairs + (prec == IFAC_FP64_SPLIT ? 2 : 1), acache, bcache, bpre, avmap, bvmap, out32,
                    b32);
  }
  Mat R = compact(ctx, std::move(C), P.row.p, tau, nocopy);
  R.f32 = out32;
  ctx->products += 1;
  return R;
}

// the low-precision copy of a sum's result (op(A) layout, one zero block appended)
static void* lp_copy_alloc(ifac_ctx* ctx, const ifac_bsr& C, int lp_prec, OperandCache* lpc, int* elt) {
  *elt = 0;
  if (!lpc || (lp_prec != IFAC_TF32 && lp_prec != IFAC_BF16)) return nullptr;
  *elt = lp_prec == IFAC_BF16 ? 2 : 4;
  const size_t bb = (size_t)C.bs * C.bs * (*elt);
  lpc->reset();
  lpc->conv = Buf<uint8_t>(ctx, (size_t)(C.nnzb + 1) * bb);
  lpc->conv_elt = *elt;
  IFAC_CK(cudaMemsetAsync(lpc->conv.p + (size_t)C.nnzb * bb, 0, bb, ctx->stream));
  return lpc->conv.p;
}

Mat sym_sum(ifac_ctx* ctx, double alpha, const ifac_bsr& U, double beta, const ifac_bsr* B, double gamma,
            const int32_t* umap, bool mirror, int lp_prec, OperandCache* lpc, bool u32) {
  Pattern P = sym_pattern(ctx, U, B, gamma != 0.0);
  Mat C(ctx);
  C.m.n = U.n;
  C.m.bs = U.bs;
  C.m.nb = U.nb;
  C.m.nnzb = P.nnzb;
  C.m.row_ptr = P.rp.release();
  C.m.col_idx = P.ci.release();
  C.m.val = static_cast<double*>(dalloc(ctx, sizeof(double) * (size_t)(P.nnzb ? P.nnzb : 1) * U.bs * U.bs));
  C.m.norms = static_cast<double*>(dalloc(ctx, sizeof(double) * (P.nnzb ? P.nnzb : 1)));
  int elt = 0;
  void* lp = lp_copy_alloc(ctx, C.m, lp_prec, lpc, &elt);
  sym_numeric(ctx, alpha, U, beta, B, gamma, C.m, P.row.p, umap, mirror, lp, elt, u32);
  if (lp && mirror) {
    lpc->tpos = Buf<int32_t>(ctx, (size_t)(C.m.nnzb ? C.m.nnzb : 1));
    transposed_positions(ctx, C.m, P.row.p, lpc->tpos.p);
  }
  return C;
}

Mat poly2_operand(ifac_ctx* ctx, const ifac_bsr& U, const ifac_bsr& D, double b1, double b2, int prec,
                  OperandCache* pc, const int32_t* umap, bool u32) {
  Pattern Pp = sym_pattern(ctx, U, &D, false);
  Mat P(ctx);
  P.m.n = U.n;
  P.m.bs = U.bs;
  P.m.nb = U.nb;
  P.m.nnzb = Pp.nnzb;
  P.m.row_ptr = Pp.rp.release();
  P.m.col_idx = Pp.ci.release();
  const int elt = prec == IFAC_BF16 ? 2 : 4;
  pc->reset();
  pc->conv = Buf<uint8_t>(ctx, (size_t)(Pp.nnzb + 1) * U.bs * U.bs * elt);
  pc->conv_elt = elt;
  pc->b_ready = true;
  poly2_lp(ctx, elt, U, D, b1, b2, P.m, Pp.row.p, pc->conv.p, umap, u32);
  return P;
}

Mat add(ifac_ctx* ctx, double alpha, const ifac_bsr& A, double beta, const ifac_bsr* B, double gamma,
        const int32_t* bmap, int lp_prec, OperandCache* lpc, bool b32) {
  Pattern P = union_pattern(ctx, A, B, gamma != 0.0);
  Mat C(ctx);
  C.m.n = A.n;
  C.m.bs = A.bs;
  C.m.nb = A.nb;
  C.m.nnzb = P.nnzb;
  C.m.row_ptr = P.rp.release();
  C.m.col_idx = P.ci.release();
  C.m.val = static_cast<double*>(dalloc(ctx, sizeof(double) * (size_t)(P.nnzb ? P.nnzb : 1) * A.bs * A.bs));
  C.m.norms = static_cast<double*>(dalloc(ctx, sizeof(double) * (P.nnzb ? P.nnzb : 1)));
  int elt = 0;
  void* lp = lp_copy_alloc(ctx, C.m, lp_prec, lpc, &elt);
  add_numeric(ctx, alpha, A, beta, B, gamma, C.m, P.row.p, bmap, lp, elt, b32);
  return C;
}

__global__ void k_keep_norm(const double* __restrict__ norms, int64_t n, double tau, uint8_t* __restrict__ keep) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p < n) keep[p] = (norms[p] < tau) ? 0 : 1;
}

Mat truncate(ifac_ctx* ctx, const ifac_bsr& A, double tau) {
  Buf<double> tmp;
  const double* norms = A.norms;
  if (!norms) {
    tmp = Buf<double>(ctx, A.nnzb);
    block_norms(ctx, A, tmp.p);
    norms = tmp.p;
  }
  ifac_bsr a = A;
  a.norms = const_cast<double*>(norms);
  Buf<uint8_t> keep(ctx, A.nnzb);
  if (A.nnzb) {
    k_keep_norm<<<cdiv(A.nnzb, 256), 256, 0, ctx->stream>>>(norms, A.nnzb, tau, keep.p);
    IFAC_CK_LAUNCH();
  }
  return select_blocks(ctx, a, nullptr, keep.p);
}

Mat copy_mat(ifac_ctx* ctx, const ifac_bsr& A) {
  Mat C = mat_alloc(ctx, A.n, A.bs, A.nb, A.nnzb);
  IFAC_CK(cudaMemcpyAsync(C.m.row_ptr, A.row_ptr, sizeof(int32_t) * (A.nb + 1), cudaMemcpyDeviceToDevice, ctx->stream));
  if (A.nnzb) {
    IFAC_CK(cudaMemcpyAsync(C.m.col_idx, A.col_idx, sizeof(int32_t) * A.nnzb, cudaMemcpyDeviceToDevice, ctx->stream));
    IFAC_CK(cudaMemcpyAsync(C.m.val, A.val, sizeof(double) * (size_t)A.nnzb * A.bs * A.bs, cudaMemcpyDeviceToDevice,
                            ctx->stream));
    if (A.norms)
      IFAC_CK(cudaMemcpyAsync(C.m.norms, A.norms, sizeof(double) * A.nnzb, cudaMemcpyDeviceToDevice, ctx->stream));
    else
      block_norms(ctx, C.m, C.m.norms);
  }
  return C;
}

}  // namespace ifac
