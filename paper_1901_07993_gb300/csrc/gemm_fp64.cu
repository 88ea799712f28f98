// gemm_fp64.cu -- FP64 numeric phase of C = alpha op(A) op(B) (Section 5's
// block-sparse product; each block product is a dense bs x bs contraction).
//
// One CTA of 256 threads per output block C_IJ (grid-stride over the output
// pattern).  The K indices common to row I of op(A) and column J of op(B)
// are found 32 at a time by one warp (binary search of each K of the sorted
// op(A) row in the sorted op(B) column); for every matching K the two blocks
// are staged in shared memory (transposed on the way in when the operand is
// used transposed) and each thread accumulates an R x R register tile,
// R = bs/16.  Epilogue: scale by alpha, FP64 Frobenius norm by warp shuffles,
// then the block and its norm are written.  GB300 issues about two FP64 FMAs
// per clock per SM, so this kernel is bound by the FP64 pipe; staging costs
// are far below it.
#include "internal.cuh"

namespace ifac {

template <int BS>
__global__ void __launch_bounds__(256) k_gemm_fp64(
    const int32_t* __restrict__ crow, const int32_t* __restrict__ cci, int64_t cnnz,
    const int32_t* __restrict__ arp, const int32_t* __restrict__ aci, const int32_t* __restrict__ asrc, int tA,
    const double* __restrict__ aval,
    const int32_t* __restrict__ brp, const int32_t* __restrict__ bci, const int32_t* __restrict__ bsrc, int tB,
    const double* __restrict__ bval, double alpha, double* __restrict__ cval, double* __restrict__ cnorm,
    unsigned long long* __restrict__ pairs) {
  constexpr int R = BS / 16;
  extern __shared__ double smem[];
  double* As = smem;            // op(A)_IK, row-major [i][k]
  double* Bs = smem + BS * BS;  // op(B)_KJ, row-major [k][j]
  __shared__ int pa[32], pb[32];
  __shared__ int npairs;
  __shared__ double red[8];
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15, lane = tid & 31, wid = tid >> 5;
  unsigned long long mypairs = 0;

  for (int64_t p = blockIdx.x; p < cnnz; p += gridDim.x) {
    const int I = crow[p], J = cci[p];
    double acc[R][R];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int c = 0; c < R; ++c) acc[r][c] = 0.0;
    const int a0 = arp[I], a1 = arp[I + 1], b0 = brp[J], b1 = brp[J + 1];
    for (int base = a0; base < a1; base += 32) {
      if (wid == 0) {
        int q = base + lane, hit = -1;
        if (q < a1) {
          int K = aci[q], lo = b0, hi = b1;
          while (lo < hi) {
            int mid = (lo + hi) >> 1;
            if (bci[mid] < K) lo = mid + 1;
            else hi = mid;
          }
          if (lo < b1 && bci[lo] == K) hit = lo;
        }
        unsigned m = __ballot_sync(0xffffffffu, hit >= 0);
        if (hit >= 0) {
          int slot = __popc(m & ((1u << lane) - 1u));
          pa[slot] = asrc ? asrc[q] : q;
          pb[slot] = bsrc ? bsrc[hit] : hit;
        }
        if (lane == 0) npairs = __popc(m);
      }
      __syncthreads();
      const int np = npairs;
      for (int k = 0; k < np; ++k) {
        const double* ga = aval + (size_t)pa[k] * (BS * BS);
        const double* gb = bval + (size_t)pb[k] * (BS * BS);
        for (int e = tid; e < BS * BS; e += 256) {
          int r = e / BS, c = e % BS;
          double va = ga[e], vb = gb[e];
          As[tA ? c * BS + r : e] = va;
          Bs[tB ? c * BS + r : e] = vb;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < BS; ++kk) {
          double av[R], bv[R];
#pragma unroll
          for (int r = 0; r < R; ++r) av[r] = As[(ty * R + r) * BS + kk];
#pragma unroll
          for (int c = 0; c < R; ++c) bv[c] = Bs[kk * BS + tx * R + c];
#pragma unroll
          for (int r = 0; r < R; ++r)
#pragma unroll
            for (int c = 0; c < R; ++c) acc[r][c] = fma(av[r], bv[c], acc[r][c]);
        }
        __syncthreads();
      }
      mypairs += np;
      __syncthreads();  // pa/pb/npairs are rewritten by the next chunk
    }
    // epilogue: alpha, norm, store
    double ss = 0.0;
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int c = 0; c < R; ++c) {
        acc[r][c] *= alpha;
        ss = fma(acc[r][c], acc[r][c], ss);
      }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if (lane == 0) red[wid] = ss;
    double* out = cval + (size_t)p * (BS * BS);
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int c = 0; c < R; ++c) out[(ty * R + r) * BS + tx * R + c] = acc[r][c];
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < 8; ++w) t += red[w];
      cnorm[p] = sqrt(t);
    }
    __syncthreads();
  }
  // per-CTA pair count (only thread 0 tallied through npairs; every thread saw the same)
  if (tid == 0 && mypairs) atomicAdd(pairs, mypairs);
}

template <int BS>
static void launch(ifac_ctx* ctx, const View& arows, bool tA, const ifac_bsr& A, const View& bcols, bool tB,
                   const ifac_bsr& B, double alpha, ifac_bsr& C, const int32_t* crow, unsigned long long* pairs) {
  size_t smem = sizeof(double) * 2 * BS * BS;
  static std::atomic<unsigned long long> attr_set{0};
  if (first_on_device(attr_set, ctx->device))
    IFAC_CK(cudaFuncSetAttribute(k_gemm_fp64<BS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
  int per_sm = BS >= 64 ? 3 : 8;
  int64_t grid = std::min<int64_t>(C.nnzb, (int64_t)sms * per_sm);
  prof_begin(ctx, 0);
  k_gemm_fp64<BS><<<(int)grid, 256, smem, ctx->stream>>>(crow, C.col_idx, C.nnzb, arows.rp, arows.ci, arows.src,
                                                          tA ? 1 : 0, A.val, bcols.rp, bcols.ci, bcols.src,
                                                          tB ? 1 : 0, B.val, alpha, C.val, C.norms, pairs);
  IFAC_CK_LAUNCH();
  prof_end(ctx);
  ++ctx->gemm_launches;
}

void gemm_numeric_fp64(ifac_ctx* ctx, const View& arows, bool tA_blocks, const ifac_bsr& A, const View& bcols,
                       bool tB_blocks, const ifac_bsr& B, double alpha, ifac_bsr& C, const int32_t* crow,
                       unsigned long long* pairs_dev) {
  if (C.nnzb == 0) return;
  switch (A.bs) {
    case 16: launch<16>(ctx, arows, tA_blocks, A, bcols, tB_blocks, B, alpha, C, crow, pairs_dev); break;
    case 32: launch<32>(ctx, arows, tA_blocks, A, bcols, tB_blocks, B, alpha, C, crow, pairs_dev); break;
    case 64: launch<64>(ctx, arows, tA_blocks, A, bcols, tB_blocks, B, alpha, C, crow, pairs_dev); break;
    default: fail(IFAC_ERR_UNSUPPORTED, "FP64 block product built for bs in {16, 32, 64}");
  }
}

}  // namespace ifac
