// gemm_band.cu -- TF32 / BF16 block products of banded patterns on narrow
// tiles.
//
// A banded product (a 1D chain: a few stored blocks per block row) gives
// every output tile only a few K steps, and the wide super-tiles of
// gemm_tc.cu (up to 4 x 4 blocks) then multiply mostly zero blocks.  Here a
// tile is 128 x 64: two block rows I0, I0 + 1 of C and one block column J;
// its K steps are the K's at which op(B)_KJ is stored (the 2 x 1 tile plan).
// The operands are the low-precision K-major copies gemm_tc.cu makes (one
// zero block appended to each):
//
//   warp 0      : TMA producer -- per K step, op(A)_{I0,K}, op(A)_{I0+1,K}
//                 and op(B)_{K,J} (64-row boxes, one per 128-byte atom,
//                 128-byte swizzle) into one stage of a ring;
//   warp 1      : tensor-memory allocation and the single MMA-issuing thread
//                 (accumulate in TMEM, commit releases the stage; a double
//                 buffered accumulator lets the epilogue of one tile overlap
//                 the next tile's MMAs);
//   warps 2..9  : epilogue -- tcgen05.ld, alpha, block Frobenius norms
//                 (compensated FP32 sums, about 2^-42), FP64 stores through a
//                 shared-memory transpose so that stores are row segments.
//
// The inputs are the same rounded copies as the super-tile kernel's, so the
// results are the same products.  Every mbarrier wait is bounded; on expiry
// the CTA records the error flag and returns.
#include "internal.cuh"
#include "tc_common.cuh"

namespace ifac {
namespace tc {
namespace bandlp {

constexpr int BS = 64;
constexpr int TMB = 2;                  // block rows per tile
constexpr int M = TMB * BS;             // 128 accumulator rows
constexpr int N = BS;                   // 64 accumulator columns
constexpr int NEPI = 8;                 // epilogue warps: two per tensor-memory lane quarter
constexpr int MMA_WARP = 1;
constexpr int EPI0 = 2;                 // first epilogue warp
constexpr int NTHREADS = 32 * (2 + NEPI);
constexpr uint32_t TMEM_COLS = 2 * N;   // double-buffered FP32 accumulator

template <int ELT>
struct LP {
  static constexpr int ATOMS = BS * ELT / 128;  // 128-byte atoms along K per block (TF32 2, BF16 1)
  static constexpr int A_ATOM = M * 128;        // one atom column of the A tile
  static constexpr int B_ATOM = N * 128;
  static constexpr int A_BYTES = ATOMS * A_ATOM;
  static constexpr int B_BYTES = ATOMS * B_ATOM;
  static constexpr int STAGE = A_BYTES + B_BYTES;  // TF32 48 KB, BF16 24 KB (multiples of 1024)
  static constexpr int STAGES = (ELT == 4) ? 4 : 8;
  static constexpr int ATOM_ELEMS = 128 / ELT;
  static constexpr uint32_t TX = (uint32_t)STAGE;
  static constexpr int SMEM = STAGES * STAGE + 1024;
  static constexpr int KSTEPS = BS * ELT / 32;     // MMAs of 32 bytes of K per block
  static constexpr uint32_t IDESC = idesc_of<ELT, N, M>();
};

}  // namespace bandlp

struct BandLpArgs {
  const int32_t* tiles;     // [2t] pair of block rows, [2t+1] block column
  const int* ntiles;        // device: number of tiles
  const int32_t* tile_nk;   // device: K steps of each tile
  const int32_t* rec;       // plan: per K step, copy indices of op(A)_{I0,K}, op(A)_{I0+1,K}, op(B)_{K,J}
  const int32_t* rec_off;   // first record of each tile
  const int32_t* crp;       // C pattern
  const int32_t* cci;
  double* cval;
  double* cnorm;
  int nb;
  double alpha;
  int* err;
};

template <int ELT>
__global__ void __launch_bounds__(bandlp::NTHREADS, 1) k_gemm_band_lp(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, BandLpArgs args) {
  using namespace bandlp;
  using L = LP<ELT>;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[L::STAGES], empty_bar[L::STAGES];
  __shared__ __align__(8) uint64_t acc_full[2], acc_empty[2], drain_bar;
  __shared__ uint32_t tmem_base_slot;
  __shared__ volatile int abort_flag;
  __shared__ double partial[4][2];
  __shared__ float ep_stage[NEPI][32 * 17];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t smem_base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const int ntiles = *args.ntiles;
  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < L::STAGES; ++s) {
      mbar_init(smem_u32(&full_bar[s]), 1);   // the producer's expect_tx; the copies complete it
      mbar_init(smem_u32(&empty_bar[s]), 1);  // released by the MMAs' commit
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&acc_full[b]), 1);
      mbar_init(smem_u32(&acc_empty[b]), 1);
    }
    mbar_init(smem_u32(&drain_bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_slot;
  // this CTA's tiles: blockIdx.x, blockIdx.x + gridDim.x, ...
  const int mt = ntiles > (int)blockIdx.x ? (ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;

  if (warp == 0) {
    // ------------------------------ TMA producer ------------------------------
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      uint32_t issued_mask = 0, last_parity = 0;  // stages filled / parity of their last fill
      bool ok = true;
      for (int it = 0; it < mt && ok; ++it) {
        const int t = (int)blockIdx.x + it * (int)gridDim.x;
        const int nk = args.tile_nk[t];
        const int32_t* r = args.rec + (size_t)args.rec_off[t] * 3;
        for (int j = 0; j < nk; ++j, r += 3) {
          if (!mbar_wait(smem_u32(&empty_bar[stage]), phase ^ 1u, &abort_flag, args.err)) {
            ok = false;
            break;
          }
          const uint32_t fb = smem_u32(&full_bar[stage]);
          mbar_expect_tx(fb, L::TX);
          issued_mask |= 1u << stage;
          last_parity = (last_parity & ~(1u << stage)) | (phase << stage);
          const uint32_t sa = smem_base + (uint32_t)(stage * L::STAGE);
          const uint32_t sb = sa + L::A_BYTES;
#pragma unroll
          for (int a = 0; a < L::ATOMS; ++a) {
            tma_load_2d(sa + a * L::A_ATOM, &mapA, a * L::ATOM_ELEMS, r[0] * BS, fb);
            tma_load_2d(sa + a * L::A_ATOM + BS * 128, &mapA, a * L::ATOM_ELEMS, r[1] * BS, fb);
            tma_load_2d(sb + a * L::B_ATOM, &mapB, a * L::ATOM_ELEMS, r[2] * BS, fb);
          }
          if (++stage == L::STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      // before the CTA exits: the copies issued have landed and the MMAs have
      // released every stage
      for (int s = 0; s < L::STAGES; ++s)
        if (issued_mask & (1u << s)) {
          mbar_wait(smem_u32(&full_bar[s]), (last_parity >> s) & 1u, &abort_flag, args.err, false);
          mbar_wait(smem_u32(&empty_bar[s]), (last_parity >> s) & 1u, &abort_flag, args.err, false);
        }
    }
  } else if (warp == MMA_WARP) {
    // ------------------------------ MMA issuer ------------------------------
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int it = 0; it < mt && ok; ++it) {
        const int t = (int)blockIdx.x + it * (int)gridDim.x;
        const int nk = args.tile_nk[t];
        const int ab = it & 1;
        const uint32_t aphase = (uint32_t)(it >> 1) & 1u;
        const uint32_t tacc = tmem + (uint32_t)(ab * N);
        if (!mbar_wait(smem_u32(&acc_empty[ab]), aphase ^ 1u, &abort_flag, args.err)) break;
        tc_fence_after();
        for (int j = 0; j < nk; ++j) {
          if (!mbar_wait(smem_u32(&full_bar[stage]), phase, &abort_flag, args.err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = smem_base + (uint32_t)(stage * L::STAGE);
          const uint32_t sb = sa + L::A_BYTES;
#pragma unroll
          for (int kk = 0; kk < L::KSTEPS; ++kk) {
            const int atom = kk / 4, off = (kk % 4) * 32;
            mma_kstep<ELT>(tacc, smem_desc(sa + atom * L::A_ATOM + off), smem_desc(sb + atom * L::B_ATOM + off),
                           L::IDESC, (j > 0 || kk > 0) ? 1u : 0u);
          }
          mma_commit(smem_u32(&empty_bar[stage]));
          if (++stage == L::STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (!ok) break;
        mma_commit(smem_u32(&acc_full[ab]));
      }
      // every MMA this thread issued completes before tensor memory is released
      mma_commit(smem_u32(&drain_bar));
      mbar_wait(smem_u32(&drain_bar), 0, &abort_flag, args.err, false);
    }
  } else {
    // ------------------------------ epilogue ------------------------------
    const int ew = warp - EPI0;              // 0 .. NEPI - 1
    const int q = warp & 3;                  // tensor-memory lane quarter of this warp
    const int half = ew >> 2;                // columns 32 half .. 32 half + 31 of the block
    const int row = q * 32 + lane;           // accumulator row 0..127
    const int rb = row / BS;                 // block row of the tile (warp-uniform)
    const int et = threadIdx.x - 32 * EPI0;  // 0 .. 32 NEPI - 1
    const float alpha_f = (float)args.alpha;
    for (int it = 0; it < mt; ++it) {
      const int t = (int)blockIdx.x + it * (int)gridDim.x;
      const int ab = it & 1;
      const uint32_t aphase = (uint32_t)(it >> 1) & 1u;
      const int I0 = args.tiles[2 * t] * TMB, J = args.tiles[2 * t + 1];
      const int I = I0 + rb;
      int p = -1;  // position of C_IJ in C
      if (I < args.nb && J < args.nb) {
        const int lo = args.crp[I], hi = args.crp[I + 1];
        const int k = lower_bound_i32(args.cci, lo, hi, J);
        if (k < hi && args.cci[k] == J) p = k;
      }
      const bool got = mbar_wait(smem_u32(&acc_full[ab]), aphase, &abort_flag, args.err);
      if (!epi_all<32 * NEPI>(got)) break;  // all epilogue warps go on, or all stop
      tc_fence_after();
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(ab * N + half * 32), v);
      SqAcc sq;
      if (p >= 0) {  // warp-uniform
#pragma unroll
        for (int e = 0; e < 32; ++e) v[e] *= alpha_f;
        sq.add32(v);
        // 32 rows x 16 columns at a time through shared memory, so that each
        // store instruction writes two 128-byte row segments
        float* sw = ep_stage[ew];
        double* blk = args.cval + (size_t)p * BS * BS + (size_t)((q & 1) * 32) * BS + half * 32;
        const int cc = lane & 15, rr = lane >> 4;
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
#pragma unroll
          for (int e = 0; e < 16; ++e) sw[lane * 17 + e] = v[hh * 16 + e];
          __syncwarp();
#pragma unroll 4
          for (int k = 0; k < 32; k += 2)
            blk[(size_t)(k + rr) * BS + hh * 16 + cc] = f32_to_f64(sw[(k + rr) * 17 + cc]);
          __syncwarp();
        }
      }
      double ss = sq.value();
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
      if (lane == 0) partial[q][half] = ss;
      tc_fence_before();
      epi_bar<32 * NEPI>();
      // norms: block row b of the tile is covered by lane quarters 2b, 2b + 1
      if (et < TMB) {
        const int Ib = I0 + et;
        if (Ib < args.nb && J < args.nb) {
          const int lo = args.crp[Ib], hi = args.crp[Ib + 1];
          const int k = lower_bound_i32(args.cci, lo, hi, J);
          if (k < hi && args.cci[k] == J)
            args.cnorm[k] = sqrt((partial[2 * et][0] + partial[2 * et][1]) +
                                 (partial[2 * et + 1][0] + partial[2 * et + 1][1]));
        }
      }
      epi_bar<32 * NEPI>();
      if (et == 0) mbar_arrive(smem_u32(&acc_empty[ab]));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == MMA_WARP) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
  }
}

template <int ELT>
void launch_band_lp(ifac_ctx* ctx, const CUtensorMap& mapA, const CUtensorMap& mapB, const BandLpArgs& args,
                    int tiles_bound) {
  static std::atomic<unsigned long long> attr{0};
  if (first_on_device(attr, ctx->device))
    IFAC_CK(cudaFuncSetAttribute(k_gemm_band_lp<ELT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 bandlp::LP<ELT>::SMEM));
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
  const int grid = (int)std::min<int64_t>(std::max(tiles_bound, 1), sms);
  k_gemm_band_lp<ELT><<<grid, bandlp::NTHREADS, bandlp::LP<ELT>::SMEM, ctx->stream>>>(mapA, mapB, args);
  IFAC_CK_LAUNCH();
}

}  // namespace tc

// the host entry used by gemm_tc.cu's dispatcher
void band_lp_product(ifac_ctx* ctx, int elt, const void* mapA, const void* mapB, const int32_t* tiles,
                     const int* ntiles, const int32_t* tile_nk, const int32_t* rec, const int32_t* rec_off,
                     int tiles_bound, double alpha, ifac_bsr& C) {
  tc::BandLpArgs a{};
  a.tiles = tiles;
  a.ntiles = ntiles;
  a.tile_nk = tile_nk;
  a.rec = rec;
  a.rec_off = rec_off;
  a.crp = C.row_ptr;
  a.cci = C.col_idx;
  a.cval = C.val;
  a.cnorm = C.norms;
  a.nb = C.nb;
  a.alpha = alpha;
  a.err = ctx->dev_err;
  const CUtensorMap& mA = *static_cast<const CUtensorMap*>(mapA);
  const CUtensorMap& mB = *static_cast<const CUtensorMap*>(mapB);
  if (elt == 2) tc::launch_band_lp<2>(ctx, mA, mB, a, tiles_bound);
  else tc::launch_band_lp<4>(ctx, mA, mB, a, tiles_bound);
}

}  // namespace ifac
