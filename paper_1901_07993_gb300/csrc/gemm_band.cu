// gemm_band.cu -- TF32 / BF16 block products on narrow tiles, for block
// sizes 32, 64 and 128.
//
// A banded product (a 1D chain: a few stored blocks per block row) gives
// every output tile only a few K steps, and the wide super-tiles of
// gemm_tc.cu (up to 4 x 4 blocks of 64) then multiply mostly zero blocks.
// Here a tile is 128 x N accumulator elements: 128 / bs block rows I0.. of C
// and N / bs block columns J0.. (N = 64 for bs 32 and 64, N = 128 for bs 128),
// and its K steps are the K's at which some op(B)_KJ of its columns is stored
// (the tile plan of gemm_tc.cu).  A K block is streamed in chunks of at most
// 64 K elements, one chunk per ring stage.  The operands are K-major
// low-precision copies of op(A) and op(B) (one zero block appended to each),
// 128-byte swizzled, or 64-byte swizzled where a chunk row is 64 bytes (BF16
// at bs 32).  This kernel serves every TF32/BF16 product at bs 32 and 128, and
// the banded ones at bs 64.
//
//   warp 0      : TMA producer -- per chunk, one box per block and swizzle
//                 atom of the tile's op(A) block rows and op(B) block columns
//                 into one stage of a ring;
//   warp 1      : tensor-memory allocation and the single MMA-issuing thread
//                 (accumulate in TMEM, commit releases the stage; a double
//                 buffered accumulator lets the epilogue of one tile overlap
//                 the next tile's MMAs);
//   warps 2..17 : epilogue -- four warps per tensor-memory lane quarter,
//                 each on a quarter of the tile's columns: tcgen05.ld, alpha,
//                 block Frobenius norms (compensated FP32 sums, about 2^-42),
//                 FP64 (or, for the mixed refinement's intermediates, FP32)
//                 stores through a shared-memory transpose so that stores
//                 are row segments; one named barrier per tile.
//
// Every mbarrier wait is bounded; on expiry the CTA records the error flag and
// all its warps leave their loops together.
#include "internal.cuh"
#include "tc_common.cuh"

namespace ifac {
namespace tc {
namespace bandlp {

// epilogue warps: four per tensor-memory lane quarter, each on a quarter of
// the tile's columns.  The epilogue (tensor-memory reads, block norms, FP64
// stores) sets the pace of a banded product -- with eight warps the MMA
// thread waited two thirds of its time for a free accumulator -- so it has
// twice the warps of the MMA-bound kernels
constexpr int NEPI = 16;
constexpr int MMA_WARP = 1;
constexpr int EPI0 = 2;                 // first epilogue warp
constexpr int NTHREADS = 32 * (2 + NEPI);

template <int ELT, int BS>
struct LP {
  static constexpr int M = 128;
  static constexpr int TMB = M / BS;               // block rows per tile (4, 2, 1)
  static constexpr int N = BS < 64 ? 64 : BS;      // accumulator columns (64, 64, 128)
  static constexpr int TNB = N / BS;               // block columns per tile (2, 1, 1)
  static constexpr int KC = BS < 64 ? BS : 64;     // K elements per ring stage
  static constexpr int KCH = BS / KC;              // stages per K block
  static constexpr int ROWB = KC * ELT;            // bytes of one operand row's chunk (64, 128, 256)
  static constexpr int ATOM = ROWB < 128 ? ROWB : 128;  // swizzle atom row: 64 or 128 bytes
  static constexpr int ATOMS = ROWB / ATOM;        // atom columns per chunk
  static constexpr int ATOM_ELEMS = ATOM / ELT;
  static constexpr int A_ATOM = M * ATOM;          // one atom column of the op(A) tile
  static constexpr int B_ATOM = N * ATOM;
  static constexpr int A_BYTES = ATOMS * A_ATOM;
  static constexpr int B_BYTES = ATOMS * B_ATOM;
  static constexpr int STAGE = A_BYTES + B_BYTES;  // a multiple of 1024
  static constexpr int STAGES = (196608 / STAGE) < 8 ? (196608 / STAGE) : 8;
  static constexpr int SMEM = STAGES * STAGE + 1024;
  static constexpr int KSTEPS = ROWB / 32;         // MMAs of 32 bytes of K per chunk
  static constexpr uint32_t SBO = 8 * ATOM;        // 8-row group stride of the swizzled layout
  static constexpr uint32_t SWZ = ATOM == 128 ? 2 : 4;  // descriptor layout: 128- / 64-byte swizzle
  static constexpr uint32_t IDESC = idesc_of<ELT, N, M>();
  static constexpr uint32_t TMEM_COLS = 2 * N;     // double-buffered FP32 accumulator
  static constexpr uint32_t TX = (uint32_t)STAGE;
  static constexpr int RECW = TMB + TNB;           // plan record: op(A) rows, then op(B) columns
  static_assert(STAGES >= 2, "ring too shallow");
  static_assert(STAGE % 1024 == 0, "stages must keep the swizzle alignment");
};

}  // namespace bandlp

struct BandLpArgs {
  const int32_t* tiles;     // [2t] tile row (of TMB block rows), [2t+1] tile column (of TNB block columns)
  const int* ntiles;        // device: number of tiles
  const int32_t* tile_nk;   // device: K steps of each tile
  const int32_t* rec;       // plan: per K step, copy indices of the tile's op(A)_IK and op(B)_KJ
  const int32_t* rec_off;   // first record of each tile
  const int32_t* cpos;      // per tile, the C positions of its TMB x TNB blocks (-1: not in C)
  double* cval;
  float* cval32;  // non-null: C's values as FP32 (the accumulators exactly) in place of cval
  double* cnorm;
  int nb;
  double alpha;
  int* err;
};

template <int ELT, int BS>
__global__ void __launch_bounds__(bandlp::NTHREADS, 1)
    k_gemm_band_lp(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                   BandLpArgs args) {
  using namespace bandlp;
  using L = LP<ELT, BS>;
  constexpr int N = L::N, TMB = L::TMB, TNB = L::TNB;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[L::STAGES], empty_bar[L::STAGES];
  __shared__ __align__(8) uint64_t acc_full[2], acc_empty[2], drain_bar;
  __shared__ uint32_t tmem_base_slot;
  __shared__ volatile int abort_flag;
  __shared__ double partial[2][4][4];       // per tile parity: lane quarter x column quarter
  __shared__ float ep_stage[NEPI][32 * 9];  // 32 rows x 8 columns per warp
  __shared__ int32_t srec[32 * L::RECW];  // the producer's current chunk of plan records

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
                 "r"(L::TMEM_COLS));
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
    // the warp loads the next chunk of plan records while lane 0 issues the
    // copies of the current one
    int stage = 0;
    uint32_t phase = 0;
    uint32_t issued_mask = 0, last_parity = 0;  // stages filled / parity of their last fill
    bool ok = true;
    RecStream<L::RECW> rs;
    rs.init(args.rec, args.rec_off, args.tile_nk, (int)blockIdx.x, (int)gridDim.x, mt, 1);
    int32_t cur[L::RECW], nxt[L::RECW];
    int c_it, c_rep, c_j0, c_cnt, n_it, n_rep, n_j0, n_cnt;
    bool have = rs.next(lane, cur, c_it, c_rep, c_j0, c_cnt);
    while (have && ok) {
      if (lane < c_cnt) {
#pragma unroll
        for (int w = 0; w < L::RECW; ++w) srec[lane * L::RECW + w] = cur[w];
      }
      __syncwarp();
      const bool nhave = rs.next(lane, nxt, n_it, n_rep, n_j0, n_cnt);
      if (lane == 0) {
        for (int j = 0; j < c_cnt && ok; ++j) {
          const int32_t* r = srec + j * L::RECW;
          for (int c = 0; c < L::KCH; ++c) {
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
              const int x = c * L::KC + a * L::ATOM_ELEMS;
#pragma unroll
              for (int i = 0; i < TMB; ++i) tma_load_2d(sa + a * L::A_ATOM + i * BS * L::ATOM, &mapA, x, r[i] * BS, fb);
#pragma unroll
              for (int jb = 0; jb < TNB; ++jb)
                tma_load_2d(sb + a * L::B_ATOM + jb * BS * L::ATOM, &mapB, x, r[TMB + jb] * BS, fb);
            }
            if (++stage == L::STAGES) {
              stage = 0;
              phase ^= 1u;
            }
          }
        }
      }
      ok = __shfl_sync(0xffffffffu, ok, 0);
      __syncwarp();  // srec is rewritten next round
#pragma unroll
      for (int w = 0; w < L::RECW; ++w) cur[w] = nxt[w];
      c_it = n_it;
      c_rep = n_rep;
      c_j0 = n_j0;
      c_cnt = n_cnt;
      have = nhave;
    }
    // before the CTA exits: the copies issued have landed and the MMAs have
    // released every stage
    if (lane == 0)
      for (int s = 0; s < L::STAGES; ++s)
        if (issued_mask & (1u << s)) {
          mbar_wait(smem_u32(&full_bar[s]), (last_parity >> s) & 1u, &abort_flag, args.err, false);
          mbar_wait(smem_u32(&empty_bar[s]), (last_parity >> s) & 1u, &abort_flag, args.err, false);
        }
  } else if (warp == MMA_WARP) {
    // ------------------------------ MMA issuer ------------------------------
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      int nk_next = mt > 0 ? args.tile_nk[blockIdx.x] : 0;  // loaded a tile ahead
      for (int it = 0; it < mt && ok; ++it) {
        const int t = (int)blockIdx.x + it * (int)gridDim.x;
        const int nk = nk_next;
        if (it + 1 < mt) nk_next = args.tile_nk[t + (int)gridDim.x];
        const int ab = it & 1;
        const uint32_t aphase = (uint32_t)(it >> 1) & 1u;
        const uint32_t tacc = tmem + (uint32_t)(ab * N);
        if (!mbar_wait(smem_u32(&acc_empty[ab]), aphase ^ 1u, &abort_flag, args.err)) break;
        tc_fence_after();
        for (int j = 0; j < nk * L::KCH; ++j) {
          if (!mbar_wait(smem_u32(&full_bar[stage]), phase, &abort_flag, args.err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = smem_base + (uint32_t)(stage * L::STAGE);
          const uint32_t sb = sa + L::A_BYTES;
#pragma unroll
          for (int kk = 0; kk < L::KSTEPS; ++kk) {
            const int atom = (kk * 32) / L::ATOM, off = (kk * 32) % L::ATOM;
            mma_kstep<ELT>(tacc, smem_desc_sw(sa + atom * L::A_ATOM + off, L::SBO, L::SWZ),
                           smem_desc_sw(sb + atom * L::B_ATOM + off, L::SBO, L::SWZ), L::IDESC,
                           (j > 0 || kk > 0) ? 1u : 0u);
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
    constexpr int CW = N / 4;                // columns per warp (16, or 32 at N = 128)
    const int ew = warp - EPI0;              // 0 .. NEPI - 1
    const int q = warp & 3;                  // tensor-memory lane quarter of this warp
    const int cg = ew >> 2;                  // columns CW cg .. CW cg + CW - 1 of the tile
    const int rb = (q * 32) / BS;            // block row of the tile (a warp's rows lie in one)
    const int rin = (q * 32) % BS;           // first row of the warp within that block
    const int cb = (cg * CW) / BS;           // block column (a warp's columns lie in one)
    const int et = threadIdx.x - 32 * EPI0;  // 0 .. 32 NEPI - 1
    const float alpha_f = (float)args.alpha;
    // C positions of this warp's block and (threads et < TMB TNB) of the block
    // whose norm it writes, loaded a tile ahead
    constexpr int CP = TMB * TNB;
    int p_next = -1, kn_next = -1;
    if (mt > 0) {
      p_next = args.cpos[(size_t)blockIdx.x * CP + rb * TNB + cb];
      if (et < CP) kn_next = args.cpos[(size_t)blockIdx.x * CP + et];
    }
    for (int it = 0; it < mt; ++it) {
      const int t = (int)blockIdx.x + it * (int)gridDim.x;
      const int ab = it & 1;
      const uint32_t aphase = (uint32_t)(it >> 1) & 1u;
      const int p = p_next;  // position of this warp's block of C (-1: not in C)
      const int kn = kn_next;
      if (it + 1 < mt) {
        const size_t tn = (size_t)(t + (int)gridDim.x) * CP;
        p_next = args.cpos[tn + rb * TNB + cb];
        if (et < CP) kn_next = args.cpos[tn + et];
      }
      // a wait that failed is voted on after the tile (its reads of tensor
      // memory are harmless; the call returns the error)
      const bool got = mbar_wait(smem_u32(&acc_full[ab]), aphase, &abort_flag, args.err);
      tc_fence_after();
      SqAcc sq;
#pragma unroll 1
      for (int ch = 0; ch < CW / 8; ++ch) {
        const int col0 = cg * CW + ch * 8;  // tile column of this chunk
        float v[8];
        tmem_ld8(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(ab * N + col0), v);
        if (p >= 0) {  // warp-uniform
#pragma unroll
          for (int e = 0; e < 8; ++e) v[e] *= alpha_f;
          sq.add<8>(v);
          // 32 rows x 8 columns through shared memory, so that each store
          // instruction writes eight 64-byte row segments, two values per lane
          float* sw = ep_stage[ew];
          const size_t boff = (size_t)p * BS * BS + (size_t)rin * BS + (col0 % BS);
          const int c2 = (lane & 3) * 2, r8 = lane >> 2;
#pragma unroll
          for (int e = 0; e < 8; ++e) sw[lane * 9 + e] = v[e];
          __syncwarp();
          if (args.cval32) {  // kernel-uniform: FP32 values, eight 32-byte row segments per store
            float* blk = args.cval32 + boff;
#pragma unroll
            for (int k = 0; k < 32; k += 8) {
              const float* qv = sw + (k + r8) * 9 + c2;
              *reinterpret_cast<float2*>(blk + (size_t)(k + r8) * BS + c2) = make_float2(qv[0], qv[1]);
            }
          } else {
            double* blk = args.cval + boff;
#pragma unroll
            for (int k = 0; k < 32; k += 8) {
              const float* qv = sw + (k + r8) * 9 + c2;
              *reinterpret_cast<double2*>(blk + (size_t)(k + r8) * BS + c2) =
                  make_double2(f32_to_f64(qv[0]), f32_to_f64(qv[1]));
            }
          }
          __syncwarp();
        }
      }
      const double ss = sq.warp_total();
      if (lane == 0) partial[ab][q][cg] = ss;
      tc_fence_before();
      // one barrier per tile: every warp has read the accumulator and written
      // its partial norm (the partials alternate between two buffers, so the
      // next tile's writes cannot meet this tile's reads)
      if (!epi_all<32 * NEPI>(got)) break;  // all epilogue warps go on, or all stop
      if (et == 0) mbar_arrive(smem_u32(&acc_empty[ab]));
      // norms: block (br, bc) of the tile sums the warps of its lane quarters
      // and column quarters, in a fixed order
      if (et < CP && kn >= 0) {
        const int br = et / TNB, bc = et % TNB;
        // the lane quarters qq with (32 qq) / BS == br and column quarters cc
        // with (CW cc) / BS == bc, in increasing order
        const int q1 = (br + 1) * BS / 32 < 4 ? (br + 1) * BS / 32 : 4;
        const int c1 = (bc + 1) * BS / CW < 4 ? (bc + 1) * BS / CW : 4;
        double sum = 0.0;
        for (int qq = br * BS / 32; qq < q1; ++qq)
          for (int cc = bc * BS / CW; cc < c1; ++cc) sum += partial[ab][qq][cc];
        args.cnorm[kn] = sqrt(sum);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == MMA_WARP) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(L::TMEM_COLS));
  }
}

template <int ELT, int BS>
void launch_band_lp(ifac_ctx* ctx, const CUtensorMap& mapA, const CUtensorMap& mapB, const BandLpArgs& args,
                    int tiles_bound) {
  using L = bandlp::LP<ELT, BS>;
  static std::atomic<unsigned long long> attr{0};
  if (first_on_device(attr, ctx->device))
    IFAC_CK(cudaFuncSetAttribute(k_gemm_band_lp<ELT, BS>, cudaFuncAttributeMaxDynamicSharedMemorySize, L::SMEM));
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
  const int grid = (int)std::min<int64_t>(std::max(tiles_bound, 1), sms);
  k_gemm_band_lp<ELT, BS><<<grid, bandlp::NTHREADS, L::SMEM, ctx->stream>>>(mapA, mapB, args);
  IFAC_CK_LAUNCH();
}

template <typename L>
static void shape_of(BandShape* s) {
  s->tmb = L::TMB;
  s->tnb = L::TNB;
  s->atom_elems = L::ATOM_ELEMS;
  s->atom_bytes = L::ATOM;
}

}  // namespace tc

// the host entry used by gemm_tc.cu's dispatcher
void band_lp_product(ifac_ctx* ctx, int elt, int bs, const void* mapA, const void* mapB, const int32_t* tiles,
                     const int* ntiles, const int32_t* tile_nk, const int32_t* rec, const int32_t* rec_off,
                     const int32_t* cpos, int tiles_bound, double alpha, ifac_bsr& C, bool out32) {
  tc::BandLpArgs a{};
  a.tiles = tiles;
  a.ntiles = ntiles;
  a.tile_nk = tile_nk;
  a.rec = rec;
  a.rec_off = rec_off;
  a.cpos = cpos;
  a.cval = out32 ? nullptr : C.val;
  a.cval32 = out32 ? reinterpret_cast<float*>(C.val) : nullptr;
  a.cnorm = C.norms;
  a.nb = C.nb;
  a.alpha = alpha;
  a.err = ctx->dev_err;
  const CUtensorMap& mA = *static_cast<const CUtensorMap*>(mapA);
  const CUtensorMap& mB = *static_cast<const CUtensorMap*>(mapB);
  if (elt == 2) {
    if (bs == 32) tc::launch_band_lp<2, 32>(ctx, mA, mB, a, tiles_bound);
    else if (bs == 64) tc::launch_band_lp<2, 64>(ctx, mA, mB, a, tiles_bound);
    else if (bs == 128) tc::launch_band_lp<2, 128>(ctx, mA, mB, a, tiles_bound);
    else fail(IFAC_ERR_UNSUPPORTED, "tensor-core products: bs 32, 64 or 128");
  } else {
    if (bs == 32) tc::launch_band_lp<4, 32>(ctx, mA, mB, a, tiles_bound);
    else if (bs == 64) tc::launch_band_lp<4, 64>(ctx, mA, mB, a, tiles_bound);
    else if (bs == 128) tc::launch_band_lp<4, 128>(ctx, mA, mB, a, tiles_bound);
    else fail(IFAC_ERR_UNSUPPORTED, "tensor-core products: bs 32, 64 or 128");
  }
}

BandShape band_lp_shape(int elt, int bs) {
  BandShape s{};
  if (elt == 2) {
    if (bs == 32) tc::shape_of<tc::bandlp::LP<2, 32>>(&s);
    else if (bs == 64) tc::shape_of<tc::bandlp::LP<2, 64>>(&s);
    else if (bs == 128) tc::shape_of<tc::bandlp::LP<2, 128>>(&s);
    else fail(IFAC_ERR_UNSUPPORTED, "tensor-core products: bs 32, 64 or 128");
  } else {
    if (bs == 32) tc::shape_of<tc::bandlp::LP<4, 32>>(&s);
    else if (bs == 64) tc::shape_of<tc::bandlp::LP<4, 64>>(&s);
    else if (bs == 128) tc::shape_of<tc::bandlp::LP<4, 128>>(&s);
    else fail(IFAC_ERR_UNSUPPORTED, "tensor-core products: bs 32, 64 or 128");
  }
  return s;
}

}  // namespace ifac
