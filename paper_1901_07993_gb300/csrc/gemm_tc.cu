// gemm_tc.cu -- tensor-core numeric phase of C = alpha op(A) op(B) for
// 64 x 64 blocks, with BF16 or TF32 inputs and FP32 accumulation in tensor
// memory (the low-precision products of the mixed-precision schedule).
//
// Operands.  op(A) and op(B) are first copied in their own CSR order to a
// low-precision array, each block stored K-major (op(A)_IK as [i][k],
// op(B)_KJ as [j][k]), so that a transposed use of an FP64 matrix costs only
// a transposed copy; one all-zero block is appended to each copy.
//
// Tiles.  The output is cut into tiles of TM x TN blocks (M = 128 rows, N =
// 256 (BF16) or 128 (TF32) columns); only tiles that hold a block of C's
// pattern are visited, by a persistent grid.  For a tile, K runs over the
// union of the stored K's of its TM op(A) block rows; a block missing inside
// the tile (op(A)_IK or op(B)_KJ not stored) is read from the zero block, so
// every K step is one dense M x N x 64 contraction.
//
// Pairs.  Two CTAs take one super-tile of 2 TM x TN blocks: each computes
// TM block rows against the same op(B) panel and walks the same K set (the
// union over the super-tile's rows), so the panel is read from HBM once and
// from L2 by the second CTA.  Each CTA loads its own copy of every tile it
// contracts (no cluster, no cross-CTA signalling).
//
// Roles (320 threads, one CTA per SM):
//   warp 0      : TMA producer -- one 64-row box per block and 128-byte
//                 atom, 128-byte swizzle, into a STAGES-deep ring;
//   warp 1      : tensor-memory allocation and the single MMA-issuing
//                 thread (tcgen05.mma, accumulate in TMEM, tcgen05.commit
//                 releases ring slots and hands the accumulator over);
//   warps 2..9  : epilogue, two warps per tensor-memory lane quarter, each
//                 on half of the tile's column blocks -- tcgen05.ld of the
//                 accumulator, alpha, Frobenius norm per output block, FP64
//                 store into C.
// Every mbarrier wait is bounded; on expiry the CTA records an error flag,
// drains its own copies and MMAs, releases tensor memory and returns.
#include <cuda.h>
#include <climits>
#include <type_traits>
#include <cuda_bf16.h>

#include "internal.cuh"
#include "tc_common.cuh"

namespace ifac {
namespace tc {

constexpr int BS = 64;
constexpr int TM = 2;
constexpr int PAIR = 2;                    // CTAs per super-tile (consecutive blockIdx.x)
constexpr int NEPI = 8;                    // epilogue warps: two per tensor-memory lane quarter
constexpr int NTHREADS = 64 + 32 * NEPI;
// split mode: K steps per exact FP32 window, table sizes
constexpr int KW = 16;
constexpr int MAX_UNITS = 16;
constexpr int MAX_PAIRS = 40;

template <int ELT>
struct Cfg {
  static constexpr int ATOM_ELEMS = 128 / ELT;          // elements in one 128-byte row
  static constexpr int ATOMS = BS / ATOM_ELEMS;         // 128-byte atoms along K per block
  static constexpr int MMA_K = 32 / ELT;                // 32 bytes of K per tcgen05.mma
  static constexpr int KSTEPS = BS / MMA_K;             // MMAs per K block
  static constexpr int TN = (ELT == 2) ? 4 : 2;         // block columns per tile
  static constexpr int N = TN * BS;
  static constexpr int M = TM * BS;
  static constexpr int A_ATOM_BYTES = M * 128;          // one K atom of the A tile
  static constexpr int B_ATOM_BYTES = N * 128;
  static constexpr int A_BYTES = ATOMS * A_ATOM_BYTES;
  static constexpr int B_BYTES = ATOMS * B_ATOM_BYTES;
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int STAGES = (ELT == 2) ? 4 : 3;
  static constexpr int TMEM_COLS = 2 * N;               // two FP32 accumulators (double buffer)
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024;
  static constexpr uint32_t TX_BYTES = (uint32_t)(TM + TN) * BS * BS * ELT;
};

template <int ELT>
__host__ __device__ constexpr uint32_t instr_desc() {
  return idesc_of<ELT, Cfg<ELT>::N, Cfg<ELT>::M>();
}

template <int ELT>
__device__ __forceinline__ void mma_issue(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  mma_kstep<ELT>(tmem_d, adesc, bdesc, instr_desc<ELT>(), accumulate);
}

__device__ __forceinline__ void epi_bar() { epi_bar<32 * NEPI>(); }

// ---------------------------------------------------------------------------
// the kernel
// ---------------------------------------------------------------------------
struct TileArgs {
  const int32_t* tiles;      // [2*t] tile row, [2*t+1] tile column
  const int* ntiles;         // device: number of tiles
  const int* tile_nk;        // device: K steps of each tile
  int nwin;                  // split mode: the largest number of K windows of a tile
  int nb;
  const int32_t* rec;        // plan: per K step, copy indices of op(A)_IK (super-tile rows) and op(B)_KJ
  const int32_t* rec_off;    // first record of each tile
  const int32_t* crp;    // C pattern
  const int32_t* cci;
  double* cval;
  float* cval32;  // TF32/BF16 products: non-null, C's values as FP32 (the
                  // accumulators exactly, half the bytes of cval) in place of cval
  double* cnorm;
  // split mode: fixed-point sums, per C block 2048 longlong2 in hand-over
  // order ((row half, column half, pair e) x 32 lanes), so that a warp's
  // read-modify-write of one register pair covers 512 contiguous bytes
  longlong2* cpart;
  double alpha;
  int* err;
  // split mode (FP64-accurate products): the copies of op(A) and op(B) hold
  // NS BF16 slices each; pair p multiplies the slices starting at rows
  // pair_ya[p] / pair_yb[p] of the tensor maps; the pairs of unit u,
  // [unit_end[u-1], unit_end[u]), share one FP32 accumulator and its weight
  // weight 2^sh_u in the 64-bit fixed-point sums that the epilogue keeps in
  // C's value array (no norms; converted after the kernel)
  int split;
  int nunits;
  int unit_end[MAX_UNITS];
  int pair_ya[MAX_PAIRS], pair_yb[MAX_PAIRS];
  int unit_sh[MAX_UNITS];
  int* ovf;  // set to 2 on a fixed-point overflow (reported as an error by the host)
  // failure-path self-test only (0 in every product): the producer and the MMA
  // issuer do no work, so the epilogue's first accumulator wait expires after
  // wait_limit polls and the kernel reports a timeout
  int stall;
  long long wait_limit;
};

template <int ELT>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, TileArgs args) {
  using C = Cfg<ELT>;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[C::STAGES], empty_bar[C::STAGES];
  __shared__ __align__(8) uint64_t acc_full[2], acc_empty[2], drain_bar;
  __shared__ uint32_t tmem_base_slot;
  __shared__ volatile int abort_flag;
  __shared__ double partial[4][C::TN];
  __shared__ int s_unit_end[MAX_UNITS], s_pair_ya[MAX_PAIRS], s_pair_yb[MAX_PAIRS];
  __shared__ int s_unit_sh[MAX_UNITS];
  __shared__ float ep_stage[NEPI][32 * 17];  // plain epilogue: per-warp transpose for coalesced stores

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long wl = args.wait_limit;
  const uint32_t smem_base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const int ntiles = *args.ntiles;
  // CTAs 2c and 2c + 1 (pair c of ncl) take one super-tile of PAIR*TM x TN
  // blocks; CTA `crank` of the pair computes block rows (super row * PAIR +
  // crank) * TM.  Both step through the same K set (the union over the
  // super-tile's rows) and load the whole op(B) panel into their own shared
  // memory.
  const int crank = (int)(blockIdx.x % PAIR);
  const int cid = (int)(blockIdx.x / PAIR), ncl = (int)(gridDim.x / PAIR);

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int u = 0; u < MAX_UNITS; ++u) {
      s_unit_end[u] = args.unit_end[u];
      s_unit_sh[u] = args.unit_sh[u];
    }
    for (int p = 0; p < MAX_PAIRS; ++p) {
      s_pair_ya[p] = args.pair_ya[p];
      s_pair_yb[p] = args.pair_yb[p];
    }
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(smem_u32(&full_bar[s]), 1);
      mbar_init(smem_u32(&empty_bar[s]), 1);  // released by this CTA's MMAs
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&acc_full[b]), 1);
      mbar_init(smem_u32(&acc_empty[b]), 1);
    }
    mbar_init(smem_u32(&drain_bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_slot)),
                 "r"((uint32_t)C::TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_slot;

  // work items: this pair's tiles (cid, cid + ncl, ...), in split mode once
  // per K window, window-major: every pair runs window w of its tiles before
  // window w + 1, so the slices of one K range are shared through L2, while a
  // tile's fixed-point sums are only ever updated by the one CTA that owns its rows
  const int mt = ntiles > cid ? (ntiles - cid + ncl - 1) / ncl : 0;
  const int nitems = mt * (args.split ? args.nwin : 1);
  auto item = [&](int j, int& t, int& kb, int& cnt) -> bool {
    t = cid + (j % mt) * ncl;
    const int nk = args.tile_nk[t];
    if (!args.split) {
      kb = 0;
      cnt = nk;
      return cnt > 0;
    }
    kb = (j / mt) * KW;
    if (kb >= nk) return false;
    cnt = min(KW, nk - kb);
    return true;
  };

  if (warp == 0) {
    // ------------------------------ TMA producer ------------------------------
    // The warp reads the tile's K-step records from the plan 32 at a time,
    // lane-parallel; lane 0 then issues the loads of each record into the next
    // ring slot.  In split mode the records come in windows of KW, and every
    // window is loaded once per slice pair, unit by unit.
    __shared__ int rec[32][TM + Cfg<ELT>::TN];
    __shared__ int wrec[KW][TM + Cfg<ELT>::TN];
    int stage = 0;
    uint32_t phase = 0;
    uint32_t issued_mask = 0, last_parity = 0;  // lane 0: stages filled / parity of their last fill
    bool ok = true;
    // lane 0: one ring slot with the blocks of record r, slices at rows ya / yb
    auto issue = [&](const int* r, int ya, int yb) -> bool {
      if (!mbar_wait(smem_u32(&empty_bar[stage]), phase ^ 1u, &abort_flag, args.err, true, wl)) return false;
      const uint32_t fb = smem_u32(&full_bar[stage]);
      mbar_expect_tx(fb, C::TX_BYTES);
      issued_mask |= 1u << stage;
      last_parity = (last_parity & ~(1u << stage)) | (phase << stage);
      const uint32_t sa = smem_base + stage * C::STAGE_BYTES;
      const uint32_t sb = sa + C::A_BYTES;
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int a = 0; a < C::ATOMS; ++a)
          tma_load_2d(sa + a * C::A_ATOM_BYTES + i * BS * 128, &mapA, a * C::ATOM_ELEMS, ya + r[i] * BS, fb);
#pragma unroll
      for (int c = 0; c < C::TN; ++c)
#pragma unroll
        for (int a = 0; a < C::ATOMS; ++a)
          tma_load_2d(sb + a * C::B_ATOM_BYTES + c * BS * 128, &mapB, a * C::ATOM_ELEMS, yb + r[TM + c] * BS, fb);
      if (++stage == C::STAGES) { stage = 0; phase ^= 1u; }
      return true;
    };
    // lane 0, split mode: the cnt records of the open window for every slice pair
    auto issue_window = [&](int cnt) -> bool {
      int p = 0;
      for (int u = 0; u < args.nunits; ++u)
        for (; p < s_unit_end[u]; ++p)
          for (int j = 0; j < cnt; ++j)
            if (!issue(wrec[j], s_pair_ya[p], s_pair_yb[p])) return false;
      return true;
    };
    constexpr int RECW = PAIR * TM + C::TN;  // plan record: op(A) rows of the super-tile, then op(B) columns
    for (int it = 0; it < nitems && ok && !args.stall; ++it) {
      int t, kb, cnt;
      if (!item(it, t, kb, cnt)) continue;
      const int32_t* base = args.rec + (size_t)(args.rec_off[t] + kb) * RECW;
      if (!args.split) {
        for (int k0 = 0; k0 < cnt && ok; k0 += 32) {
          const int n = min(32, cnt - k0);
          if (lane < n) {
            const int32_t* r = base + (size_t)(k0 + lane) * RECW;
#pragma unroll
            for (int i = 0; i < TM; ++i) rec[lane][i] = r[crank * TM + i];
#pragma unroll
            for (int c = 0; c < C::TN; ++c) rec[lane][TM + c] = r[PAIR * TM + c];
          }
          __syncwarp();
          if (lane == 0)
            for (int j = 0; j < n && ok; ++j) ok = issue(rec[j], 0, 0);
          ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
          __syncwarp();
        }
      } else {
        if (lane < cnt) {
          const int32_t* r = base + (size_t)lane * RECW;
#pragma unroll
          for (int i = 0; i < TM; ++i) wrec[lane][i] = r[crank * TM + i];
#pragma unroll
          for (int c = 0; c < C::TN; ++c) wrec[lane][TM + c] = r[PAIR * TM + c];
        }
        __syncwarp();
        if (lane == 0) ok = issue_window(cnt);
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
        __syncwarp();
      }
    }
    // before the CTA exits: the copies lane 0 issued have landed and the MMAs
    // have released every slot
    if (lane == 0)
      for (int s = 0; s < C::STAGES; ++s)
        if (issued_mask & (1u << s)) {
          mbar_wait(smem_u32(&full_bar[s]), (last_parity >> s) & 1u, &abort_flag, args.err, false, wl);
          mbar_wait(smem_u32(&empty_bar[s]), (last_parity >> s) & 1u, &abort_flag, args.err, false, wl);
        }
  } else if (warp == 1) {
    // ------------------------------ MMA issuer ------------------------------
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int tl = 0;  // accumulator hand-overs so far: buffer tl & 1, its phase (tl >> 1) & 1
      bool ok = true;
      // nsteps ring slots contracted into one accumulator, then handed to the epilogue
      auto run_acc = [&](int nsteps) -> bool {
        const int ab = tl & 1;
        const uint32_t aphase = (uint32_t)(tl >> 1) & 1u;
        const uint32_t tacc = tmem + (uint32_t)(ab * C::N);
        if (!mbar_wait(smem_u32(&acc_empty[ab]), aphase ^ 1u, &abort_flag, args.err, true, wl)) return false;
        tc_fence_after();
        for (int k = 0; k < nsteps; ++k) {
          if (!mbar_wait(smem_u32(&full_bar[stage]), phase, &abort_flag, args.err, true, wl)) return false;
          tc_fence_after();
          const uint32_t sa = smem_base + stage * C::STAGE_BYTES;
          const uint32_t sb = sa + C::A_BYTES;
#pragma unroll
          for (int kk = 0; kk < C::KSTEPS; ++kk) {
            const int atom = kk / (C::ATOM_ELEMS / C::MMA_K), off = (kk % (C::ATOM_ELEMS / C::MMA_K)) * 32;
            mma_issue<ELT>(tacc, smem_desc(sa + atom * C::A_ATOM_BYTES + off),
                           smem_desc(sb + atom * C::B_ATOM_BYTES + off), (k > 0 || kk > 0) ? 1u : 0u);
          }
          mma_commit(smem_u32(&empty_bar[stage]));
          if (++stage == C::STAGES) { stage = 0; phase ^= 1u; }
        }
        mma_commit(smem_u32(&acc_full[ab]));
        ++tl;
        return true;
      };
      for (int it = 0; it < nitems && ok && !args.stall; ++it) {
        int t, kb, cnt;
        if (!item(it, t, kb, cnt)) continue;  // (a tile holds a block of C's pattern, so nk >= 1)
        if (!args.split) {
          ok = run_acc(cnt);
        } else {
          int p = 0;
          for (int u = 0; u < args.nunits && ok; ++u) {
            ok = run_acc((s_unit_end[u] - p) * cnt);
            p = s_unit_end[u];
          }
        }
      }
      // every MMA this thread issued completes before tensor memory is released
      mma_commit(smem_u32(&drain_bar));
      mbar_wait(smem_u32(&drain_bar), 0, &abort_flag, args.err, false, wl);
    }
  } else {
    // ------------------------------ epilogue ------------------------------
    const int q = warp & 3;            // tensor-memory lane quarter of this warp
    const int c0 = ((warp - 2) >> 2) * (C::TN / 2), c1 = c0 + C::TN / 2;  // this warp's column blocks
    const int row = q * 32 + lane;     // accumulator row 0..127
    const int r_blk = row / BS;
    const int et = threadIdx.x - 64;   // 0 .. 32 NEPI - 1
    const float alpha_f = (float)args.alpha;
    int tl = 0;
    bool good = true;
    for (int it = 0; it < nitems && good; ++it) {
      int t, kb, cnt;
      if (!item(it, t, kb, cnt)) continue;
      const int I0 = (args.tiles[2 * t] * PAIR + crank) * TM, J0 = args.tiles[2 * t + 1] * C::TN;
      const int I = I0 + r_blk;  // warp-uniform: a warp's 32 rows lie in one block row
      int pc[C::TN];             // position of C_{I, J0+c} in C, or -1
#pragma unroll
      for (int c = 0; c < C::TN; ++c) {
        const int J = J0 + c;
        pc[c] = -1;
        if (I < args.nb && J < args.nb) {
          const int lo = args.crp[I], hi = args.crp[I + 1];
          const int k = lower_bound_i32(args.cci, lo, hi, J);
          if (k < hi && args.cci[k] == J) pc[c] = k;
        }
      }
      if (!args.split) {
        const int ab = tl & 1;
        const uint32_t aphase = (uint32_t)(tl >> 1) & 1u;
        ++tl;
        const bool got = mbar_wait(smem_u32(&acc_full[ab]), aphase, &abort_flag, args.err, true, wl);
        if (!epi_all<32 * NEPI>(got)) break;  // all epilogue warps go on, or all stop
        tc_fence_after();
#pragma unroll 1
        for (int c = c0; c < c1; ++c) {
          const int p = pc[c];
          SqAcc sq;  // this thread's 64 squares, accurate to about 2^-42 (FP32 pipe)
#pragma unroll
          for (int h = 0; h < BS / 32; ++h) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(ab * C::N + c * BS + h * 32), v);
            if (p >= 0) {  // warp-uniform
#pragma unroll
              for (int e = 0; e < 32; ++e) v[e] *= alpha_f;
              sq.add32(v);
              // 32 rows x 16 columns at a time through shared memory, so that
              // each store instruction writes two 128-byte row segments
              float* sw = ep_stage[warp - 2];
              const size_t boff = (size_t)p * BS * BS + (size_t)((q & 1) * 32) * BS + h * 32;
              const int cc = lane & 15, rr = lane >> 4;
#pragma unroll
              for (int half = 0; half < 2; ++half) {
#pragma unroll
                for (int e = 0; e < 16; ++e) sw[lane * 17 + e] = v[half * 16 + e];
                __syncwarp();
                if (args.cval32) {  // kernel-uniform
                  float* blk = args.cval32 + boff;
#pragma unroll 4
                  for (int k = 0; k < 32; k += 2) blk[(size_t)(k + rr) * BS + half * 16 + cc] = sw[(k + rr) * 17 + cc];
                } else {
                  double* blk = args.cval + boff;
#pragma unroll 4
                  for (int k = 0; k < 32; k += 2)
                    blk[(size_t)(k + rr) * BS + half * 16 + cc] = f32_to_f64(sw[(k + rr) * 17 + cc]);
                }
                __syncwarp();
              }
            }
          }
          const double ss = sq.warp_total();
          if (lane == 0) partial[q][c] = ss;
        }
        tc_fence_before();
        epi_bar();
        // norms: block row rb is covered by lane quarters 2rb and 2rb+1, summed in that order
        if (et < TM * C::TN) {
          const int rb = et / C::TN, c = et % C::TN;
          const int Ib = I0 + rb, J = J0 + c;
          if (Ib < args.nb && J < args.nb) {
            const int lo = args.crp[Ib], hi = args.crp[Ib + 1];
            const int k = lower_bound_i32(args.cci, lo, hi, J);
            if (k < hi && args.cci[k] == J) args.cnorm[k] = sqrt(partial[2 * rb][c] + partial[2 * rb + 1][c]);
          }
        }
        epi_bar();
        if (et == 0) mbar_arrive(smem_u32(&acc_empty[ab]));
      } else {
        // C_int += acc 2^sh_u, one hand-over per unit of this window; C is held
        // as 64-bit fixed point (scale 2^-f relative to sigma_i tau_j) until the
        // conversion after the kernel
        for (int u = 0; u < args.nunits; ++u) {
          const int ab = tl & 1;
          const uint32_t aphase = (uint32_t)(tl >> 1) & 1u;
          ++tl;
          const bool got = mbar_wait(smem_u32(&acc_full[ab]), aphase, &abort_flag, args.err, true, wl);
          if (!epi_all<32 * NEPI>(got)) { good = false; break; }
          tc_fence_after();
          const int sh = s_unit_sh[u];
#pragma unroll 1
          for (int c = c0; c < c1; ++c) {
            const int p = pc[c];
#pragma unroll
            for (int h = 0; h < BS / 32; ++h) {
              longlong2 dv[16];
              longlong2* dst = args.cpart + (size_t)(p < 0 ? 0 : p) * (BS * BS / 2) +
                               (size_t)(((q & 1) * 2 + h) * 16) * 32 + lane;
              if (p >= 0) {
#pragma unroll
                for (int e = 0; e < 16; ++e) dv[e] = dst[e * 32];
              }
              float v[32];
              tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(ab * C::N + c * BS + h * 32), v);
              if (p >= 0) {
                bool bad = false;
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                  dv[e].x = fixed_add(dv[e].x, __float2int_rn(v[2 * e]), sh, bad);
                  dv[e].y = fixed_add(dv[e].y, __float2int_rn(v[2 * e + 1]), sh, bad);
                  dst[e * 32] = dv[e];
                }
                if (bad) *args.ovf = 2;
              }
            }
          }
          tc_fence_before();
          epi_bar();
          if (et == 0) mbar_arrive(smem_u32(&acc_empty[ab]));
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)C::TMEM_COLS));
  }
}

// ---------------------------------------------------------------------------
// operand conversion and tile list
// ---------------------------------------------------------------------------
// dst[q] = low-precision copy of block src[q] of X (B x B blocks; K-major:
// transposed when tr).  Reads are coalesced; a transposed copy goes through
// shared memory in 32 x 32 sub-blocks.  X's values are FP64 (V = double) or
// the FP32 results of a TF32/BF16 product (V = float), rounded alike.
template <int ELT, int B, typename V>
__global__ void __launch_bounds__(256) k_convert(const V* __restrict__ val, const int32_t* __restrict__ src,
                                                 int64_t nblk, int tr, void* __restrict__ dst) {
  constexpr int BSZ = B * B;
  using T = typename std::conditional<ELT == 2, uint16_t, uint32_t>::type;
  __shared__ T tile[32][33];
  auto conv = [](V x) -> T {
    if constexpr (std::is_same<V, float>::value) {
      if constexpr (ELT == 2) return f32_to_bf16_bits_rne(x);
      else return f32_to_tf32(f32_flush(x));
    } else {
      if constexpr (ELT == 2) return f64_to_bf16_bits_rne(x);
      else return f32_to_tf32(__uint_as_float(f64_to_f32_bits_rne(x)));
    }
  };
  T* out = reinterpret_cast<T*>(dst);
  for (int64_t qb = blockIdx.x; qb < nblk; qb += gridDim.x) {
    const V* s = val + (size_t)(src ? src[qb] : qb) * BSZ;
    T* d = out + (size_t)qb * BSZ;
    if (!tr) {
      for (int e = threadIdx.x; e < BSZ; e += blockDim.x) d[e] = conv(s[e]);
      continue;
    }
    for (int ti = 0; ti < B / 32; ++ti)
      for (int tj = 0; tj < B / 32; ++tj) {
        // stored rows 32 ti.., columns 32 tj.. -> copy rows 32 tj.., columns 32 ti..
        for (int e = threadIdx.x; e < 1024; e += blockDim.x) {
          const int r = e >> 5, c = e & 31;
          tile[r][c] = conv(s[(size_t)(ti * 32 + r) * B + tj * 32 + c]);
        }
        __syncthreads();
        for (int e = threadIdx.x; e < 1024; e += blockDim.x) {
          const int r = e >> 5, c = e & 31;
          d[(size_t)(tj * 32 + r) * B + ti * 32 + c] = tile[c][r];
        }
        __syncthreads();
      }
  }
}

// out[q] = vmap[src[q]] (src null: identity): the value position of view entry
// q of a matrix whose kept blocks stayed in place after truncation
__global__ void k_compose(const int32_t* __restrict__ src, const int32_t* __restrict__ vmap, int64_t n,
                          int32_t* __restrict__ out) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q < n) out[q] = vmap[src ? src[q] : q];
}

static const int32_t* value_src(ifac_ctx* ctx, const int32_t* src, const int32_t* vmap, int64_t n,
                                Buf<int32_t>& keep) {
  if (!vmap) return src;
  keep = Buf<int32_t>(ctx, (size_t)std::max<int64_t>(n, 1));
  if (n > 0) {
    k_compose<<<cdiv(n, 256), 256, 0, ctx->stream>>>(src, vmap, n, keep.p);
    IFAC_CK_LAUNCH();
  }
  return keep.p;
}

// P = b1 D + b2 W, the correction polynomial of Eq. (2.1) at m = 2 in the
// mixed schedule, written straight into the low-precision op(B) copy that
// M = Z P reads (P itself is never stored in FP64): block p of P's pattern,
// (I, J), is stored transposed ([j][k], as op(B) blocks are), W_IJ = U_IJ for
// J >= I and U_JI^T below, U the upper block triangle of delta^2.  The block
// is assembled in FP32 in shared memory (inputs rounded to FP32 on their bit
// patterns, one FMA per element), then rounded to TF32 / BF16 as k_convert
// rounds.  One CTA per block (grid-stride).  U's values are FP64 or the FP32
// results of its TF32/BF16 product (UV = float), rounded alike.
template <int ELT, typename UV>
__global__ void __launch_bounds__(256)
    k_poly2_lp(const int32_t* __restrict__ prow, const int32_t* __restrict__ pci, int64_t pnnz,
               const int32_t* __restrict__ urp, const int32_t* __restrict__ uci, const UV* __restrict__ uval,
               const int32_t* __restrict__ umap, const int32_t* __restrict__ drp, const int32_t* __restrict__ dci,
               const double* __restrict__ dval, float b1, float b2, void* __restrict__ dst) {
  constexpr int B = 64, BSZ = B * B;
  using T = typename std::conditional<ELT == 2, uint16_t, uint32_t>::type;
  __shared__ float t[B][B + 1];
  __shared__ int sq[2];
  const auto f32 = [](double x) { return __uint_as_float(f64_to_f32_bits_rne(x)); };
  const auto u32 = [](UV x) {
    if constexpr (std::is_same<UV, float>::value) return f32_flush(x);
    else return __uint_as_float(f64_to_f32_bits_rne(x));
  };
  T* out = reinterpret_cast<T*>(dst);
  for (int64_t p = blockIdx.x; p < pnnz; p += gridDim.x) {
    const int I = prow[p], J = pci[p];
    if (threadIdx.x == 0) {
      int k = lower_bound_i32(dci, drp[I], drp[I + 1], J);
      sq[0] = (k < drp[I + 1] && dci[k] == J) ? k : -1;
      const int r = I < J ? I : J, c = I < J ? J : I;
      k = lower_bound_i32(uci, urp[r], urp[r + 1], c);
      sq[1] = (k < urp[r + 1] && uci[k] == c) ? (umap ? umap[k] : k) : -1;
    }
    __syncthreads();
    const int qd = sq[0], qu = sq[1];
    for (int e = threadIdx.x; e < BSZ; e += blockDim.x)
      t[e >> 6][e & 63] = qd >= 0 ? b1 * f32(dval[(size_t)qd * BSZ + e]) : 0.0f;
    __syncthreads();
    if (qu >= 0) {
      const UV* u = uval + (size_t)qu * BSZ;
      if (J >= I) {
        for (int e = threadIdx.x; e < BSZ; e += blockDim.x)
          t[e >> 6][e & 63] = fmaf(b2, u32(u[e]), t[e >> 6][e & 63]);
      } else {  // U_JI read in its stored order, added transposed
        for (int e = threadIdx.x; e < BSZ; e += blockDim.x)
          t[e & 63][e >> 6] = fmaf(b2, u32(u[e]), t[e & 63][e >> 6]);
      }
      __syncthreads();
    }
    // row c of the copy is column c of P_IJ
    T* d = out + (size_t)p * BSZ;
    for (int e = threadIdx.x; e < BSZ; e += blockDim.x) {
      const float v = t[e & 63][e >> 6];
      if constexpr (ELT == 2) d[e] = __bfloat16_as_ushort(__float2bfloat16_rn(v));
      else d[e] = f32_to_tf32(v);
    }
    __syncthreads();  // t is rewritten for the next block
  }
}

// flag[tile] = 1 for every tile holding a block of C's pattern
__global__ void k_tile_flags(const int32_t* __restrict__ row, const int32_t* __restrict__ ci, int64_t nnz, int tm,
                             int tn, int ntc, uint8_t* __restrict__ flag) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= nnz) return;
  flag[(size_t)(row[p] / tm) * ntc + ci[p] / tn] = 1;
}

// Tiles of a sparse C in one pass over its blocks: block p owns its tile
// (I / tm, J / tn) when the tile holds no earlier block, i.e. neither the block
// before it in row I nor a block of the tile's earlier rows lies in the tile's
// column range.  The owners, in C's order, list every tile once.
__global__ void k_tile_owner(const int32_t* __restrict__ row, const int32_t* __restrict__ rp,
                             const int32_t* __restrict__ ci, int64_t nnz, int tm, int tn, int32_t* __restrict__ own) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= nnz) return;
  const int I = row[p], c0 = (ci[p] / tn) * tn;
  int o = (p > rp[I] && ci[p - 1] >= c0) ? 0 : 1;
  for (int I2 = (I / tm) * tm; o && I2 < I; ++I2) {
    const int hi = rp[I2 + 1];
    const int q = lower_bound_i32(ci, rp[I2], hi, c0);
    if (q < hi && ci[q] < c0 + tn) o = 0;
  }
  own[p] = o;
}

__global__ void k_tile_owner_write(const int32_t* __restrict__ row, const int32_t* __restrict__ ci, int64_t nnz,
                                   int tm, int tn, const int32_t* __restrict__ off, int32_t* __restrict__ out) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= nnz || off[p + 1] == off[p]) return;
  out[2 * (size_t)off[p]] = row[p] / tm;
  out[2 * (size_t)off[p] + 1] = ci[p] / tn;
}

// Tile compaction in grouped order: linear index li runs over groups of GROUP
// tile rows, column by column inside a group, so that CTAs running at the same
// time share op(B) panels in L2.  Three passes: count per chunk, scan, write.
constexpr int GROUP = 8;
constexpr int CHUNK = 1024;

__device__ __forceinline__ int64_t grouped_to_rowmajor(int64_t li, int ntr, int ntc) {
  const int64_t g = li / ((int64_t)GROUP * ntc);
  const int64_t rows = min((int64_t)GROUP, (int64_t)ntr - g * GROUP);
  const int64_t off = li - g * GROUP * ntc;
  return (g * GROUP + off % rows) * ntc + off / rows;
}

__global__ void k_tile_count(const uint8_t* __restrict__ flag, int ntr, int ntc, int32_t* __restrict__ cnt) {
  __shared__ int red[32];
  const int64_t tot = (int64_t)ntr * ntc;
  const int64_t li = (int64_t)blockIdx.x * CHUNK + threadIdx.x;
  const int f = (li < tot && flag[grouped_to_rowmajor(li, ntr, ntc)]) ? 1 : 0;
  const unsigned m = __ballot_sync(0xffffffffu, f);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = __popc(m);
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < CHUNK / 32; ++w) t += red[w];
    cnt[blockIdx.x] = t;
  }
}

__global__ void k_tile_write(const uint8_t* __restrict__ flag, int ntr, int ntc, const int32_t* __restrict__ off,
                             int32_t* __restrict__ out) {
  __shared__ int wbase[32];
  const int64_t tot = (int64_t)ntr * ntc;
  const int64_t li = (int64_t)blockIdx.x * CHUNK + threadIdx.x;
  const int64_t i = li < tot ? grouped_to_rowmajor(li, ntr, ntc) : 0;
  const bool f = li < tot && flag[i];
  const unsigned m = __ballot_sync(0xffffffffu, f);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) wbase[w] = __popc(m);
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int k = 0; k < CHUNK / 32; ++k) {
      const int c = wbase[k];
      wbase[k] = acc;
      acc += c;
    }
  }
  __syncthreads();
  if (f) {
    const int pos = off[blockIdx.x] + wbase[w] + __popc(m & ((1u << lane) - 1u));
    out[2 * pos] = (int32_t)(i / ntc);
    out[2 * pos + 1] = (int32_t)(i % ntc);
  }
}

// dense block-index map of a CSR pattern: map[I*nb + J] = q for block q, else zero_idx
__global__ void k_map_fill(int32_t* __restrict__ map, int64_t n, int32_t zero_idx) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) map[i] = zero_idx;
}

__global__ void k_map_scatter(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, int nb,
                              int32_t* __restrict__ map) {
  const int row = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (row >= nb) return;
  for (int p = rp[row] + lane; p < rp[row + 1]; p += 32) map[(size_t)row * nb + ci[p]] = p;
}

// pairs += |row K of op(B)| for every stored block (I, K) of op(A): the number
// of (I, K, J) block triples, i.e. of stored-block products
// stored block pairs (op(A)_IK, op(B)_KJ) of the product: all of them, or
// with upper only those with J >= I (found by binary search in the sorted
// op(B) row K).  wpairs (nullable) also gets w per pair.  Warp per row I.
__global__ void k_count_pairs(const int32_t* __restrict__ arp, const int32_t* __restrict__ aci, int nb,
                              const int32_t* __restrict__ brp, const int32_t* __restrict__ bci, int upper,
                              unsigned long long* __restrict__ pairs, unsigned long long* __restrict__ wpairs,
                              int w) {
  const int row = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  unsigned long long c = 0;
  if (row < nb)
    for (int p = arp[row] + lane; p < arp[row + 1]; p += 32) {
      const int K = aci[p];
      int lo = brp[K];
      const int hi = brp[K + 1];
      if (upper) {
        int h = hi;
        while (lo < h) {
          const int mid = (lo + h) >> 1;
          if (bci[mid] < row) lo = mid + 1;
          else h = mid;
        }
      }
      c += (unsigned long long)(hi - lo);
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if (lane == 0 && c) {
    atomicAdd(pairs, c);
    if (wpairs) atomicAdd(wpairs, c * (unsigned long long)w);
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encoder() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    IFAC_CK(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !p) fail(IFAC_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// 2D view of a low-precision block array: rows = (nblk) * 64, 64 elements per
// row; boxes of one 128-byte atom x 64 rows, 128-byte swizzle

// Plan records of every super-tile: for each K of the union of its rows'
// bitmaps at which some op(B)_KJ of its columns is stored, the copy index of
// op(A)_IK for each of its ROWS block rows and of op(B)_KJ for each of its
// COLS block columns (the zero block when absent); K steps whose op(B) blocks
// are all absent contribute nothing and are left out.  One warp per tile,
// candidate K's 32 at a time, lane-parallel.  COUNT: the number of records
// into nk[t] (and the largest into *kmax); else the records, from off[t] on,
// and (cpos non-null) the position in C's pattern of each of the tile's
// ROWS x COLS blocks (-1 where C holds none), so that a product's epilogue
// finds its output blocks with one load instead of a search.
template <int ROWS, int COLS, bool COUNT>
__global__ void k_tile_plan(const int32_t* __restrict__ tiles, const int* __restrict__ ntiles,
                            const int32_t* __restrict__ off, const uint32_t* __restrict__ bm, int nb, int W,
                            const int32_t* __restrict__ mapA, const int32_t* __restrict__ mapB,
                            const int32_t* __restrict__ arp, const int32_t* __restrict__ aci,
                            const int32_t* __restrict__ brp, const int32_t* __restrict__ bci, int a_zero, int b_zero,
                            const int32_t* __restrict__ amap, int32_t* __restrict__ rec, int32_t* __restrict__ nk_out,
                            int* __restrict__ kmax, const int32_t* __restrict__ crp = nullptr,
                            const int32_t* __restrict__ cci = nullptr, int32_t* __restrict__ cpos = nullptr,
                            const int32_t* __restrict__ bmap = nullptr) {
  static_assert(ROWS * COLS <= 32, "one lane per block of the tile");
  const int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= *ntiles) {  // the grid covers an upper bound of the tile count
    if (COUNT && lane == 0) nk_out[t] = 0;
    return;
  }
  const int I0 = tiles[2 * t] * ROWS, J0 = tiles[2 * t + 1] * COLS;
  if (!COUNT && cpos && lane < ROWS * COLS) {
    const int I = I0 + lane / COLS, J = J0 + lane % COLS;
    int pos = -1;
    if (I < nb && J < nb) {
      const int hi = crp[I + 1];
      const int q = lower_bound_i32(cci, crp[I], hi, J);
      if (q < hi && cci[q] == J) pos = q;
    }
    cpos[(size_t)t * (ROWS * COLS) + lane] = pos;
  }
  int e = COUNT ? 0 : off[t];
  for (int wbase = 0; wbase < W; wbase += 32) {
    const int w = wbase + lane;
    uint32_t word = 0;
    if (w < W) {
#pragma unroll
      for (int r = 0; r < ROWS; ++r)
        if (I0 + r < nb) word |= bm[(size_t)(I0 + r) * W + w];
    }
    while (__any_sync(0xffffffffu, word != 0u)) {
      int ra[ROWS], rb[COLS];
      bool valid = false;
      if (word != 0u) {
        const int K = w * 32 + __ffs(word) - 1;
        word &= word - 1u;
        if (mapA) {
#pragma unroll
          for (int c = 0; c < COLS; ++c) rb[c] = (J0 + c < nb) ? mapB[(size_t)K * nb + J0 + c] : b_zero;
        } else {
          const int hi = brp[K + 1];
          int q = lower_bound_i32(bci, brp[K], hi, J0);
#pragma unroll
          for (int c = 0; c < COLS; ++c) {
            int idx = b_zero;
            if (q < hi && bci[q] == J0 + c) idx = q++;
            rb[c] = idx;
          }
        }
#pragma unroll
        for (int c = 0; c < COLS; ++c) valid |= rb[c] != b_zero;
        if (!COUNT && valid) {
          if (mapA) {
#pragma unroll
            for (int r = 0; r < ROWS; ++r) ra[r] = (I0 + r < nb) ? mapA[(size_t)(I0 + r) * nb + K] : a_zero;
          } else {
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
              int idx = a_zero;
              if (I0 + r < nb) {
                const int hi = arp[I0 + r + 1];
                const int q = lower_bound_i32(aci, arp[I0 + r], hi, K);
                if (q < hi && aci[q] == K) idx = q;
              }
              ra[r] = idx;
            }
          }
        }
      }
      const unsigned m = __ballot_sync(0xffffffffu, valid);
      if (!COUNT && valid) {
        int32_t* out = rec + (size_t)(e + __popc(m & ((1u << lane) - 1u))) * (ROWS + COLS);
#pragma unroll
        for (int r = 0; r < ROWS; ++r) out[r] = (amap && ra[r] != a_zero) ? amap[ra[r]] : ra[r];
#pragma unroll
        for (int c = 0; c < COLS; ++c) out[ROWS + c] = (bmap && rb[c] != b_zero) ? bmap[rb[c]] : rb[c];
      }
      e += __popc(m);
    }
  }
  if (COUNT && lane == 0) {
    nk_out[t] = e;
    if (kmax) atomicMax(kmax, e);
  }
}

// The tile plan of a product: super-tiles of ROWS x COLS blocks holding a
// block of C's pattern (grouped order), their K-step counts and records.
struct Plan {
  Buf<int32_t> tiles, coff, tnk, off, rec, cpos;  // cpos: C positions of each tile's blocks
  int nchunk = 0;
  int64_t ntot = 0;
  int ntiles = 0;  // upper bound of the tile count (the count itself stays on the device)
  int kmax = 0;
};

template <int ROWS, int COLS>
static Plan make_plan(ifac_ctx* ctx, const View& arows, const ifac_bsr& A, bool tA, const View& brows,
                      const ifac_bsr& B, const ifac_bsr& C, const int32_t* crow, bool want_kmax,
                      int kmax_limit = 0, const int32_t* amap = nullptr, const HostRead* extra = nullptr,
                      const int32_t* bmap = nullptr) {
  // amap (nullable): copy index of each op(A) view position, when op(A)'s
  // low-precision copy is not in view order (a shared copy of a transposed
  // operand, held in the stored order).  bmap (nullable): the same for
  // op(B) (a symmetric op(B) read from its op(A) copy).  extra (nullable): one more small
  // read-back the caller needs, taken with the plan's sizes in one
  // synchronisation.
  // kmax_limit > 0: a plan whose longest tile has more K steps is not wanted;
  // it returns after the count pass with kmax set and no records
  const int nb = A.nb, W = words_per_row(nb);
  Plan P;
  // K sets (bitmap rows of op(A)); dense block-index maps of op(A), op(B)
  // while they stay small, binary searches in the CSR patterns beyond that
  Buf<uint32_t> bmA = pattern_bitmap(ctx, A, tA);
  const int64_t nb2 = (int64_t)nb * nb;
  const bool dense_maps = nb2 <= (int64_t)4 << 20;
  Buf<int32_t> imA, imB;
  if (dense_maps) {
    imA = Buf<int32_t>(ctx, nb2);
    imB = Buf<int32_t>(ctx, nb2);
    k_map_fill<<<cdiv(nb2, 256), 256, 0, ctx->stream>>>(imA.p, nb2, (int32_t)A.nnzb);
    IFAC_CK_LAUNCH();
    k_map_fill<<<cdiv(nb2, 256), 256, 0, ctx->stream>>>(imB.p, nb2, (int32_t)B.nnzb);
    IFAC_CK_LAUNCH();
    k_map_scatter<<<cdiv((int64_t)nb * 32, 256), 256, 0, ctx->stream>>>(arows.rp, arows.ci, nb, imA.p);
    IFAC_CK_LAUNCH();
    k_map_scatter<<<cdiv((int64_t)nb * 32, 256), 256, 0, ctx->stream>>>(brows.rp, brows.ci, nb, imB.p);
    IFAC_CK_LAUNCH();
  }
  const int ntr = cdiv(nb, ROWS), ntc = cdiv(nb, COLS);
  P.ntot = (int64_t)ntr * ntc;
  if ((int64_t)C.nnzb * 16 < P.ntot) {
    // a sparse C (a banded product): its tiles from its blocks, in C's order
    P.nchunk = (int)C.nnzb;
    P.tiles = Buf<int32_t>(ctx, (size_t)2 * std::max<int64_t>(C.nnzb, 1));
    P.coff = Buf<int32_t>(ctx, (size_t)C.nnzb + 1);
    Buf<int32_t> own(ctx, (size_t)std::max<int64_t>(C.nnzb, 1));
    if (C.nnzb) {
      k_tile_owner<<<cdiv(C.nnzb, 256), 256, 0, ctx->stream>>>(crow, C.row_ptr, C.col_idx, C.nnzb, ROWS, COLS,
                                                               own.p);
      IFAC_CK_LAUNCH();
    }
    scan_counts(ctx, own.p, P.coff.p, (int)C.nnzb, false);
    if (C.nnzb) {
      k_tile_owner_write<<<cdiv(C.nnzb, 256), 256, 0, ctx->stream>>>(crow, C.col_idx, C.nnzb, ROWS, COLS,
                                                                     P.coff.p, P.tiles.p);
      IFAC_CK_LAUNCH();
    }
  } else {
    P.nchunk = cdiv(P.ntot, CHUNK);
    Buf<uint8_t> flags(ctx, (size_t)P.ntot);
    Buf<int32_t> ccnt(ctx, P.nchunk);
    P.tiles = Buf<int32_t>(ctx, (size_t)2 * P.ntot);
    P.coff = Buf<int32_t>(ctx, P.nchunk + 1);
    IFAC_CK(cudaMemsetAsync(flags.p, 0, (size_t)P.ntot, ctx->stream));
    k_tile_flags<<<cdiv(C.nnzb, 256), 256, 0, ctx->stream>>>(crow, C.col_idx, C.nnzb, ROWS, COLS, ntc, flags.p);
    IFAC_CK_LAUNCH();
    k_tile_count<<<P.nchunk, CHUNK, 0, ctx->stream>>>(flags.p, ntr, ntc, ccnt.p);
    IFAC_CK_LAUNCH();
    scan_counts(ctx, ccnt.p, P.coff.p, P.nchunk, false);
    k_tile_write<<<P.nchunk, CHUNK, 0, ctx->stream>>>(flags.p, ntr, ntc, P.coff.p, P.tiles.p);
    IFAC_CK_LAUNCH();
  }
  const int* ntiles = P.coff.p + P.nchunk;
  // the per-tile kernels and arrays are sized by a bound of the tile count
  // (every tile holds a block of C), not by all ntr x ntc positions
  const int nt = (int)std::min<int64_t>(P.ntot, C.nnzb);
  P.ntiles = nt;
  P.tnk = Buf<int32_t>(ctx, (size_t)std::max(nt, 1));
  P.off = Buf<int32_t>(ctx, (size_t)nt + 1);
  Buf<int> dk(ctx, 1);
  IFAC_CK(cudaMemsetAsync(dk.p, 0, sizeof(int), ctx->stream));
  int64_t total = 0;
  if (nt > 0) {
    k_tile_plan<ROWS, COLS, true><<<cdiv((int64_t)nt * 32, 256), 256, 0, ctx->stream>>>(
        P.tiles.p, ntiles, nullptr, bmA.p, nb, W, dense_maps ? imA.p : nullptr, dense_maps ? imB.p : nullptr,
        arows.rp, arows.ci, brows.rp, brows.ci, (int)A.nnzb, (int)B.nnzb, nullptr, nullptr, P.tnk.p,
        want_kmax ? dk.p : nullptr);
    IFAC_CK_LAUNCH();
    scan_counts(ctx, P.tnk.p, P.off.p, nt, false);
  }
  {
    // the record count, the longest tile and the caller's extra read-back
    // behind one synchronisation
    int32_t tot32 = 0;
    const HostRead none{nullptr, nullptr, 0};
    const HostRead ex = extra ? *extra : none;
    if (ex.bytes) {
      to_host_many(ctx, {{&tot32, nt > 0 ? (const void*)(P.off.p + nt) : (const void*)dk.p, sizeof(int32_t)},
                         {&P.kmax, dk.p, sizeof(int)},
                         ex});
    } else {
      to_host_many(ctx, {{&tot32, nt > 0 ? (const void*)(P.off.p + nt) : (const void*)dk.p, sizeof(int32_t)},
                         {&P.kmax, dk.p, sizeof(int)}});
    }
    total = nt > 0 ? tot32 : 0;
    if (!want_kmax) P.kmax = 0;
  }
  if (total > (int64_t)0x7fffffff / (ROWS + COLS))
    fail(IFAC_ERR_TOO_LARGE, "tensor-core product: tile plan exceeds 2^31 entries");
  if (want_kmax && kmax_limit > 0 && P.kmax > kmax_limit) return P;
  P.rec = Buf<int32_t>(ctx, (size_t)std::max<int64_t>(total, 1) * (ROWS + COLS));
  P.cpos = Buf<int32_t>(ctx, (size_t)std::max(nt, 1) * (ROWS * COLS));
  if (nt > 0) {
    k_tile_plan<ROWS, COLS, false><<<cdiv((int64_t)nt * 32, 256), 256, 0, ctx->stream>>>(
        P.tiles.p, ntiles, P.off.p, bmA.p, nb, W, dense_maps ? imA.p : nullptr, dense_maps ? imB.p : nullptr,
        arows.rp, arows.ci, brows.rp, brows.ci, (int)A.nnzb, (int)B.nnzb, amap, P.rec.p, nullptr, nullptr,
        C.row_ptr, C.col_idx, P.cpos.p, bmap);
    IFAC_CK_LAUNCH();
  }
  // the plan kernel has read the maps and the bitmap before they are freed
  // (stream-ordered frees)
  return P;
}

template <int ELT>
static CUtensorMap make_map(void* base, int64_t nblk) {
  CUtensorMap m;
  cuuint64_t dims[2] = {(cuuint64_t)BS, (cuuint64_t)nblk * BS};
  cuuint64_t strides[1] = {(cuuint64_t)BS * ELT};
  cuuint32_t box[2] = {(cuuint32_t)Cfg<ELT>::ATOM_ELEMS, (cuuint32_t)BS};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encoder()(&m, ELT == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base,
                         dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) fail(IFAC_ERR_CUDA, "cuTensorMapEncodeTiled failed with code " + std::to_string((int)r));
  return m;
}

// the same for bs x bs blocks (rows = nblk * bs, bs elements per row) with
// boxes of one swizzle atom (atom_elems elements, 64- or 128-byte swizzle) by
// bs rows, as the narrow-tile kernel reads them
static CUtensorMap make_map_bs(int elt, int bs, void* base, int64_t nblk, const BandShape& sh) {
  CUtensorMap m;
  cuuint64_t dims[2] = {(cuuint64_t)bs, (cuuint64_t)nblk * bs};
  cuuint64_t strides[1] = {(cuuint64_t)bs * elt};
  cuuint32_t box[2] = {(cuuint32_t)sh.atom_elems, (cuuint32_t)bs};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encoder()(&m, elt == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base,
                         dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         sh.atom_bytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) fail(IFAC_ERR_CUDA, "cuTensorMapEncodeTiled failed with code " + std::to_string((int)r));
  return m;
}

// BF16 slices of bs x bs blocks with boxes of inner x rows elements, 64- or
// 128-byte swizzle (inner * 2 bytes)
static CUtensorMap make_map_box(int bs, void* base, int64_t nblk, int inner, int rows) {
  CUtensorMap m;
  cuuint64_t dims[2] = {(cuuint64_t)bs, (cuuint64_t)nblk * bs};
  cuuint64_t strides[1] = {(cuuint64_t)bs * 2};
  cuuint32_t box[2] = {(cuuint32_t)inner, (cuuint32_t)rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encoder()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE,
                         inner * 2 == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) fail(IFAC_ERR_CUDA, "cuTensorMapEncodeTiled failed with code " + std::to_string((int)r));
  return m;
}

template <int ELT, typename V = double>
static void convert_blocks(ifac_ctx* ctx, int bs, const V* val, const int32_t* src, int64_t nblk, bool tr,
                           void* dst) {
  const int grid = (int)std::min<int64_t>(nblk, 152 * 16);
  if (bs == 32) k_convert<ELT, 32, V><<<grid, 256, 0, ctx->stream>>>(val, src, nblk, tr ? 1 : 0, dst);
  else if (bs == 64) k_convert<ELT, 64, V><<<grid, 256, 0, ctx->stream>>>(val, src, nblk, tr ? 1 : 0, dst);
  else k_convert<ELT, 128, V><<<grid, 256, 0, ctx->stream>>>(val, src, nblk, tr ? 1 : 0, dst);
  IFAC_CK_LAUNCH();
}

// the narrow-tile plan of a block size (tile of 128 / bs x max(64, bs) / bs blocks)
static Plan band_plan(ifac_ctx* ctx, int bs, const View& arows, const ifac_bsr& A, bool tA, const View& brows,
                      const ifac_bsr& B, const ifac_bsr& C, const int32_t* crow, int kmax_limit,
                      const int32_t* amap, const HostRead* extra = nullptr, const int32_t* bmap = nullptr) {
  if (bs == 32) return make_plan<4, 2>(ctx, arows, A, tA, brows, B, C, crow, true, kmax_limit, amap, extra, bmap);
  if (bs == 64) return make_plan<2, 1>(ctx, arows, A, tA, brows, B, C, crow, true, kmax_limit, amap, extra, bmap);
  return make_plan<1, 1>(ctx, arows, A, tA, brows, B, C, crow, true, kmax_limit, amap, extra, bmap);
}

// out32: C's values are written as FP32 (C.val holds floats); b32: B's values
// are FP32 (an earlier product's out32 result)
template <int ELT>
static void run(ifac_ctx* ctx, const View& arows, bool tA, const ifac_bsr& A, const View& brows, bool tB,
                const ifac_bsr& B, double alpha, ifac_bsr& C, const int32_t* crow, bool upper,
                unsigned long long* pairs, OperandCache* ac, OperandCache* bc, const OperandCache* bpre,
                const int32_t* avmap, const int32_t* bvmap, bool out32, bool b32) {
  using Cf = Cfg<ELT>;
  const int nb = A.nb, bs = A.bs;
  const size_t bbytes = (size_t)bs * bs * ELT;
  // a cache filled by an earlier product's op(B) holds transposed blocks in
  // the stored order: it serves op(A) = that matrix transposed, through the
  // view's source indices, and nothing else
  if (ac && ac->from_b && !(tA && ac->conv_elt == ELT)) ac = nullptr;
  const int32_t* amap = (ac && ac->from_b) ? arows.src : nullptr;
  // low-precision, K-major copies of op(A) and op(B) plus one zero block each
  // (op(A)'s taken from the cache when it holds one of this format, op(B)'s
  // from bpre when its producer wrote it in this format)
  const bool bhit = bpre && bpre->b_ready && bpre->conv_elt == ELT && !tB;
  // an exactly symmetric op(B) = B whose op(A) copy is at hand: block (K, J)
  // of the op(B) copy, B_KJ^T = B_JK, is that copy's block at tpos
  const bool bsym = !bhit && bpre && bpre->tpos.p && bpre->conv_elt == ELT && !tB;
  const int32_t* bmap = bsym ? bpre->tpos.p : nullptr;
  Buf<uint8_t> la, lb;
  const bool hit = ac && ac->conv_elt == ELT;
  if (!hit) {
    la = Buf<uint8_t>(ctx, (size_t)(A.nnzb + 1) * bbytes);
    IFAC_CK(cudaMemsetAsync(la.p + (size_t)A.nnzb * bbytes, 0, bbytes, ctx->stream));
    Buf<int32_t> asrc;
    if (A.nnzb) convert_blocks<ELT>(ctx, bs, A.val, value_src(ctx, arows.src, avmap, A.nnzb, asrc), A.nnzb, tA, la.p);
    if (ac) {
      ac->conv = std::move(la);
      ac->conv_elt = ELT;
    }
  }
  uint8_t* const la_p = ac ? ac->conv.p : la.p;
  if (!bhit && !bsym) {
    lb = Buf<uint8_t>(ctx, (size_t)(B.nnzb + 1) * bbytes);
    IFAC_CK(cudaMemsetAsync(lb.p + (size_t)B.nnzb * bbytes, 0, bbytes, ctx->stream));
    Buf<int32_t> bsrc;
    if (B.nnzb) {
      const int32_t* vs = value_src(ctx, brows.src, bvmap, B.nnzb, bsrc);
      if (b32) convert_blocks<ELT, float>(ctx, bs, reinterpret_cast<const float*>(B.val), vs, B.nnzb, !tB, lb.p);
      else convert_blocks<ELT>(ctx, bs, B.val, vs, B.nnzb, !tB, lb.p);
    }
  }
  uint8_t* const lb_p = (bhit || bsym) ? bpre->conv.p : lb.p;
  if (bc && !tB && !bhit && !bsym) {  // op(B) = B in its stored order: keep the copy for a later op(A) = B^T
    bc->reset();
    bc->conv = std::move(lb);
    bc->conv_elt = ELT;
    bc->from_b = true;
  }
  k_count_pairs<<<cdiv((int64_t)nb * 32, 256), 256, 0, ctx->stream>>>(arows.rp, arows.ci, nb, brows.rp, brows.ci,
                                                                      upper ? 1 : 0, pairs, nullptr, 0);
  IFAC_CK_LAUNCH();
  // narrow tiles (gemm_band.cu) for every product at bs 32 and 128, and for
  // the banded ones at bs 64 (no 128 x 64 tile with more than KW K steps);
  // the super-tiles below for the other bs-64 products
  // (the context's schedule can ask for super-tiles only, or narrow tiles up
  // to another K length)
  const int nk_lim = ctx->narrow_kmax < 0 ? KW : ctx->narrow_kmax;
  if (bs != 64 || nk_lim > 0) {
    const BandShape sh = band_lp_shape(ELT, bs);
    Plan Pb = band_plan(ctx, bs, arows, A, tA, brows, B, C, crow, bs == 64 ? nk_lim : 0, amap, nullptr, bmap);
    if (bs != 64 || (Pb.kmax >= 1 && Pb.kmax <= nk_lim)) {
      const CUtensorMap mapA = make_map_bs(ELT, bs, la_p, A.nnzb + 1, sh);
      const CUtensorMap mapB = make_map_bs(ELT, bs, lb_p, B.nnzb + 1, sh);
      prof_begin(ctx, 1);
      band_lp_product(ctx, ELT, bs, &mapA, &mapB, Pb.tiles.p, Pb.coff.p + Pb.nchunk, Pb.tnk.p, Pb.rec.p, Pb.off.p,
                      Pb.cpos.p, Pb.ntiles, alpha, C, out32);
      prof_end(ctx);
      ++ctx->tc_launches;
      return;
    }
  }
  const CUtensorMap mapA = make_map<ELT>(la_p, A.nnzb + 1);
  const CUtensorMap mapB = make_map<ELT>(lb_p, B.nnzb + 1);
  Plan P = make_plan<PAIR * TM, Cf::TN>(ctx, arows, A, tA, brows, B, C, crow, false, 0, amap, nullptr, bmap);
  static std::atomic<unsigned long long> attr{0};
  if (first_on_device(attr, ctx->device))
    IFAC_CK(cudaFuncSetAttribute(k_gemm_tc<ELT>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cf::SMEM_BYTES));
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
  TileArgs args;
  args.tiles = P.tiles.p;
  args.ntiles = P.coff.p + P.nchunk;  // the scan's total
  args.tile_nk = P.tnk.p;
  args.nwin = 1;
  args.nb = nb;
  args.rec = P.rec.p;
  args.rec_off = P.off.p;
  args.crp = C.row_ptr;
  args.cci = C.col_idx;
  args.cval = out32 ? nullptr : C.val;
  args.cval32 = out32 ? reinterpret_cast<float*>(C.val) : nullptr;
  args.cnorm = C.norms;
  args.alpha = alpha;
  args.err = ctx->dev_err;
  args.split = 0;
  args.cpart = nullptr;
  args.ovf = nullptr;
  args.nunits = 0;
  for (int u = 0; u < MAX_UNITS; ++u) args.unit_end[u] = args.unit_sh[u] = 0;
  for (int p = 0; p < MAX_PAIRS; ++p) args.pair_ya[p] = args.pair_yb[p] = 0;
  args.stall = 0;
  args.wait_limit = WAIT_LIMIT;
  // one CTA per SM, in pairs; at most one pair per tile (idle pairs return at once)
  const int64_t pairs_grid = std::min<int64_t>(std::max(P.ntiles, 1), sms / PAIR);
  prof_begin(ctx, 1);
  k_gemm_tc<ELT><<<(unsigned)(pairs_grid * PAIR), NTHREADS, Cf::SMEM_BYTES, ctx->stream>>>(mapA, mapB, args);
  IFAC_CK_LAUNCH();
  prof_end(ctx);
  ++ctx->tc_launches;
}

// ---------------------------------------------------------------------------
// FP64-accurate products on the tensor cores by error-free splitting
// (Ozaki, Ogita, Oishi, Rump, "Error-free transformations of matrix
// multiplication by using fast routines of matrix multiplication and its
// applications", Numer. Algorithms 59, 2012): every row i of op(A) is scaled
// by a power of two sigma_i >= its largest magnitude and split into NS slices
// of 7-bit integers (exact in BF16), a = sigma_i sum_s q_s 2^(-7 s) + rest;
// likewise the columns of op(B) with tau_j.  A product of two slices
// (first slices |q| <= 128, later ones |q| <= 64) is a sum of integers, exact
// in FP32 while its magnitude bound stays <= 2^24.  Slice pairs with equal
// weight 2^(-7(s+t)), s + t <= NS + 1, are packed greedily into units whose
// bound over a window stays <= 2^24.  A window holds KW = 16 K blocks (1024
// terms), or fewer when the product's longest tile has fewer K steps: for
// NS = 7, 13 units at full windows, 7 when no tile has more than 7 K steps
// (banded patterns such as a 1D chain).  Per tile and window, each unit is
// one accumulator that the epilogue adds, scaled, into the FP64 result.
// ---------------------------------------------------------------------------
constexpr int SPLIT_BITS = 7;

// GB300's FP64 pipe is narrow, so the splitting below works on the bit
// patterns of the FP64 inputs with integer arithmetic only.

// exponent e of sigma = 2^e for every scalar row of a (possibly transposed)
// row view: max_k |x_rk| = m 2^e with m in [0.5, 1) (e = 0 for an all-zero row);
// the largest scaled row 1-norm sum_k |x_rk| / sigma (FP32, magnitudes
// truncated to 24 bits) into *l1max and the largest scaled row 2-norm
// (sum_k x_rk^2)^(1/2) / sigma (FP64 sum, rounded up) into *l2max, both as
// FP32 bits
__device__ __forceinline__ void row_scale_out(unsigned long long m, float l1, double sq, int nscalars, int* eout,
                                              unsigned int* l1max, unsigned int* l2max) {
  const int ea = (int)(m >> 52);
  int e = 0;
  if (ea > 0) e = ea - 1022;                       // [2^(ea-1023), 2^(ea-1022))
  else if (m != 0) e = (64 - __clzll((long long)m)) - 1074;  // subnormal: [2^(L-1075), 2^(L-1074))
  *eout = e;
  if (m != 0) {
    // entries below 2^-126 were left out: add their largest possible share
    const float s = ldexpf(l1, -e) + (float)nscalars * ldexpf(1.0f, -126 - e);
    atomicMax(l1max, __float_as_uint(fminf(s, 3.0e38f)));
    const float s2 = (float)(ldexp(sqrt(sq), -e) * 1.0001) + 1e-30f;
    atomicMax(l2max, __float_as_uint(fminf(s2, 3.0e38f)));
  }
}

__device__ __forceinline__ void row_scale_acc(double x, unsigned long long& m, float& l1, double& sq) {
  sq = fma(x, x, sq);
  const unsigned long long u = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
  m = u > m ? u : m;
  const int e32 = (int)(u >> 52) - 896;  // FP32 exponent field of |x|
  if (e32 > 0)
    l1 += __uint_as_float(e32 > 254 ? 0x7f7fffffu : (((uint32_t)e32 << 23) | (uint32_t)((u >> 29) & 0x7fffffu)));
}

// transposed views: one CTA of B threads per block row; thread r takes
// column r of each stored block (op(X) row r), reads coalesced across threads
template <int B>
__global__ void __launch_bounds__(B) k_row_scale_t(const int32_t* __restrict__ rp, const int32_t* __restrict__ src,
                                                   int nb, const double* __restrict__ val, int* __restrict__ eout,
                                                   unsigned int* __restrict__ l1max, unsigned int* __restrict__ l2max) {
  const int I = blockIdx.x, r = threadIdx.x;
  if (I >= nb) return;
  // four independent accumulators (rows k mod 4 of each block) so that the
  // FP64 FMA and FP32 add chains overlap; combined at the end
  unsigned long long m[4] = {0, 0, 0, 0};
  float l1[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  double sq[4] = {0.0, 0.0, 0.0, 0.0};
  for (int q = rp[I]; q < rp[I + 1]; ++q) {
    const double* blk = val + (size_t)(src ? src[q] : q) * B * B;
#pragma unroll 4
    for (int k = 0; k < B; k += 4) {
#pragma unroll
      for (int j = 0; j < 4; ++j) row_scale_acc(blk[(k + j) * B + r], m[j], l1[j], sq[j]);
    }
  }
  const unsigned long long m01 = m[0] > m[1] ? m[0] : m[1], m23 = m[2] > m[3] ? m[2] : m[3];
  row_scale_out(m01 > m23 ? m01 : m23, (l1[0] + l1[1]) + (l1[2] + l1[3]), (sq[0] + sq[1]) + (sq[2] + sq[3]),
                (rp[I + 1] - rp[I]) * B, eout + (size_t)I * B + r, l1max, l2max);
}

// rows stored as rows: one warp per scalar row, lanes along the row (coalesced)
template <int B>
__global__ void k_row_scale(const int32_t* __restrict__ rp, const int32_t* __restrict__ src, int nb,
                            const double* __restrict__ val, int* __restrict__ eout, unsigned int* __restrict__ l1max,
                            unsigned int* __restrict__ l2max) {
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= (int64_t)nb * B) return;
  const int I = (int)(w / B), r = (int)(w % B);
  unsigned long long m = 0;  // |x| bit patterns order like the magnitudes
  float l1 = 0.0f;
  double sq = 0.0;
  for (int q = rp[I]; q < rp[I + 1]; ++q) {
    const double* blk = val + (size_t)(src ? src[q] : q) * B * B;
    for (int c = lane; c < B; c += 32) row_scale_acc(blk[r * B + c], m, l1, sq);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long u = __shfl_xor_sync(0xffffffffu, m, o);
    m = u > m ? u : m;
    l1 += __shfl_xor_sync(0xffffffffu, l1, o);
    sq += __shfl_xor_sync(0xffffffffu, sq, o);
  }
  if (lane == 0) row_scale_out(m, l1, sq, (rp[I + 1] - rp[I]) * B, eout + w, l1max, l2max);
}

// sigma exponents (and the scaled 1-norm bound) of the rows of a row view
static void row_scales(ifac_ctx* ctx, int bs, const int32_t* rp, const int32_t* src, int nb, bool tr,
                       const double* val, int* eout, unsigned int* l1max, unsigned int* l2max) {
  const int g = cdiv((int64_t)nb * bs * 32, 256);
  if (bs == 32) {
    if (tr) k_row_scale_t<32><<<nb, 32, 0, ctx->stream>>>(rp, src, nb, val, eout, l1max, l2max);
    else k_row_scale<32><<<g, 256, 0, ctx->stream>>>(rp, src, nb, val, eout, l1max, l2max);
  } else if (bs == 64) {
    if (tr) k_row_scale_t<64><<<nb, 64, 0, ctx->stream>>>(rp, src, nb, val, eout, l1max, l2max);
    else k_row_scale<64><<<g, 256, 0, ctx->stream>>>(rp, src, nb, val, eout, l1max, l2max);
  } else {
    if (tr) k_row_scale_t<128><<<nb, 128, 0, ctx->stream>>>(rp, src, nb, val, eout, l1max, l2max);
    else k_row_scale<128><<<g, 256, 0, ctx->stream>>>(rp, src, nb, val, eout, l1max, l2max);
  }
  IFAC_CK_LAUNCH();
}

// NS BF16 slice copies (K-major, op() CSR order) of a view; row r of block qb
// has scale exponent sexp[sblk[qb] * B + r].  With Y = x 2^(62 - e) held as a
// 64-bit integer (|Y| < 2^62; bits below 2^-62 of sigma dropped by rounding),
// digit k is q_k = round(Y_k / 2^(62 - 7k)) (ties up), Y_{k+1} = Y_k - q_k 2^(62 - 7k).
__device__ __forceinline__ void split_digits(double x, int e, int ns, int (&q)[8]) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int ea = (int)((u >> 52) & 0x7ff);
  unsigned long long mant = u & 0xfffffffffffffull;
  int eb = ea;
  if (ea) mant |= 1ull << 52;
  else eb = 1;
  // |x| = mant 2^(eb - 1075);  |Y| = mant 2^(eb - 1013 - e)
  const int sh = eb - 1013 - e;
  unsigned long long Y = 0;
  if (sh >= 0) Y = mant << sh;  // sh <= 9 since |x| < sigma
  else if (sh > -63) Y = (mant + (1ull << (-sh - 1))) >> (-sh);
  const long long y = (u >> 63) ? -(long long)Y : (long long)Y;
  // the digits in closed form: with R_k = floor((y + 2^(d_k - 1)) / 2^d_k),
  // y rounded (half up) to a multiple of 2^d_k, the digits so far sum to
  // R_k 2^d_k, so q_1 = R_1 and q_k = R_k - 2^7 R_(k-1).  Each q_k is small,
  // so 32-bit arithmetic on the low words of the R_k suffices.
  int rprev = 0;
#pragma unroll
  for (int k = 1; k <= 8; ++k) {
    if (k > ns) break;
    const int d = 62 - SPLIT_BITS * k;
    const unsigned long long t = (unsigned long long)y + (1ull << (d - 1));
    const uint32_t lo = (uint32_t)t, hi = (uint32_t)(t >> 32);
    const int r = d >= 32 ? ((int)hi >> (d - 32)) : (int)__funnelshift_r(lo, hi, d);
    q[k - 1] = k == 1 ? r : (int)((uint32_t)r - ((uint32_t)rprev << 7));
    rprev = r;
  }
}

// digits of elements (r, c) and (r, c + 1) of op(X)'s block into the slices
__device__ __forceinline__ void split_pair(double x0, double x1, int e, int ns, __nv_bfloat16* dst,
                                           size_t slice_stride) {
  int q0[8], q1[8];
  split_digits(x0, e, ns, q0);
  split_digits(x1, e, ns, q1);
  // |q| <= 128 is exact in BF16: the upper half of its FP32 pattern, formed
  // with one integer and one FP32 add (2^23 + 2^22 + q, minus that offset)
  const auto bf = [](int q) -> uint32_t {
    return __float_as_uint(__int_as_float(0x4B400000 + q) - 12582912.0f) >> 16;
  };
  for (int k = 0; k < ns; ++k)
    *reinterpret_cast<uint32_t*>(dst + (size_t)k * slice_stride) = bf(q0[k]) | (bf(q1[k]) << 16);
}

template <int B>
__global__ void __launch_bounds__(256) k_split(const double* __restrict__ val, const int32_t* __restrict__ src,
                                               int64_t nblk, int tr, const int32_t* __restrict__ sblk,
                                               const int* __restrict__ sexp, int ns,
                                               __nv_bfloat16* __restrict__ dst) {
  constexpr int BSZ = B * B;
  __shared__ double tile[32][33];  // transposed views: 32 x 32 sub-blocks
  const size_t slice_stride = (size_t)(nblk + 1) * BSZ;
  for (int64_t qb = blockIdx.x; qb < nblk; qb += gridDim.x) {
    const double* s = val + (size_t)(src ? src[qb] : qb) * BSZ;
    const int* se = sexp + (size_t)sblk[qb] * B;
    __nv_bfloat16* d = dst + (size_t)qb * BSZ;
    if (!tr) {
      for (int e2 = threadIdx.x; e2 < BSZ / 2; e2 += blockDim.x) {
        const int e = 2 * e2, r = e / B;
        split_pair(s[e], s[e + 1], se[r], ns, d + e, slice_stride);
      }
      continue;
    }
    // op(X) row r = stored column r: stored rows 32 ti.., columns 32 tj.. give
    // op rows 32 tj.., columns 32 ti.. (coalesced reads through shared memory)
    for (int ti = 0; ti < B / 32; ++ti)
      for (int tj = 0; tj < B / 32; ++tj) {
        for (int e = threadIdx.x; e < 1024; e += blockDim.x) {
          const int r = e >> 5, c = e & 31;
          tile[r][c] = s[(size_t)(ti * 32 + r) * B + tj * 32 + c];
        }
        __syncthreads();
        for (int e2 = threadIdx.x; e2 < 512; e2 += blockDim.x) {
          const int r = (2 * e2) >> 5, c = (2 * e2) & 31;  // op sub-block element (r, c), (r, c + 1)
          const int orow = tj * 32 + r, ocol = ti * 32 + c;
          split_pair(tile[c][r], tile[c + 1][r], se[orow], ns, d + (size_t)orow * B + ocol, slice_stride);
        }
        __syncthreads();
      }
  }
}

static void split_blocks(ifac_ctx* ctx, int bs, const double* val, const int32_t* src, int64_t nblk, bool tr,
                         const int32_t* sblk, const int* sexp, int ns, void* dst) {
  const int grid = (int)std::min<int64_t>(nblk, 152 * 16);
  __nv_bfloat16* d = reinterpret_cast<__nv_bfloat16*>(dst);
  if (bs == 32) k_split<32><<<grid, 256, 0, ctx->stream>>>(val, src, nblk, tr ? 1 : 0, sblk, sexp, ns, d);
  else if (bs == 64) k_split<64><<<grid, 256, 0, ctx->stream>>>(val, src, nblk, tr ? 1 : 0, sblk, sexp, ns, d);
  else k_split<128><<<grid, 256, 0, ctx->stream>>>(val, src, nblk, tr ? 1 : 0, sblk, sexp, ns, d);
  IFAC_CK_LAUNCH();
}

// x 2^E rounded to nearest (ties to even), built from the integer's bits;
// results outside the normal range take the FP64 pipe
__device__ __forceinline__ double i64_ldexp(long long x, int E) {
  if (x == 0) return 0.0;
  const unsigned long long sgn = x < 0 ? (1ull << 63) : 0ull;
  const unsigned long long ux = x < 0 ? (unsigned long long)(-x) : (unsigned long long)x;
  int len = 64 - __clzll((long long)ux);
  unsigned long long mant;
  if (len > 53) {
    const int sh = len - 53;
    mant = ux >> sh;
    const unsigned long long rem = ux & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (mant & 1ull))) {
      if (++mant == (1ull << 53)) {
        mant >>= 1;
        ++len;
      }
    }
  } else {
    mant = ux << (53 - len);
  }
  const int field = len - 1 + E + 1023;  // value = mant 2^(len - 53 + E), mant in [2^52, 2^53)
  if (field < 1 || field > 2046) return (double)x * ldexp(1.0, E);
  return __longlong_as_double((long long)(sgn | ((unsigned long long)field << 52) | (mant & 0xfffffffffffffull)));
}

// C_IJ = S_int 2^(e_i + e_j + ea) * am from the fixed-point sums of the
// split kernel (alpha = am 2^ea; am = +-1 when alpha is a signed power of
// two): coalesced reads in hand-over order, a transpose through shared
// memory, row-major FP64 writes, then the FP64 block norms
__global__ void __launch_bounds__(256) k_split_finish(const int32_t* __restrict__ crow,
                                                      const int32_t* __restrict__ cci, int64_t nnzb,
                                                      const longlong2* __restrict__ part, double* __restrict__ cval,
                                                      const int* __restrict__ sige, const int* __restrict__ taue,
                                                      int ea, double am, double* __restrict__ cnorm) {
  __shared__ double tile[BS][BS + 1];
  __shared__ double red[8];
  const bool unit = (am == 1.0 || am == -1.0);
  for (int64_t p = blockIdx.x; p < nnzb; p += gridDim.x) {
    const int I = crow[p], J = cci[p];
    const longlong2* src = part + (size_t)p * (BS * BS / 2);
    for (int i = threadIdx.x; i < BS * BS / 2; i += blockDim.x) {
      const int lane = i & 31, e = (i >> 5) & 15, h = (i >> 9) & 1, qq = i >> 10;
      const int r = qq * 32 + lane, col = h * 32 + 2 * e;
      longlong2 x = src[i];
      if (unit && am < 0.0) {
        x.x = -x.x;
        x.y = -x.y;
      }
      const int er = ea + sige[(size_t)I * BS + r];
      double v0 = i64_ldexp(x.x, er + taue[(size_t)J * BS + col]);
      double v1 = i64_ldexp(x.y, er + taue[(size_t)J * BS + col + 1]);
      if (!unit) {
        v0 *= am;
        v1 *= am;
      }
      tile[r][col] = v0;
      tile[r][col + 1] = v1;
    }
    __syncthreads();
    double* c = cval + (size_t)p * BS * BS;
    double ss = 0.0;
    for (int k = threadIdx.x; k < BS * BS; k += blockDim.x) {
      const double v = tile[k / BS][k % BS];
      c[k] = v;
      ss = fma(v, v, ss);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if (lane == 0) red[wid] = ss;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < 8; ++w) t += red[w];
      cnorm[p] = sqrt(t);
    }
  }
}

// ---------------------------------------------------------------------------
// Split products on narrow tiles (bs 32, 64, 128).  A tile is 128 x 64
// accumulator elements: 128 / bs block rows of C by 64 columns (two block
// columns at bs 32, one at bs 64, half of one at bs 128, whose two halves the
// same CTA takes one after the other).  Each K block is streamed in chunks of
// at most 64 K elements; a chunk's slices are loaded once -- slice k of the
// tile's op(A) rows and op(B) columns share one ring slot -- and, as soon as
// slot k has landed, the MMAs of the slice pairs (a, b) with max(a, b) = k
// are issued; a slot is released after the last pair that reads it.  Every
// accumulation unit keeps its own FP32 accumulator in tensor memory (up to 8
// units x 64 columns).  A window of K blocks is as long as every weight class
// fits one unit; after each window the epilogue adds the units, scaled, into
// 64-bit fixed-point sums held in registers, so a tile may span any number of
// windows.  After the tile's last window the epilogue writes
// S_ij 2^(ea + e_i + e_j) * am in FP64 and the block norms.
// ---------------------------------------------------------------------------
namespace band {
constexpr int MAX_U = 8;                    // units live at once: 8 x 64 = 512 columns
// 16 epilogue warps, four per tensor-memory lane quarter, each on 16 of the
// tile's 64 columns: the epilogue's adds of the units into the fixed-point
// sums stand between the MMAs of consecutive tiles (the accumulators hold
// every unit, so they are not double-buffered), and twice the warps of the
// other kernels halve that time
constexpr int EPW = 16;
constexpr int NTB = 32 * (2 + EPW);
constexpr uint32_t TMEM_COLS = 512;
// FP32 accumulate, A = B = BF16, both K-major, N = 64, M = 128
constexpr uint32_t IDESC = idesc_of<2, 64, 128>();

template <int B>
struct SB {
  static constexpr int M = 128, N = 64;
  static constexpr int TMB = M / B;                 // block rows per tile (4, 2, 1)
  static constexpr int TNB = B <= N ? N / B : 1;    // block columns per tile (2, 1, 1)
  static constexpr int NSUB = B > N ? B / N : 1;    // column sub-tiles per block column (1, 1, 2)
  static constexpr int BROWS = B < N ? B : N;       // rows of one op(B) box (32, 64, 64)
  // K chunks of 64 elements (32 at bs 32); halving them at bs 64 and 128 was
  // measured slower: the per-slot waits, copies and commits double while the
  // products stay the same
  static constexpr int KC = B < 64 ? B : 64;        // K elements per chunk
  static constexpr int KCH = B / KC;                // chunks per K block (1, 1, 2)
  static constexpr int ATOM = KC * 2;               // bytes of one BF16 row chunk: one swizzle atom (64 or 128)
  static constexpr int SLOT_A = M * ATOM;           // one slice of the tile's op(A) rows: 8, 16, 16 KB
  static constexpr int SLOT_B = N * ATOM;           // one slice of its op(B) columns: 4, 8, 8 KB
  static constexpr int MAXS = 8;                    // slices per operand at most
  // every op(B) slice of a chunk stays in one of two buffers while the op(A)
  // slices stream through a ring: slice a of op(A) meets slices 0 .. ns-1-a
  // of op(B), and its slot is released as soon as those products are issued
  static constexpr int B_BUF = MAXS * SLOT_B;
  static constexpr int RA_FIT = (216 * 1024 - 2 * B_BUF) / SLOT_A;
  static constexpr int RA = RA_FIT < 16 ? RA_FIT : 16;  // op(A) ring slots: 16, 5, 5
  static constexpr int SMEM_BYTES = 2 * B_BUF + RA * SLOT_A + 1024;
  static constexpr int KSTEPS = ATOM / 32;          // MMAs per slice pair and chunk
  static constexpr uint32_t SBO = 8 * ATOM;
  static constexpr uint32_t SWZ = ATOM == 128 ? 2 : 4;
  static constexpr int RECW = TMB + TNB;
  static_assert(SLOT_A % 1024 == 0 && SLOT_B % 1024 == 0, "slots must keep the swizzle alignment");
  static_assert(RA >= 2, "op(A) ring too shallow");
};
}  // namespace band

struct BandArgs {
  const int32_t* tiles;    // [2t] tile row (of TMB block rows), [2t+1] tile column (of TNB block columns)
  const int* ntiles;       // device: number of tiles
  const int* tile_nk;      // device: K blocks of each tile
  const int32_t* rec;      // plan: per K block, copy indices of the tile's op(A)_IK, then op(B)_KJ
  const int32_t* rec_off;  // first record of each tile
  const int32_t* cpos;     // per tile, the C positions of its TMB x TNB blocks (-1: not in C)
  double* cval;            // C's values and block norms (FP64)
  double* cnorm;
  const int* sige;         // scale exponents of the scalar rows of op(A) and columns of op(B)
  const int* taue;
  int ea;                  // C_ij = S_ij 2^(ea + e_i + e_j) * am, S_ij the 64-bit fixed-point sum
  double am;               // +-1 (applied to the integer) or the mantissa of alpha
  int nb;
  int ns;                  // slices per operand (1..8)
  int kwin;                // K blocks per window (every weight class exact in one FP32 accumulator)
  int slice_rows_a;        // tensor-map rows between consecutive slices of op(A): (nnzb_A + 1) bs
  int slice_rows_b;
  int nunits;
  int unit_sh[band::MAX_U];
  // Horner groups of units: unit u with unit_step[u] >= 0 enters its group's
  // 64-bit accumulator as g = (g << unit_step[u]) + x_u (the first unit of a
  // group, bit u of unit_first, starts it); at the group's last unit (bit u of
  // unit_last) g is added into the sums at scale 2^unit_sh[u].  A unit with
  // unit_step[u] < 0 (below the fixed-point scale) is rounded into the sums
  // on its own.
  int unit_step[band::MAX_U];
  uint32_t unit_first, unit_last;
  int8_t unit_ab[band::SB<64>::MAXS * band::SB<64>::MAXS];  // unit of slice pair (a, b), a + b <= ns - 1
  int* err;
  int* ovf;
};

template <int B>
__global__ void __launch_bounds__(band::NTB, 1)
    k_gemm_split_band(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                      BandArgs args) {
  using namespace band;
  using L = SB<B>;
  constexpr int N = L::N, TMB = L::TMB, TNB = L::TNB, RA = L::RA;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t afull[RA], aempty[RA], bfull[2], bempty[2];
  __shared__ __align__(8) uint64_t acc_full, acc_empty, drain_bar;
  __shared__ uint32_t tmem_base_slot;
  __shared__ volatile int abort_flag;
  __shared__ double partial[4][EPW / 4];
  __shared__ int32_t srec[32 * L::RECW];  // the producer's current chunk of plan records

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t smem_base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const uint32_t bbase = smem_base, abase = smem_base + 2u * (uint32_t)L::B_BUF;
  const int ntiles = *args.ntiles;
  const int ns = args.ns;
  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < RA; ++s) {
      mbar_init(smem_u32(&afull[s]), 1);
      mbar_init(smem_u32(&aempty[s]), 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(smem_u32(&bfull[s]), 1);
      mbar_init(smem_u32(&bempty[s]), 1);
    }
    mbar_init(smem_u32(&acc_full), 1);
    mbar_init(smem_u32(&acc_empty), 1);
    mbar_init(smem_u32(&drain_bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
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
    // the warp loads the next chunk of plan records while lane 0 issues the
    // copies of the current one (column sub-tile h = the chunk's repetition).
    // Per K chunk: every op(B) slice into the next buffer, then the op(A)
    // slices one ring slot each.
    int slot = 0, bb = 0;
    uint32_t phase = 0, bphase = 0;
    uint32_t issued_mask = 0, last_parity = 0, b_issued = 0, b_parity = 0;
    bool ok = true;
    RecStream<L::RECW> rs;
    rs.init(args.rec, args.rec_off, args.tile_nk, (int)blockIdx.x, (int)gridDim.x, mt, L::NSUB);
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
        const int h = c_rep;
        for (int j = 0; j < c_cnt && ok; ++j) {
          const int32_t* r = srec + j * L::RECW;
          for (int c = 0; c < L::KCH && ok; ++c) {
            if (!mbar_wait(smem_u32(&bempty[bb]), bphase ^ 1u, &abort_flag, args.err)) {
              ok = false;
              break;
            }
            const uint32_t fbb = smem_u32(&bfull[bb]);
            mbar_expect_tx(fbb, (uint32_t)(ns * L::SLOT_B));
            b_issued |= 1u << bb;
            b_parity = (b_parity & ~(1u << bb)) | (bphase << bb);
            const uint32_t sb = bbase + (uint32_t)(bb * L::B_BUF);
            for (int k = 0; k < ns; ++k) {
              const int yb = k * args.slice_rows_b;
#pragma unroll
              for (int jb = 0; jb < TNB; ++jb)
                tma_load_2d(sb + k * L::SLOT_B + jb * L::BROWS * L::ATOM, &mapB, c * L::KC,
                            yb + r[TMB + jb] * B + h * N, fbb);
            }
            if (++bb == 2) {
              bb = 0;
              bphase ^= 1u;
            }
            for (int k = 0; k < ns; ++k) {
              if (!mbar_wait(smem_u32(&aempty[slot]), phase ^ 1u, &abort_flag, args.err)) {
                ok = false;
                break;
              }
              const uint32_t fb = smem_u32(&afull[slot]);
              mbar_expect_tx(fb, (uint32_t)L::SLOT_A);
              issued_mask |= 1u << slot;
              last_parity = (last_parity & ~(1u << slot)) | (phase << slot);
              const uint32_t sa = abase + (uint32_t)(slot * L::SLOT_A);
              const int ya = k * args.slice_rows_a;
#pragma unroll
              for (int i = 0; i < TMB; ++i) tma_load_2d(sa + i * B * L::ATOM, &mapA, c * L::KC, ya + r[i] * B, fb);
              if (++slot == RA) {
                slot = 0;
                phase ^= 1u;
              }
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
    // the copies issued have landed and the MMAs have released every slot
    if (lane == 0) {
      for (int s = 0; s < RA; ++s)
        if (issued_mask & (1u << s)) {
          mbar_wait(smem_u32(&afull[s]), (last_parity >> s) & 1u, &abort_flag, args.err, false);
          mbar_wait(smem_u32(&aempty[s]), (last_parity >> s) & 1u, &abort_flag, args.err, false);
        }
      for (int s = 0; s < 2; ++s)
        if (b_issued & (1u << s)) {
          mbar_wait(smem_u32(&bfull[s]), (b_parity >> s) & 1u, &abort_flag, args.err, false);
          mbar_wait(smem_u32(&bempty[s]), (b_parity >> s) & 1u, &abort_flag, args.err, false);
        }
    }
  } else if (warp == 1) {
    // ------------------------------ MMA issuer ------------------------------
    if (lane == 0) {
      int slot = 0, bb = 0;  // ring position of the next op(A) slot, op(B) buffer
      uint32_t phase = 0, bphase = 0, acc_phase = 0;
      bool ok = true;
      int nk_next = mt > 0 ? args.tile_nk[blockIdx.x] : 0;  // loaded a tile ahead
      for (int it = 0; it < mt && ok; ++it) {
        const int t = (int)blockIdx.x + it * (int)gridDim.x;
        const int nk = nk_next;
        if (it + 1 < mt) nk_next = args.tile_nk[t + (int)gridDim.x];
        for (int h = 0; h < L::NSUB && ok; ++h) {
          for (int w0 = 0; w0 < nk && ok; w0 += args.kwin) {
            const int w1 = min(nk, w0 + args.kwin);
            // the epilogue has read the previous window's accumulators
            if (!mbar_wait(smem_u32(&acc_empty), acc_phase ^ 1u, &abort_flag, args.err)) {
              ok = false;
              break;
            }
            tc_fence_after();
            uint32_t started = 0;  // units whose accumulator holds this window's sum
            for (int j = w0; j < w1 && ok; ++j) {
              for (int c = 0; c < L::KCH && ok; ++c) {
                if (!mbar_wait(smem_u32(&bfull[bb]), bphase, &abort_flag, args.err)) {
                  ok = false;
                  break;
                }
                tc_fence_after();
                // descriptors: the start-address field (bits 0-13, address / 16)
                // of a slot's or a K step's operand is the base descriptor plus
                // its byte offset / 16 (shared addresses stay below 2^18)
                const uint64_t db0 = smem_desc_sw(bbase + (uint32_t)(bb * L::B_BUF), L::SBO, L::SWZ);
                for (int a = 0; a < ns; ++a) {
                  if (!mbar_wait(smem_u32(&afull[slot]), phase, &abort_flag, args.err)) {
                    ok = false;
                    break;
                  }
                  tc_fence_after();
                  const uint64_t da = smem_desc_sw(abase + (uint32_t)(slot * L::SLOT_A), L::SBO, L::SWZ);
                  for (int b = 0; b < ns - a; ++b) {
                    const int u = args.unit_ab[a * L::MAXS + b];
                    const uint32_t tacc = tmem + (uint32_t)(u * N);
                    const uint64_t db = db0 + (uint64_t)(b * (L::SLOT_B >> 4));
                    const uint32_t acc0 = (started >> u) & 1u;
#pragma unroll
                    for (int kk = 0; kk < L::KSTEPS; ++kk)
                      mma_kstep<2>(tacc, da + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2), IDESC, kk > 0 ? 1u : acc0);
                    started |= 1u << u;
                  }
                  mma_commit(smem_u32(&aempty[slot]));  // op(A) slice a is used up
                  if (++slot == RA) {
                    slot = 0;
                    phase ^= 1u;
                  }
                }
                if (!ok) break;
                mma_commit(smem_u32(&bempty[bb]));  // the chunk's op(B) slices are used up
                if (++bb == 2) {
                  bb = 0;
                  bphase ^= 1u;
                }
              }
            }
            if (!ok) break;
            mma_commit(smem_u32(&acc_full));
            acc_phase ^= 1u;
          }
        }
      }
      // every MMA this thread issued completes before tensor memory is released
      mma_commit(smem_u32(&drain_bar));
      mbar_wait(smem_u32(&drain_bar), 0, &abort_flag, args.err, false);
    }
  } else {
    // ------------------------------ epilogue ------------------------------
    constexpr int CW = N / (EPW / 4);        // columns per warp (16)
    const int q = warp & 3;                  // tensor-memory lane quarter
    const int cg = (warp - 2) >> 2;          // columns CW cg .. CW cg + CW - 1 of the tile
    const int rb = (q * 32) / B;             // block row of the tile (a warp's rows lie in one)
    const int rin = (q * 32) % B + lane;     // this thread's row within that block
    const int cb = (cg * CW) / B;            // block column of the tile (at bs <= 64)
    const int et = threadIdx.x - 64;
    uint32_t acc_phase = 0;
    const bool unit = (args.am == 1.0 || args.am == -1.0), neg = args.am < 0.0;
    bool good = true;
    // the tile's K-step count, its block coordinates, and the C positions of
    // this warp's block and (threads et < TMB TNB) of the block whose norm it
    // writes, loaded a tile ahead
    constexpr int CP = TMB * TNB;
    int nk_n = 0, ti_n = 0, tj_n = 0, p_n = -1, kn_n = -1;
    const auto load_next = [&](int tn) {
      nk_n = args.tile_nk[tn];
      ti_n = args.tiles[2 * tn];
      tj_n = args.tiles[2 * tn + 1];
      p_n = args.cpos[(size_t)tn * CP + rb * TNB + cb];
      if (et < CP) kn_n = args.cpos[(size_t)tn * CP + et];
    };
    if (mt > 0) load_next((int)blockIdx.x);
    for (int it = 0; it < mt && good; ++it) {
      const int t = (int)blockIdx.x + it * (int)gridDim.x;
      const int nk = nk_n;
      const int I0 = ti_n * TMB, J0 = tj_n * TNB;
      const int I = I0 + rb, J = J0 + cb;
      const int p = p_n;  // position of C_IJ in C (warp-uniform; -1: not in C)
      const int kn = kn_n;
      if (it + 1 < mt) load_next(t + (int)gridDim.x);
      SqAcc sq;  // this thread's squares over the tile's column sub-tiles
      for (int h = 0; h < L::NSUB && good; ++h) {
        const int cin = (h * N + cg * CW) % B;  // first column of this warp within block J
        long long s[CW];
#pragma unroll
        for (int e = 0; e < CW; ++e) s[e] = 0;
        bool bad = false;
        for (int w0 = 0; w0 < nk; w0 += args.kwin) {
          const bool got = mbar_wait(smem_u32(&acc_full), acc_phase, &abort_flag, args.err);
          acc_phase ^= 1u;
          if (!epi_all<32 * EPW>(got)) {  // all epilogue warps go on, or all stop
            good = false;
            break;
          }
          tc_fence_after();
          // units of equal or adjacent weight combine in 64-bit Horner
          // groups first, so a group costs one checked shift-and-add into
          // the sums instead of one per unit (8 columns at a time)
#pragma unroll
          for (int hf = 0; hf < CW / 8; ++hf) {
            long long g[8];
#pragma unroll 1
            for (int u = 0; u < args.nunits; ++u) {
              float v[8];
              tmem_ld8(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(u * N + cg * CW + hf * 8), v);
              const int sh = args.unit_sh[u], st = args.unit_step[u];
              if (st < 0) {
#pragma unroll
                for (int e = 0; e < 8; ++e) s[hf * 8 + e] = fixed_add(s[hf * 8 + e], __float2int_rn(v[e]), sh, bad);
              } else {
                if ((args.unit_first >> u) & 1u) {
#pragma unroll
                  for (int e = 0; e < 8; ++e) g[e] = (long long)__float2int_rn(v[e]);
                } else {
#pragma unroll
                  for (int e = 0; e < 8; ++e)
                    g[e] = (long long)((unsigned long long)g[e] << st) + (long long)__float2int_rn(v[e]);
                }
                if ((args.unit_last >> u) & 1u) {
#pragma unroll
                  for (int e = 0; e < 8; ++e) s[hf * 8 + e] = fixed_add64(s[hf * 8 + e], g[e], sh, bad);
                }
              }
            }
          }
          // the accumulators are read: the next window's MMAs may overwrite them
          tc_fence_before();
          epi_bar<32 * EPW>();
          if (et == 0) mbar_arrive(smem_u32(&acc_empty));
        }
        if (!good) break;
        // every K of the tile is in these sums: the FP64 result,
        // S_ij 2^(ea + e_i + e_j) * am rounded once, and its squares for the norm
        if (p >= 0) {
          const int er = args.ea + args.sige[(size_t)I * B + rin];
          const int* tj = args.taue + (size_t)J * B + cin;
          double* dst = args.cval + (size_t)p * B * B + (size_t)rin * B + cin;
#pragma unroll
          for (int e = 0; e < CW; e += 2) {
            const long long x0 = (unit && neg) ? -s[e] : s[e], x1 = (unit && neg) ? -s[e + 1] : s[e + 1];
            double v0 = i64_ldexp(x0, er + tj[e]), v1 = i64_ldexp(x1, er + tj[e + 1]);
            if (!unit) {
              v0 *= args.am;
              v1 *= args.am;
            }
            sq.add_f64(v0);
            sq.add_f64(v1);
            *reinterpret_cast<double2*>(dst + e) = make_double2(v0, v1);
          }
          if (bad) *args.ovf = 2;
        }
      }
      if (!good) break;
      const double ss = sq.warp_total();
      if (lane == 0) partial[q][cg] = ss;
      epi_bar<32 * EPW>();
      // norms: block (br, bc) of the tile sums the warps of its lane quarters
      // and column groups, in a fixed order
      if (et < CP && kn >= 0) {
        const int br = et / TNB, bc = et % TNB;
        // the lane quarters qq with (32 qq) / B == br and column groups cc
        // with (CW cc) / B == bc, in increasing order
        const int q1 = (br + 1) * B / 32 < 4 ? (br + 1) * B / 32 : 4;
        const int c1 = (bc + 1) * B / CW < EPW / 4 ? (bc + 1) * B / CW : EPW / 4;
        double sum = 0.0;
        for (int qq = br * B / 32; qq < q1; ++qq)
          for (int cc = bc * B / CW; cc < c1; ++cc) sum += partial[qq][cc];
        args.cnorm[kn] = sqrt(sum);
      }
      epi_bar<32 * EPW>();
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(band::TMEM_COLS));
  }
}

// Accumulation units of a split product with ns slices per operand: slice
// pairs (s, t), s + t <= ns + 1, of equal weight 2^(-7 (s + t)) packed
// greedily while sum over the unit of max|q_s| max|q_t| * 64 * kw stays
// <= 2^24, kw = the K blocks a window holds (KW, or the longest tile's K
// steps when fewer), so that every FP32 accumulator sums integers exactly.
struct UnitTable {
  int nunits = 0, npairs = 0;
  int unit_end[MAX_UNITS] = {};  // pairs of unit u: [unit_end[u - 1], unit_end[u])
  int unit_g[MAX_UNITS] = {};    // weight class s + t of unit u
  int si[MAX_PAIRS] = {}, ti[MAX_PAIRS] = {}, pu[MAX_PAIRS] = {};  // slices (1-based) and unit of each pair
};

static UnitTable unit_table(int ns, int kw, int bs) {
  UnitTable t;
  const auto qmax = [](int s) { return s == 1 ? 128 : 64; };
  const int64_t cap = ((int64_t)1 << 24) / ((int64_t)bs * std::max(1, kw));
  for (int g = 2; g <= ns + 1; ++g) {
    int64_t used = 0;
    bool open = false;
    for (int s = 1; s < g; ++s) {
      const int u = g - s;
      if (s > ns || u > ns) continue;
      const int64_t cost = (int64_t)qmax(s) * qmax(u);
      if (open && used + cost > cap) {
        t.unit_end[t.nunits++] = t.npairs;
        used = 0;
        open = false;
      }
      if (!open) {
        if (t.nunits >= MAX_UNITS) fail(IFAC_ERR_UNSUPPORTED, "split product: too many accumulation units");
        t.unit_g[t.nunits] = g;
        open = true;
      }
      if (t.npairs >= MAX_PAIRS) fail(IFAC_ERR_UNSUPPORTED, "split product: too many slice pairs");
      t.si[t.npairs] = s;
      t.ti[t.npairs] = u;
      t.pu[t.npairs] = t.nunits;
      ++t.npairs;
      used += cost;
    }
    if (open) t.unit_end[t.nunits++] = t.npairs;
  }
  return t;
}

template <int B>
static void launch_split_band(ifac_ctx* ctx, const CUtensorMap& mA, const CUtensorMap& mB, const BandArgs& ba,
                              int tiles_bound, int sms) {
  using L = band::SB<B>;
  static std::atomic<unsigned long long> attr{0};
  if (first_on_device(attr, ctx->device))
    IFAC_CK(cudaFuncSetAttribute(k_gemm_split_band<B>, cudaFuncAttributeMaxDynamicSharedMemorySize, L::SMEM_BYTES));
  const int grid = (int)std::min<int64_t>(std::max(tiles_bound, 1), sms);
  k_gemm_split_band<B><<<grid, band::NTB, L::SMEM_BYTES, ctx->stream>>>(mA, mB, ba);
  IFAC_CK_LAUNCH();
}

static void run_split(ifac_ctx* ctx, int ns, const View& arows, bool tA, const ifac_bsr& A, const View& brows,
                      bool tB, const ifac_bsr& B, double alpha, ifac_bsr& C, const int32_t* crow, bool upper,
                      unsigned long long* pairs, OperandCache* ac, OperandCache* bc, const int32_t* avmap,
                      const int32_t* bvmap) {
  Buf<int32_t> asrc, bsrc;  // value positions of op(A) / op(B) view entries under value maps
  using Cf = Cfg<2>;
  const int nb = A.nb, bs = A.bs;
  const int64_t rows = (int64_t)nb * bs;
  if (ns < 1 || ns > 8) fail(IFAC_ERR_UNSUPPORTED, "split product: 1 to 8 slices");
  // a cache filled by an earlier product's op(B) (transposed blocks in the
  // stored order, with that operand's column scales) serves op(A) = that
  // matrix transposed, through the view's source indices, and nothing else
  if (ac && ac->from_b && !(tA && ac->split_ns >= ns)) ac = nullptr;
  const int32_t* amap = (ac && ac->from_b) ? arows.src : nullptr;
  // scales: sigma (rows of op(A)), tau (columns of op(B) = rows of op(B)^T);
  // op(A)'s scales and slices come from the cache when it holds at least ns
  const bool hit = ac && ac->split_ns >= ns;
  const int nsa = hit ? ac->split_ns : (ac ? std::min(8, std::max(ns, ac->want_ns)) : ns);
  Buf<int> sige, taue(ctx, rows);
  // [0] / [1]: scaled 1-norm bounds of op(A) rows / op(B) columns, [2] / [3]: 2-norm bounds
  Buf<unsigned int> l1(ctx, 4);
  IFAC_CK(cudaMemsetAsync(l1.p, 0, 4 * sizeof(unsigned int), ctx->stream));
  if (!hit) {
    sige = Buf<int>(ctx, rows);
    row_scales(ctx, bs, arows.rp, value_src(ctx, arows.src, avmap, A.nnzb, asrc), nb, tA, A.val, sige.p, l1.p,
               l1.p + 2);
  }
  {
    View bt = view_rows(ctx, B, !tB);
    Buf<int32_t> btsrc;
    row_scales(ctx, bs, bt.rp, value_src(ctx, bt.src, bvmap, B.nnzb, btsrc), nb, !tB, B.val, taue.p, l1.p + 1,
               l1.p + 3);
  }
  // slices: row scale block of an op(A) entry is its CSR row; of an op(B) entry its CSR column
  const size_t bbytes = (size_t)bs * bs * 2;
  Buf<uint8_t> la, lb(ctx, (size_t)ns * (B.nnzb + 1) * bbytes);
  for (int k = 0; k < ns; ++k)
    IFAC_CK(cudaMemsetAsync(lb.p + ((size_t)k * (B.nnzb + 1) + B.nnzb) * bbytes, 0, bbytes, ctx->stream));
  if (!hit) {
    la = Buf<uint8_t>(ctx, (size_t)nsa * (A.nnzb + 1) * bbytes);
    for (int k = 0; k < nsa; ++k)
      IFAC_CK(cudaMemsetAsync(la.p + ((size_t)k * (A.nnzb + 1) + A.nnzb) * bbytes, 0, bbytes, ctx->stream));
    if (A.nnzb) {
      Buf<int32_t> arow(ctx, A.nnzb);
      expand_rows(ctx, arows.rp, nb, arow.p);
      split_blocks(ctx, bs, A.val, value_src(ctx, arows.src, avmap, A.nnzb, asrc), A.nnzb, tA, arow.p, sige.p, nsa,
                   la.p);
    }
  }
  uint8_t* const la_p = hit ? ac->split.p : la.p;
  const int* const sige_p = hit ? ac->sexp.p : sige.p;
  const int* const taue_p = taue.p;
  if (B.nnzb)
    split_blocks(ctx, bs, B.val, value_src(ctx, brows.src, bvmap, B.nnzb, bsrc), B.nnzb, !tB, brows.ci, taue.p, ns,
                 lb.p);
  // one tensor map over all slices of each operand (slice s at row s (nnzb + 1) bs)
  if ((int64_t)ns * (std::max(A.nnzb, B.nnzb) + 1) * bs > (int64_t)0x7fffffff)
    fail(IFAC_ERR_TOO_LARGE, "split product: slice copies exceed the 2^31-row tensor-map range");
  // tile plans: narrow tiles (128 x 64) first.  At bs 64 a product whose
  // tiles all fit one window with at most band::MAX_U units runs on the
  // narrow kernel, every other one on the windowed super-tile kernel; at bs
  // 32 and 128 every product runs on the narrow kernel, window by window.
  // The context's schedule can ask for super-tiles only at bs 64, or narrow
  // tiles (window by window) up to another K length.
  float l1h[4] = {0.f, 0.f, 0.f, 0.f};  // scaled 1- and 2-norm bounds (as l1 above)
  const HostRead l1read{l1h, l1.p, sizeof(l1h)};
  // the default (-1): narrow tiles for every product; with the op(B) slices
  // of a chunk resident and the op(A) slices streamed they are faster than
  // super-tiles on dense products too (3D cluster, n = 16,384: 1.77 s
  // against 2.26 s of split kernel per refinement)
  const int nk_lim = ctx->narrow_kmax_split < 0 ? INT_MAX : ctx->narrow_kmax_split;
  Plan Pb;
  bool banded = bs != 64;
  if (bs != 64 || nk_lim > 0) {
    Pb = band_plan(ctx, bs, arows, A, tA, brows, B, C, crow, bs == 64 && nk_lim < INT_MAX ? nk_lim : 0, amap,
                   &l1read);
    if (bs == 64) banded = Pb.kmax >= 1 && Pb.kmax <= nk_lim;
  } else {
    to_host(ctx, l1h, l1.p, sizeof(l1h));
  }
  Plan P;
  if (!banded) P = make_plan<PAIR * TM, Cf::TN>(ctx, arows, A, tA, brows, B, C, crow, true, 0, amap);
  // block pairs, and block pairs times the ns (ns + 1) / 2 slice pairs
  k_count_pairs<<<cdiv((int64_t)nb * 32, 256), 256, 0, ctx->stream>>>(arows.rp, arows.ci, nb, brows.rp, brows.ci,
                                                                      upper ? 1 : 0, pairs, pairs + 1,
                                                                      ns * (ns + 1) / 2);
  IFAC_CK_LAUNCH();
  const int kmax = banded ? Pb.kmax : P.kmax;
  if (hit) {
    l1h[0] = ac->l1;
    l1h[2] = ac->l2;
  } else if (ac) {
    ac->l1 = l1h[0];
    ac->l2 = l1h[2];
    ac->split = std::move(la);
    ac->sexp = std::move(sige);
    ac->split_ns = nsa;
  }
  uint8_t* const lb_p = lb.p;
  if (bc && !tB) {  // op(B) = B in its stored order: keep its slices for a later op(A) = B^T
    bc->reset();
    bc->split = std::move(lb);
    bc->sexp = std::move(taue);
    bc->l1 = l1h[1];
    bc->l2 = l1h[3];
    bc->split_ns = ns;
    bc->from_b = true;
  }
  // window of the narrow kernel: the K blocks (at most 1024 K elements) for
  // which every unit stays exact, as long as at most band::MAX_U units
  // result; the longest tile's K blocks when fewer
  int kwin = std::min(1024 / bs, std::max(kmax, 1));
  while (kwin > 1 && unit_table(ns, kwin, bs).nunits > band::MAX_U) --kwin;
  // the windowed kernel adds into zeroed 64-bit sums that a second kernel
  // converts; the narrow kernel holds each tile's complete sums and writes FP64
  Buf<longlong2> part;
  if (!banded) {
    part = Buf<longlong2>(ctx, (size_t)C.nnzb * (BS * BS / 2));
    IFAC_CK(cudaMemsetAsync(part.p, 0, sizeof(longlong2) * (size_t)C.nnzb * (BS * BS / 2), ctx->stream));
  }
  int ea_alpha = 0;
  const double am = std::frexp(alpha, &ea_alpha) * 2.0;  // alpha = am 2^(ea_alpha - 1), am in [1, 2)
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
  // fixed point, scale 2^-f relative to sigma_i tau_j, with every partial sum
  // below 2^62: |sum_ij| <= min(sum_k |a_ik| / sigma_i, sum_k |b_kj| / tau_j)
  // (|a / sigma|, |b / tau| < 1), bounded by the largest scaled row / column
  // 1-norm (FP32, so with a margin), by the scalar inner length K of the
  // longest tile, and (Cauchy-Schwarz) by the product of the largest scaled
  // row and column 2-norms, each widened by 0.0125 sqrt(K) for the slices'
  // rounding (sum_s |q_s| 2^-7s exceeds |a / sigma| by at most 0.0125).  The
  // 2-norm bound is the tight one for dense operands, where every bit of f
  // saved is a rounding the finest accumulation units escape in each window.
  // f <= 56 keeps every weight 2^(f - 7g) of the 7-slice product integral.
  // An overflow would still be detected and reported.
  int lgK = 0;
  while (((int64_t)1 << lgK) < (int64_t)std::max(kmax, 1) * bs) ++lgK;
  const double rk = 0.0125 * std::sqrt((double)std::max(kmax, 1) * bs);
  const double l2b = ((double)l1h[2] + rk) * ((double)l1h[3] + rk);
  const double l1b = std::min(std::min((double)l1h[0], (double)l1h[1]), l2b) * 1.125 + 2.0;
  int lgB = 0;
  while (std::ldexp(1.0, lgB) < l1b && lgB < 62) ++lgB;
  const int fbits = std::min(56, 62 - std::min(lgK, lgB));
  // units: a window of kw K blocks (every window of every tile has at most kw
  // blocks, so each FP32 accumulator sums integers of magnitude <= 2^24
  // exactly)
  const UnitTable ut = banded ? unit_table(ns, kwin, bs) : unit_table(ns, std::min(KW, std::max(kmax, 1)), bs);
  prof_begin(ctx, 2);
  if (banded) {
    BandArgs ba{};
    ba.tiles = Pb.tiles.p;
    ba.ntiles = Pb.coff.p + Pb.nchunk;
    ba.tile_nk = Pb.tnk.p;
    ba.rec = Pb.rec.p;
    ba.rec_off = Pb.off.p;
    ba.cpos = Pb.cpos.p;
    ba.cval = C.val;
    ba.cnorm = C.norms;
    ba.sige = sige_p;
    ba.taue = taue_p;
    ba.ea = ea_alpha - 1 - fbits;
    ba.am = am;
    ba.nb = nb;
    ba.ns = ns;
    ba.kwin = kwin;
    ba.slice_rows_a = (int)(A.nnzb + 1) * bs;
    ba.slice_rows_b = (int)(B.nnzb + 1) * bs;
    ba.nunits = ut.nunits;
    if (ut.nunits > band::MAX_U) fail(IFAC_ERR_UNSUPPORTED, "split product: too many units for the narrow kernel");
    for (int u = 0; u < ut.nunits; ++u) ba.unit_sh[u] = fbits - SPLIT_BITS * ut.unit_g[u];
    // Horner groups: consecutive units with shifts >= 0 (descending, so each
    // step is 0 or 7 bits); a group's value is below ngroup 2^(24 + span),
    // kept within int64 by a span of at most 35 bits with at most 8 units
    {
      ba.unit_first = ba.unit_last = 0u;
      int start = -1;
      for (int u = 0; u < ut.nunits; ++u) {
        const int sh = ba.unit_sh[u];
        if (sh < 0) {
          if (start >= 0) ba.unit_last |= 1u << (u - 1);
          start = -1;
          ba.unit_step[u] = -1;
          continue;
        }
        if (start >= 0 && ba.unit_sh[start] - sh <= 35) {
          ba.unit_step[u] = ba.unit_sh[u - 1] - sh;
        } else {
          if (start >= 0) ba.unit_last |= 1u << (u - 1);
          start = u;
          ba.unit_first |= 1u << u;
          ba.unit_step[u] = 0;
        }
      }
      if (start >= 0) ba.unit_last |= 1u << (ut.nunits - 1);
    }
    // the unit of each slice pair (a, b) with a + b <= ns - 1 (0-based)
    for (int k = 0; k < band::SB<64>::MAXS * band::SB<64>::MAXS; ++k) ba.unit_ab[k] = -1;
    for (int p = 0; p < ut.npairs; ++p) {
      const int a = ut.si[p] - 1, b = ut.ti[p] - 1;
      if (a < 0 || b < 0 || a + b > ns - 1) fail(IFAC_ERR_CUDA, "split product: slice pair outside the table");
      ba.unit_ab[a * band::SB<64>::MAXS + b] = (int8_t)ut.pu[p];
    }
    for (int a = 0; a < ns; ++a)
      for (int b = 0; b < ns - a; ++b)
        if (ba.unit_ab[a * band::SB<64>::MAXS + b] < 0)
          fail(IFAC_ERR_CUDA, "split product: inconsistent banded issue table");
    ba.err = ctx->dev_err;
    ba.ovf = ctx->dev_err;
    const int kc = bs < 64 ? bs : 64;  // K elements per chunk (band::SB<bs>::KC)
    const CUtensorMap mA = make_map_box(bs, la_p, (int64_t)ns * (A.nnzb + 1), kc, bs);
    const CUtensorMap mB = make_map_box(bs, lb_p, (int64_t)ns * (B.nnzb + 1), kc, bs < 64 ? bs : 64);
    if (bs == 32) launch_split_band<32>(ctx, mA, mB, ba, Pb.ntiles, sms);
    else if (bs == 64) launch_split_band<64>(ctx, mA, mB, ba, Pb.ntiles, sms);
    else launch_split_band<128>(ctx, mA, mB, ba, Pb.ntiles, sms);
  } else {
    const CUtensorMap mA = make_map<2>(la_p, (int64_t)ns * (A.nnzb + 1));
    const CUtensorMap mB = make_map<2>(lb_p, (int64_t)ns * (B.nnzb + 1));
    static std::atomic<unsigned long long> attr{0};
    if (first_on_device(attr, ctx->device))
      IFAC_CK(cudaFuncSetAttribute(k_gemm_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cf::SMEM_BYTES));
    TileArgs args{};
    args.tiles = P.tiles.p;
    args.ntiles = P.coff.p + P.nchunk;
    args.tile_nk = P.tnk.p;
    args.nwin = cdiv(std::max(kmax, 1), KW);
    args.nb = nb;
    args.rec = P.rec.p;
    args.rec_off = P.off.p;
    args.crp = C.row_ptr;
    args.cci = C.col_idx;
    args.cval = C.val;
    args.cnorm = C.norms;
    args.alpha = 1.0;
    args.err = ctx->dev_err;
    args.split = 1;
    args.cpart = part.p;
    args.stall = 0;
    args.wait_limit = WAIT_LIMIT;
    args.nunits = ut.nunits;
    for (int u = 0; u < ut.nunits; ++u) {
      args.unit_end[u] = ut.unit_end[u];
      args.unit_sh[u] = fbits - SPLIT_BITS * ut.unit_g[u];
    }
    for (int p = 0; p < ut.npairs; ++p) {
      args.pair_ya[p] = (ut.si[p] - 1) * (int)(A.nnzb + 1) * BS;
      args.pair_yb[p] = (ut.ti[p] - 1) * (int)(B.nnzb + 1) * BS;
    }
    args.ovf = ctx->dev_err;
    const int64_t pairs_grid = std::min<int64_t>(std::max(P.ntiles, 1), sms / PAIR);
    k_gemm_tc<2><<<(unsigned)(pairs_grid * PAIR), NTHREADS, Cf::SMEM_BYTES, ctx->stream>>>(mA, mB, args);
    IFAC_CK_LAUNCH();
  }
  prof_end(ctx);
  ++ctx->split_launches;
  if (!banded) {
    k_split_finish<<<(int)std::min<int64_t>(C.nnzb, 152 * 16), 256, 0, ctx->stream>>>(
        crow, C.col_idx, C.nnzb, part.p, C.val, sige_p, taue_p, ea_alpha - 1 - fbits, am, C.norms);
    IFAC_CK_LAUNCH();
  }
}

// Failure-path self-test of the bounded waits: one pair of CTAs over a
// one-tile product (1 x 1 blocks of a 64-row matrix) whose producer and MMA
// issuer do no work, so the epilogue's accumulator wait expires after
// wait_limit polls.  Nothing is copied or multiplied; every CTA releases its
// tensor memory and returns, and the host sees the device error flag.
static void stall_selftest(ifac_ctx* ctx, long long wait_limit) {
  using Cf = Cfg<2>;
  Buf<uint8_t> zeros(ctx, (size_t)2 * BS * BS * 2);
  IFAC_CK(cudaMemsetAsync(zeros.p, 0, zeros.n, ctx->stream));
  const CUtensorMap m = make_map<2>(zeros.p, 2);
  // tiles {0, 0}; one tile; one K step; plan records all zero; C pattern: one block
  Buf<int32_t> small(ctx, 32);
  const int32_t host[32] = {0, 0, /*ntiles*/ 1, /*nk*/ 1, /*rec_off*/ 0, 1, /*crp*/ 0, 1, /*cci*/ 0};
  IFAC_CK(cudaMemcpyAsync(small.p, host, sizeof(host), cudaMemcpyHostToDevice, ctx->stream));
  Buf<double> cval(ctx, (size_t)BS * BS + 1);
  TileArgs args{};
  args.tiles = small.p;
  args.ntiles = small.p + 2;
  args.tile_nk = small.p + 3;
  args.nwin = 1;
  args.nb = 1;
  args.rec = small.p + 9;  // zeros
  args.rec_off = small.p + 4;
  args.crp = small.p + 6;
  args.cci = small.p + 8;
  args.cval = cval.p;
  args.cnorm = cval.p + BS * BS;
  args.alpha = 1.0;
  args.err = ctx->dev_err;
  args.split = 0;
  args.stall = 1;
  args.wait_limit = wait_limit;
  static std::atomic<unsigned long long> attr{0};
  if (first_on_device(attr, ctx->device))
    IFAC_CK(cudaFuncSetAttribute(k_gemm_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cf::SMEM_BYTES));
  k_gemm_tc<2><<<PAIR, NTHREADS, Cf::SMEM_BYTES, ctx->stream>>>(m, m, args);
  IFAC_CK_LAUNCH();
  IFAC_CK(cudaStreamSynchronize(ctx->stream));
}

}  // namespace tc

void tc_wait_timeout_selftest(ifac_ctx* ctx, long long wait_limit) { tc::stall_selftest(ctx, wait_limit); }

void gemm_numeric_tc(ifac_ctx* ctx, int prec, const View& arows, bool tA, const ifac_bsr& A, const View& brows,
                     bool tB, const ifac_bsr& B, double alpha, ifac_bsr& C, const int32_t* crow, bool upper,
                     unsigned long long* pairs_dev, OperandCache* acache, OperandCache* bcache,
                     const OperandCache* bpre, const int32_t* avmap, const int32_t* bvmap, bool out32, bool b32) {
  if (C.nnzb == 0) return;
  if ((out32 || b32) && prec != IFAC_TF32 && prec != IFAC_BF16)
    fail(IFAC_ERR_INVALID, "FP32 values: TF32/BF16 products only");
  if (A.bs != 32 && A.bs != 64 && A.bs != 128) fail(IFAC_ERR_UNSUPPORTED, "tensor-core block products: bs 32, 64 or 128");
  if (!B.val && !(bpre && bpre->b_ready)) fail(IFAC_ERR_INVALID, "tensor-core product: op(B) has no values");
  if (prec == IFAC_BF16)
    tc::run<2>(ctx, arows, tA, A, brows, tB, B, alpha, C, crow, upper, pairs_dev, acache, bcache, bpre, avmap, bvmap,
               out32, b32);
  else if (prec == IFAC_TF32)
    tc::run<4>(ctx, arows, tA, A, brows, tB, B, alpha, C, crow, upper, pairs_dev, acache, bcache, bpre, avmap, bvmap,
               out32, b32);
  else if (prec == IFAC_FP64_SPLIT)
    tc::run_split(ctx, ctx->split_slices, arows, tA, A, brows, tB, B, alpha, C, crow, upper, pairs_dev, acache,
                  bcache, avmap, bvmap);
  else fail(IFAC_ERR_UNSUPPORTED, "unknown precision");
}

// the mixed schedule's P at m = 2 as a low-precision op(B) copy (k_poly2_lp)
void poly2_lp(ifac_ctx* ctx, int elt, const ifac_bsr& U, const ifac_bsr& D, double b1, double b2,
              const ifac_bsr& P, const int32_t* prow, void* out, const int32_t* umap, bool u32) {
  if (U.bs != 64) fail(IFAC_ERR_UNSUPPORTED, "correction operand: bs 64");
  const size_t bb = (size_t)64 * 64 * elt;
  IFAC_CK(cudaMemsetAsync(static_cast<uint8_t*>(out) + (size_t)P.nnzb * bb, 0, bb, ctx->stream));
  if (P.nnzb == 0) return;
  const int grid = (int)std::min<int64_t>(P.nnzb, 152 * 8);
  const float* u32v = reinterpret_cast<const float*>(U.val);
  if (elt == 2 && u32)
    tc::k_poly2_lp<2, float><<<grid, 256, 0, ctx->stream>>>(prow, P.col_idx, P.nnzb, U.row_ptr, U.col_idx, u32v, umap,
                                                             D.row_ptr, D.col_idx, D.val, (float)b1, (float)b2, out);
  else if (elt == 2)
    tc::k_poly2_lp<2, double><<<grid, 256, 0, ctx->stream>>>(prow, P.col_idx, P.nnzb, U.row_ptr, U.col_idx, U.val,
                                                              umap, D.row_ptr, D.col_idx, D.val, (float)b1, (float)b2,
                                                              out);
  else if (u32)
    tc::k_poly2_lp<4, float><<<grid, 256, 0, ctx->stream>>>(prow, P.col_idx, P.nnzb, U.row_ptr, U.col_idx, u32v, umap,
                                                             D.row_ptr, D.col_idx, D.val, (float)b1, (float)b2, out);
  else
    tc::k_poly2_lp<4, double><<<grid, 256, 0, ctx->stream>>>(prow, P.col_idx, P.nnzb, U.row_ptr, U.col_idx, U.val,
                                                              umap, D.row_ptr, D.col_idx, D.val, (float)b1, (float)b2,
                                                              out);
  IFAC_CK_LAUNCH();
}

}  // namespace ifac
