// tc_common.cuh -- device helpers shared by the tensor-core product kernels
// (gemm_tc.cu, gemm_band.cu): mbarrier waits with a poll bound, TMA loads,
// shared-memory and instruction descriptors of tcgen05.mma (K-major
// operands, 128-byte swizzle), tensor-memory loads, and the integer-only
// conversions between FP64, FP32, TF32 and BF16 bit patterns.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cstdint>

namespace ifac {
namespace tc {

constexpr long long WAIT_LIMIT = 1ll << 27;  // polls of one bounded wait

// ---------------------------------------------------------------------------
// PTX helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: true when the phase of `parity` completed; false on the CTA's
// abort flag or (after `limit` polls) on timeout, which raises both flags.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* gerr,
                                          bool honour_abort = true, long long limit = WAIT_LIMIT) {
  for (long long i = 0; i < limit; ++i) {
    if (mbar_try(bar, parity)) return true;
    if (honour_abort && *abort_flag) return false;
  }
  *abort_flag = 1;
  atomicExch(gerr, 1);
  return false;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;                   // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;         // stride byte offset
  d |= (uint64_t)1 << 46;                   // version
  d |= (uint64_t)2 << 61;                   // 128-byte swizzle
  return d;
}

// the same for another swizzle: sbo = the 8-row group stride (8 x the atom
// row), swz = descriptor layout type (2: 128-byte swizzle, 4: 64-byte)
__device__ __forceinline__ uint64_t smem_desc_sw(uint32_t addr, uint32_t sbo, uint32_t swz) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;                   // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(sbo >> 4) << 32;          // stride byte offset: 8-row groups
  d |= (uint64_t)1 << 46;                   // version
  d |= (uint64_t)swz << 61;                 // swizzle mode
  return d;
}

// Instruction descriptor: FP32 accumulate, A/B format (ELT bytes: 2 BF16,
// 4 TF32), both K-major, N x M.
template <int ELT, int N, int M>
__host__ __device__ constexpr uint32_t idesc_of() {
  return (1u << 4)                                       // D = F32
         | ((ELT == 2 ? 1u : 2u) << 7)                   // A = BF16 / TF32
         | ((ELT == 2 ? 1u : 2u) << 10)                  // B = BF16 / TF32
         | ((uint32_t)(N >> 3) << 17)                    // N
         | ((uint32_t)(M >> 4) << 24);                   // M
}

// D (tensor memory) (+)= A B for one K step of 32 bytes, single CTA
template <int ELT>
__device__ __forceinline__ void mma_kstep(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  if constexpr (ELT == 2) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
  }
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 lanes x 32 columns of FP32 from tensor memory into 32 registers
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// FP32 -> FP64 by moving the fields (exact, subnormals normalised; inf and
// NaN take the conversion instruction), keeping the epilogue off the FP64 pipe
__device__ __forceinline__ double f32_to_f64(float f);

// f 2^-64 as FP64 (exact: the result is far inside FP64's normal range), on
// the bit pattern for zeros and normal values; subnormal, inf and NaN inputs
// (never seen in the sums below) take the general route
__device__ __forceinline__ double f32_to_f64_m64(float f) {
  const uint32_t u = __float_as_uint(f);
  if ((u & 0x7fffffffu) == 0u) return __hiloint2double((int)(u & 0x80000000u), 0);
  const uint32_t ex = (u >> 23) & 0xffu;
  if (ex == 0u || ex == 0xffu) return f32_to_f64(f) * 5.421010862427522e-20;  // 2^-64
  const uint32_t hi = (u & 0x80000000u) | ((ex + 896u - 64u) << 20) | ((u & 0x7fffffu) >> 3);
  return __hiloint2double((int)hi, (int)(u << 29));
}

__device__ __forceinline__ double f32_to_f64(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t sign = u & 0x80000000u, ex = (u >> 23) & 0xffu, man = u & 0x7fffffu;
  if (ex == 0xffu) return (double)f;  // inf, NaN
  if (ex == 0u) {
    if (man == 0u) return __hiloint2double((int)sign, 0);
    // subnormal: man 2^-149 with man < 2^23, normal in FP64
    const int len = 32 - __clz((int)man);                       // bit length, 1..23
    const uint32_t e64 = (uint32_t)(len - 1 - 149 + 1023);      // exponent field
    const unsigned long long m52 = ((unsigned long long)man << (53 - len)) & 0xfffffffffffffull;
    return __hiloint2double((int)(sign | (e64 << 20) | (uint32_t)(m52 >> 32)), (int)(uint32_t)m52);
  }
  const uint32_t hi = sign | ((ex + 896u) << 20) | (man >> 3);
  return __hiloint2double((int)hi, (int)(u << 29));
}

// d + x 2^sh in 64-bit integers, x 2^sh rounded half up when sh < 0
// (|x| <= 2^24); `bad` records a signed overflow of the term or the sum
__device__ __forceinline__ long long fixed_add(long long d, int x, int sh, bool& bad) {
  long long t;
  if (sh >= 0) {
    t = (long long)((unsigned long long)(long long)x << sh);
    bad |= (t >> sh) != (long long)x;
  } else {
    t = (sh < -30) ? 0 : (long long)((x + (1 << (-sh - 1))) >> (-sh));
  }
  const long long r = (long long)((unsigned long long)d + (unsigned long long)t);
  bad |= ((d ^ r) & (t ^ r)) < 0;
  return r;
}

// d + (x << sh) for a 64-bit x, sh >= 0, flagging a shift or sum that
// overflows
__device__ __forceinline__ long long fixed_add64(long long d, long long x, int sh, bool& bad) {
  const long long t = (long long)((unsigned long long)x << sh);
  bad |= (t >> sh) != x;
  const long long r = (long long)((unsigned long long)d + (unsigned long long)t);
  bad |= ((d ^ r) & (t ^ r)) < 0;
  return r;
}

// Sum of squares of FP32 values for the block norms that truncation tests,
// accurate to about 2^-42 relative without the FP64 pipe: each square of
// x 2^32 is split exactly into p + e (FMA), p is added to the running sum with
// an error-free two-sum, and the errors are collected in a second FP32 word.
// The scale 2^32 keeps squares of |x| in [2^-95, 2^28) normal, and 64 of
// them finite; larger magnitudes (rare) are squared in FP64, smaller ones
// contribute below 2^-190 each.
struct SqAcc {
  float hi = 0.0f, lo = 0.0f;
  double big = 0.0;
  // |x| < 2^28 (the caller checks a whole chunk first)
  __device__ __forceinline__ void add_small(float x) {
    const float y = x * 4294967296.0f;
    const float p = y * y;
    const float e = fmaf(y, y, -p);
    const float s = hi + p;
    const float bp = s - hi;
    const float err = (hi - (s - bp)) + (p - bp);
    hi = s;
    lo += err + e;
  }
  // K values: the FP32 path when all are below 2^28 (the usual case), else
  // FP64 squares (a separate branch of K FP64 FMAs)
  template <int K>
  __device__ __forceinline__ void add(const float (&v)[K]) {
    float mx = 0.0f;
#pragma unroll
    for (int i = 0; i < K; ++i) mx = fmaxf(mx, fabsf(v[i]));
    if (mx < 268435456.0f) {
#pragma unroll
      for (int i = 0; i < K; ++i) add_small(v[i]);
    } else {
#pragma unroll
      for (int i = 0; i < K; ++i) big = fma((double)v[i], (double)v[i], big);
    }
  }
  __device__ __forceinline__ void add32(const float (&v)[32]) { add<32>(v); }
  // an FP64 value, squared through FP32 without the FP64 pipe: its top 24
  // significand bits hi and the next 29 bits lo (rounded to 24) give
  // v^2 = hi^2 + 2 hi lo + lo^2 with lo^2 < 2^-46 v^2 left out.  |v| in
  // [2^-95, 2^28): FP32 path (lo dropped below 2^-74); larger: FP64; smaller:
  // below 2^-190 each, left out.
  __device__ __forceinline__ void add_f64(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int f = (int)((b >> 52) & 0x7ffu);
    if (f >= 1023 - 95 && f < 1023 + 28) {
      // hi 2^32 and lo 2^32 (exponent fields offset by +32)
      const float y = __uint_as_float(((uint32_t)(f - 896 + 32) << 23) | (uint32_t)((b >> 29) & 0x7fffffu));
      const float z = f >= 949 ? __int2float_rn((int)(b & 0x1fffffffu)) *
                                     __uint_as_float((uint32_t)(f - 948 + 32) << 23)
                               : 0.0f;
      const float p = y * y;
      const float e = fmaf(y, y, -p);
      const float c = 2.0f * y * z;
      const float s = hi + p;
      const float bp = s - hi;
      const float err = (hi - (s - bp)) + (p - bp);
      hi = s;
      lo += err + (e + c);
    } else if (f >= 1023 + 28) {
      big = fma(v, v, big);
    }
  }
  // the sum over the warp's 32 lanes (every lane gets it): hi and lo reduced
  // in FP32 with error-free two-sums, converted once; the FP64 part only when
  // some lane holds one
  __device__ __forceinline__ double warp_total() const {
    float h = hi, l = lo;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float h2 = __shfl_xor_sync(0xffffffffu, h, o), l2 = __shfl_xor_sync(0xffffffffu, l, o);
      const float s = h + h2;
      const float bp = s - h;
      const float err = (h - (s - bp)) + (h2 - bp);
      h = s;
      l = l + l2 + err;
    }
    // (h + l) 2^-64 rounded once, as ((double)h + (double)l) 2^-64: the
    // scaling moves to the exponent fields, so one FP64 add remains
    double r = f32_to_f64_m64(h) + f32_to_f64_m64(l);
    if (__any_sync(0xffffffffu, __double_as_longlong(big) != 0)) {  // big >= +0
      double bsum = big;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) bsum += __shfl_xor_sync(0xffffffffu, bsum, o);
      r += bsum;
    }
    return r;
  }
  __device__ __forceinline__ double value() const {
    return (f32_to_f64_m64(hi) + f32_to_f64_m64(lo)) + big;  // (hi + lo) 2^-64 + big
  }
};

// named barrier 1 over the NT epilogue threads
template <int NT>
__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory"); }

// the same barrier with a vote: true on every epilogue thread iff `v` is true
// on all of them, so that all leave a loop together (a named barrier that only
// some of its threads reach would never complete)
template <int NT>
__device__ __forceinline__ bool epi_all(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
      "bar.red.and.pred q, 1, %2, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(NT)
      : "memory");
  return r != 0;
}

__device__ __forceinline__ int lower_bound_i32(const int32_t* __restrict__ a, int lo, int hi, int v) {
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (a[mid] < v) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Plan records streamed to a producer warp.  A CTA's tiles are t0, t0 + tstep,
// ... (mt of them); each tile's records are visited `reps` times in a row (the
// column sub-tiles of a split product at bs 128) in chunks of up to 32 K
// steps.  next() has the 32 lanes load one chunk (lane j: the record of K step
// j0 + j) into registers and moves on; the producer calls it for the following
// chunk before lane 0 issues the copies of the current one, so the loads are
// in flight while lane 0 waits on the ring, and no record load sits on the
// issue path.  The next tile's K-step count and record offset are loaded as
// soon as its predecessor's last chunk has been handed out.
template <int RECW>
struct RecStream {
  const int32_t* rec;
  const int32_t* rec_off;
  const int32_t* tile_nk;
  int t0, tstep, mt, reps;
  int it, rep, j0, nk;  // the next chunk to load, and the K-step count of its tile
  const int32_t* base;  // first record of tile it

  __device__ __forceinline__ void meta() {
    if (it < mt) {
      const int t = t0 + it * tstep;
      nk = tile_nk[t];
      base = rec + (size_t)rec_off[t] * RECW;
    }
  }
  __device__ __forceinline__ void init(const int32_t* rec_, const int32_t* rec_off_, const int32_t* tile_nk_, int t0_,
                                       int tstep_, int mt_, int reps_) {
    rec = rec_;
    rec_off = rec_off_;
    tile_nk = tile_nk_;
    t0 = t0_;
    tstep = tstep_;
    mt = mt_;
    reps = reps_;
    it = rep = j0 = nk = 0;
    base = nullptr;
    meta();
  }
  // false past the last chunk; else the chunk's tile (position it in the
  // CTA's list), repetition, first K step and record count
  __device__ __forceinline__ bool next(int lane, int32_t (&v)[RECW], int& c_it, int& c_rep, int& c_j0, int& c_cnt) {
    if (it >= mt) return false;
    c_it = it;
    c_rep = rep;
    c_j0 = j0;
    c_cnt = nk - j0 < 32 ? nk - j0 : 32;
    if (lane < c_cnt) {
      const int32_t* r = base + (size_t)(j0 + lane) * RECW;
#pragma unroll
      for (int w = 0; w < RECW; ++w) v[w] = r[w];
    }
    j0 += 32;
    if (j0 >= nk) {
      j0 = 0;
      if (++rep >= reps) {
        rep = 0;
        ++it;
        meta();
      }
    }
    return true;
  }
};

__device__ __forceinline__ uint32_t f32_to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// FP64 -> BF16 (round to nearest even) and FP64 -> FP32 (round to nearest
// even) -> TF32 (round half away from zero at 10 fraction bits), on the bit
// patterns: GB300's FP64 pipe is narrow.  Magnitudes below 2^-126 become
// zero (the tensor-core formats' normal range starts there; the products of
// such inputs would be below FP32's normal range as well).
__device__ __forceinline__ uint32_t f64_to_f32_bits_rne(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const uint32_t sign = (uint32_t)(u >> 32) & 0x80000000u;
  const int ex = (int)((u >> 52) & 0x7ff);
  if (ex == 0x7ff) return sign | 0x7f800000u | (((u & 0xfffffffffffffull) != 0) ? 0x400000u : 0u);
  const int e32 = ex - 1023 + 127;
  if (e32 < 1) return sign;  // below the normal range: zero
  const unsigned long long m = u & 0xfffffffffffffull;
  uint32_t mant = (uint32_t)(m >> 29);
  const uint32_t rem = (uint32_t)(m & 0x1fffffffull);
  uint32_t bits = ((uint32_t)e32 << 23) | mant;
  if (rem > 0x10000000u || (rem == 0x10000000u && (mant & 1u))) ++bits;  // carries into the exponent
  if (e32 > 254 || bits >= 0x7f800000u) return sign | 0x7f800000u;
  return sign | bits;
}

// The same roundings from FP32 values (the FP32 results of TF32/BF16
// products): identical to the FP64 routines above applied to the same value,
// FP32 subnormals included (they become zero).
__device__ __forceinline__ float f32_flush(float x) {
  const uint32_t u = __float_as_uint(x);
  return ((u & 0x7f800000u) == 0u) ? __uint_as_float(u & 0x80000000u) : x;
}

__device__ __forceinline__ uint16_t f32_to_bf16_bits_rne(float x) {
  const uint32_t u = __float_as_uint(x);
  const uint16_t sign = (uint16_t)((u >> 16) & 0x8000u);
  const uint32_t ex = (u >> 23) & 0xffu;
  if (ex == 0xffu) return sign | 0x7f80u | (((u & 0x7fffffu) != 0) ? 0x40u : 0u);
  if (ex == 0u) return sign;
  const uint32_t mant = (u >> 16) & 0x7fu, rem = u & 0xffffu;
  uint32_t bits = (ex << 7) | mant;
  if (rem > 0x8000u || (rem == 0x8000u && (mant & 1u))) ++bits;
  if (bits >= 0x7f80u) return sign | 0x7f80u;
  return sign | (uint16_t)bits;
}

__device__ __forceinline__ uint16_t f64_to_bf16_bits_rne(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const uint16_t sign = (uint16_t)((u >> 48) & 0x8000u);
  const int ex = (int)((u >> 52) & 0x7ff);
  if (ex == 0x7ff) return sign | 0x7f80u | (((u & 0xfffffffffffffull) != 0) ? 0x40u : 0u);
  const int e8 = ex - 1023 + 127;
  if (e8 < 1) return sign;
  const unsigned long long m = u & 0xfffffffffffffull;
  const uint32_t mant = (uint32_t)(m >> 45);
  const unsigned long long rem = m & 0x1fffffffffffull, half = 0x100000000000ull;
  uint32_t bits = ((uint32_t)e8 << 7) | mant;
  if (rem > half || (rem == half && (mant & 1u))) ++bits;
  if (e8 > 254 || bits >= 0x7f80u) return sign | 0x7f80u;
  return sign | (uint16_t)bits;
}

}  // namespace tc
}  // namespace ifac
