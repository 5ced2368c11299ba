// Shared pieces of the sliced tensor-core kernels: the fixed-point slicing of FP64
// values into BF16 digits, and the inline-PTX wrappers for mbarriers, bulk copies and
// tcgen05 MMAs (sm_100 family).
#pragma once
#include <stdint.h>

#include "vrte_internal.cuh"

namespace vrte {

constexpr long long WAIT_LIMIT = 1ll << 22;      // polls before a wait is declared stuck

__device__ __host__ inline int pad_to(int x, int m) { return (x + m - 1) / m * m; }

// Exponent field of a float64 for the scale search: 0 for zero and subnormals; a
// non-finite value counts as zero and sets *bad.
__device__ inline int exp_field(double x, bool* bad) {
  int E = (int)((__double_as_longlong(x) >> 52) & 0x7FF);
  if (E == 0x7FF) {
    *bad = true;
    return 0;
  }
  return E;
}
// Scale exponent from the largest exponent field of a row or column: max |x| < 2^e.
__device__ inline int scale_exp(int Emax) { return Emax ? Emax - 1022 : 0; }

// Slices of v 2^-e in (-1, 1) in integer arithmetic: X = round(v 2^(6 + 7(S-1) - e)) is
// cut into signed base-128 digits q_p in [-64, 64] (most significant first), and slice p
// is q_p 2^-7p, written as its (exact) BF16 bit pattern. Subnormals and non-finite
// values give zero slices.
template <int S>
__device__ inline void slice_bits(double v, int e, unsigned short* bf) {
  long long b = __double_as_longlong(v);
  int E = (int)((b >> 52) & 0x7FF);
  long long X = 0;
  if (E != 0 && E != 0x7FF) {
    long long mant = (b & 0xFFFFFFFFFFFFFll) | (1ll << 52);
    int sh = E - 1075 + 6 + 7 * (S - 1) - e;  // |v| < 2^e keeps X below 2^(6 + 7(S-1))
    if (sh >= 0) X = mant << sh;
    else if (sh > -63) X = (mant + (1ll << (-sh - 1))) >> (-sh);
    if (b < 0) X = -X;
  }
  float scale = 1.0f;
#pragma unroll
  for (int p = 1; p < S; ++p) scale *= 1.0f / 128.0f;
#pragma unroll
  for (int p = S - 1; p >= 1; --p) {
    int d = (int)(((X + 64) & 127) - 64);
    X = (X - d) >> 7;  // exact: X - d is a multiple of 128
    bf[p] = (unsigned short)(__float_as_uint((float)d * scale) >> 16);
    scale *= 128.0f;
  }
  bf[0] = (unsigned short)(__float_as_uint((float)X) >> 16);
}

// Writes the S slices of 8 consecutive K entries (one 16-byte chunk per slice).
template <int S>
__device__ inline void put_chunk(const double* v, int e, unsigned short* dst0,
                                 size_t slice_stride) {
  uint32_t w[S][4];
#pragma unroll
  for (int t = 0; t < 8; t += 2) {
    unsigned short lo[S], hi[S];
    slice_bits<S>(v[t], e, lo);
    slice_bits<S>(v[t + 1], e, hi);
#pragma unroll
    for (int p = 0; p < S; ++p) w[p][t >> 1] = (uint32_t)lo[p] | ((uint32_t)hi[p] << 16);
  }
#pragma unroll
  for (int p = 0; p < S; ++p)
    *(uint4*)(dst0 + p * slice_stride) = make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
}

// ------------------------------------------------------------------ PTX helpers
__device__ inline uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ inline void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ inline void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes) : "memory");
}
__device__ inline bool mbar_try_wait(uint64_t* bar, unsigned phase) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok) : "r"(smem_u32(bar)), "r"(phase) : "memory");
  return ok != 0;
}
// bounded wait: returns false if the barrier did not complete within WAIT_LIMIT polls
__device__ inline bool mbar_wait(uint64_t* bar, unsigned phase) {
  for (long long it = 0; it < WAIT_LIMIT; ++it)
    if (mbar_try_wait(bar, phase)) return true;
  return false;
}
__device__ inline void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
// D (+)= A B, BF16 in, FP32 accumulate in TMEM, one M = 128 x N tile per the instruction
// descriptor (cta_group::1, kind::f16); the shared-memory descriptors are given as their
// (low, high) 32-bit words:
// the address field sits in the low word and shared-memory offsets never carry out of it,
// so unrolled issue loops step descriptors with 32-bit adds of constants.
__device__ __forceinline__ void mma_bf16_w(uint32_t dtmem, uint32_t alo, uint32_t ahi,
                                           uint32_t blo, uint32_t bhi, uint32_t idesc,
                                           uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n .reg .b64 da, db;\n setp.ne.b32 p, %6, 0;\n"
      " mov.b64 da, {%1, %2};\n mov.b64 db, {%3, %4};\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], da, db, %5, p;\n}\n" ::"r"(dtmem),
      "r"(alo), "r"(ahi), "r"(blo), "r"(bhi), "r"(idesc), "r"(acc));
}
__device__ inline void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::
                   "r"(smem_u32(bar)) : "memory");
}

// Byte offset of element (row r, k) in a 64B-swizzled K-major tile of 32 BF16 per row:
// 8-row groups of 512 bytes, 64 bytes per row, 16-byte chunk index XOR ((row / 2) mod 4).
__device__ inline int swz64_offset(int r, int k) {
  int chunk = k >> 3, within = k & 7;
  return (r >> 3) * 512 + (r & 7) * 64 + ((chunk ^ ((r >> 1) & 3)) << 4) + within * 2;
}

__device__ inline uint64_t smem_desc_sw64(const void* p) {
  uint64_t a = (uint64_t)(smem_u32(p) >> 4) & 0x3FFF;
  return a | ((uint64_t)1 << 16)         // leading byte offset (unused for swizzled K-major)
         | ((uint64_t)(512 >> 4) << 32)  // stride byte offset: 8 rows x 64 bytes
         | ((uint64_t)1 << 46)           // descriptor version for sm_100-family
         | ((uint64_t)4 << 61);          // 64-byte swizzle
}

__device__ inline void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

}  // namespace vrte
