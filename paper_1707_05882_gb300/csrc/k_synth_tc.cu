// Azimuthal synthesis of the mixed form on the tcgen05 tensor cores (Eqs. 7, 12).
//
// The table is F[pair][j][el] = sum_m w_c(el)[m][j] I^m[pair][el] for the n_in x n_out
// (incident, outgoing) pairs, the 16 Mueller elements el and the azimuths phi_j, where the
// weight table w_c is the cosine table for the elements of the (IQ, IQ) and (UV, UV) blocks
// (class 0) and the sine table for the off-diagonal blocks (class 1, with a minus sign for
// the IQ rows). Each class is a GEMM with rows (pair, element of the class), columns
// azimuths and K = orders, computed exactly as in the sliced FP64 product (fixed-point BF16
// digits of every row and column, see tc_common.cuh) with five slices and four TMEM
// accumulators: the slice-pair diagonals d = 0, 1, 2 each in an exact one (at most three
// pairs of 2^12-bounded integers, K <= 1365), the diagonals 3 and 4 sharing a fourth whose
// FP32 rounding lies about 2^-37 below the leading term.
//
// Kernel structure (one persistent CTA per SM, 320 threads):
//   warp 0    bulk-copies the slice tiles of A (rows) and B (azimuths) for one 32-order K
//             block into one of three 60 KB shared-memory stages;
//   warp 1    owns the TMEM allocation (512 columns = two buffers of 4 x 64) and issues
//             the 15 slice-pair MMAs of every K block into the tile's buffer;
//   warps 2-9 drain a finished buffer (TMEM -> registers -> error-free FP32 sum ->
//             scaled store; two warps per TMEM lane quarter, 32 columns each) while
//             warp 1 already fills the other one.
// Only one azimuth of every mirror pair (phi, -phi) of the grid is computed: the cosine class
// is even and the sine class odd in the azimuth, so the epilogue stores each value at both
// (for the uniform 360-azimuth grid, 181 computed columns in three tiles instead of six).
// Tiles run azimuth-tile fastest, so the azimuth tiles of one row tile are in flight
// together and its slices come from L2 after the first read. Every wait is bounded: on
// timeout the kernel records ST_TIMEOUT, waits (bounded) for its copies and MMAs, frees
// TMEM and returns.
#include <stdint.h>

#include <algorithm>

#include "tc_common.cuh"

namespace vrte {
namespace {

constexpr int SY_M = 128;    // tile rows: 16 pairs x 8 elements of one class
constexpr int SY_N = 64;     // tile columns: azimuths
constexpr int SY_KB = 32;    // orders per stage: one 64-byte swizzle row of BF16
constexpr int SY_S = 5;      // slices per operand
constexpr int SY_NACC = 4;   // TMEM accumulators per buffer
constexpr int SY_STAGES = 3;
constexpr int SY_A_TILE = SY_M * SY_KB * 2;                      // 8 KiB
constexpr int SY_B_TILE = SY_N * SY_KB * 2;                      // 4 KiB
constexpr int SY_STAGE_BYTES = SY_S * (SY_A_TILE + SY_B_TILE);   // 60 KiB
constexpr int SY_SMEM = SY_STAGES * SY_STAGE_BYTES + 1024;
constexpr int SY_EPI_WARPS = 8;  // two per TMEM lane quarter, each draining 32 columns
constexpr int SY_THREADS = 64 + 32 * SY_EPI_WARPS;
constexpr uint32_t SY_TMEM_COLS = 2 * SY_NACC * SY_N;            // 512
constexpr int SY_PAIRS_PER_TILE = SY_M / 8;

// class of each Mueller element (row-major 4x4) and its position within the class
__constant__ int c_el_class[16] = {0, 0, 1, 1, 0, 0, 1, 1, 1, 1, 0, 0, 1, 1, 0, 0};
__constant__ int c_el_pos[16] = {0, 1, 0, 1, 2, 3, 2, 3, 4, 5, 4, 5, 6, 7, 6, 7};
__constant__ int c_class_el[2][8] = {{0, 1, 4, 5, 10, 11, 14, 15}, {2, 3, 6, 7, 8, 9, 12, 13}};

// accumulator of slice pair (p, q)
__device__ inline int sy_acc(int p, int q) { return min(p + q, SY_NACC - 1); }

struct SynthLayout {
  int P, MT, NT, Kp, KB;
  size_t a_bytes, e_bytes, b_bytes, f_bytes;
};

// P pairs per launch, M orders, n_phi azimuths
SynthLayout synth_layout(int P, int M, int n_phi) {
  SynthLayout L;
  L.P = P;
  L.MT = (P + SY_PAIRS_PER_TILE - 1) / SY_PAIRS_PER_TILE;
  L.NT = (n_phi + SY_N - 1) / SY_N;
  L.Kp = pad_to(M, SY_KB);
  L.KB = L.Kp / SY_KB;
  auto al = [](size_t b) { return (b + 1023) / 1024 * 1024; };
  L.a_bytes = al((size_t)2 * SY_S * L.MT * L.KB * SY_A_TILE);
  L.e_bytes = al((size_t)2 * L.MT * SY_M * sizeof(int));
  L.b_bytes = al((size_t)2 * SY_S * L.NT * L.KB * SY_B_TILE);
  L.f_bytes = al((size_t)2 * L.NT * SY_N * sizeof(int));
  return L;
}

// Rows of both classes for P pairs starting at pair0: one CTA per 16 pairs (grid-strided),
// thread t -> (pair 16 mt + t / 16, element t % 16), so that every load of one order
// reads 2 KB of I^m contiguously. Row exponent from the integer maximum of the exponent
// fields over the orders, then the slices of 8 orders per 16-byte chunk.
__global__ void __launch_bounds__(256) k_synth_slice_rows(int P, long long pair0,
                                                          long long pairs_total, int M, int MT,
                                                          int KB, const double* __restrict__ Isyn,
                                                          unsigned short* As, int* ea,
                                                          unsigned* status) {
  const int pl = threadIdx.x >> 4, el = threadIdx.x & 15;
  const int cls = c_el_class[el], e = c_el_pos[el];
  const bool neg = cls == 1 && e < 4;
  const int r = pl * 8 + e;
  const size_t mstride = (size_t)pairs_total * 16;
  const size_t tile_elems = (size_t)SY_M * SY_KB;
  const size_t slice_stride = (size_t)MT * KB * tile_elems;
  bool bad = false;
  for (int mt = blockIdx.x; mt < MT; mt += gridDim.x) {
    const int pr = mt * SY_PAIRS_PER_TILE + pl;
    const bool valid = pr < P;
    const double* src = Isyn + (size_t)(pair0 + (valid ? pr : 0)) * 16 + el;
    int Em = 0;
    if (valid) {
      int m = 0;
      for (; m + 8 <= M; m += 8) {
        double v[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) v[t] = src[(size_t)(m + t) * mstride];
#pragma unroll
        for (int t = 0; t < 8; ++t) Em = max(Em, exp_field(v[t], &bad));
      }
      for (; m < M; ++m) Em = max(Em, exp_field(src[(size_t)m * mstride], &bad));
    }
    const int ee = scale_exp(Em);
    ea[(size_t)cls * MT * SY_M + (size_t)mt * SY_M + r] = ee;
    unsigned short* dst_t = As + (size_t)cls * SY_S * slice_stride + (size_t)mt * KB * tile_elems;
    for (int k0 = 0; k0 < KB * SY_KB; k0 += 8) {
      double v[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        double x = (valid && k0 + t < M) ? src[(size_t)(k0 + t) * mstride] : 0.0;
        v[t] = neg ? -x : x;
      }
      const int kb = k0 / SY_KB;
      put_chunk<SY_S>(v, ee, dst_t + (size_t)kb * tile_elems + (swz64_offset(r, k0 - kb * SY_KB) >> 1),
                      slice_stride);
    }
  }
  if (bad) atomicOr(status, ST_NONFINITE);
}

// Columns of both weight tables: grid (NT, 2 classes), thread = column c of the computed
// azimuths, the grid's azimuth rep[c] (c < n_rep).
__global__ void __launch_bounds__(SY_N) k_synth_slice_cols(int M, int n_phi, int n_rep,
                                                           const int* __restrict__ rep, int NT,
                                                           int KB, const double* __restrict__ wc,
                                                           const double* __restrict__ ws,
                                                           unsigned short* Bs, int* fb,
                                                           unsigned* status) {
  const int nt = blockIdx.x, cls = blockIdx.y, c = threadIdx.x;
  const int jc = nt * SY_N + c;
  const bool in = jc < n_rep;
  const int j = in ? rep[jc] : 0;
  const double* W = cls ? ws : wc;
  bool bad = false;
  int Em = 0;
  if (in)
    for (int m = 0; m < M; ++m) Em = max(Em, exp_field(W[(size_t)m * n_phi + j], &bad));
  const int ee = scale_exp(Em);
  fb[(size_t)cls * NT * SY_N + jc] = ee;
  const size_t tile_elems = (size_t)SY_N * SY_KB;
  const size_t slice_stride = (size_t)NT * KB * tile_elems;
  unsigned short* dst_t = Bs + (size_t)cls * SY_S * slice_stride + (size_t)nt * KB * tile_elems;
  for (int k0 = 0; k0 < KB * SY_KB; k0 += 8) {
    double v[8];
#pragma unroll
    for (int t = 0; t < 8; ++t)
      v[t] = (in && k0 + t < M) ? W[(size_t)(k0 + t) * n_phi + j] : 0.0;
    const int kb = k0 / SY_KB;
    put_chunk<SY_S>(v, ee, dst_t + (size_t)kb * tile_elems + (swz64_offset(c, k0 - kb * SY_KB) >> 1),
                    slice_stride);
  }
  if (bad) atomicOr(status, ST_NONFINITE);
}

// scaled value of one output element from the four accumulators (FP32 table)
__device__ inline float synth_value(const uint32_t* x, int E2, float*) {
  // error-free FP32 sum (hi + lo), largest diagonal first, rounded once
  float hi = 0.0f, lo = 0.0f;
#pragma unroll
  for (int a = 0; a < SY_NACC; ++a) {
    float v = __uint_as_float(x[a]);
    float sm = hi + v, bb = sm - hi;
    lo += (hi - (sm - bb)) + (v - bb);
    hi = sm;
  }
  float w = hi + lo;
  return (E2 > -120 && E2 < 120) ? w * __int_as_float((E2 + 127) << 23) : ldexpf(w, E2);
}
// (FP64 table) the exact accumulators hold integers times 2^-7d: combine them in an int64
// in units of 2^-14, then one FP64 fma adds the rounded fourth
__device__ inline double synth_value(const uint32_t* x, int E2, double*) {
  long long I = 0;
#pragma unroll
  for (int a = 0; a < SY_NACC - 1; ++a)
    I += (long long)__float2int_rn(__uint_as_float(x[a]) * (float)(1 << (7 * a)))
         << (7 * (SY_NACC - 2 - a));
  double w = fma((double)I, 0x1p-14, (double)__uint_as_float(x[SY_NACC - 1]));
  return (E2 > -1000 && E2 < 1000) ? w * __longlong_as_double((long long)(E2 + 1023) << 52)
                                   : ldexp(w, E2);
}

template <typename T>
__global__ void __launch_bounds__(SY_THREADS, 1)
    k_synth_mma(int P, long long pair0, int n_phi, int n_rep, const int* __restrict__ map,
                int MT, int NT, int KB, const unsigned short* __restrict__ As,
                const int* __restrict__ ea, const unsigned short* __restrict__ Bs,
                const int* __restrict__ fb, T* out, unsigned* status) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ uint64_t full_bar[SY_STAGES], empty_bar[SY_STAGES], tfull_bar[2], tempty_bar[2],
      fin_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tiles = 2 * MT * NT;
  const size_t a_tile_elems = (size_t)SY_M * SY_KB, b_tile_elems = (size_t)SY_N * SY_KB;
  const size_t a_slice = (size_t)MT * KB * a_tile_elems, b_slice = (size_t)NT * KB * b_tile_elems;

  if (threadIdx.x == 0) {
    for (int s = 0; s < SY_STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull_bar[b], 1);
      mbar_init(&tempty_bar[b], SY_EPI_WARPS);
    }
    mbar_init(&fin_bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(SY_TMEM_COLS) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  auto fail = [&]() {
    abort_flag = 1;
    atomicOr(status, ST_TIMEOUT);
  };

  bool issued[SY_STAGES] = {};   // producer: stages with copies issued, and their round
  int round_of[SY_STAGES] = {};
  if (warp == 0) {
    // ---- producer: one thread issues the bulk copies of every K block
    if (lane == 0) {
      int g = 0;
      for (int t = blockIdx.x; t < tiles && !abort_flag; t += gridDim.x) {
        const int nt = t % NT, cls = (t / NT) & 1, mt = t / (2 * NT);
        const unsigned short* a0 = As + (size_t)cls * SY_S * a_slice + (size_t)mt * KB * a_tile_elems;
        const unsigned short* b0 = Bs + (size_t)cls * SY_S * b_slice + (size_t)nt * KB * b_tile_elems;
        bool ok = true;
        for (int kb = 0; kb < KB; ++kb, ++g) {
          const int s = g % SY_STAGES, r = g / SY_STAGES;
          if (!mbar_wait(&empty_bar[s], (r & 1) ^ 1)) { ok = false; break; }
          unsigned char* st = smem + (size_t)s * SY_STAGE_BYTES;
          mbar_expect_tx(&full_bar[s], (unsigned)SY_STAGE_BYTES);
          for (int p = 0; p < SY_S; ++p)
            bulk_g2s(st + p * SY_A_TILE, a0 + p * a_slice + (size_t)kb * a_tile_elems, SY_A_TILE,
                     &full_bar[s]);
          for (int q = 0; q < SY_S; ++q)
            bulk_g2s(st + SY_S * SY_A_TILE + q * SY_B_TILE,
                     b0 + q * b_slice + (size_t)kb * b_tile_elems, SY_B_TILE, &full_bar[s]);
          issued[s] = true;
          round_of[s] = r;
        }
        if (!ok) { fail(); break; }
      }
    }
  } else if (warp == 1) {
    // ---- MMA issue: one thread, 15 slice-pair products per K block
    if (lane == 0) {
      // D = F32, A = B = BF16, both K-major, N = 64, M = 128
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) |
                             ((uint32_t)(SY_N >> 3) << 17) | ((uint32_t)(SY_M >> 4) << 24);
      int g = 0, lt = 0;
      for (int t = blockIdx.x; t < tiles && !abort_flag; t += gridDim.x, ++lt) {
        const int b = lt & 1, use = lt >> 1;
        if (!mbar_wait(&tempty_bar[b], (use & 1) ^ 1)) { fail(); break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t dbase = tmem + (uint32_t)(b * SY_NACC * SY_N);
        bool ok = true;
        for (int kb = 0; kb < KB; ++kb, ++g) {
          const int s = g % SY_STAGES, r = g / SY_STAGES;
          if (!mbar_wait(&full_bar[s], r & 1)) { ok = false; break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          unsigned char* st = smem + (size_t)s * SY_STAGE_BYTES;
          const uint64_t adesc = smem_desc_sw64(st);
          const uint32_t alo = (uint32_t)adesc, dhi = (uint32_t)(adesc >> 32);
          const uint32_t blo = (uint32_t)smem_desc_sw64(st + SY_S * SY_A_TILE);
          const uint32_t later = kb > 0 ? 1u : 0u;
#pragma unroll
          for (int p = 0; p < SY_S; ++p)
#pragma unroll
            for (int q = 0; p + q < SY_S; ++q) {
              const int a = sy_acc(p, q);
              // first pair (in this order) of its accumulator: overwrite in K block 0
              const bool first = p == 0 && q < SY_NACC;
#pragma unroll
              for (int k16 = 0; k16 < SY_KB / 16; ++k16)
                mma_bf16_w(dbase + (uint32_t)(a * SY_N),
                           alo + (uint32_t)(p * (SY_A_TILE >> 4) + k16 * 2), dhi,
                           blo + (uint32_t)(q * (SY_B_TILE >> 4) + k16 * 2), dhi, idesc,
                           (k16 > 0 || !first) ? 1u : later);
            }
          mma_commit(&empty_bar[s]);  // the stage is free once these MMAs have read it
        }
        if (!ok) { fail(); break; }
        mma_commit(&tfull_bar[b]);    // the buffer is ready once every MMA has completed
      }
      // every MMA issued has completed before TMEM is released (bounded)
      mma_commit(&fin_bar);
      if (!mbar_wait(&fin_bar, 0)) fail();
    }
  } else {
    // ---- epilogue: warp w drains TMEM lanes 32 (w mod 4) .. + 31 (tile rows), columns
    // 32 h .. 32 h + 31 with h = (w - 2) / 4
    const int quad = warp & 3;
    const int cbeg = ((warp - 2) >> 2) * (SY_N / 2);
    const int r = quad * 32 + lane;
    const int pl = r >> 3, e = r & 7;
    int lt = 0;
    for (int t = blockIdx.x; t < tiles && !abort_flag; t += gridDim.x, ++lt) {
      const int b = lt & 1, use = lt >> 1;
      if (!mbar_wait(&tfull_bar[b], use & 1)) { fail(); break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int nt = t % NT, cls = (t / NT) & 1, mt = t / (2 * NT);
      const int pr = mt * SY_PAIRS_PER_TILE + pl;
      const bool valid = pr < P;
      const int erow = ea[(size_t)cls * MT * SY_M + (size_t)mt * SY_M + r] - 12;
      const int el = c_class_el[cls][e];
      T* orow = out + (size_t)(pair0 + (valid ? pr : 0)) * n_phi * 16 + el;
      const int* fcol = fb + (size_t)cls * NT * SY_N + nt * SY_N;
      const uint32_t tbase = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(b * SY_NACC * SY_N);
      bool bad = false;
      for (int c0 = cbeg; c0 < cbeg + SY_N / 2; c0 += 16) {
        __syncwarp();
        uint32_t x[SY_NACC][16];
#pragma unroll
        for (int a = 0; a < SY_NACC; ++a) {
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,"
              "%12,%13,%14,%15}, [%16];\n"
              : "=r"(x[a][0]), "=r"(x[a][1]), "=r"(x[a][2]), "=r"(x[a][3]), "=r"(x[a][4]),
                "=r"(x[a][5]), "=r"(x[a][6]), "=r"(x[a][7]), "=r"(x[a][8]), "=r"(x[a][9]),
                "=r"(x[a][10]), "=r"(x[a][11]), "=r"(x[a][12]), "=r"(x[a][13]), "=r"(x[a][14]),
                "=r"(x[a][15])
              : "r"(tbase + (uint32_t)(a * SY_N + c0)));
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (c0 + 16 >= cbeg + SY_N / 2) {
          // this warp's last reads of the buffer are done: hand its share back
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          __syncwarp();
          if (lane == 0) mbar_arrive(&tempty_bar[b]);
        }
#pragma unroll
        for (int t16 = 0; t16 < 16; ++t16) {
          const int jc = nt * SY_N + c0 + t16;
          if (valid && jc < n_rep) {
            uint32_t xs[SY_NACC];
#pragma unroll
            for (int a = 0; a < SY_NACC; ++a) xs[a] = x[a][t16];
            T v = synth_value(xs, erow + fcol[c0 + t16], (T*)nullptr);
            bad |= !isfinite((double)v);
            // the table streams out (evict-first), at the azimuth and at its mirror (the
            // cosine class even, the sine class odd in the azimuth)
            __stcs(orow + (size_t)map[jc] * 16, v);
            const int jm = map[n_phi + jc];
            if (jm >= 0) __stcs(orow + (size_t)jm * 16, cls ? -v : v);
          }
        }
      }
      if (bad) atomicOr(status, ST_NONFINITE);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // after an abort, let the copies still in flight land before the CTA exits (bounded)
  if (warp == 0 && lane == 0 && abort_flag)
    for (int s = 0; s < SY_STAGES; ++s)
      if (issued[s]) mbar_wait(&full_bar[s], round_of[s] & 1);
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(SY_TMEM_COLS) : "memory");
}

int sm_count() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
      sms = 1;
  }
  return sms;
}

}  // namespace

size_t tc_synthesis_workspace(int M, int n_in, int n_out, int n_phi, int k_block) {
  SynthLayout L = synth_layout(std::min(k_block, n_in) * n_out, M, n_phi);
  return L.a_bytes + L.e_bytes + L.b_bytes + L.f_bytes;
}

void tc_synthesis(int M, int n_in, int n_out, int n_phi, int n_rep, const int* map,
                  const double* Isyn, const double* wc, const double* ws, void* out,
                  int out_dtype, int k_block, void* work, unsigned* status, cudaStream_t s,
                  const SynthHook* hook, int k_lo, int k_hi, bool slice_weights) {
  if (k_hi < 0 || k_hi > n_in) k_hi = n_in;
  const long long pairs_total = (long long)n_in * n_out;
  const SynthLayout Lmax = synth_layout(std::min(k_block, n_in) * n_out, M, n_rep);
  unsigned char* w = (unsigned char*)work;
  unsigned short* As = (unsigned short*)w;
  int* ea = (int*)(w + Lmax.a_bytes);
  unsigned short* Bs = (unsigned short*)(w + Lmax.a_bytes + Lmax.e_bytes);
  int* fb = (int*)(w + Lmax.a_bytes + Lmax.e_bytes + Lmax.b_bytes);
  const int sms = sm_count();
  if (slice_weights)
    k_synth_slice_cols<<<dim3(Lmax.NT, 2), SY_N, 0, s>>>(M, n_phi, n_rep, map, Lmax.NT, Lmax.KB,
                                                         wc, ws, Bs, fb, status);
  if (out_dtype == VRTE_OUT_F64)
    cudaFuncSetAttribute(k_synth_mma<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, SY_SMEM);
  else
    cudaFuncSetAttribute(k_synth_mma<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, SY_SMEM);
  for (int k0 = k_lo; k0 < k_hi; k0 += k_block) {
    const int kb = std::min(k_block, k_hi - k0);
    const SynthLayout L = synth_layout(kb * n_out, M, n_rep);
    const long long pair0 = (long long)k0 * n_out;
    k_synth_slice_rows<<<std::min(L.MT, 2 * sms), 256, 0, s>>>(L.P, pair0, pairs_total, M, L.MT,
                                                               L.KB, Isyn, As, ea, status);
    const int tiles = 2 * L.MT * L.NT;
    const int grid = std::min(tiles, sms);
    if (out_dtype == VRTE_OUT_F64)
      k_synth_mma<double><<<grid, SY_THREADS, SY_SMEM, s>>>(L.P, pair0, n_phi, n_rep, map, L.MT,
                                                            L.NT, L.KB, As, ea, Bs, fb,
                                                            (double*)out, status);
    else
      k_synth_mma<float><<<grid, SY_THREADS, SY_SMEM, s>>>(L.P, pair0, n_phi, n_rep, map, L.MT,
                                                           L.NT, L.KB, As, ea, Bs, fb, (float*)out,
                                                           status);
    if (hook) hook->fn(hook->user, hook->layer, k0, k0 + kb, s);
  }
}

}  // namespace vrte
