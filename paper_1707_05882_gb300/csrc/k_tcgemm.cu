// FP64-accurate batched GEMM on the tcgen05 tensor cores by exact fixed-point slicing.
//
// Every row i of A is scaled by 2^-e_i (e_i: the exponent of max_k |A_ik|) and written as
//   A_ik 2^-e_i = 2^-6 sum_p a_ikp,   a_ikp = 2^(-7p) x integer of magnitude <= 64,
// likewise every column j of B with 2^-f_j and slices b_kjq. Each slice is a 7-bit integer
// times a power of two, which BF16 represents exactly, and every product a_ikp b_kjq is an
// integer of magnitude <= 2^12 times 2^(-7(p+q)). Products on one diagonal d = p + q share
// a scale, so a FP32 accumulator that collects them sums them exactly as long as its
// integer total stays within 2^24, i.e. at most 4 pairs for K <= 1024: diagonals 0 .. 3
// get one TMEM accumulator each, diagonal 4 two (3 + 2 pairs), and the diagonals
// 5 .. S-1 share a seventh whose rounding sits 2^-35 below the leading term. Pairs with
// p + q >= S are dropped. The epilogue combines the exact accumulators in an int64,
// adds the last in FP64 and scales by 2^(e_i + f_j - 12):
//   C_ij = 2^(e_i + f_j - 12) (acc_0 + ... + acc_6),
// so the error is the slices dropped: relative to max|A_i| max|B_j| per term ~3e-9 at
// S = 4, ~3e-13 at S = 6, ~2e-15 at S = 7.
//
// Data flow: `k_slice_rows` / `k_slice_cols` write the slices directly as the shared-
// memory image of 64B-swizzled K-major tiles ([unit][tile][k-block][slice] blocks of
// 128 x 32 or 64 x 32 BF16), so the GEMM kernel loads each tile with one bulk copy. The
// persistent GEMM kernel computes 128 x 64 output tiles with up to seven accumulators of
// 64 columns in TMEM. It is warp-specialised: one warp keeps a ring of shared-memory
// stages (S = 7: two of 84 KB; S <= 5: three or four) filled with bulk copies, one warp
// issues the MMAs as stages fill, and eight warps drain the accumulators; with S <= 4 two
// TMEM buffers let the next tile's MMAs run during the epilogue. Every mbarrier wait is
// bounded; on timeout the kernel records ST_TIMEOUT, waits (bounded) for its copies and
// MMAs, frees TMEM and returns.
#include <stdint.h>

#include <algorithm>

#include "tc_common.cuh"

namespace vrte {

constexpr int TC_M = 128;       // output rows per CTA (MMA M)
constexpr int TC_N = 64;        // output columns per CTA (MMA N)
static_assert(TC_N == kTcTileCols, "column tiles of TcRange");
constexpr int TC_KB = 32;       // K per stage (one 64-byte swizzle row of BF16)
constexpr int TC_MAXS = 8;      // maximum number of slices
constexpr int TC_NACC = 7;      // TMEM accumulators (see acc_index)
constexpr int TC_STAGES = 4;    // shared-memory stages (at most)
constexpr int TC_EPI_WARPS = 8; // epilogue warps: two per TMEM lane quarter, 32 columns each
constexpr int TC_THREADS = 64 + 32 * TC_EPI_WARPS;  // warp 0 copies, warp 1 MMAs
constexpr int TC_GROUP_M = 8;   // row tiles per group of the tile order
constexpr int TC_SMEM_MAX = 227 * 1024;
constexpr int A_TILE_BYTES = TC_M * TC_KB * 2;   // 8 KiB
constexpr int B_TILE_BYTES = TC_N * TC_KB * 2;   // 4 KiB

// Accumulator of slice pair (p, q): diagonals d = p + q < 4 one each; diagonal 4 split by
// p <= 2 (3 pairs) and p >= 3 (2 pairs) so that each stays exact for K <= 1024; the
// diagonals 5 .. S-1 share the last one (rounded; 2^-35 below the leading term).
__device__ __host__ inline int acc_index(int p, int q) {
  int d = p + q;
  return d < 4 ? d : (d == 4 ? (p <= 2 ? 4 : 5) : 6);
}
// diagonal (scale 2^-7d) of exact accumulator a
__device__ __host__ inline int acc_diag(int a) { return a < 4 ? a : 4; }
__device__ __host__ inline int acc_count(int S) { return S <= 4 ? S : (S == 5 ? 6 : 7); }
// as many stages (up to four) of S slices of A and B tiles as fit in shared memory
__device__ __host__ inline int tc_stages(int S) {
  int n = (TC_SMEM_MAX - 2048) / (S * (A_TILE_BYTES + B_TILE_BYTES));
  return n < 1 ? 1 : (n > TC_STAGES ? TC_STAGES : n);
}
__device__ __host__ inline int tc_smem_bytes(int S) {
  return tc_stages(S) * S * (A_TILE_BYTES + B_TILE_BYTES) + 1024;
}

// A rows: A[u][i][k] (row-major, lda, unit stride sA), M x K. Writes
//   out[u][mt][kb][p] tiles (128 x 32 BF16 images) and e[u][i] (int exponent).
// One CTA per (row block of TR, unit); each thread slices 8 consecutive k of one row. TR = TC_M
// for the A operand; TR = TC_N slices the rows of a matrix stored N x K as the B operand (B^T).
template <int S, int TR = TC_M>
__global__ void k_slice_rows(int M, int K, const double* __restrict__ A, int lda,
                             long long sA, unsigned short* out, int* e_out, unsigned* status) {
  int mt = blockIdx.x, u = blockIdx.y;
  int Mp = pad_to(M, TR), Kp = pad_to(K, TC_KB), KB = Kp / TC_KB, MT = Mp / TR;
  __shared__ int ex[TR];
  const double* Ab = A + (size_t)u * sA;
  bool bad = false;
  // per-row exponent: warp per row, integer max of the exponent fields
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int r = warp; r < TR; r += nw) {
    int i = mt * TR + r;
    int Em = 0;
    if (i < M)
      for (int k = lane; k < K; k += 32) Em = max(Em, exp_field(Ab[(size_t)i * lda + k], &bad));
    Em = __reduce_max_sync(0xffffffffu, Em);
    if (lane == 0) {
      ex[r] = scale_exp(Em);
      if (i < M) e_out[(size_t)u * Mp + i] = ex[r];
    }
  }
  __syncthreads();
  const size_t tile_elems = (size_t)TR * TC_KB;
  const size_t slice_stride = tile_elems;  // the S slices of a tile block are adjacent
  const int chunks = Kp / 8;
  for (int idx = threadIdx.x; idx < TR * chunks; idx += blockDim.x) {
    int r = idx / chunks, k0 = 8 * (idx - r * chunks);
    int i = mt * TR + r;
    double v[8];
    for (int t = 0; t < 8; ++t)
      v[t] = (i < M && k0 + t < K) ? Ab[(size_t)i * lda + k0 + t] : 0.0;
    int kb = k0 / TC_KB;
    size_t base = ((((size_t)u * MT + mt) * KB + kb) * S) * tile_elems;
    put_chunk<S>(v, ex[r], out + base + (swz64_offset(r, k0 - kb * TC_KB) >> 1), slice_stride);
  }
  if (bad) atomicOr(status, ST_NONFINITE);
}

// B columns: B[u][k][j] (row-major, ldb, unit stride sB), K x N, sliced per column j
// into K-major tiles out[u][nt][kb][q] (64 x 32 BF16 images, row = j) and f[u][j].
// Each thread slices 8 consecutive k of one column (consecutive threads: consecutive
// columns, so every global load is coalesced).
// TR = TC_N for the B operand; TR = TC_M slices the columns of a matrix stored K x M as the A
// operand (A^T). blockDim = 512 = (512 / TR) row groups x TR columns.
template <int S, int TR = TC_N>
__global__ void k_slice_cols(int N, int K, const double* __restrict__ B, int ldb,
                             long long sB, unsigned short* out, int* f_out, unsigned* status) {
  constexpr int G = 512 / TR;
  int nt = blockIdx.x, u = blockIdx.y;
  int Np = pad_to(N, TR), Kp = pad_to(K, TC_KB), KB = Kp / TC_KB, NT = Np / TR;
  __shared__ int ex[TR];
  __shared__ int red[G][TR];
  const double* Bb = B + (size_t)u * sB;
  bool bad = false;
  // per-column max exponent: threads over columns (coalesced rows), G row groups
  int c = threadIdx.x % TR, g = threadIdx.x / TR;
  int j = nt * TR + c;
  int Em = 0;
  if (j < N) {
    // eight independent loads in flight per thread
    int k = g;
    for (; k + 7 * G < K; k += 8 * G) {
      double v[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) v[t] = Bb[(size_t)(k + G * t) * ldb + j];
#pragma unroll
      for (int t = 0; t < 8; ++t) Em = max(Em, exp_field(v[t], &bad));
    }
    for (; k < K; k += G) Em = max(Em, exp_field(Bb[(size_t)k * ldb + j], &bad));
  }
  red[g][c] = Em;
  __syncthreads();
  if (g == 0) {
    int m2 = 0;
    for (int q = 0; q < G; ++q) m2 = max(m2, red[q][c]);
    ex[c] = scale_exp(m2);
    if (j < N) f_out[(size_t)u * Np + j] = ex[c];
  }
  __syncthreads();
  const size_t tile_elems = (size_t)TR * TC_KB;
  const size_t slice_stride = tile_elems;  // the S slices of a tile block are adjacent
  const int chunks = Kp / 8;
  for (int idx = threadIdx.x; idx < TR * chunks; idx += blockDim.x) {
    int k0 = 8 * (idx / TR), cc = idx % TR;
    int jj = nt * TR + cc;
    double v[8];
    for (int t = 0; t < 8; ++t)
      v[t] = (jj < N && k0 + t < K) ? Bb[(size_t)(k0 + t) * ldb + jj] : 0.0;
    int kb = k0 / TC_KB;
    size_t base = ((((size_t)u * NT + nt) * KB + kb) * S) * tile_elems;
    put_chunk<S>(v, ex[cc], out + base + (swz64_offset(cc, k0 - kb * TC_KB) >> 1), slice_stride);
  }
  if (bad) atomicOr(status, ST_NONFINITE);
}

// slicers are compiled for each slice count; the host picks one at run time
#define VRTE_SLICE_DISPATCH(S, CALL) \
  switch (S) {                       \
    case 1: CALL(1); break;          \
    case 2: CALL(2); break;          \
    case 3: CALL(3); break;          \
    case 4: CALL(4); break;          \
    case 5: CALL(5); break;          \
    case 6: CALL(6); break;          \
    case 7: CALL(7); break;          \
    default: CALL(8); break;         \
  }

// TMEM columns of one accumulator buffer, buffers per CTA, and the allocation
__device__ __host__ inline int tc_buf_cols(int S) { return acc_count(S) * TC_N; }
__device__ __host__ inline int tc_nbuf(int S) { return 2 * tc_buf_cols(S) <= 512 ? 2 : 1; }
__device__ __host__ inline uint32_t tc_tmem_cols(int S) {
  int c = tc_nbuf(S) * tc_buf_cols(S);
  return c <= 32 ? 32 : (c <= 64 ? 64 : (c <= 128 ? 128 : (c <= 256 ? 256 : 512)));
}

// tile t of the persistent sequence -> (unit, row tile, column tile): per unit, groups of
// TC_GROUP_M row tiles with every column tile, row tile fastest inside a group, so that
// the tiles in flight at one time share few slice panels (L2 reuse)
__device__ inline void tc_decode(int t, int MT, int NT, int& u, int& mt, int& nt) {
  const int per_unit = MT * NT;
  u = t / per_unit;
  const int tl = t - u * per_unit;
  const int gsz = TC_GROUP_M * NT;
  const int g = tl / gsz, idx = tl - g * gsz;
  const int gm = min(TC_GROUP_M, MT - g * TC_GROUP_M);
  mt = g * TC_GROUP_M + idx % gm;
  nt = idx / gm;
}

// K blocks that are zero in both operands of unit u (see TcKSkip) and are skipped: the
// blocks lying entirely in [zk0, zk0 + zbase + zstep u); at least one block stays, so that
// every accumulator is written.
__device__ inline void tc_skip_range(const TcKSkip& z, int u, int KB, int& zb0, int& zb1) {
  const int len = z.zbase + z.zstep * u;
  zb0 = (z.zk0 + TC_KB - 1) / TC_KB;
  zb1 = len > 0 ? min((z.zk0 + len) / TC_KB, KB) : 0;
  if (zb1 <= zb0) zb0 = zb1 = 0;
  if (zb0 == 0 && zb1 >= KB) zb1 = KB - 1;
}

template <class Epi>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_tc_gemm(int M, int N, int K, int S, const unsigned short* __restrict__ As,
              const int* __restrict__ ea, const unsigned short* __restrict__ Bs,
              const int* __restrict__ fb, float* scratch, Epi epi, unsigned* status,
              int batch, TcKSkip zskip, int nt_lo, int nt_cnt) {
  // Persistent: CTA b takes tiles b, b + gridDim.x, ... Warp 0 bulk-copies the slice
  // tiles of each 32-wide K block into a ring of shared-memory stages, warp 1 (owner of
  // the TMEM allocation) issues the slice-pair MMAs as the stages fill, and warps 2-9
  // drain the finished accumulators (two per TMEM lane quarter); with two TMEM buffers (S <= 4) the next tile's MMAs
  // run during the epilogue, with one the copies for it do.
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ uint64_t full_bar[TC_STAGES], empty_bar[TC_STAGES], tfull_bar[2], tempty_bar[2],
      fin_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int Mp = pad_to(M, TC_M), Np = pad_to(N, TC_N), Kp = pad_to(K, TC_KB);
  const int KB = Kp / TC_KB, MT = Mp / TC_M, NT = Np / TC_N;
  // the column tiles nt_lo .. nt_lo + nt_cnt - 1 of every unit (all: 0, NT)
  const int NTr = nt_cnt > 0 ? nt_cnt : NT;
  const int tiles = MT * NTr * batch;
  const int stage_bytes = S * (A_TILE_BYTES + B_TILE_BYTES);
  const int nst = tc_stages(S);
  const int nacc = acc_count(S);
  const int buf_cols = tc_buf_cols(S), nbuf = tc_nbuf(S);
  const uint32_t ncols = tc_tmem_cols(S);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const size_t a_unit = (size_t)S * MT * KB * (A_TILE_BYTES / 2);
  const size_t b_unit = (size_t)S * NT * KB * (B_TILE_BYTES / 2);

  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull_bar[b], 1);
      mbar_init(&tempty_bar[b], TC_EPI_WARPS);
    }
    mbar_init(&fin_bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(ncols) : "memory");
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

  bool issued[TC_STAGES] = {};  // producer: stages with copies issued, and their round
  int round_of[TC_STAGES] = {};
  if (warp == 0) {
    // ---- producer
    if (lane == 0) {
      int g = 0;
      for (int t = blockIdx.x; t < tiles && !abort_flag; t += gridDim.x) {
        int u, mt, nt;
        tc_decode(t, MT, NTr, u, mt, nt);
        nt += nt_lo;
        // the S slice tiles of a (tile, K block) are adjacent: one bulk copy per operand
        const unsigned short* a0 =
            As + (size_t)u * a_unit + (size_t)mt * KB * S * (A_TILE_BYTES / 2);
        const unsigned short* b0 =
            Bs + (size_t)u * b_unit + (size_t)nt * KB * S * (B_TILE_BYTES / 2);
        int zb0, zb1;
        tc_skip_range(zskip, u, KB, zb0, zb1);
        bool ok = true;
        for (int kb = 0; kb < KB; ++kb) {
          if (kb >= zb0 && kb < zb1) continue;  // zero in both operands of this unit
          const int s = g % nst, r = g / nst;
          ++g;
          if (!mbar_wait(&empty_bar[s], (r & 1) ^ 1)) { ok = false; break; }
          unsigned char* st = smem + (size_t)s * stage_bytes;
          mbar_expect_tx(&full_bar[s], (unsigned)stage_bytes);
          bulk_g2s(st, a0 + (size_t)kb * S * (A_TILE_BYTES / 2), S * A_TILE_BYTES, &full_bar[s]);
          bulk_g2s(st + S * A_TILE_BYTES, b0 + (size_t)kb * S * (B_TILE_BYTES / 2),
                   S * B_TILE_BYTES, &full_bar[s]);
          issued[s] = true;
          round_of[s] = r;
        }
        if (!ok) { fail(); break; }
      }
    }
  } else if (warp == 1) {
    // ---- MMA issue
    if (lane == 0) {
      // D = F32, A = B = BF16, both K-major, N = 64, M = 128
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) |
                             ((uint32_t)(TC_N >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
      int g = 0, lt = 0;
      for (int t = blockIdx.x; t < tiles && !abort_flag; t += gridDim.x, ++lt) {
        const int b = nbuf == 2 ? (lt & 1) : 0, use = nbuf == 2 ? (lt >> 1) : lt;
        if (!mbar_wait(&tempty_bar[b], (use & 1) ^ 1)) { fail(); break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t dbase = tmem + (uint32_t)(b * buf_cols);
        int u, mt, nt;
        tc_decode(t, MT, NTr, u, mt, nt);
        nt += nt_lo;
        int zb0, zb1;
        tc_skip_range(zskip, u, KB, zb0, zb1);
        const int kfirst = (zb0 == 0 && zb1 > 0) ? zb1 : 0;  // first K block issued
        bool ok = true;
        for (int kb = 0; kb < KB; ++kb) {
          if (kb >= zb0 && kb < zb1) continue;
          const int s = g % nst, r = g / nst;
          ++g;
          if (!mbar_wait(&full_bar[s], r & 1)) { ok = false; break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          unsigned char* st = smem + (size_t)s * stage_bytes;
          // descriptors differ only in the start-address field (bits 0-13, 16-byte units):
          // the fully unrolled issue steps their low words by constants
          const uint64_t adesc = smem_desc_sw64(st);
          const uint32_t alo = (uint32_t)adesc, dhi = (uint32_t)(adesc >> 32);
          const uint32_t blo = (uint32_t)smem_desc_sw64(st + S * A_TILE_BYTES);
          const uint32_t later = kb != kfirst ? 1u : 0u;
#pragma unroll
          for (int p = 0; p < TC_MAXS; ++p)
#pragma unroll
            for (int q = 0; q < TC_MAXS - p; ++q) {
              if (p + q >= S) continue;
              const int a = acc_index(p, q);
              // first pair (in this order) of its accumulator: overwrite in K block 0
              const bool first = (p == 0 && q <= 5) || (p == 3 && q == 1);
#pragma unroll
              for (int k16 = 0; k16 < TC_KB / 16; ++k16)
                mma_bf16_w(dbase + (uint32_t)(a * TC_N),
                           alo + (uint32_t)(p * (A_TILE_BYTES >> 4) + k16 * 2), dhi,
                           blo + (uint32_t)(q * (B_TILE_BYTES >> 4) + k16 * 2), dhi, idesc,
                           (k16 > 0 || !first) ? 1u : later);
            }
          mma_commit(&empty_bar[s]);  // the stage is free once these MMAs have read it
        }
        if (!ok) { fail(); break; }
        mma_commit(&tfull_bar[b]);    // the accumulators are final once every MMA is done
      }
      // every MMA issued has completed before TMEM is released (bounded)
      mma_commit(&fin_bar);
      if (!mbar_wait(&fin_bar, 0)) fail();
    }
  } else {
    // ---- epilogue: warp w drains TMEM lanes 32 (w mod 4) .. + 31 (output rows), columns
    // 32 h .. 32 h + 31 with h = (w - 2) / 4
    const int quad = warp & 3;
    const int cbeg = ((warp - 2) >> 2) * (TC_N / 2), cend = cbeg + TC_N / 2;
    int lt = 0;
    for (int t = blockIdx.x; t < tiles && !abort_flag; t += gridDim.x, ++lt) {
      const int b = nbuf == 2 ? (lt & 1) : 0, use = nbuf == 2 ? (lt >> 1) : lt;
      if (!mbar_wait(&tfull_bar[b], use & 1)) { fail(); break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      int u, mt, nt;
      tc_decode(t, MT, NTr, u, mt, nt);
      nt += nt_lo;
      const int i = mt * TC_M + quad * 32 + lane;
      const int erow = (i < M) ? ea[(size_t)u * Mp + i] : 0;
      const uint32_t tbase = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(b * buf_cols);
      // the exact accumulators hold integers in units of 2^-7d: combine them in an int64
      // in units of 2^-28 (|I| < 2^53), then one FP64 fma adds the rounded last one
      auto finish = [&](int c0, const uint32_t (&regs)[TC_NACC][16]) {
#pragma unroll
        for (int t2 = 0; t2 < 16; ++t2) {
          const int j = nt * TC_N + c0 + t2;
          if (j >= N) continue;
          long long I = 0;
#pragma unroll
          for (int a = 0; a < TC_NACC - 1; ++a)
            I += (long long)__float2int_rn(__uint_as_float(regs[a][t2]) *
                                           (float)(1 << (7 * acc_diag(a))))
                 << (7 * (4 - acc_diag(a)));
          double w = fma((double)I, 0x1p-28, (double)__uint_as_float(regs[TC_NACC - 1][t2]));
          int E2 = erow + fb[(size_t)u * Np + j] - 12;
          // 2^E2 from its bit pattern while it is a normal number
          double v = (E2 > -1000 && E2 < 1000)
                         ? w * __longlong_as_double((long long)(E2 + 1023) << 52)
                         : ldexp(w, E2);
          epi(u, i, j, v);
        }
      };
      auto load_tmem = [&](int c0, uint32_t (&regs)[TC_NACC][16]) {
#pragma unroll
        for (int a = 0; a < TC_NACC; ++a) {
          if (a >= nacc) {
#pragma unroll
            for (int t2 = 0; t2 < 16; ++t2) regs[a][t2] = 0u;  // +0.0f
            continue;
          }
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,"
              "%12,%13,%14,%15}, [%16];\n"
              : "=r"(regs[a][0]), "=r"(regs[a][1]), "=r"(regs[a][2]), "=r"(regs[a][3]),
                "=r"(regs[a][4]), "=r"(regs[a][5]), "=r"(regs[a][6]), "=r"(regs[a][7]),
                "=r"(regs[a][8]), "=r"(regs[a][9]), "=r"(regs[a][10]), "=r"(regs[a][11]),
                "=r"(regs[a][12]), "=r"(regs[a][13]), "=r"(regs[a][14]), "=r"(regs[a][15])
              : "r"(tbase + (uint32_t)(a * TC_N + c0)));
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (c0 + 16 >= cend) {
          // this warp's last reads of the buffer are done: hand its share back
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          __syncwarp();
          if (lane == 0) mbar_arrive(&tempty_bar[b]);
        }
      };
      if (nbuf == 2) {
        // two TMEM buffers: the next tile's MMAs already run in the other one
        for (int c0 = cbeg; c0 < cend; c0 += 16) {
          __syncwarp();
          uint32_t regs[TC_NACC][16];
          load_tmem(c0, regs);
          if (i < M) finish(c0, regs);
        }
      } else {
        // one TMEM buffer: park the raw accumulators in this CTA's (L2-resident) scratch,
        // layout [acc][column / 4][row] of float4 so that every warp store is coalesced,
        // hand TMEM back at once, and combine from the scratch while the MMAs of the next
        // tile run (each thread reads back only what it wrote)
        float4* sc = (float4*)scratch + (size_t)blockIdx.x * (TC_NACC * (TC_N / 4) * TC_M);
        const int row = quad * 32 + lane;
        for (int c0 = cbeg; c0 < cend; c0 += 16) {
          __syncwarp();
          uint32_t regs[TC_NACC][16];
          load_tmem(c0, regs);
#pragma unroll
          for (int a = 0; a < TC_NACC; ++a) {
            if (a >= nacc) continue;
#pragma unroll
            for (int g4 = 0; g4 < 4; ++g4)
              sc[((size_t)a * (TC_N / 4) + c0 / 4 + g4) * TC_M + row] =
                  make_float4(__uint_as_float(regs[a][4 * g4]), __uint_as_float(regs[a][4 * g4 + 1]),
                              __uint_as_float(regs[a][4 * g4 + 2]),
                              __uint_as_float(regs[a][4 * g4 + 3]));
          }
        }
        if (i < M)
          for (int c0 = cbeg; c0 < cend; c0 += 16) {
            uint32_t regs[TC_NACC][16];
#pragma unroll
            for (int a = 0; a < TC_NACC; ++a) {
#pragma unroll
              for (int g4 = 0; g4 < 4; ++g4) {
                float4 v4 = a < nacc ? sc[((size_t)a * (TC_N / 4) + c0 / 4 + g4) * TC_M + row]
                                     : make_float4(0.f, 0.f, 0.f, 0.f);
                regs[a][4 * g4] = __float_as_uint(v4.x);
                regs[a][4 * g4 + 1] = __float_as_uint(v4.y);
                regs[a][4 * g4 + 2] = __float_as_uint(v4.z);
                regs[a][4 * g4 + 3] = __float_as_uint(v4.w);
              }
            }
            finish(c0, regs);
          }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // after an abort, let the copies still in flight land before the CTA exits (bounded)
  if (warp == 0 && lane == 0 && abort_flag)
    for (int s = 0; s < TC_STAGES; ++s)
      if (issued[s]) mbar_wait(&full_bar[s], round_of[s] & 1);
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols)
                 : "memory");
}


// one persistent CTA per SM (each holds up to 512 TMEM columns and most of shared memory)
static int tc_grid(long long tiles) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
      sms = 1;
  }
  return (int)std::min<long long>(tiles, sms);
}

struct TcLayout {
  int Mp, Np, Kp, MT, NT, KB;
  size_t a_bytes, b_bytes, e_bytes, f_bytes, s_bytes;
};

// epilogue scratch of one persistent CTA: the raw accumulators of one tile
constexpr size_t TC_SCRATCH_PER_CTA = (size_t)TC_NACC * TC_M * TC_N * sizeof(float);

static TcLayout tc_layout(int M, int N, int K, int batch, int S) {
  TcLayout L;
  L.Mp = pad_to(M, TC_M);
  L.Np = pad_to(N, TC_N);
  L.Kp = pad_to(K, TC_KB);
  L.MT = L.Mp / TC_M;
  L.NT = L.Np / TC_N;
  L.KB = L.Kp / TC_KB;
  auto al = [](size_t b) { return (b + 1023) / 1024 * 1024; };
  L.a_bytes = al((size_t)batch * S * L.Mp * L.Kp * 2);
  L.b_bytes = al((size_t)batch * S * L.Np * L.Kp * 2);
  L.e_bytes = al((size_t)batch * L.Mp * 4);
  L.f_bytes = al((size_t)batch * L.Np * 4);
  L.s_bytes = tc_scratch_bytes();
  return L;
}

size_t tc_scratch_bytes() { return (size_t)tc_grid(1ll << 40) * TC_SCRATCH_PER_CTA; }

size_t tc_workspace_bytes(int M, int N, int K, int batch, int S) {
  TcLayout L = tc_layout(M, N, K, batch, S);
  return L.a_bytes + L.b_bytes + L.e_bytes + L.f_bytes + L.s_bytes;
}

bool tc_shape_ok(int K, int S) { return S >= 1 && S <= TC_MAXS && K >= 1 && K <= 1024; }

template <class Epi>
void tc_gemm(int M, int N, int K, const double* A, int lda, long long sA, const double* B, int ldb,
             long long sB, Epi epi, int batch, int S, void* work, unsigned* status,
             cudaStream_t s, TcKSkip zskip = TcKSkip{}, int max_ctas = 0, bool tA = false,
             bool tB = false, TcRange rg = TcRange{}) {
  if (M <= 0 || N <= 0 || batch <= 0) return;
  TcLayout L = tc_layout(M, N, K, batch, S);
  unsigned char* w = (unsigned char*)work;
  unsigned short* As = (unsigned short*)w;
  unsigned short* Bs = (unsigned short*)(w + L.a_bytes);
  int* ea = (int*)(w + L.a_bytes + L.b_bytes);
  int* fb = (int*)(w + L.a_bytes + L.b_bytes + L.e_bytes);
  float* scratch = (float*)(w + L.a_bytes + L.b_bytes + L.e_bytes + L.f_bytes);
  // A rows (A^T: the columns of A stored K x M) and B columns (B^T: the rows of B stored N x K)
#define VRTE_SLICE_AB(SS)                                                                       \
  if (tA)                                                                                       \
    k_slice_cols<SS, TC_M><<<dim3(L.MT, batch), 512, 0, s>>>(M, K, A, lda, sA, As, ea, status);  \
  else                                                                                          \
    k_slice_rows<SS, TC_M><<<dim3(L.MT, batch), 256, 0, s>>>(M, K, A, lda, sA, As, ea, status);  \
  if (tB)                                                                                       \
    k_slice_rows<SS, TC_N><<<dim3(L.NT, batch), 256, 0, s>>>(N, K, B, ldb, sB, Bs, fb, status);  \
  else                                                                                          \
    k_slice_cols<SS, TC_N><<<dim3(L.NT, batch), 512, 0, s>>>(N, K, B, ldb, sB, Bs, fb, status)
  if (rg.slice) VRTE_SLICE_DISPATCH(S, VRTE_SLICE_AB)
#undef VRTE_SLICE_AB
  if (!rg.run) return;
  const int nt_lo = rg.nt_cnt > 0 ? rg.nt_lo : 0;
  const int nt_cnt = rg.nt_cnt > 0 ? std::min(rg.nt_cnt, L.NT - nt_lo) : L.NT;
  if (nt_lo < 0 || nt_cnt <= 0) return;
  int smem = tc_smem_bytes(S);
  cudaFuncSetAttribute(k_tc_gemm<Epi>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  int grid = tc_grid((long long)L.MT * nt_cnt * batch);
  if (max_ctas > 0) grid = std::min(grid, max_ctas);
  k_tc_gemm<Epi><<<grid, TC_THREADS, smem, s>>>(
      M, N, K, S, As, ea, Bs, fb, scratch, epi, status, batch, zskip, nt_lo, nt_cnt);
}

struct TcEpiStore {
  double* C;
  int ldc;
  long long sC;
  double beta;
  double alpha = 1.0;
  __device__ void operator()(int u, int i, int j, double v) const {
    double* c = C + (size_t)u * sC + (size_t)i * ldc + j;
    *c = beta == 0.0 ? alpha * v : fma(alpha, v, beta * *c);
  }
};

void tc_gemm_store(int M, int N, int K, const double* A, int lda, long long sA, const double* B,
                   int ldb, long long sB, double beta, double* C, int ldc, long long sC,
                   int batch, int S, void* work, unsigned* status, cudaStream_t s,
                   TcKSkip zskip, int max_ctas, TcRange rg) {
  tc_gemm(M, N, K, A, lda, sA, B, ldb, sB, TcEpiStore{C, ldc, sC, beta}, batch, S, work, status,
          s, zskip, max_ctas, false, false, rg);
}

void tc_gemm_store_t(bool tA, bool tB, int M, int N, int K, double alpha, const double* A,
                     int lda, long long sA, const double* B, int ldb, long long sB, double beta,
                     double* C, int ldc, long long sC, int batch, int S, void* work,
                     unsigned* status, cudaStream_t s) {
  tc_gemm(M, N, K, A, lda, sA, B, ldb, sB, TcEpiStore{C, ldc, sC, beta, alpha}, batch, S, work,
          status, s, TcKSkip{}, 0, tA, tB);
}

void tc_gemm_part(const OrderBatch& b, int K, const double* A, int lda, long long sA,
                  const double* B, long long sB, const double* T1, const double* g0tab,
                  double* Isyn, int S, void* work, cudaStream_t s, TcKSkip zskip,
                  int* nonfinite, TcRange rg) {
  EpiPart e{T1, Isyn, g0tab, b.N, b.n_in, b.n_out, b.m0, nonfinite};
  tc_gemm(4 * b.n_out, 4 * b.n_in, K, A, lda, sA, B, 4 * b.n_in, sB, e, b.n_units, S, work,
          b.status, s, zskip, 0, false, false, rg);
}

// First half of a reconstruction contraction too deep for one exact accumulation
// (K > 1024): T1[u][i][j] += g0(o, k) acc, the second half then goes through EpiPart.
struct EpiPartAccum {
  double* T1;
  const double* g0tab;
  int n_in, n_out;
  __device__ void operator()(int u, int i, int j, double acc) const {
    int R = 4 * n_in;
    double* t = T1 + (size_t)u * (4 * n_out) * R + (size_t)i * R + j;
    *t = fma(g0tab[(size_t)(i >> 2) * n_in + (j >> 2)], acc, *t);
  }
};

void tc_gemm_part_accum(const OrderBatch& b, int K, const double* A, int lda, long long sA,
                        const double* B, long long sB, double* T1, const double* g0tab, int S,
                        void* work, cudaStream_t s, TcKSkip zskip) {
  EpiPartAccum e{T1, g0tab, b.n_in, b.n_out};
  tc_gemm(4 * b.n_out, 4 * b.n_in, K, A, lda, sA, B, 4 * b.n_in, sB, e, b.n_units, S, work,
          b.status, s, zskip);
}

}  // namespace vrte

extern "C" size_t vrte_gemm_sliced_workspace(int M, int N, int K, int batch, int slices) {
  if (M < 1 || N < 1 || batch < 1 || !vrte::tc_shape_ok(K, slices)) return 0;
  return vrte::tc_workspace_bytes(M, N, K, batch, slices);
}

extern "C" vrte_status vrte_gemm_sliced(int M, int N, int K, const double* d_A, int lda,
                                        long long stride_a, const double* d_B, int ldb,
                                        long long stride_b, double* d_C, int ldc,
                                        long long stride_c, int batch, int slices,
                                        void* d_workspace, size_t workspace_bytes,
                                        unsigned* d_status, void* stream) {
  if (M < 1 || N < 1 || batch < 1 || !vrte::tc_shape_ok(K, slices) || !d_A || !d_B || !d_C ||
      !d_workspace || !d_status || lda < K || ldb < N || ldc < N)
    return VRTE_ERR_INVALID_ARG;
  if (workspace_bytes < vrte::tc_workspace_bytes(M, N, K, batch, slices))
    return VRTE_ERR_INVALID_ARG;
  vrte::tc_gemm_store(M, N, K, d_A, lda, stride_a, d_B, ldb, stride_b, 0.0, d_C, ldc, stride_c,
                      batch, slices, d_workspace, d_status, (cudaStream_t)stream);
  return cudaGetLastError() == cudaSuccess ? VRTE_OK : VRTE_ERR_CUDA;
}
