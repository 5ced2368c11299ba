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
// memory image of 128B-swizzled K-major tiles ([unit][slice][tile][k-block] blocks of
// 128 x 64 or 64 x 64 BF16), so the GEMM kernel loads each tile with one bulk copy. The
// GEMM kernel computes a 128 x 64 output tile per CTA with up to seven accumulators of 64
// columns in TMEM, as many shared-memory stages as fit (S = 7: one of 168 KB; S <= 4: two
// or three; a 32-wide K block with two stages at S = 7 measured slower), one thread issuing
// bulk copies and MMAs, and four warps draining TMEM in the epilogue. Every mbarrier wait
// is bounded; on timeout the kernel records ST_TIMEOUT, waits (bounded) for its copies,
// frees TMEM and returns.
#include <stdint.h>

#include <algorithm>

#include "tc_common.cuh"

namespace vrte {

constexpr int TC_M = 128;       // output rows per CTA (MMA M)
constexpr int TC_N = 64;        // output columns per CTA (MMA N)
constexpr int TC_KB = 64;       // K per stage (one 128-byte swizzle row of BF16)
constexpr int TC_MAXS = 8;      // maximum number of slices
constexpr int TC_NACC = 7;      // TMEM accumulators (see acc_index)
constexpr int TC_STAGES = 3;    // shared-memory stages (at most)
constexpr int TC_SMEM_MAX = 227 * 1024;
constexpr int A_TILE_BYTES = TC_M * TC_KB * 2;   // 16 KiB
constexpr int B_TILE_BYTES = TC_N * TC_KB * 2;   // 8 KiB

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
// as many stages (up to three) of S slices of A and B tiles as fit in shared memory
__device__ __host__ inline int tc_stages(int S) {
  int n = (TC_SMEM_MAX - 1024) / (S * (A_TILE_BYTES + B_TILE_BYTES));
  return n < 1 ? 1 : (n > TC_STAGES ? TC_STAGES : n);
}
__device__ __host__ inline int tc_smem_bytes(int S) {
  return tc_stages(S) * S * (A_TILE_BYTES + B_TILE_BYTES) + 1024;
}

// Byte offset of element (row r, k) inside a 128B-swizzled K-major tile of 64 BF16 per row:
// 8-row groups of 1024 bytes, 128 bytes per row, 16-byte chunk index XOR (row mod 8).
__device__ inline int swz_offset(int r, int k) {
  int chunk = k >> 3, within = k & 7;
  return (r >> 3) * 1024 + (r & 7) * 128 + ((chunk ^ (r & 7)) << 4) + within * 2;
}

// A rows: A[u][i][k] (row-major, lda, unit stride sA), M x K. Writes
//   out[u][p][mt][kb] tiles (128 x 64 BF16 images) and e[u][i] (int exponent).
// One CTA per (row block of 128, unit); each thread slices 8 consecutive k of one row.
template <int S>
__global__ void k_slice_rows(int M, int K, const double* __restrict__ A, int lda,
                             long long sA, unsigned short* out, int* e_out, unsigned* status) {
  int mt = blockIdx.x, u = blockIdx.y;
  int Mp = pad_to(M, TC_M), Kp = pad_to(K, TC_KB), KB = Kp / TC_KB, MT = Mp / TC_M;
  __shared__ int ex[TC_M];
  const double* Ab = A + (size_t)u * sA;
  bool bad = false;
  // per-row exponent: warp per row, integer max of the exponent fields
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int r = warp; r < TC_M; r += nw) {
    int i = mt * TC_M + r;
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
  const size_t tile_elems = (size_t)TC_M * TC_KB;
  const size_t slice_stride = (size_t)MT * KB * tile_elems;
  const int chunks = Kp / 8;
  for (int idx = threadIdx.x; idx < TC_M * chunks; idx += blockDim.x) {
    int r = idx / chunks, k0 = 8 * (idx - r * chunks);
    int i = mt * TC_M + r;
    double v[8];
    for (int t = 0; t < 8; ++t)
      v[t] = (i < M && k0 + t < K) ? Ab[(size_t)i * lda + k0 + t] : 0.0;
    int kb = k0 / TC_KB;
    size_t base = ((((size_t)u * S) * MT + mt) * KB + kb) * tile_elems;
    put_chunk<S>(v, ex[r], out + base + (swz_offset(r, k0 - kb * TC_KB) >> 1), slice_stride);
  }
  if (bad) atomicOr(status, ST_NONFINITE);
}

// B columns: B[u][k][j] (row-major, ldb, unit stride sB), K x N, sliced per column j
// into K-major tiles out[u][q][nt][kb] (64 x 64 BF16 images, row = j) and f[u][j].
// Each thread slices 8 consecutive k of one column (consecutive threads: consecutive
// columns, so every global load is coalesced).
template <int S>
__global__ void k_slice_cols(int N, int K, const double* __restrict__ B, int ldb,
                             long long sB, unsigned short* out, int* f_out, unsigned* status) {
  int nt = blockIdx.x, u = blockIdx.y;
  int Np = pad_to(N, TC_N), Kp = pad_to(K, TC_KB), KB = Kp / TC_KB, NT = Np / TC_N;
  __shared__ int ex[TC_N];
  __shared__ int red[8][TC_N];
  const double* Bb = B + (size_t)u * sB;
  bool bad = false;
  // per-column max exponent: threads over columns (coalesced rows), 8 row groups
  int c = threadIdx.x % TC_N, g = threadIdx.x / TC_N;  // blockDim = 512 -> 8 groups
  int j = nt * TC_N + c;
  int Em = 0;
  if (j < N)
    for (int k = g; k < K; k += 8) Em = max(Em, exp_field(Bb[(size_t)k * ldb + j], &bad));
  red[g][c] = Em;
  __syncthreads();
  if (g == 0) {
    int m2 = 0;
    for (int q = 0; q < 8; ++q) m2 = max(m2, red[q][c]);
    ex[c] = scale_exp(m2);
    if (j < N) f_out[(size_t)u * Np + j] = ex[c];
  }
  __syncthreads();
  const size_t tile_elems = (size_t)TC_N * TC_KB;
  const size_t slice_stride = (size_t)NT * KB * tile_elems;
  const int chunks = Kp / 8;
  for (int idx = threadIdx.x; idx < TC_N * chunks; idx += blockDim.x) {
    int k0 = 8 * (idx / TC_N), cc = idx % TC_N;
    int jj = nt * TC_N + cc;
    double v[8];
    for (int t = 0; t < 8; ++t)
      v[t] = (jj < N && k0 + t < K) ? Bb[(size_t)(k0 + t) * ldb + jj] : 0.0;
    int kb = k0 / TC_KB;
    size_t base = ((((size_t)u * S) * NT + nt) * KB + kb) * tile_elems;
    put_chunk<S>(v, ex[cc], out + base + (swz_offset(cc, k0 - kb * TC_KB) >> 1), slice_stride);
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

template <class Epi>
__global__ void __launch_bounds__(128) k_tc_gemm(int M, int N, int K, int S,
                                                 const unsigned short* __restrict__ As,
                                                 const int* __restrict__ ea,
                                                 const unsigned short* __restrict__ Bs,
                                                 const int* __restrict__ fb, Epi epi,
                                                 unsigned* status, int batch) {
  // Persistent: CTA b takes tiles b, b + gridDim.x, ... (tile t = mt + MT (nt + NT u)).
  // Thread 0 issues bulk copies and MMAs; once a tile's MMAs are done it starts the next
  // tile's first copies, which land while the four warps drain TMEM.
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ uint64_t full_bar[TC_STAGES], empty_bar[TC_STAGES], done_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  // align the dynamic region to 1024 bytes (128B swizzle atoms)
  unsigned char* smem =
      (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int Mp = pad_to(M, TC_M), Np = pad_to(N, TC_N), Kp = pad_to(K, TC_KB);
  const int KB = Kp / TC_KB, MT = Mp / TC_M, NT = Np / TC_N;
  const int tiles = MT * NT * batch;
  const int stage_bytes = S * (A_TILE_BYTES + B_TILE_BYTES);
  const int nst = tc_stages(S);
  const int nacc = acc_count(S);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t ncols = (nacc * TC_N <= 128) ? 128 : (nacc * TC_N <= 256 ? 256 : 512);

  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&done_bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(ncols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  // instruction descriptor: D = F32, A = B = BF16, K-major, N = 64, M = 128
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_N >> 3) << 17) |
                         ((uint32_t)(TC_M >> 4) << 24);
  const size_t a_unit = (size_t)S * MT * KB * (A_TILE_BYTES / 2);
  const size_t b_unit = (size_t)S * NT * KB * (B_TILE_BYTES / 2);

  // thread-0 pipeline state (barrier phases carry over from tile to tile)
  bool pending[TC_STAGES] = {};
  bool unwaited[TC_STAGES] = {};
  uint32_t full_phase[TC_STAGES] = {}, empty_phase[TC_STAGES] = {}, done_phase = 0;
  int issued = 0;
  auto issue_copies = [&](int t, int kb, int s) {
    const int tmt = t % MT, tnt = (t / MT) % NT, tu = t / (MT * NT);
    unsigned char* st = smem + (size_t)s * stage_bytes;
    mbar_expect_tx(&full_bar[s], (unsigned)stage_bytes);
    for (int p = 0; p < S; ++p) {
      const unsigned short* src =
          As + (size_t)tu * a_unit + (((size_t)p * MT + tmt) * KB + kb) * (A_TILE_BYTES / 2);
      bulk_g2s(st + p * A_TILE_BYTES, src, A_TILE_BYTES, &full_bar[s]);
    }
    for (int q = 0; q < S; ++q) {
      const unsigned short* src =
          Bs + (size_t)tu * b_unit + (((size_t)q * NT + tnt) * KB + kb) * (B_TILE_BYTES / 2);
      bulk_g2s(st + S * A_TILE_BYTES + q * B_TILE_BYTES, src, B_TILE_BYTES, &full_bar[s]);
    }
    pending[s] = true;
  };
  auto prologue = [&](int t) {
    for (issued = 0; issued < KB && issued < nst; ++issued) issue_copies(t, issued, issued);
  };
  if (threadIdx.x == 0 && (int)blockIdx.x < tiles) prologue(blockIdx.x);

  for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int mt = tile % MT, nt = (tile / MT) % NT, u = tile / (MT * NT);
    if (threadIdx.x == 0) {
      bool ok = true;
      unsigned written = 0;  // accumulators that hold a value (the first MMA overwrites)
      for (int kb = 0; kb < KB && ok; ++kb) {
        int s = kb % nst;
        if (!mbar_wait(&full_bar[s], full_phase[s])) { ok = false; break; }
        full_phase[s] ^= 1;
        pending[s] = false;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        unsigned char* st = smem + (size_t)s * stage_bytes;
        // descriptors differ only in the start-address field (bits 0-13, 16-byte units)
        const uint64_t abase = smem_desc_sw128(st);
        const uint64_t bbase = smem_desc_sw128(st + S * A_TILE_BYTES);
        for (int p = 0; p < S; ++p)
          for (int q = 0; p + q < S; ++q) {
            int a = acc_index(p, q);
            uint32_t dt = tmem + (uint32_t)(a * TC_N);
#pragma unroll
            for (int k16 = 0; k16 < TC_KB / 16; ++k16) {
              uint64_t ad = abase + (uint64_t)(p * (A_TILE_BYTES >> 4) + k16 * 2);
              uint64_t bd = bbase + (uint64_t)(q * (B_TILE_BYTES >> 4) + k16 * 2);
              uint32_t acc = (k16 == 0 && !((written >> a) & 1u)) ? 0u : 1u;
              mma_bf16(dt, ad, bd, idesc, acc);
            }
            written |= 1u << a;
          }
        mma_commit(&empty_bar[s]);
        unwaited[s] = true;
        // refill the previous block's stage once its MMAs are done, so that the MMAs just
        // issued keep the tensor pipe busy meanwhile (with one stage: this block's stage)
        const int lag = nst > 1 ? 1 : 0;
        if (kb >= lag && issued < KB) {
          int ps = (kb - lag) % nst;
          if (!mbar_wait(&empty_bar[ps], empty_phase[ps])) { ok = false; break; }
          empty_phase[ps] ^= 1;
          unwaited[ps] = false;
          issue_copies(tile, issued, ps);
          ++issued;
        }
      }
      // every MMA issued so far has completed once done_bar fires (also before an abort)
      mma_commit(&done_bar);
      if (!mbar_wait(&done_bar, done_phase)) ok = false;
      done_phase ^= 1;
      // the stage releases not waited for have completed too: keep the phases in step
      for (int s2 = 0; s2 < TC_STAGES; ++s2)
        if (unwaited[s2]) { empty_phase[s2] ^= 1; unwaited[s2] = false; }
      if (ok && tile + (int)gridDim.x < tiles) prologue(tile + gridDim.x);
      if (!ok) {
        abort_flag = 1;
        atomicOr(status, ST_TIMEOUT);
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (abort_flag) break;

    // epilogue: warp w drains TMEM lanes 32w..32w+31 (output rows), 16 columns at a time
    const int r = warp * 32 + lane;
    const int i = mt * TC_M + r;
    const int erow = (i < M) ? ea[(size_t)u * Mp + i] : 0;
    for (int c0 = 0; c0 < TC_N; c0 += 16) {
      uint32_t regs[TC_NACC][16];
#pragma unroll
      for (int a = 0; a < TC_NACC; ++a) {
        if (a >= nacc) {
#pragma unroll
          for (int t = 0; t < 16; ++t) regs[a][t] = 0u;  // +0.0f
          continue;
        }
        uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(a * TC_N + c0);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
            "%13,%14,%15}, [%16];\n"
            : "=r"(regs[a][0]), "=r"(regs[a][1]), "=r"(regs[a][2]), "=r"(regs[a][3]),
              "=r"(regs[a][4]), "=r"(regs[a][5]), "=r"(regs[a][6]), "=r"(regs[a][7]),
              "=r"(regs[a][8]), "=r"(regs[a][9]), "=r"(regs[a][10]), "=r"(regs[a][11]),
              "=r"(regs[a][12]), "=r"(regs[a][13]), "=r"(regs[a][14]), "=r"(regs[a][15])
            : "r"(taddr));
      }
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (i >= M) continue;
      if constexpr (Epi::kF32) {
        // FP32 output: an error-free FP32 sum (hi + lo) of the accumulators, largest first,
        // rounded once; no FP64 instruction
#pragma unroll
        for (int t = 0; t < 16; ++t) {
          float hi = 0.0f, lo = 0.0f;
#pragma unroll
          for (int a = 0; a < TC_NACC; ++a) {
            float x = __uint_as_float(regs[a][t]);
            float sm = hi + x, bb = sm - hi;
            lo += (hi - (sm - bb)) + (x - bb);
            hi = sm;
          }
          int j = nt * TC_N + c0 + t;
          if (j < N) {
            int E2 = erow + fb[(size_t)u * Np + j] - 12;
            float w = hi + lo;
            float v = (E2 > -120 && E2 < 120) ? w * __int_as_float((E2 + 127) << 23)
                                              : ldexpf(w, E2);
            epi.put32(u, i, j, v);
          }
        }
      } else {
        // the exact accumulators hold integers in units of 2^-7d: combine them in an int64
        // in units of 2^-28 (|I| < 2^53), then one FP64 fma adds the rounded last one
#pragma unroll
        for (int t = 0; t < 16; ++t) {
          long long I = 0;
          float r4 = 0.0f;
#pragma unroll
          for (int a = 0; a < TC_NACC; ++a) {
            float x = __uint_as_float(regs[a][t]);
            if (a < TC_NACC - 1)  // exact: an integer times 2^-7d, d = acc_diag(a)
              I += (long long)__float2int_rn(x * (float)(1 << (7 * acc_diag(a))))
                   << (7 * (4 - acc_diag(a)));
            else
              r4 = x;
          }
          int j = nt * TC_N + c0 + t;
          if (j < N) {
            double w = fma((double)I, 0x1p-28, (double)r4);
            int E2 = erow + fb[(size_t)u * Np + j] - 12;
            // 2^E2 from its bit pattern while it is a normal number
            double v = (E2 > -1000 && E2 < 1000)
                           ? w * __longlong_as_double((long long)(E2 + 1023) << 52)
                           : ldexp(w, E2);
            epi(u, i, j, v);
          }
        }
      }
    }
    // TMEM is free for the next tile's MMAs once every warp has read it
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  if (threadIdx.x == 0 && abort_flag) {
    // let the copies still in flight land before the CTA exits (bounded)
    for (int s = 0; s < TC_STAGES; ++s)
      if (pending[s]) mbar_wait(&full_bar[s], full_phase[s]);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
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
  size_t a_bytes, b_bytes, e_bytes, f_bytes;
};

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
  return L;
}

size_t tc_workspace_bytes(int M, int N, int K, int batch, int S) {
  TcLayout L = tc_layout(M, N, K, batch, S);
  return L.a_bytes + L.b_bytes + L.e_bytes + L.f_bytes;
}

bool tc_shape_ok(int K, int S) { return S >= 1 && S <= TC_MAXS && K >= 1 && K <= 1024; }

template <class Epi>
void tc_gemm(int M, int N, int K, const double* A, int lda, long long sA, const double* B, int ldb,
             long long sB, Epi epi, int batch, int S, void* work, unsigned* status,
             cudaStream_t s) {
  if (M <= 0 || N <= 0 || batch <= 0) return;
  TcLayout L = tc_layout(M, N, K, batch, S);
  unsigned char* w = (unsigned char*)work;
  unsigned short* As = (unsigned short*)w;
  unsigned short* Bs = (unsigned short*)(w + L.a_bytes);
  int* ea = (int*)(w + L.a_bytes + L.b_bytes);
  int* fb = (int*)(w + L.a_bytes + L.b_bytes + L.e_bytes);
#define VRTE_SLICE_AB(SS)                                                                  \
  k_slice_rows<SS><<<dim3(L.MT, batch), 256, 0, s>>>(M, K, A, lda, sA, As, ea, status);  \
  k_slice_cols<SS><<<dim3(L.NT, batch), 512, 0, s>>>(N, K, B, ldb, sB, Bs, fb, status)
  VRTE_SLICE_DISPATCH(S, VRTE_SLICE_AB)
#undef VRTE_SLICE_AB
  int smem = tc_smem_bytes(S);
  cudaFuncSetAttribute(k_tc_gemm<Epi>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  k_tc_gemm<Epi><<<tc_grid((long long)L.MT * L.NT * batch), 128, smem, s>>>(
      M, N, K, S, As, ea, Bs, fb, epi, status, batch);
}

struct TcEpiStore {
  static constexpr bool kF32 = false;
  double* C;
  int ldc;
  long long sC;
  double beta;
  __device__ void operator()(int u, int i, int j, double v) const {
    double* c = C + (size_t)u * sC + (size_t)i * ldc + j;
    *c = beta == 0.0 ? v : v + beta * *c;
  }
};

void tc_gemm_store(int M, int N, int K, const double* A, int lda, long long sA, const double* B,
                   int ldb, long long sB, double beta, double* C, int ldc, long long sC,
                   int batch, int S, void* work, unsigned* status, cudaStream_t s) {
  tc_gemm(M, N, K, A, lda, sA, B, ldb, sB, TcEpiStore{C, ldc, sC, beta}, batch, S, work, status,
          s);
}

void tc_gemm_part(const OrderBatch& b, int K, const double* A, int lda, long long sA,
                  const double* B, long long sB, const double* T1, const double* g0tab,
                  double* Isyn, int S, void* work, cudaStream_t s) {
  EpiPart e{T1, Isyn, g0tab, b.N, b.n_in, b.n_out, b.m0};
  tc_gemm(4 * b.n_out, 4 * b.n_in, K, A, lda, sA, B, 4 * b.n_in, sB, e, b.n_units, S, work,
          b.status, s);
}

// First half of a reconstruction contraction too deep for one exact accumulation
// (K > 1024): T1[u][i][j] += g0(o, k) acc, the second half then goes through EpiPart.
struct EpiPartAccum {
  static constexpr bool kF32 = false;
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
                        void* work, cudaStream_t s) {
  EpiPartAccum e{T1, g0tab, b.n_in, b.n_out};
  tc_gemm(4 * b.n_out, 4 * b.n_in, K, A, lda, sA, B, 4 * b.n_in, sB, e, b.n_units, S, work,
          b.status, s);
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
