// Dense FP64 linear algebra on CUDA cores: batched GEMM (with an epilogue hook for the
// reconstruction) and batched in-place Gauss-Jordan inversion with partial pivoting.
// FP64 stays on the CUDA cores: sm_103a has no FP64 tensor-core path worth using.
#include "vrte_internal.cuh"

namespace vrte {

constexpr int GB_M = 64, GB_N = 64, GB_K = 16;

struct EpiStore {
  double alpha, beta;
  double* C;
  int ldc;
  long long sC;
  __device__ void operator()(int u, int i, int j, double acc) const {
    double* c = C + (size_t)u * sC + (size_t)i * ldc + j;
    *c = beta == 0.0 ? alpha * acc : alpha * acc + beta * *c;
  }
};

// Tiled FP64 GEMM: 64x64 output tile, 256 threads, 4x4 outputs per thread (strided by 16
// so shared-memory reads are conflict free), K staged 16 at a time. Row-major operands;
// tA / tB select op(A) = A^T (A stored K x M) and op(B) = B^T (B stored N x K).
template <class Epi>
__global__ void __launch_bounds__(256) k_dgemm(int M, int N, int K, const double* __restrict__ A,
                                               int lda, long long sA, bool tA,
                                               const double* __restrict__ B, int ldb,
                                               long long sB, bool tB, Epi epi, const int* mask) {
  __shared__ double As[GB_K][GB_M + 1];
  __shared__ double Bs[GB_K][GB_N + 1];
  int u = blockIdx.z;
  if (mask && !mask[u]) return;
  int m0 = blockIdx.y * GB_M, n0 = blockIdx.x * GB_N;
  int tid = threadIdx.x;
  int tx = tid & 15, ty = tid >> 4;
  const double* Ab = A + (size_t)u * sA;
  const double* Bb = B + (size_t)u * sB;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  for (int k0 = 0; k0 < K; k0 += GB_K) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int row, kk;
      if (!tA) { kk = tid & 15; row = (tid >> 4) + 16 * q; }
      else { row = tid & 63; kk = (tid >> 6) + 4 * q; }
      int gi = m0 + row, gk = k0 + kk;
      double v = 0.0;
      if (gi < M && gk < K) v = tA ? Ab[(size_t)gk * lda + gi] : Ab[(size_t)gi * lda + gk];
      As[kk][row] = v;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int col, kk;
      if (!tB) { col = tid & 63; kk = (tid >> 6) + 4 * q; }
      else { kk = tid & 15; col = (tid >> 4) + 16 * q; }
      int gj = n0 + col, gk = k0 + kk;
      double v = 0.0;
      if (gj < N && gk < K) v = tB ? Bb[(size_t)gj * ldb + gk] : Bb[(size_t)gk * ldb + gj];
      Bs[kk][col] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GB_K; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int gi = m0 + ty + 16 * i, gj = n0 + tx + 16 * j;
      if (gi < M && gj < N) epi(u, gi, gj, acc[i][j]);
    }
}

template <class Epi>
static void run_dgemm(int M, int N, int K, const double* A, int lda, long long sA, bool tA,
                      const double* B, int ldb, long long sB, bool tB, Epi epi, int batch,
                      cudaStream_t s, const int* mask = nullptr) {
  if (M <= 0 || N <= 0 || batch <= 0) return;
  dim3 grid((N + GB_N - 1) / GB_N, (M + GB_M - 1) / GB_M, batch);
  k_dgemm<Epi><<<grid, 256, 0, s>>>(M, N, K, A, lda, sA, tA, B, ldb, sB, tB, epi, mask);
}

void dgemm_batched_mask(bool tA, bool tB, int M, int N, int K, double alpha, const double* A,
                        int lda, long long sA, const double* B, int ldb, long long sB, double beta,
                        double* C, int ldc, long long sC, int batch, const int* mask,
                        cudaStream_t s) {
  EpiStore e{alpha, beta, C, ldc, sC};
  run_dgemm(M, N, K, A, lda, sA, tA, B, ldb, sB, tB, e, batch, s, mask);
}

void dgemm_batched_t(bool tA, bool tB, int M, int N, int K, double alpha, const double* A,
                     int lda, long long sA, const double* B, int ldb, long long sB, double beta,
                     double* C, int ldc, long long sC, int batch, cudaStream_t s) {
  EpiStore e{alpha, beta, C, ldc, sC};
  run_dgemm(M, N, K, A, lda, sA, tA, B, ldb, sB, tB, e, batch, s);
}

void dgemm_batched(int M, int N, int K, double alpha, const double* A, int lda, long long sA,
                   const double* B, int ldb, long long sB, double beta, double* C, int ldc,
                   long long sC, int batch, cudaStream_t s) {
  dgemm_batched_t(false, false, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, batch, s);
}

void dgemm_part_epilogue(const OrderBatch& b, const double* A, const double* B, const double* T1,
                         const double* g0tab, double* Isyn, cudaStream_t s) {
  int Ro = 4 * b.n_out, R = 4 * b.n_in, n2 = 2 * b.n;
  EpiPart e{T1, Isyn, g0tab, b.N, b.n_in, b.n_out, b.m0};
  run_dgemm(Ro, R, n2, A, b.ldU, (long long)Ro * b.ldU, false, B, R, b.sSD, false, e,
            b.n_units, s);
}

// Gauss-Jordan inversion with partial (row) pivoting, blocked, one CTA per matrix.
// The unblocked algorithm's step k picks the largest |W[i][k]|, i >= k, swaps rows,
// scales the pivot row and subtracts multiples of it from every other row, the pivot
// column taking the inverse's column; row swaps are undone at the end by swapping
// columns in reverse order. Here the steps run BI columns at a time: the panel of BI
// columns is eliminated in shared memory (recording each step's column C_c and the
// swaps), and the other columns receive the BI steps at once. With the swaps applied
// first, an outside column v maps to v + Z v[blk], where over the block rows
// (pivots D, strictly lower part Lw and strictly upper part Up of C[blk])
//   Q = (D + Lw)^-1,  Z[blk] = (I - Up) Q - I,  Z[other] = -C[other] Q,
// a rank-BI update read from and written to global memory once per block (the
// unblocked form reads and writes the whole matrix at every step).
// A zero or non-finite pivot sets ST_SINGULAR (the matrix is still processed).
constexpr int BI = 16;   // panel width
constexpr int TJ = 32;   // column tile of the outside update

__global__ void __launch_bounds__(512) k_inverse(int n, const double* __restrict__ A,
                                                 double* __restrict__ Ainv, unsigned* status) {
  extern __shared__ double sh[];
  double* P = sh;                  // [n][BI] panel
  double* Cb = P + (size_t)n * BI; // [n][BI] step columns, then Z
  double* Wb = Cb + (size_t)n * BI;// [BI][TJ] block rows of a column tile
  int* perm = (int*)(Wb + BI * TJ);
  __shared__ double red_v[16];
  __shared__ int red_i[16];
  __shared__ double rk[BI];
  __shared__ double Q[BI][BI], G[BI][BI];
  const int u = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const double* Ab = A + (size_t)u * n * n;
  double* W = Ainv + (size_t)u * n * n;
  for (size_t e = tid; e < (size_t)n * n; e += nt) W[e] = Ab[e];
  __syncthreads();
  for (int k0 = 0; k0 < n; k0 += BI) {
    const int bb = min(BI, n - k0);
    for (int e = tid; e < n * bb; e += nt) {
      int i = e / bb, c = e - i * bb;
      P[i * BI + c] = W[(size_t)i * n + k0 + c];
    }
    __syncthreads();
    // ---- panel elimination
    for (int c = 0; c < bb; ++c) {
      const int k = k0 + c;
      double best = -1.0;
      int bi = k;
      for (int i = k + tid; i < n; i += nt) {
        double v = fabs(P[i * BI + c]);
        if (v > best) { best = v; bi = i; }
      }
      for (int off = 16; off > 0; off >>= 1) {
        double ov = __shfl_down_sync(0xffffffffu, best, off);
        int oi = __shfl_down_sync(0xffffffffu, bi, off);
        if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
      }
      if ((tid & 31) == 0) { red_v[tid >> 5] = best; red_i[tid >> 5] = bi; }
      __syncthreads();
      if (tid < 32) {
        int nw = (nt + 31) >> 5;
        best = tid < nw ? red_v[tid] : -1.0;
        bi = tid < nw ? red_i[tid] : k;
        for (int off = 16; off > 0; off >>= 1) {
          double ov = __shfl_down_sync(0xffffffffu, best, off);
          int oi = __shfl_down_sync(0xffffffffu, bi, off);
          if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
        }
        if (tid == 0) { red_i[0] = bi; perm[k] = bi; }
      }
      __syncthreads();
      const int p = red_i[0];
      if (p != k && tid < BI) {
        // the panel row, and the recorded columns of earlier steps, follow the swap
        double t = P[k * BI + tid];
        P[k * BI + tid] = P[p * BI + tid];
        P[p * BI + tid] = t;
        if (tid < c) {
          t = Cb[k * BI + tid];
          Cb[k * BI + tid] = Cb[p * BI + tid];
          Cb[p * BI + tid] = t;
        }
      }
      __syncthreads();
      for (int i = tid; i < n; i += nt) Cb[i * BI + c] = P[i * BI + c];
      __syncthreads();
      const double piv = P[k * BI + c];
      if (tid == 0 && (piv == 0.0 || !isfinite(piv))) atomicOr(status, ST_SINGULAR);
      const double pinv = 1.0 / piv;
      if (tid < bb) rk[tid] = (tid == c) ? pinv : P[k * BI + tid] * pinv;
      __syncthreads();
      for (int e = tid; e < n * bb; e += nt) {
        int i = e / bb, cc = e - i * bb;
        if (i == k) {
          P[i * BI + cc] = rk[cc];
        } else {
          double w = (cc == c) ? 0.0 : P[i * BI + cc];
          P[i * BI + cc] = w - Cb[i * BI + c] * rk[cc];
        }
      }
      __syncthreads();
    }
    for (int e = tid; e < n * bb; e += nt) {
      int i = e / bb, c = e - i * bb;
      W[(size_t)i * n + k0 + c] = P[i * BI + c];
    }
    // ---- the block's swaps on the outside columns, in order
    for (int c = 0; c < bb; ++c) {
      const int k = k0 + c, p = perm[k];
      if (p != k)
        for (int j = tid; j < n; j += nt) {
          if (j >= k0 && j < k0 + bb) continue;
          double t = W[(size_t)k * n + j];
          W[(size_t)k * n + j] = W[(size_t)p * n + j];
          W[(size_t)p * n + j] = t;
        }
      __syncthreads();
    }
    // ---- Q = (D + Lw)^-1 (forward substitution per column), G = (I - Up) Q
    if (tid < bb) {
      const int col = tid;
      for (int r = 0; r < bb; ++r) {
        double acc = (r == col) ? 1.0 : 0.0;
        for (int c2 = 0; c2 < r; ++c2) acc -= Cb[(k0 + r) * BI + c2] * Q[c2][col];
        Q[r][col] = acc / Cb[(k0 + r) * BI + r];
      }
    }
    __syncthreads();
    if (tid < bb * bb) {
      const int r = tid / bb, c = tid - r * bb;
      double g = Q[r][c];
      for (int c2 = r + 1; c2 < bb; ++c2) g -= Cb[(k0 + r) * BI + c2] * Q[c2][c];
      G[r][c] = g;
    }
    __syncthreads();
    // Z overwrites C row by row (each row only reads its own entries)
    for (int i = tid; i < n; i += nt) {
      double z[BI];
      if (i >= k0 && i < k0 + bb) {
        const int r = i - k0;
#pragma unroll
        for (int c = 0; c < BI; ++c) z[c] = (c < bb) ? G[r][c] - (r == c ? 1.0 : 0.0) : 0.0;
      } else {
        double ci[BI];
#pragma unroll
        for (int c = 0; c < BI; ++c) ci[c] = (c < bb) ? Cb[i * BI + c] : 0.0;
#pragma unroll
        for (int c = 0; c < BI; ++c) {
          double acc = 0.0;
#pragma unroll
          for (int c2 = c; c2 < BI; ++c2)
            if (c2 < bb) acc -= ci[c2] * Q[c2][c];
          z[c] = acc;
        }
      }
#pragma unroll
      for (int c = 0; c < BI; ++c)
        if (c < bb) Cb[i * BI + c] = z[c];
    }
    __syncthreads();
    // ---- W[:, out] += Z W[blk, out], one tile of TJ columns at a time
    for (int j0 = 0; j0 < n; j0 += TJ) {
      for (int e = tid; e < bb * TJ; e += nt) {
        int c = e / TJ, jj = e - c * TJ;
        int j = j0 + jj;
        Wb[c * TJ + jj] = (j < n) ? W[(size_t)(k0 + c) * n + j] : 0.0;
      }
      __syncthreads();
      for (int e = tid; e < n * TJ; e += nt) {
        int i = e / TJ, jj = e - i * TJ;
        int j = j0 + jj;
        if (j >= n || (j >= k0 && j < k0 + bb)) continue;
        double acc = W[(size_t)i * n + j];
        for (int c = 0; c < bb; ++c) acc = fma(Cb[i * BI + c], Wb[c * TJ + jj], acc);
        W[(size_t)i * n + j] = acc;
      }
      __syncthreads();
    }
  }
  for (int k = n - 1; k >= 0; --k) {
    int p = perm[k];
    if (p != k) {
      for (int i = tid; i < n; i += nt) {
        double t = W[(size_t)i * n + k];
        W[(size_t)i * n + k] = W[(size_t)i * n + p];
        W[(size_t)i * n + p] = t;
      }
    }
    __syncthreads();
  }
}

void batched_inverse(int n, double* A, double* Ainv, int batch, unsigned* status, cudaStream_t s) {
  // static shared memory (reductions, Q, G) comes on top: always raise the dynamic limit
  size_t smem = (2 * (size_t)n * BI + BI * TJ) * sizeof(double) + n * sizeof(int);
  cudaFuncSetAttribute(k_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_inverse<<<batch, 512, smem, s>>>(n, A, Ainv, status);
}

}  // namespace vrte
