// Dense FP64 linear algebra on CUDA cores: batched GEMM (with an epilogue hook for the
// reconstruction) and batched in-place Gauss-Jordan inversion with partial pivoting.
// FP64 stays on the CUDA cores: sm_103a has no FP64 tensor-core path worth using.
#include <algorithm>

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

// T = double: the FP64 inverse. T = float: the same elimination in FP32 (the starting
// inverse of the mixed form's Newton refinement), W an FP32 workspace. Orders u with
// skip && !skip[u] return at once. CTAs from nb1 on invert a second batch (n2, A2, Ainv2),
// so that two batches of matrices share one launch.
template <typename T>
__global__ void __launch_bounds__(512) k_inverse(int n, const double* __restrict__ A,
                                                 T* __restrict__ Ainv, unsigned* status,
                                                 const int* __restrict__ skip, int nb1, int n2,
                                                 const double* __restrict__ A2,
                                                 T* __restrict__ Ainv2) {
  extern __shared__ __align__(16) unsigned char sh_raw[];
  T* sh = (T*)sh_raw;
  T* P = sh;                  // [n][BI] panel
  T* Cb = P + (size_t)n * BI; // [n][BI] step columns, then Z
  T* Wb = Cb + (size_t)n * BI;// [BI][TJ] block rows of a column tile
  int* perm = (int*)(Wb + BI * TJ);
  __shared__ T red_v[16];
  __shared__ int red_i[16];
  __shared__ T rk[BI];
  __shared__ T Q[BI][BI], G[BI][BI];
  int u = blockIdx.x;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (u >= nb1) {
    u -= nb1;
    n = n2;
    A = A2;
    Ainv = Ainv2;
  } else if (skip && !skip[u]) {
    return;
  }
  const double* Ab = A + (size_t)u * n * n;
  T* W = Ainv + (size_t)u * n * n;
  for (size_t e = tid; e < (size_t)n * n; e += nt) W[e] = (T)Ab[e];
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
      T best = -1;
      int bi = k;
      for (int i = k + tid; i < n; i += nt) {
        T v = fabs(P[i * BI + c]);
        if (v > best) { best = v; bi = i; }
      }
      for (int off = 16; off > 0; off >>= 1) {
        T ov = __shfl_down_sync(0xffffffffu, best, off);
        int oi = __shfl_down_sync(0xffffffffu, bi, off);
        if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
      }
      if ((tid & 31) == 0) { red_v[tid >> 5] = best; red_i[tid >> 5] = bi; }
      __syncthreads();
      if (tid < 32) {
        int nw = (nt + 31) >> 5;
        best = tid < nw ? red_v[tid] : (T)-1;
        bi = tid < nw ? red_i[tid] : k;
        for (int off = 16; off > 0; off >>= 1) {
          T ov = __shfl_down_sync(0xffffffffu, best, off);
          int oi = __shfl_down_sync(0xffffffffu, bi, off);
          if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
        }
        if (tid == 0) { red_i[0] = bi; perm[k] = bi; }
      }
      __syncthreads();
      const int p = red_i[0];
      if (p != k && tid < BI) {
        // the panel row, and the recorded columns of earlier steps, follow the swap
        T t = P[k * BI + tid];
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
      const T piv = P[k * BI + c];
      if (tid == 0 && (piv == (T)0 || !isfinite(piv))) atomicOr(status, ST_SINGULAR);
      const T pinv = (T)1 / piv;
      if (tid < bb) rk[tid] = (tid == c) ? pinv : P[k * BI + tid] * pinv;
      __syncthreads();
      for (int e = tid; e < n * bb; e += nt) {
        int i = e / bb, cc = e - i * bb;
        if (i == k) {
          P[i * BI + cc] = rk[cc];
        } else {
          T w = (cc == c) ? (T)0 : P[i * BI + cc];
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
          T t = W[(size_t)k * n + j];
          W[(size_t)k * n + j] = W[(size_t)p * n + j];
          W[(size_t)p * n + j] = t;
        }
      __syncthreads();
    }
    // ---- Q = (D + Lw)^-1 (forward substitution per column), G = (I - Up) Q
    if (tid < bb) {
      const int col = tid;
      for (int r = 0; r < bb; ++r) {
        T acc = (r == col) ? (T)1 : (T)0;
        for (int c2 = 0; c2 < r; ++c2) acc -= Cb[(k0 + r) * BI + c2] * Q[c2][col];
        Q[r][col] = acc / Cb[(k0 + r) * BI + r];
      }
    }
    __syncthreads();
    if (tid < bb * bb) {
      const int r = tid / bb, c = tid - r * bb;
      T g = Q[r][c];
      for (int c2 = r + 1; c2 < bb; ++c2) g -= Cb[(k0 + r) * BI + c2] * Q[c2][c];
      G[r][c] = g;
    }
    __syncthreads();
    // Z overwrites C row by row (each row only reads its own entries)
    for (int i = tid; i < n; i += nt) {
      T z[BI];
      if (i >= k0 && i < k0 + bb) {
        const int r = i - k0;
#pragma unroll
        for (int c = 0; c < BI; ++c) z[c] = (c < bb) ? G[r][c] - (r == c ? (T)1 : (T)0) : (T)0;
      } else {
        T ci[BI];
#pragma unroll
        for (int c = 0; c < BI; ++c) ci[c] = (c < bb) ? Cb[i * BI + c] : (T)0;
#pragma unroll
        for (int c = 0; c < BI; ++c) {
          T acc = 0;
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
        Wb[c * TJ + jj] = (j < n) ? W[(size_t)(k0 + c) * n + j] : (T)0;
      }
      __syncthreads();
      for (int e = tid; e < n * TJ; e += nt) {
        int i = e / TJ, jj = e - i * TJ;
        int j = j0 + jj;
        if (j >= n || (j >= k0 && j < k0 + bb)) continue;
        T acc = W[(size_t)i * n + j];
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
        T t = W[(size_t)i * n + k];
        W[(size_t)i * n + k] = W[(size_t)i * n + p];
        W[(size_t)i * n + p] = t;
      }
    }
    __syncthreads();
  }
}

void batched_inverse(int n, double* A, double* Ainv, int batch, unsigned* status, cudaStream_t s,
                     const int* skip) {
  // static shared memory (reductions, Q, G) comes on top: always raise the dynamic limit
  size_t smem = (2 * (size_t)n * BI + BI * TJ) * sizeof(double) + n * sizeof(int);
  cudaFuncSetAttribute(k_inverse<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_inverse<double><<<batch, 512, smem, s>>>(n, A, Ainv, status, skip, batch, 0, nullptr, nullptr);
}

// FP32 inverses of two batches in one launch (the second may be empty: nb = 0)
static void batched_inverse_f32_pair(int na, const double* A, float* Ainv, int nb,
                                     const double* B, float* Binv, int batch, unsigned* status,
                                     cudaStream_t s) {
  const int nm = std::max(na, nb);
  size_t smem = (2 * (size_t)nm * BI + BI * TJ) * sizeof(float) + nm * sizeof(int);
  cudaFuncSetAttribute(k_inverse<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_inverse<float><<<(nb > 0 ? 2 : 1) * batch, 512, smem, s>>>(na, A, Ainv, status, nullptr, batch,
                                                               nb, B, Binv);
}

void batched_inverse_f32(int n, const double* A, float* Ainv, int batch, unsigned* status,
                         cudaStream_t s) {
  batched_inverse_f32_pair(n, A, Ainv, 0, nullptr, nullptr, batch, status, s);
}

}  // namespace vrte

namespace vrte {

// ------------------------------------------------------------------ Newton inverse
// Inverse of a batch of FP64 matrices with the O(n^3) work on the tensor cores: a starting
// inverse X0 from the FP32 elimination above, then Newton-Schulz steps
//   E_k = I - A X_k,   X_{k+1} = X_k + X_k E_k,
// whose residual squares at every step (||E_{k+1}|| <= ||E_k||^2) while ||E_0|| < 1, each
// step two sliced FP64-accurate products (k_tcgemm.cu). A matrix whose final max|E| is not
// below `tol` (an FP32 start too poor or non-finite) is inverted again by the FP64
// elimination, masked to those matrices.

__global__ void k_widen(size_t count, const float* __restrict__ x, double* __restrict__ y) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
       i += (size_t)gridDim.x * blockDim.x)
    y[i] = (double)x[i];
}

// E = I - R in place, err[u] = max |E| as the bit pattern of a non-negative double (those
// order like the doubles; a NaN compares above every finite value)
__global__ void k_eye_minus(int n, double* R, unsigned long long* err) {
  const int u = blockIdx.y;
  const size_t nn = (size_t)n * n;
  double* Ru = R + (size_t)u * nn;
  unsigned long long m = 0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nn;
       e += (size_t)gridDim.x * blockDim.x) {
    const size_t i = e / n, j = e - i * n;
    const double v = (i == j ? 1.0 : 0.0) - Ru[e];
    Ru[e] = v;
    const unsigned long long b = (unsigned long long)__double_as_longlong(fabs(v));
    m = b > m ? b : m;
  }
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long o = __shfl_down_sync(0xffffffffu, m, off);
    m = o > m ? o : m;
  }
  if ((threadIdx.x & 31) == 0 && m) atomicMax(err + u, m);
}

__global__ void k_newton_flag(int batch, const unsigned long long* err, double tol, int* flag,
                              int* count) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= batch) return;
  const double e = __longlong_as_double((long long)err[u]);
  const int f = !(e <= tol);
  flag[u] = f;
  if (f) atomicAdd(count, 1);
}

size_t newton_inverse_scratch_bytes(int na, int nb, int batch) {
  const size_t a = (size_t)na * na * batch, b = (size_t)nb * nb * batch;
  return std::max(a, b) * sizeof(double) + (a + b + 2) * sizeof(float) +
         (size_t)batch * sizeof(int) + sizeof(unsigned);
}

void newton_inverse(int na, const double* A, double* XA, int nb, const double* B, double* XB,
                    int batch, int steps, double tol, void* scratch, unsigned long long* err,
                    int* fallback_count, void* tcw, int slices, unsigned* status, cudaStream_t s) {
  const size_t nna = (size_t)na * na * batch, nnb = (size_t)nb * nb * batch;
  double* Rm = (double*)scratch;
  float* xa32 = (float*)(Rm + std::max(nna, nnb));
  float* xb32 = xa32 + nna + (nna & 1);
  int* flag = (int*)(xb32 + nnb + 1);
  // the FP32 elimination's pivot findings do not enter the plan's status: a failed start is
  // caught by the residual below
  unsigned* st32 = (unsigned*)(flag + batch);
  batched_inverse_f32_pair(na, A, xa32, nb, B, xb32, batch, st32, s);
  for (int q = 0; q < (nb > 0 ? 2 : 1); ++q) {
    const int n = q ? nb : na;
    const double* M = q ? B : A;
    double* X = q ? XB : XA;
    unsigned long long* e = err + (size_t)q * batch;
    const size_t nn = (size_t)n * n;
    k_widen<<<1024, 256, 0, s>>>(nn * batch, q ? xb32 : xa32, X);
    const dim3 eg((unsigned)std::min<size_t>((nn + 255) / 256, 64), batch);
    for (int k = 0; k <= steps; ++k) {
      tc_gemm_store(n, n, n, M, n, (long long)nn, X, n, (long long)nn, 0.0, Rm, n,
                    (long long)nn, batch, slices, tcw, status, s);
      cudaMemsetAsync(e, 0, batch * sizeof(unsigned long long), s);
      k_eye_minus<<<eg, 256, 0, s>>>(n, Rm, e);
      if (k == steps) break;
      // X <- X E + X: the product reads X only through its slices, taken before the
      // epilogue writes X
      tc_gemm_store(n, n, n, X, n, (long long)nn, Rm, n, (long long)nn, 1.0, X, n,
                    (long long)nn, batch, slices, tcw, status, s);
    }
    k_newton_flag<<<(batch + 127) / 128, 128, 0, s>>>(batch, e, tol, flag, fallback_count);
    batched_inverse(n, const_cast<double*>(M), X, batch, status, s, flag);
  }
}

}  // namespace vrte
