// Mixed form: FP64 recomputation of ill-conditioned reconstruction columns.
//
// Near a resonance between an incident cosine and a mode (mu0 kappa_j ~ 1) the
// eigenbasis particular solution (Sec. 3.B, Eq. 47) grows like 1 / (kappa_j^2 - mu0^-2)
// and the boundary solve answers with a homogeneous coefficient that cancels it
// (Eqs. 45-46), so the exiting radiance of that incident column is a small difference
// of two large contractions (Eq. 38). The sliced tensor-core product is accurate to
// ~eps K max|row| max|column| per element; this pass estimates that bound for every
// (order, incident) column block from the row and column maxima of the operands,
// compares it with the order-0 radiance I_00 of the same pair, and recomputes the flagged column
// blocks in FP64 from the FP64 operators (boundary coefficients from K^-1 and the
// right-hand side, written over those columns of C, then both reconstruction contractions),
// overwriting I^m.
#include "vrte_internal.cuh"

namespace vrte {

// out[u][r / 4] = max over the four rows r of a group and c < cols of |A[u][r][c]| (zeroed
// before): one warp per row, the group's maximum by an integer max of the bit patterns
// (non-negative doubles order like them).
__global__ void k_row_absmax(int rows, int cols, const double* __restrict__ A, int lda,
                             long long sA, double* __restrict__ out) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  int u = blockIdx.y;
  if (warp >= rows) return;
  const double* a = A + (size_t)u * sA + (size_t)warp * lda;
  double m = 0.0;
  for (int c = lane; c < cols; c += 32) m = fmax(m, fabs(a[c]));
  for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
  if (lane == 0 && m > 0.0)
    atomicMax((unsigned long long*)out + (size_t)u * (rows / 4) + warp / 4,
              (unsigned long long)__double_as_longlong(m));
}

// out[u][c / 4] = max over the four columns c of a group and r < rows of |B[u][r][c]| (zeroed
// before): one thread per column (coalesced rows).
__global__ void k_col_absmax(int rows, int cols, const double* __restrict__ B, int ldb,
                             long long sB, double* __restrict__ out) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  int u = blockIdx.y;
  if (c >= cols) return;
  const double* b = B + (size_t)u * sB + c;
  double m = 0.0;
  for (int r = 0; r < rows; ++r) m = fmax(m, fabs(b[(size_t)r * ldb]));
  if (m > 0.0)
    atomicMax((unsigned long long*)out + (size_t)u * (cols / 4) + c / 4,
              (unsigned long long)__double_as_longlong(m));
}

// The error bound of the sliced contractions against tol |I^0_00(o, k)| (order 0 sets the
// scale of the synthesized radiance at that pair), from the row maxima per outgoing o
// (rmH, rmU: [U][n_out]) and column maxima per incident k (cmC, cmSD: [U][n_in]), each over
// the four Stokes rows or columns: one thread per (outgoing o, incident k = k0 + blockIdx.y),
// which reads the order-0 reference once and tests every order u of the batch, marking the
// column blocks (u, k) that fail in `flags` (already set for a non-finite result by the
// reconstruction's epilogue).
__global__ void k_flag_columns(OrderBatch b, const double* __restrict__ rmH,
                               const double* __restrict__ rmU, const double* __restrict__ cmC,
                               const double* __restrict__ cmSD, const double* __restrict__ g0tab,
                               const double* __restrict__ Isyn, double epsK1, double epsK2,
                               double tol, int k0, int* flags) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = k0 + blockIdx.y;
  if (o >= b.n_out) return;
  const double ref = Isyn[((size_t)k * b.n_out + o) * 16];
  const double lim = isfinite(ref) ? tol * fabs(ref) : -1.0;
  const double g0 = g0tab[(size_t)o * b.n_in + k];
  for (int u = 0; u < b.n_units; ++u) {
    const double rH = rmH[(size_t)u * b.n_out + o], rU = rmU[(size_t)u * b.n_out + o];
    const double cC = cmC[(size_t)u * b.n_in + k], cS = cmSD[(size_t)u * b.n_in + k];
    const double bound = epsK1 * rH * cC + epsK2 * g0 * rU * cS;
    if (!(bound <= lim) && !flags[(size_t)u * b.n_in + k]) flags[(size_t)u * b.n_in + k] = 1;
  }
}

// The flagged column blocks with incident k0 <= k < k1 into the work list of k_fix_columns.
__global__ void k_collect_columns(int n_in, int k0, int k1, int U, const int* __restrict__ flags,
                                  int* count, int* total, int2* list, int cap) {
  const int k = k0 + blockIdx.x * blockDim.x + threadIdx.x;
  const int u = blockIdx.y;
  if (k >= k1 || u >= U || !flags[(size_t)u * n_in + k]) return;
  const int slot = atomicAdd(count, 1);
  atomicAdd(total, 1);
  if (slot < cap) list[slot] = make_int2(u, k);
}

// The flagged column blocks are recomputed in two persistent passes over work items, so that
// the FP64 work spreads over the SMs however few columns are flagged:
// k_fix_coeffs: the FP64 boundary coefficients C'[:, 4k..4k+3] = K^-1 RHS[:, 4k..4k+3] of a
//   flagged (u, k), FIX_CROWS rows per work item (one warp per row), written over the sliced
//   product's columns of C;
// k_fix_columns: FIX_ROWS output rows r = 4o + a per work item (one warp per row), with the
//   block's C' and beam columns SD[:, 4k..4k+3] staged in shared memory:
//   I^m[k][o][a][s] = sum_i Hhat[r][i] C'[i][s] + g0(o, k) sum_i U[r][i] SD[i][4k + s].
constexpr int FIX_CROWS = 64;   // coefficient rows per work item of k_fix_coeffs
constexpr int FIX_ROWS = 64;    // output rows per work item of k_fix_columns
constexpr int FIX_THREADS = 256;

__global__ void __launch_bounds__(FIX_THREADS) k_fix_coeffs(
    OrderBatch b, const double* __restrict__ Kinv, const double* __restrict__ RHS,
    const int* __restrict__ count, const int2* __restrict__ list, int cap, double* __restrict__ C) {
  extern __shared__ double Rs[];  // [2n][4]: the right-hand side's column block
  const int n2 = 2 * b.n, R = 4 * b.n_in;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int items = min(*count, cap);
  const int nblk = (n2 + FIX_CROWS - 1) / FIX_CROWS;
  for (int wi = blockIdx.x; wi < items * nblk; wi += gridDim.x) {
    const int it = wi / nblk, i0 = (wi - it * nblk) * FIX_CROWS;
    const int2 e = list[it];
    const int u = e.x, k = e.y;
    const double* rh = RHS + (size_t)u * n2 * R + 4 * k;
    __syncthreads();  // Rs of the previous item is no longer read
    for (int t = threadIdx.x; t < 4 * n2; t += blockDim.x) Rs[t] = rh[(size_t)(t >> 2) * R + (t & 3)];
    __syncthreads();
    const double* Ki = Kinv + (size_t)u * n2 * n2;
    for (int i = i0 + warp; i < min(n2, i0 + FIX_CROWS); i += nw) {
      double acc[4] = {0.0, 0.0, 0.0, 0.0};
      for (int j = lane; j < n2; j += 32) {
        const double kv = Ki[(size_t)i * n2 + j];
        for (int s = 0; s < 4; ++s) acc[s] = fma(kv, Rs[4 * j + s], acc[s]);
      }
      for (int s = 0; s < 4; ++s)
        for (int off = 16; off > 0; off >>= 1) acc[s] += __shfl_xor_sync(0xffffffffu, acc[s], off);
      if (lane == 0) {
        double* dst = C + (size_t)u * n2 * R + (size_t)i * R + 4 * k;
        for (int s = 0; s < 4; ++s) dst[s] = acc[s];
      }
    }
  }
}

// staged: the beam columns (Kpart x 4) fit in shared memory beside C' (else read from SD)
__global__ void __launch_bounds__(FIX_THREADS) k_fix_columns(
    OrderBatch b, const double* __restrict__ C, const double* __restrict__ Hhat,
    const double* __restrict__ Uext, const double* __restrict__ SD,
    const double* __restrict__ g0tab, int Kpart, const int* __restrict__ count,
    const int2* __restrict__ list, int cap, int staged, double* __restrict__ Isyn) {
  extern __shared__ double sm[];
  const int n2 = 2 * b.n, R = 4 * b.n_in, Ro = 4 * b.n_out;
  double* Cs = sm;           // [2n][4]: C' of the block
  double* Ss = sm + 4 * n2;  // [Kpart][4]: the beam columns of the block (staged)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int items = min(*count, cap);
  const int nblk = (Ro + FIX_ROWS - 1) / FIX_ROWS;
  for (int wi = blockIdx.x; wi < items * nblk; wi += gridDim.x) {
    const int it = wi / nblk, r0 = (wi - it * nblk) * FIX_ROWS;
    const int2 e = list[it];
    const int u = e.x, k = e.y;
    const double* cb = C + (size_t)u * n2 * R + 4 * k;
    const double* sd = SD + (size_t)u * b.sSD + 4 * k;
    __syncthreads();  // the previous item's blocks are no longer read
    for (int t = threadIdx.x; t < 4 * n2; t += blockDim.x) Cs[t] = cb[(size_t)(t >> 2) * R + (t & 3)];
    if (staged)
      for (int t = threadIdx.x; t < 4 * Kpart; t += blockDim.x)
        Ss[t] = sd[(size_t)(t >> 2) * R + (t & 3)];
    __syncthreads();
    const double* H = Hhat + (size_t)u * Ro * n2;
    const double* Ub = Uext + (size_t)u * Ro * b.ldU;
    for (int r = r0 + warp; r < min(Ro, r0 + FIX_ROWS); r += nw) {
      double h[4] = {0.0, 0.0, 0.0, 0.0}, q[4] = {0.0, 0.0, 0.0, 0.0};
      for (int i = lane; i < n2; i += 32) {
        const double hv = H[(size_t)r * n2 + i];
        for (int s = 0; s < 4; ++s) h[s] = fma(hv, Cs[4 * i + s], h[s]);
      }
      for (int i = lane; i < Kpart; i += 32) {
        const double uv = Ub[(size_t)r * b.ldU + i];
        const double* col = staged ? Ss + 4 * i : sd + (size_t)i * R;
        for (int s = 0; s < 4; ++s) q[s] = fma(uv, col[s], q[s]);
      }
      for (int s = 0; s < 4; ++s)
        for (int off = 16; off > 0; off >>= 1) {
          h[s] += __shfl_xor_sync(0xffffffffu, h[s], off);
          q[s] += __shfl_xor_sync(0xffffffffu, q[s], off);
        }
      if (lane == 0) {
        const int o = r >> 2, a = r & 3;
        const double g0 = g0tab[(size_t)o * b.n_in + k];
        double* dst = Isyn + (((size_t)(b.m0 + u) * b.n_in + k) * b.n_out + o) * 16 + 4 * a;
        for (int s = 0; s < 4; ++s) dst[s] = fma(g0, q[s], h[s]);
      }
    }
  }
}

static int fix_grid() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
      sms = 1;
  }
  return 4 * sms;
}

// maxima per (unit, outgoing) and per (unit, incident), each over its four Stokes entries,
// in `scratch`: rmH, rmU [U][n_out], cmC, cmSD [U][n_in]
void refine_maxima(const OrderBatch& b, int Kpart, const double* C, const double* Hhat,
                   const double* Uext, const double* SD, double* scratch, cudaStream_t s) {
  const int U = b.n_units, n2 = 2 * b.n, R = 4 * b.n_in, Ro = 4 * b.n_out;
  double* rmH = scratch;
  double* rmU = rmH + (size_t)U * b.n_out;
  double* cmC = rmU + (size_t)U * b.n_out;
  double* cmSD = cmC + (size_t)U * b.n_in;
  cudaMemsetAsync(scratch, 0, (size_t)U * 2 * (b.n_out + b.n_in) * sizeof(double), s);
  k_row_absmax<<<dim3((Ro + 7) / 8, U), 256, 0, s>>>(Ro, n2, Hhat, n2, (long long)Ro * n2, rmH);
  k_row_absmax<<<dim3((Ro + 7) / 8, U), 256, 0, s>>>(Ro, Kpart, Uext, b.ldU,
                                                      (long long)Ro * b.ldU, rmU);
  k_col_absmax<<<dim3((R + 127) / 128, U), 128, 0, s>>>(n2, R, C, R, (long long)n2 * R, cmC);
  k_col_absmax<<<dim3((R + 127) / 128, U), 128, 0, s>>>(Kpart, R, SD, R, b.sSD, cmSD);
}

void refine_range(const OrderBatch& b, int Kpart, const double* Kinv, const double* RHS,
                  double* C, const double* Hhat, const double* Uext, const double* SD, const double* g0tab,
                  double eps, double tol, const double* scratch, int* counters, int2* list,
                  int cap, double* Isyn, int* nonfinite, int k0, int k1, cudaStream_t s) {
  const int U = b.n_units, n2 = 2 * b.n;
  if (k1 <= k0) return;
  const double* rmH = scratch;
  const double* rmU = rmH + (size_t)U * b.n_out;
  const double* cmC = rmU + (size_t)U * b.n_out;
  const double* cmSD = cmC + (size_t)U * b.n_in;
  cudaMemsetAsync(counters, 0, sizeof(int), s);
  k_flag_columns<<<dim3((b.n_out + 127) / 128, k1 - k0), 128, 0, s>>>(
      b, rmH, rmU, cmC, cmSD, g0tab, Isyn, eps * n2, eps * Kpart, tol, k0, nonfinite);
  k_collect_columns<<<dim3((k1 - k0 + 127) / 128, U), 128, 0, s>>>(
      b.n_in, k0, k1, U, nonfinite, counters, counters + 1, list, cap);
  // the coefficients first (C'), then the rows from them; the work lists are read on the GPU
  const size_t smem_c = (size_t)n2 * 4 * sizeof(double);
  if (smem_c > 48 * 1024)
    cudaFuncSetAttribute(k_fix_coeffs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_c);
  k_fix_coeffs<<<fix_grid(), FIX_THREADS, smem_c, s>>>(b, Kinv, RHS, counters, list, cap, C);
  const size_t smem_full = smem_c + (size_t)Kpart * 4 * sizeof(double);
  const int staged = smem_full <= (size_t)160 * 1024;
  const size_t smem = staged ? smem_full : smem_c;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_fix_columns, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_fix_columns<<<fix_grid(), FIX_THREADS, smem, s>>>(b, C, Hhat, Uext, SD, g0tab, Kpart,
                                                      counters, list, cap, staged, Isyn);
}

void refine_columns(const OrderBatch& b, int Kpart, const double* Kinv, const double* RHS,
                    double* C, const double* Hhat, const double* Uext, const double* SD,
                    const double* g0tab, double eps, double tol, double* scratch, int* counters,
                    int2* list, int cap, double* Isyn, int* nonfinite, cudaStream_t s) {
  refine_maxima(b, Kpart, C, Hhat, Uext, SD, scratch, s);
  refine_range(b, Kpart, Kinv, RHS, C, Hhat, Uext, SD, g0tab, eps, tol, scratch, counters,
               list, cap, Isyn, nonfinite, 0, b.n_in, s);
}

size_t refine_scratch_doubles(int U, int n_in, int n_out) {
  return (size_t)U * (8 * (size_t)n_out + 8 * (size_t)n_in);
}

}  // namespace vrte
