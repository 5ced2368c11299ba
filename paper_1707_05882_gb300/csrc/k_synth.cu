// Step a8: azimuthal Fourier synthesis of the Mueller BRDF (Sec. 2.D, Eqs. 7, 12, 39).
//
// out[k][o][j][a][s] = sum_m w_as(m, j) I^m[k][o][a][s] with the Fourier factor of the
// incident column's family (Eq. 7): cos for the (IQ, IQ) and (UV, UV) blocks, +sin for
// (UV rows, IQ columns) and -sin for (IQ rows, UV columns). wc/ws already carry
// (2 - delta_m0)/2 and the (-1)^m of the half-turn between source and beam azimuth.
// FP64 form: one CTA per (incident, outgoing) pair, the M x 16 order radiances staged in
// shared memory, one thread per azimuth.
#include "vrte_internal.cuh"

namespace vrte {

template <typename T>
__global__ void __launch_bounds__(128) k_synth_fp64(int M, int n_in, int n_out, int n_phi,
                                                    const double* __restrict__ Isyn,
                                                    const double* __restrict__ wc,
                                                    const double* __restrict__ ws, T* out,
                                                    unsigned* status) {
  extern __shared__ double Ish[];  // [M][16]
  int pair = blockIdx.x;           // k * n_out + o
  int k = pair / n_out, o = pair - k * n_out;
  for (int e = threadIdx.x; e < M * 16; e += blockDim.x) {
    int m = e >> 4, q = e & 15;
    Ish[e] = Isyn[(((size_t)m * n_in + k) * n_out + o) * 16 + q];
  }
  __syncthreads();
  bool bad = false;
  for (int j = threadIdx.x; j < n_phi; j += blockDim.x) {
    double acc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = 0.0;
    for (int m = 0; m < M; ++m) {
      double c = wc[(size_t)m * n_phi + j], s = ws[(size_t)m * n_phi + j];
      const double* I = Ish + m * 16;
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          double w = (a < 2) == (b < 2) ? c : (a < 2 ? -s : s);
          acc[4 * a + b] = fma(w, I[4 * a + b], acc[4 * a + b]);
        }
    }
    T* dst = out + ((size_t)pair * n_phi + j) * 16;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      if (!isfinite(acc[q])) bad = true;
      dst[q] = (T)acc[q];
    }
  }
  if (bad) atomicOr(status, ST_NONFINITE);
}

void launch_synthesis_fp64(int M, int n_in, int n_out, int n_phi, const double* Isyn,
                           const double* wc, const double* ws, void* out, int out_dtype,
                           unsigned* status, cudaStream_t s) {
  size_t smem = (size_t)M * 16 * sizeof(double);
  long long pairs = (long long)n_in * n_out;
  if (out_dtype == VRTE_OUT_F64) {
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(k_synth_fp64<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
    k_synth_fp64<double><<<(unsigned)pairs, 128, smem, s>>>(M, n_in, n_out, n_phi, Isyn, wc, ws,
                                                            (double*)out, status);
  } else {
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(k_synth_fp64<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
    k_synth_fp64<float><<<(unsigned)pairs, 128, smem, s>>>(M, n_in, n_out, n_phi, Isyn, wc, ws,
                                                           (float*)out, status);
  }
}

}  // namespace vrte
