// Internal declarations shared by the CUDA translation units of the VRTE library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "vrte.h"

namespace vrte {

// Device status word bits (set with atomicOr by kernels, read by vrte_plan_status).
enum : unsigned {
  ST_NO_CONVERGENCE = 1u << 0,
  ST_SINGULAR = 1u << 1,
  ST_NONFINITE = 1u << 2,
  ST_BAD_INDEX = 1u << 3,
  ST_TIMEOUT = 1u << 4,  // a bounded device wait gave up (kernel returned early)
};

constexpr double kPi = 3.14159265358979323846;

// Per-layer geometry of one batch of Fourier orders m0 .. m0 + n_units - 1.
struct OrderBatch {
  int N;        // nodes per hemisphere
  int n;        // 4N
  int L;        // expansion coefficients
  int m0;       // first order of the batch
  int n_units;  // orders in the batch
  int n_in, n_out;
  int P;        // table points: N nodes, then n_in incident, then n_out outgoing
  double tau, omega;
  const double* coef;  // [L][6]
  unsigned* status;
  int ldU;             // row stride of [U+ | U- | direct operator] (2n, or 2n + 4L when mixed)
  long long sSD;       // unit stride of [s; d; direct beams] (2n R, or (2n + 4L) R when mixed)
};

// Depth integral of exp(-t/mu0) exp(-t/mu_o) / mu_o over the layer (Eq. 38, Q term).
__host__ __device__ inline double depth_factor(double tau, double mu_o, double mu0) {
  double xs = 1.0 / mu_o + 1.0 / mu0;
  return -expm1(-tau * xs) / (mu_o * xs);
}

// Reconstruction epilogue (row i = 4o + a: outgoing o, exiting component a; column
// j = 4k + s: incident k, basis s): Isyn[m][k][o][a][s] = T1[i][j] + g0(o, k) acc with
// g0 = depth_factor from the per-layer table g0tab[o][k].
struct EpiPart {
  const double* T1;
  double* Isyn;
  const double* g0tab;
  int N, n_in, n_out, m0;
  __device__ void operator()(int u, int i, int j, double acc) const {
    int R = 4 * n_in;
    int o = i >> 2, a = i & 3, k = j >> 2, s = j & 3;
    double g0 = g0tab[(size_t)o * n_in + k];
    double v = fma(g0, acc, T1[(size_t)u * (4 * n_out) * R + (size_t)i * R + j]);
    size_t dst = (((size_t)(m0 + u) * n_in + k) * n_out + o) * 16 + 4 * a + s;
    Isyn[dst] = v;
  }
};

// ---------------------------------------------------------------- tables (k_tables.cu)
void launch_gauss_nodes(int N, double* mu, double* w, unsigned* status, cudaStream_t s);
void launch_interface(int N, int n_in, int n_out, double nif, const double* mu_nodes,
                      const double* mu_in, const double* mu_out, double* pts, double* min4,
                      double* mout4, double* rtop4, cudaStream_t s);
void launch_gsf_tables(const OrderBatch& b, const double* pts, double* p, double* r, double* t,
                       cudaStream_t s);
void launch_trig_table(int M, int n_phi, const double* phi, double* wc, double* ws, cudaStream_t s);

// ---------------------------------------------------------------- assembly (k_assemble.cu)
// Parity-split sums S+-(x, y) = sum_l P_l^m(x) B_l (I +- (-1)^(l-m) D) P_l^m(y) at
// table points, written into the operator each stage needs.
void launch_assemble_EF(const OrderBatch& b, const double* p, const double* r, const double* t,
                        const double* mu_nodes, const double* w_nodes, double* E, double* F,
                        cudaStream_t s);
void launch_assemble_beam(const OrderBatch& b, const double* p, const double* r, const double* t,
                          const double* mu_nodes, const double* min4, double* Pm, double* Rm,
                          cudaStream_t s);
void launch_assemble_U(const OrderBatch& b, const double* p, const double* r, const double* t,
                       const double* w_nodes, const double* mout4, double* U, cudaStream_t s);
void launch_assemble_direct(const OrderBatch& b, const double* p, const double* r,
                            const double* t, const double* pts, const double* min4,
                            const double* mout4, double* T1, cudaStream_t s);
// Direct (once-scattered) term as a contraction over (l, component): writes
// Adir = M_out P_l(mu_o) B_l into columns 2n.. of the [U+ | U- | Adir] rows and
// Bdir = (omega/2pi) (-1)^(l-m) D P_l(mu0) D b_k into rows 2n.. of [s; d; Bdir].
// Depth factors g0tab[o][k] = depth_factor(tau, mu_o, mu0_k) of one layer.
void launch_depth_table(int N, int n_in, int n_out, double tau, const double* pts, double* g0tab,
                        cudaStream_t s);
// Mixed form: factors of the parity-split sums over (l, component) for U+-, beam p, r.
void launch_mixed_operators(const OrderBatch& b, const double* p, const double* r,
                            const double* t, const double* mu_nodes, const double* w_nodes,
                            const double* min4, double* Ln, double* RU, double* Rp, double* Rm,
                            cudaStream_t s);
void launch_direct_operators(const OrderBatch& b, const double* p, const double* r,
                             const double* t, const double* min4, const double* mout4,
                             double* Uext, double* SDext, cudaStream_t s);

// ---------------------------------------------------------------- dense FP64 (k_linalg.cu)
// C[u] = alpha * A[u] (M x K, row-major, lda) * B[u] (K x N, ldb) + beta * C[u]
void dgemm_batched(int M, int N, int K, double alpha, const double* A, int lda, long long sA,
                   const double* B, int ldb, long long sB, double beta, double* C, int ldc,
                   long long sC, int batch, cudaStream_t s);
// Reconstruction epilogue: Isyn[m][k][o][a][s] = T1[ro][rc] + g0(o, k) * (A @ B)[ro][rc]
void dgemm_part_epilogue(const OrderBatch& b, const double* A, const double* B, const double* T1,
                         const double* g0tab, double* Isyn, cudaStream_t s);
void batched_inverse(int n, double* A, double* Ainv, int batch, unsigned* status, cudaStream_t s);
void batched_eigen(int n, const double* A, double* H, double* Z, double* V, double* X,
                   double* lam_re, double* lam_im, double* scale, int batch, unsigned* status,
                   cudaStream_t s, const int* mask = nullptr);
// Re-solves orders whose reduced eigenvectors are not accurate enough with the 2n x 2n
// block form (see k_eigen.cu); overwrites X, Y and lambda of the flagged orders.
void eigen_block_fallback(int n, int m0, const double* E, const double* F, const double* FY,
                          double* X, double* Y, double* lam_re, double* lam_im, double tol,
                          int force0, double* res, int* flag, double* B, double* Hb, double* Zb,
                          double* Vb, double* Xb, double* kb_re, double* kb_im, double* balb,
                          int batch, unsigned* status, cudaStream_t s);

// ---------------------------------------------------------------- tensor cores (k_tcgemm.cu)
// C = A B (+ beta C) with A, B FP64 sliced into S exact 7-bit BF16 slices (relative
// accuracy ~2^-7S per term); K <= 1024, 1 <= S <= 4. `work` holds tc_workspace_bytes.
size_t tc_workspace_bytes(int M, int N, int K, int batch, int S);
// the part of tc_workspace_bytes that does not grow with the batch (epilogue scratch)
size_t tc_scratch_bytes();
bool tc_shape_ok(int K, int S);
void tc_gemm_store(int M, int N, int K, const double* A, int lda, long long sA, const double* B,
                   int ldb, long long sB, double beta, double* C, int ldc, long long sC,
                   int batch, int S, void* work, unsigned* status, cudaStream_t s);
void tc_gemm_part(const OrderBatch& b, int K, const double* A, int lda, long long sA,
                  const double* B, long long sB, const double* T1, const double* g0tab,
                  double* Isyn, int S, void* work, cudaStream_t s);
// Mixed form: flags (order, incident) column blocks whose sliced reconstruction error
// bound eps K max|row| max|column| exceeds tol |I_00| and recomputes them in FP64.
void refine_columns(const OrderBatch& b, int Kpart, const double* Kinv, const double* RHS,
                    const double* C, const double* Hhat, const double* Uext, const double* SD,
                    const double* g0tab, double eps, double tol, double* scratch, int* counters,
                    int2* list, int cap, double* Isyn, cudaStream_t s);
size_t refine_scratch_doubles(int U, int n_in, int n_out);
// T1 += g0 (A @ B): the first part of a reconstruction contraction split in K.
void tc_gemm_part_accum(const OrderBatch& b, int K, const double* A, int lda, long long sA,
                        const double* B, long long sB, double* T1, const double* g0tab, int S,
                        void* work, cudaStream_t s);
// Called on the host after the kernels that complete the table rows of incident cosines
// k0 .. k1-1 of one layer have been enqueued on `s` (the host-buffer solve starts the copy
// of those rows there).
struct SynthHook {
  void (*fn)(void* user, int layer, int k0, int k1, cudaStream_t s);
  void* user;
  int layer;
};
// Synthesis of the order radiances on the tensor cores (five slices), in blocks of k_block
// incident cosines (k_synth_tc.cu).
size_t tc_synthesis_workspace(int M, int n_in, int n_out, int n_phi, int k_block);
void tc_synthesis(int M, int n_in, int n_out, int n_phi, const double* Isyn, const double* wc,
                  const double* ws, void* out, int out_dtype, int k_block, void* work,
                  unsigned* status, cudaStream_t s, const SynthHook* hook = nullptr);

// ---------------------------------------------------------------- mode algebra (k_modes.cu)
void launch_pack_Y(const OrderBatch& b, const double* EX, const double* lam_re,
                   const double* lam_im, double* Y, cudaStream_t s);
void launch_build_K(const OrderBatch& b, const double* X, const double* Y, const double* lam_re,
                    const double* lam_im, const double* rtop4, double* K, cudaStream_t s);
void launch_particular_rhs(const OrderBatch& b, const double* w_in, const double* r,
                           const double* pts, double* w_out, cudaStream_t s);
void launch_eigen_scale(const OrderBatch& b, const double* lam_re, const double* lam_im,
                        const double* pts, double* y, cudaStream_t s);
void launch_particular_sd(const OrderBatch& b, const double* pbeam, const double* Es,
                          const double* pts, double* d, cudaStream_t s);
void launch_bc_rhs(const OrderBatch& b, const double* sv, const double* d, const double* rtop4,
                   const double* pts, double* rhs, cudaStream_t s);
void launch_build_Hhat(const OrderBatch& b, const double* P1, const double* P2,
                       const double* lam_re, const double* lam_im, const double* pts,
                       double* Hhat, cudaStream_t s);

// ---------------------------------------------------------------- synthesis (k_synth.cu)
void launch_synthesis_fp64(int M, int n_in, int n_out, int n_phi, const double* Isyn,
                           const double* wc, const double* ws, void* out, int out_dtype,
                           unsigned* status, cudaStream_t s);

}  // namespace vrte
