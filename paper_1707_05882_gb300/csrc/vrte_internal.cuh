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
  int* nonfinite = nullptr;  // optional [unit][n_in]: set for a column block with a NaN or Inf
  __device__ void operator()(int u, int i, int j, double acc) const {
    int R = 4 * n_in;
    int o = i >> 2, a = i & 3, k = j >> 2, s = j & 3;
    double g0 = g0tab[(size_t)o * n_in + k];
    double v = fma(g0, acc, T1[(size_t)u * (4 * n_out) * R + (size_t)i * R + j]);
    size_t dst = (((size_t)(m0 + u) * n_in + k) * n_out + o) * 16 + 4 * a + s;
    Isyn[dst] = v;
    if (nonfinite && !isfinite(v)) atomicOr(nonfinite + (size_t)u * n_in + k, 1);
  }
};

// ---------------------------------------------------------------- complex FP64 helpers
// (modes of a complex eigenvalue pair are kept in real form in the buffers; these evaluate
// their exponentials and depth integrals)
struct cd {
  double r, i;
};
__device__ inline cd cmul(cd a, cd b) { return cd{a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r}; }
__device__ inline cd cdivv(cd a, cd b) {
  double den = b.r * b.r + b.i * b.i;
  return cd{(a.r * b.r + a.i * b.i) / den, (a.i * b.r - a.r * b.i) / den};
}
__device__ inline cd cexpv(cd z) {
  double e = exp(z.r), sn, cs;
  sincos(z.i, &sn, &cs);
  return cd{e * cs, e * sn};
}
// exp(z) - 1, by its Taylor series for |z| < 1e-2
__device__ inline cd cexpm1v(cd z) {
  if (fabs(z.r) + fabs(z.i) < 1e-2) {
    cd term = z, acc = z;
    for (int k = 2; k < 10; ++k) {
      term = cmul(term, z);
      term.r /= k;
      term.i /= k;
      acc.r += term.r;
      acc.i += term.i;
    }
    return acc;
  }
  cd e = cexpv(z);
  return cd{e.r - 1.0, e.i};
}
// principal square root of a + ib without cancellation: with r = sqrt((|a| + |z|)/2),
// sqrt(z) = (r, b/(2r)) for a >= 0 and (|b|/(2r), sign(b) r) for a < 0. (Forming
// sqrt((|z| - a)/2) instead fails for pairs with a tiny imaginary part: |z| may round
// below a.)
__device__ inline cd csqrtv(double a, double b) {
  if (b == 0.0) return a >= 0.0 ? cd{sqrt(a), 0.0} : cd{0.0, sqrt(-a)};
  double r = sqrt(0.5 * (fabs(a) + hypot(a, b)));
  if (a >= 0.0) return cd{r, 0.5 * b / r};
  return cd{0.5 * fabs(b) / r, copysign(r, b)};
}

__device__ inline cd kappa_of(const double* lr, const double* li, int j) {
  return csqrtv(lr[j], li[j]);
}


// Forward-mode dual number: value and derivative with respect to one parameter.
struct dual {
  double v, d;
};
__host__ __device__ inline dual operator+(dual a, dual b) { return dual{a.v + b.v, a.d + b.d}; }
__host__ __device__ inline dual operator-(dual a, dual b) { return dual{a.v - b.v, a.d - b.d}; }
__host__ __device__ inline dual operator-(dual a) { return dual{-a.v, -a.d}; }
__host__ __device__ inline dual operator*(dual a, dual b) { return dual{a.v * b.v, a.d * b.v + a.v * b.d}; }
__host__ __device__ inline dual operator/(dual a, dual b) {
  return dual{a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)};
}
__host__ __device__ inline dual operator+(dual a, double b) { return dual{a.v + b, a.d}; }
__host__ __device__ inline dual operator+(double a, dual b) { return dual{a + b.v, b.d}; }
__host__ __device__ inline dual operator-(dual a, double b) { return dual{a.v - b, a.d}; }
__host__ __device__ inline dual operator-(double a, dual b) { return dual{a - b.v, -b.d}; }
__host__ __device__ inline dual operator*(dual a, double b) { return dual{a.v * b, a.d * b}; }
__host__ __device__ inline dual operator*(double a, dual b) { return dual{a * b.v, a * b.d}; }
__host__ __device__ inline dual operator/(dual a, double b) { return dual{a.v / b, a.d / b}; }
__host__ __device__ inline dual operator/(double a, dual b) {
  return dual{a / b.v, -a * b.d / (b.v * b.v)};
}
__host__ __device__ inline dual dsqrt(dual a) {
  double r = sqrt(a.v);
  return dual{r, r > 0.0 ? 0.5 * a.d / r : 0.0};
}
__host__ __device__ inline dual dexp(dual a) {
  double e = exp(a.v);
  return dual{e, e * a.d};
}
__host__ __device__ inline dual dlog(dual a) { return dual{log(a.v), a.d / a.v}; }
__host__ __device__ inline double val(double a) { return a; }
__host__ __device__ inline double val(dual a) { return a.v; }
__host__ __device__ inline double dsqrt(double a) { return sqrt(a); }
__host__ __device__ inline double dexp(double a) { return exp(a); }
__host__ __device__ inline double dlog(double a) { return log(a); }

// ---------------------------------------------------------------- tables (k_tables.cu)
void launch_gauss_nodes(int N, double* mu, double* w, unsigned* status, cudaStream_t s);
void launch_interface(int N, int n_in, int n_out, double nif, const double* mu_nodes,
                      const double* mu_in, const double* mu_out, double* pts, double* min4,
                      double* mout4, double* rtop4, cudaStream_t s);
void launch_gsf_tables(const OrderBatch& b, const double* pts, double* p, double* r, double* t,
                       cudaStream_t s);
// d/dn of the interface data (dual numbers): dpts [P], dmin4, dmout4, drtop4 (k_tables.cu)
void launch_interface_dn(int N, int n_in, int n_out, double nif, const double* mu_nodes,
                         const double* mu_in, const double* mu_out, double* dpts, double* dmin4,
                         double* dmout4, double* drtop4, cudaStream_t s);
// tangent tables: table 1 = d/dn at the incident points, table 2 = at the outgoing points,
// the function values at every other point
void launch_gsf_tables_dn(const OrderBatch& b, const double* pts, const double* dpts, double* p1,
                          double* r1, double* t1, double* p2, double* r2, double* t2,
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
// Depth factors g0tab[o][k] = depth_factor(tau, mu_o, mu0_k) of one layer, followed by its
// beam table (beam_table(g0tab)): e^{-tau0/mu0_k} then 1/mu0_k, n_in each.
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
// the same with op(A) = A^T (A stored K x M) when tA and op(B) = B^T (B stored N x K) when tB
void dgemm_batched_t(bool tA, bool tB, int M, int N, int K, double alpha, const double* A,
                     int lda, long long sA, const double* B, int ldb, long long sB, double beta,
                     double* C, int ldc, long long sC, int batch, cudaStream_t s);
// Reconstruction epilogue: Isyn[m][k][o][a][s] = T1[ro][rc] + g0(o, k) * (A @ B)[ro][rc]
void dgemm_part_epilogue(const OrderBatch& b, const double* A, const double* B, const double* T1,
                         const double* g0tab, double* Isyn, cudaStream_t s);
// Ainv[u] = A[u]^-1 (FP64 Gauss-Jordan with partial pivoting, one CTA per matrix); with
// skip, only the matrices u with skip[u] != 0.
void batched_inverse(int n, double* A, double* Ainv, int batch, unsigned* status, cudaStream_t s,
                     const int* skip = nullptr);
// The same elimination in FP32 into an FP32 result (a starting inverse).
void batched_inverse_f32(int n, const double* A, float* Ainv, int batch, unsigned* status,
                         cudaStream_t s);
// Mixed form: XA[u] = A[u]^-1 (na x na) and XB[u] = B[u]^-1 (nb x nb; nb = 0: none) from
// one FP32 elimination launch and `steps` Newton-Schulz steps X <- X + X (I - A X) on the
// tensor cores (sliced products of `slices` slices, workspace tcw); err[q][u] receives the
// final max|I - A X| (bits of a non-negative double); matrices whose residual is not below
// tol are inverted again by the FP64 elimination, counted in *fallback_count. `scratch`
// holds newton_inverse_scratch_bytes(na, nb, batch).
size_t newton_inverse_scratch_bytes(int na, int nb, int batch);
void newton_inverse(int na, const double* A, double* XA, int nb, const double* B, double* XB,
                    int batch, int steps, double tol, void* scratch, unsigned long long* err,
                    int* fallback_count, void* tcw, int slices, unsigned* status, cudaStream_t s);
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
// accuracy ~2^-7S per term); K <= 1024, 1 <= S <= 8. `work` holds tc_workspace_bytes.
size_t tc_workspace_bytes(int M, int N, int K, int batch, int S);
// the part of tc_workspace_bytes that does not grow with the batch (epilogue scratch)
size_t tc_scratch_bytes();
bool tc_shape_ok(int K, int S);
// A K range on which both operands of unit u are zero: [zk0, zk0 + zbase + zstep u). The
// K blocks inside it are neither copied nor multiplied (a Fourier order m has no terms of
// degree l < m: its (l, component) contractions start at K = 4m).
struct TcKSkip {
  int zk0 = 0, zbase = 0, zstep = 0;
};
// Parts of a sliced product: `slice` writes both operands' slices into the workspace, `run`
// multiplies the column tiles [nt_lo, nt_lo + nt_cnt) of 64 columns (nt_cnt = 0: all) from the
// slices already there (the same M, N, K, batch and workspace as the slicing call).
struct TcRange {
  bool slice = true, run = true;
  int nt_lo = 0, nt_cnt = 0;
};
constexpr int kTcTileCols = 64;  // columns of one output tile of the sliced product
void tc_gemm_store(int M, int N, int K, const double* A, int lda, long long sA, const double* B,
                   int ldb, long long sB, double beta, double* C, int ldc, long long sC,
                   int batch, int S, void* work, unsigned* status, cudaStream_t s,
                   TcKSkip zskip = TcKSkip{}, int max_ctas = 0, TcRange rg = TcRange{});
// C = alpha op(A) op(B) + beta C with op = transpose where tA / tB (A stored K x M, B stored
// N x K), as the sliced product above.
void tc_gemm_store_t(bool tA, bool tB, int M, int N, int K, double alpha, const double* A,
                     int lda, long long sA, const double* B, int ldb, long long sB, double beta,
                     double* C, int ldc, long long sC, int batch, int S, void* work,
                     unsigned* status, cudaStream_t s);
void tc_gemm_part(const OrderBatch& b, int K, const double* A, int lda, long long sA,
                  const double* B, long long sB, const double* T1, const double* g0tab,
                  double* Isyn, int S, void* work, cudaStream_t s, TcKSkip zskip = TcKSkip{},
                  int* nonfinite = nullptr, TcRange rg = TcRange{});
// Mixed form: flags (order, incident) column blocks whose sliced reconstruction error
// bound eps K max|row| max|column| exceeds tol |I_00| and recomputes them in FP64 (their
// boundary coefficients, written over those columns of C, then their columns of I^m).
void refine_columns(const OrderBatch& b, int Kpart, const double* Kinv, const double* RHS,
                    double* C, const double* Hhat, const double* Uext, const double* SD,
                    const double* g0tab, double eps, double tol, double* scratch, int* counters,
                    int2* list, int cap, double* Isyn, int* nonfinite, cudaStream_t s);
// refine_columns in two parts: the operand maxima (once, when the operands are final), then the
// flag / collect / FP64 fix of the incident cosines k0 <= k < k1 (after their columns of I^m
// are reconstructed).
void refine_maxima(const OrderBatch& b, int Kpart, const double* C, const double* Hhat,
                   const double* Uext, const double* SD, double* scratch, cudaStream_t s);
void refine_range(const OrderBatch& b, int Kpart, const double* Kinv, const double* RHS,
                  double* C, const double* Hhat, const double* Uext, const double* SD, const double* g0tab,
                  double eps, double tol, const double* scratch, int* counters, int2* list,
                  int cap, double* Isyn, int* nonfinite, int k0, int k1, cudaStream_t s);
size_t refine_scratch_doubles(int U, int n_in, int n_out);
// T1 += g0 (A @ B): the first part of a reconstruction contraction split in K.
void tc_gemm_part_accum(const OrderBatch& b, int K, const double* A, int lda, long long sA,
                        const double* B, long long sB, double* T1, const double* g0tab, int S,
                        void* work, cudaStream_t s, TcKSkip zskip = TcKSkip{});
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
// map: [n_phi] computed azimuths (the first n_rep entries) and [n_phi] their mirrors at -phi
// (-1: none), written by the plan; the mirror's table entry is the computed one (cosine
// class) or its negative (sine class).
// Only the incident cosines k_lo <= k < k_hi (k_hi < 0: all); slice_weights false reuses the
// weight slices a previous call left in `work`.
void tc_synthesis(int M, int n_in, int n_out, int n_phi, int n_rep, const int* map,
                  const double* Isyn, const double* wc, const double* ws, void* out,
                  int out_dtype, int k_block, void* work, unsigned* status, cudaStream_t s,
                  const SynthHook* hook = nullptr, int k_lo = 0, int k_hi = -1,
                  bool slice_weights = true);

// ---------------------------------------------------------------- mode algebra (k_modes.cu)
void launch_pack_Y(const OrderBatch& b, const double* EX, const double* lam_re,
                   const double* lam_im, double* Y, cudaStream_t s);
void launch_build_K(const OrderBatch& b, const double* X, const double* Y, const double* lam_re,
                    const double* lam_im, const double* rtop4, double* K, cudaStream_t s);
// (btab: the layer's beam table, see launch_depth_table)
void launch_particular_rhs(const OrderBatch& b, const double* w_in, const double* r,
                           const double* btab, double* w_out, cudaStream_t s);
void launch_eigen_scale(const OrderBatch& b, const double* lam_re, const double* lam_im,
                        const double* btab, double* y, cudaStream_t s);
void launch_particular_sd(const OrderBatch& b, const double* pbeam, const double* Es,
                          const double* pts, double* d, cudaStream_t s);
void launch_bc_rhs(const OrderBatch& b, const double* sv, const double* d, const double* rtop4,
                   const double* btab, double* rhs, cudaStream_t s);
void launch_build_Hhat(const OrderBatch& b, const double* P1, const double* P2,
                       const double* lam_re, const double* lam_im, const double* pts,
                       double* Hhat, cudaStream_t s);

// ---------------------------------------------------------------- reflecting base (k_modes.cu)
// Direction-independent Mueller BRDF matrix R of a reflecting base (row-major), the sum of the
// layer's base_mueller and the Lambertian 2 rho e0 e0^T; passed to the kernels by value.
struct BaseR {
  double r[16];
};
// The base of a layer; false for a black base (R = 0).
inline bool layer_base(const vrte_layer& l, BaseR* out) {
  BaseR b;
  bool any = false;
  for (int i = 0; i < 16; ++i) {
    b.r[i] = l.base_mueller[i];
    any = any || b.r[i] != 0.0;
  }
  b.r[0] += 2.0 * l.base_albedo;
  any = any || l.base_albedo != 0.0;
  if (out) *out = b;
  return any;
}
// Buffer of the base stage per workspace slot: basev [4][2n], zb [4][R], vb [4][R] doubles.
inline size_t base_buffer_doubles(int n, int R) { return 8 * (size_t)n + 8 * (size_t)R; }
void launch_base_K(int N, int n, double tau, const BaseR& Rg, const double* X, const double* Y,
                   const double* lam_re, const double* lam_im, const double* mu_nodes,
                   const double* w_nodes, double* K, double* basev, cudaStream_t s);
void launch_base_rhs(int N, int n, int R, long long sSD, double tau, const BaseR& Rg,
                     const double* SD, const double* pts, const double* min4,
                     const double* mu_nodes, const double* w_nodes, double* RHS, double* zb,
                     int add_rhs, cudaStream_t s, double t_above = 0.0);
// Adds the base's radiance at the bottom, attenuated by e^{-tau/mu_o}, to the order-0 upward
// radiance `out` (basebuf as filled by launch_base_K and launch_base_rhs; its vb part is
// written here).
void launch_base_recon(int n, int N, int n_in, int n_out, double tau, const BaseR& Rg,
                       const double* C, double* basebuf, const double* pts,
                       const double* mout4, double* out, int isyn, cudaStream_t s);
// Multi-layer slabs (k_slab.cu): boundary blocks and right-hand side of one sub-layer, the
// beam's attenuation to a sub-layer's top, and the attenuated sum of the sub-layers'
// contributions to the upward radiance at the slab's top.
void launch_slab_blocks(const OrderBatch& b, int first, const double* X, const double* Y,
                        const double* lam_re, const double* lam_im, const double* rtop4,
                        double* D, double* Uup, double* Ldn, cudaStream_t s);
void launch_slab_rhs(const OrderBatch& b, int first, const double* SD, const double* rtop4,
                     const double* pts, const double* Pd_prev, double* rhs, double* Pd_cur,
                     double* Zt, cudaStream_t s);
void launch_slab_scale_sd(const OrderBatch& b, double t, const double* pts, double* SD,
                          cudaStream_t s);
void launch_slab_accum(const OrderBatch& b, double t, const double* pts, const double* T1,
                       const double* Tq, const double* g0tab, double* Acc, int first,
                       cudaStream_t s);
void launch_slab_store(const OrderBatch& b, const double* Acc, double* Isyn, cudaStream_t s);

// ---------------------------------------------------------------- radiance at depth tau
void launch_btdf_points(int N, int n_in, int n_out, double nif, const double* mu_out, double* pts,
                        double* mout4, double* rout4, cudaStream_t s);
void launch_assemble_direct_depth(const OrderBatch& b, double tau, int down, const double* p,
                                  const double* r, const double* t, const double* pts,
                                  const double* min4, double* T, cudaStream_t s);
void launch_build_Hdepth(const OrderBatch& b, double tau, int down, const double* P1,
                         const double* P2, const double* lam_re, const double* lam_im,
                         const double* pts, double* H, cudaStream_t s);
void launch_depth_combine(const OrderBatch& b, double tau, int down, const double* Tdep,
                          const double* Q, const double* T1, const double* Qp, const double* pts,
                          const double* rout4, double* Isyn, cudaStream_t s);

// ---------------------------------------------------------------- synthesis (k_synth.cu)
void launch_synthesis_fp64(int M, int n_in, int n_out, int n_phi, const double* Isyn,
                           const double* wc, const double* ws, void* out, int out_dtype,
                           unsigned* status, cudaStream_t s);

// ---------------------------------------------------------------- adjoint (k_adjoint.cu)
// Synthesis transpose: Ibar[m][k][o][16] from the table gradient G (FP32 or FP64).
void launch_synth_transpose(int M, int n_in, int n_out, int n_phi, const void* G, int g_dtype,
                            const double* wc, const double* ws, double* Ibar, cudaStream_t s);
// acc[0] = dL/domega, acc[1] = dL/dtau0, acc[2] = dL/dn, acc[3 + 6 l + q] = dL/dcoef
void bw_tb(const OrderBatch& b, const double* Ibar, const double* g0tab, double* Tb, double* G0,
           cudaStream_t s);
void bw_g0(const OrderBatch& b, const double* Tb, const double* Qp, const double* T1,
           const double* pts, const double* dpts, double* acc, cudaStream_t s);
void bw_kappa(const OrderBatch& b, const double* lam_re, const double* lam_im, double* kap,
              cudaStream_t s);
void bw_hhat(const OrderBatch& b, const double* Hb, const double* P1, const double* P2,
             const double* kap, const double* pts, const double* dpts, double* P1b, double* P2b,
             double* acc, cudaStream_t s);
void bw_K(const OrderBatch& b, const double* Kb, const double* X, const double* Y,
          const double* kap, const double* rtop4, const double* drtop4, double* acc,
          cudaStream_t s);
void bw_rhs(const OrderBatch& b, const double* nu, const double* SD, double* SDb,
            const double* rtop4, const double* drtop4, const double* pts, const double* dpts,
            double* acc, cudaStream_t s);
void bw_part_d(const OrderBatch& b, const double* SD, const double* SDb, const double* pts,
               const double* dpts, double* pb, double* acc, cudaStream_t s);
void bw_scale(const OrderBatch& b, const double* lam_re, const double* lam_im, const double* ys,
              double* ysb, const double* pts, const double* dpts, double* acc, cudaStream_t s);
void bw_part_w(const OrderBatch& b, const double* wb, const double* r, const double* pts,
               const double* dpts, double* rb, double* acc, cudaStream_t s);
void bw_cplx_cols(const OrderBatch& b, const double* X, const double* Y, const double* kap,
                  const double* rtop4, double* Xc, double* Yc, double* Pmc, double* Gtc,
                  cudaStream_t s);
void bw_cplx_rows(int n, int rows, int cols, long long sA, const double* A, const double* kap,
                  double* Z, int units, cudaStream_t s);
void bw_rowdiv(int n, int cols, const double* kap, double* Z, int units, cudaStream_t s);
void bw_zeta(int n, int R, const double* Ta, const double* Tz, double* zeta, int units,
             cudaStream_t s);
void bw_psi(const OrderBatch& b, const double* P1, const double* P2, const double* kap,
            const double* pts, double* PsiT1, double* PsiT2, cudaStream_t s);
void bw_gf(const OrderBatch& b, const double* kap, const double* pts, double* Ah, cudaStream_t s);
void bw_i1(int n, double tau, const double* kap, double* Om, int units, cudaStream_t s);
void bw_i2(const OrderBatch& b, const double* kap, const double* pts, const double* Dp,
           double* Dp2, cudaStream_t s);
void bw_omblk(int n, const double* Om, double* OmF, double* OmE, int units, cudaStream_t s);
void bw_dot(long long count, const double* A, long long sA, const double* B, long long sB,
            double scale, double* dst, int units, cudaStream_t s);
void bw_dot_ef(int n, int N, const double* Eb, const double* E2, const double* Fb,
               const double* F2, const double* mu_nodes, double* acc, int units, cudaStream_t s);
void bw_sbar_nn(const OrderBatch& b, const double* Eb, const double* Fb, const double* mu_nodes,
                const double* w_nodes, double* S, cudaStream_t s);
void bw_sbar_ni(const OrderBatch& b, const double* pb, const double* rb, const double* mu_nodes,
                const double* min4, double* S, cudaStream_t s);
void bw_sbar_on(const OrderBatch& b, const double* Ub, const double* w_nodes, const double* mout4,
                double* S, cudaStream_t s);
void bw_sbar_oi(const OrderBatch& b, const double* G0, const double* min4, const double* mout4,
                double* S, cudaStream_t s);
void bw_pstack(const OrderBatch& b, int y0, int ny, const double* pt, const double* rt,
               const double* tt, double* PY, cudaStream_t s);
void bw_bbar(const OrderBatch& b, int x0, int nx, const double* Qg, const double* Qd,
             long long sQ, const double* pt, const double* rt, const double* tt, double* acc,
             cudaStream_t s);
void bw_finish(int L, int Lmax, double nif, const double* acc, double* grad, cudaStream_t s);

}  // namespace vrte
