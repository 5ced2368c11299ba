/*
 * vrte.h -- C ABI of the GB300 DOM solver for the vector radiative transfer
 * equation (VRTE) of a flat particulate layer and its polarized subsurface BRDF.
 *
 * Method: Collin & Pattanaik, "GPU accelerated computation of Polarized
 * Subsurface BRDF for Flat Particulate Layers" (arXiv 1707.05882).
 *   - Sec. 2.B, Eqs. 6-15: azimuthal Fourier decomposition; every order m is an
 *     independent discrete-ordinate problem built from the phase-matrix
 *     expansion coefficients at N double-Gauss nodes per hemisphere.
 *   - Sec. 3.A, Eqs. 40-45: homogeneous solution through the 4N x 4N product FE.
 *   - Sec. 3.B, Eqs. 46-48: particular solution for a collimated beam.
 *   - Sec. 3.C, Eqs. 49-56: boundary-condition system, one per order, with every
 *     incident direction and Stokes basis vector as a right-hand side.
 *   - Sec. 2.C, Eqs. 36-38 and Sec. 3.D: source-function reconstruction at
 *     arbitrary outgoing angles.
 *   - Sec. 2.D, Eqs. 1, 12, 39: Fourier synthesis into the 4x4 Mueller BRDF.
 *
 * Conventions (the paper leaves them open; the library fixes them):
 *   - optical depth grows downward, mu > 0 is an upward propagation direction;
 *   - Stokes vectors on the meridian frame (e_theta, e_phi) of the propagation
 *     direction, V = -2 Im(E_theta E_phi*);
 *   - F[r][s] = exiting radiance component r for a unit incident Stokes basis
 *     vector s, divided by the irradiance mu_in * I0 on the horizontal surface
 *     (units 1/sr); mu_in is the cosine towards the source, mu_out towards the
 *     viewer, dphi = phi_out - phi_in, both directions pointing away from the
 *     surface;
 *   - optional smooth dielectric top of relative index n > 1 (Fresnel
 *     transmission in and out, internal specular reflection as the top boundary
 *     condition); n <= 1 means a bare top. Black lower boundary, or a reflecting
 *     base with a direction-independent Mueller BRDF matrix (vrte_layer.base_albedo
 *     for the depolarizing Lambertian base, vrte_layer.base_mueller in general).
 *
 * Threading and ownership: a plan is used by one host thread at a time. All
 * d_* pointers are device memory owned by the caller; the plan owns its
 * workspace (allocated by vrte_plan_create / vrte_set_layer, freed by
 * vrte_destroy). Every call is asynchronous on the caller's stream except where
 * stated; errors found on the device are recorded in a device status word and
 * reported by vrte_plan_status (which synchronizes) and by the next call.
 */
#ifndef VRTE_H
#define VRTE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  VRTE_OK = 0,
  VRTE_ERR_INVALID_ARG = 1,   /* rejected before any launch */
  VRTE_ERR_STATE = 2,         /* call order violated (e.g. solve before set_layer) */
  VRTE_ERR_CUDA = 3,          /* a CUDA runtime call failed */
  VRTE_ERR_OOM = 4,           /* workspace allocation failed */
  VRTE_ERR_NO_CONVERGENCE = 5,/* eigen iteration hit its sweep limit */
  VRTE_ERR_SINGULAR = 6,      /* a pivot below tolerance in an LU / inverse */
  VRTE_ERR_NONFINITE = 7,     /* a NaN or Inf reached the output */
  VRTE_ERR_UNSUPPORTED = 8    /* valid request the library does not implement */
} vrte_status;

typedef enum {
  VRTE_FP64 = 0,   /* every stage in FP64 on CUDA cores */
  VRTE_MIXED = 1   /* dense contractions on tcgen05 tensor cores, FP64 where it matters */
} vrte_precision;

typedef enum {
  VRTE_OUT_F32 = 0,
  VRTE_OUT_F64 = 1
} vrte_dtype;

/* Plan descriptor. Grids are host arrays copied at plan creation. */
typedef struct {
  int n_nodes_max;     /* N: Gauss nodes per hemisphere, 1 <= N <= 96 */
  int n_orders_max;    /* M: Fourier orders m = 0..M-1, 1 <= M <= 1024 */
  int n_coef_max;      /* L: expansion coefficients l = 0..L-1, 1 <= L <= 1024 */
  int n_layers_max;    /* independent layers solved in one call */
  int n_mu_in;         /* incident cosines (towards the source), 1..16384 */
  int n_mu_out;        /* outgoing cosines (towards the viewer), 1..16384 */
  int n_phi;           /* azimuth differences */
  const double* mu_in; /* host [n_mu_in],  each in (0, 1] */
  const double* mu_out;/* host [n_mu_out], each in (0, 1] */
  const double* phi;   /* host [n_phi], radians, dphi = phi_out - phi_in */
  int precision;       /* vrte_precision */
  unsigned flags;      /* VRTE_FLAG_* bits; unknown bits are rejected */
} vrte_plan_desc;

/* Records CUDA events around every pipeline stage on the solve stream, read back
 * with vrte_profile_stages. Adds two event records per stage and order batch. */
#define VRTE_FLAG_PROFILE 1u

/* Allocates, in vrte_set_layer, the workspace of the adjoint (vrte_brdf_backward), which
 * vrte_brdf_backward requires. The adjoint recomputes each order batch's eigen-decomposition
 * and boundary factors in FP64 from the layer parameters instead of keeping them, so the
 * workspace grows with the batch of orders processed at once, not with all orders. */
#define VRTE_FLAG_ADJOINT 2u

/* Allocates, in vrte_set_layer, the workspace of the transmission table (vrte_solve_btdf). */
#define VRTE_FLAG_TRANSMISSION 4u

/* Allocates, in vrte_set_layer, the workspace of a multi-layer slab made of the layers set
 * (vrte_solve_slab_brdf): per sub-layer and order of a batch, the block elimination's
 * factors, held once by the plan beside its workspace slots. */
#define VRTE_FLAG_SLAB 8u

/* Per-stage statistics accumulated since the last vrte_profile_reset. */
typedef struct {
  char name[24];        /* stage name, e.g. "eigen", "recon_gemm", "synthesis" */
  long long launches;   /* kernels launched by the stage (counted with or without the flag) */
  double ms;            /* summed event time (0 without VRTE_FLAG_PROFILE) */
  double flops;         /* algorithmic floating-point operations of the stage */
  double bytes;         /* algorithmic HBM bytes of the stage (compulsory traffic) */
  double tc_flops;      /* mixed form: BF16 tensor-core FLOPs the sliced products issue
                           (S (S + 1) / 2 slice products per FP64 product), else 0 */
} vrte_stage_stat;

/* Per-layer parameters (host). */
typedef struct {
  double tau;          /* optical thickness tau0 > 0 */
  double omega;        /* single-scattering albedo, 0 <= omega < 1 */
  double n_interface;  /* relative index of a smooth top; <= 1 means none; at most 3 */
  int n_nodes;         /* N of this layer, 1..n_nodes_max */
  int n_orders;        /* M of this layer, 1..n_orders_max; orders >= n_coef contribute 0 */
  int n_coef;          /* L of this layer, 1..n_coef_max */
  double base_albedo;  /* albedo rho in [0, 1] of a depolarizing Lambertian base under the
                          layer (Sec. 3.C, base reflection, R_00 = 2 rho); 0 = black base */
  double base_mueller[16]; /* direction-independent 4x4 Mueller BRDF matrix R of a reflecting
                          base under the layer, row-major, added to the Lambertian
                          2 rho e0 e0^T (Sec. 3.C, base reflection, Eqs. 57-66 with R not
                          depending on mu_i, mu_j, mu0). Scale as the paper's R: a bare base
                          reflects the table R / (2 pi). Only order 0 sees it, so its
                          (I, Q) x (U, V) entries R[0..1][2..3], R[2..3][0..1] must be 0;
                          the total R_00 must lie in [0, 2]; all zero = no extra base */
} vrte_layer;

typedef struct vrte_plan vrte_plan;

/* Creates a plan: validates the descriptor, copies the grids to the device and
 * allocates per-plan tables (the azimuth weights of the Fourier synthesis, Sec. 2.B,
 * Eqs. 7 and 12). Returns VRTE_ERR_INVALID_ARG for out-of-range sizes or cosines,
 * VRTE_ERR_OOM / VRTE_ERR_CUDA on device failures. */
vrte_status vrte_plan_create(const vrte_plan_desc* desc, vrte_plan** out);

/* Sets the layers to solve: the optical thickness, albedo and phase-matrix expansion of
 * Sec. 2.A-2.B (Eqs. 2-10; coefficients per Eq. 9's B_l). host_params: [n_layers]
 * parameters (copied).
 * d_coeffs: device FP64 [n_layers][n_coef_max][6] expansion coefficients
 * (alpha1, alpha2, alpha3, alpha4, beta1, beta2) per l, zero-padded beyond each
 * layer's n_coef; the pointer is kept and read by each solve (the caller keeps
 * it alive). Allocates the solve workspace for these layers. A VRTE_MIXED plan
 * contracts over the 4 n_coef (l, component) pairs on the tensor cores and returns
 * VRTE_ERR_UNSUPPORTED when 4 n_coef > 1024 (before touching the workspace).
 * VRTE_ERR_INVALID_ARG for a parameter out of range (see vrte_layer), including a base
 * matrix with a non-finite entry, a nonzero (I, Q) x (U, V) entry or R_00 outside [0, 2]. */
vrte_status vrte_set_layer(vrte_plan* plan, int n_layers, const vrte_layer* host_params,
                           const double* d_coeffs);

/* Solves every layer and writes the BRDF table (Sec. 2: Eq. 1's F_r from the per-order
 * solutions of Secs. 2.C and 3.A-3.D, synthesized by Eqs. 7, 12 and 39)
 *   d_brdf[n_layers][n_mu_in][n_mu_out][n_phi][4][4]   (row r = exiting Stokes
 *   component, column s = incident Stokes basis vector),
 * FP32 or FP64 per out_dtype, on `stream` (a cudaStream_t; NULL = legacy default
 * stream). Asynchronous: no host synchronization and no allocation inside. With several
 * layers the plan runs up to four layers at a time on streams of its own, forked from
 * `stream` by an event and joined back into it, so the call stays ordered on `stream`
 * and can be captured into a CUDA graph from it.
 * Accuracy against the exact DOM solution of the given N: VRTE_FP64 ~1e-10 of F_00 at
 * the same point (more near a resonance mu0 kappa_j ~ 1 of the particular solution,
 * where every FP64 formulation loses digits); VRTE_MIXED 1e-6 on the I row and 1e-5 on
 * the Q, U, V rows of F_00 (column blocks whose sliced-product error bound is large
 * are recomputed in FP64). An FP32 table is the result rounded to FP32 (VRTE_MIXED:
 * within one unit in the last place). */
vrte_status vrte_solve_brdf(vrte_plan* plan, void* d_brdf, int out_dtype, void* stream);

/* Transmission table (BTDF) of every layer: the diffuse radiance leaving the bottom of the
 * layer downward, per unit irradiance mu_in * I0 of the beam from above,
 *   d_btdf[n_layers][n_mu_in][n_mu_out][n_phi][4][4]  (layout and units as d_brdf),
 * with mu_out the cosines of the downward directions below the layer (no interface at the
 * bottom, so they are internal cosines as given), dphi = phi_out - phi_in, Stokes vectors on
 * the meridian frames of the propagation directions. The uncollided beam (a delta in
 * direction) is not included. Paper: the field at tau0 of the solution of Sec. 2.C (Eqs. 36,
 * 38 taken along the downward path) with the radiance the top sends back down (zero for a
 * bare top, R_F times the upward radiance at the same cosine under a dielectric top), and the
 * Fourier synthesis of Eq. 12. Solved in FP64 (VRTE_FP64 plans) or with the plan's mixed
 * synthesis; requires a plan created with VRTE_FLAG_TRANSMISSION (else VRTE_ERR_STATE).
 * Asynchronous; no allocation. */
vrte_status vrte_solve_btdf(vrte_plan* plan, void* d_btdf, int out_dtype, void* stream);

/* Radiance field inside every layer at depth h_tau[layer] (host, 0 <= tau <= the layer's tau0),
 * per unit irradiance mu_in * I0 of the beam from above (incident through the top interface
 * as for the BRDF), for the internal cosines mu_out of the plan, without exit factors:
 *   d_up[n_layers][n_mu_in][n_mu_out][n_phi][4][4]    directions (+mu_out, phi), upward,
 *   d_down[...]                                        directions (-mu_out, phi), downward
 * (either may be NULL; layout and Stokes frames as d_brdf, dphi = phi - phi_in). Paper:
 * Sec. 2.C reconstruction at an arbitrary tau (Eqs. 36-38 with the integration ranges
 * [tau, tau0] upward and [0, tau] downward; the boundary radiances are the reflecting base's at
 * tau0 and the top's internal reflection at 0) and Sec. 4's radiance-field experiment.
 * d_up at tau = 0 is the internal upward radiance under the top; d_down at tau0 the
 * transmission table. Solved as vrte_solve_btdf; requires VRTE_FLAG_TRANSMISSION (else
 * VRTE_ERR_STATE); a depth outside [0, tau0] gives VRTE_ERR_INVALID_ARG. */
vrte_status vrte_solve_radiance(vrte_plan* plan, const double* h_tau, void* d_up, void* d_down,
                                int out_dtype, void* stream);

/* BRDF table of ONE slab whose sub-layers are the n_layers layers of the last vrte_set_layer,
 * top first (sub-layer k spans the optical depths [t_k, t_k + tau_k], t_k the sum of the
 * thicknesses above it), each with its own expansion coefficients, albedo and thickness:
 *   d_brdf[n_mu_in][n_mu_out][n_phi][4][4]  (one table; layout and units as vrte_solve_brdf).
 * The first sub-layer's n_interface is the slab's smooth top and the last one's base_albedo
 * and base_mueller its reflecting base; the other sub-layers must have n_interface <= 1 and a
 * black base (base_albedo 0, base_mueller all 0), and
 * all must share n_nodes and n_orders (else VRTE_ERR_INVALID_ARG). Orders at or beyond a
 * sub-layer's n_coef see it as a purely attenuating layer. Paper: Sec. 2.C, multiple layer
 * materials: a homogeneous solution and a particular solution per sub-layer (for the beam
 * attenuated to the sub-layer's top), 8N more unknowns per sub-layer, and 8N continuity
 * equations of the radiance at every boundary between two sub-layers, with the top and
 * bottom conditions of Sec. 2.C; the upward radiance at the top is the sum of the
 * sub-layers' reconstructions (Eqs. 36-38), each attenuated through the sub-layers above.
 * Solved in FP64 (block elimination of the block-tridiagonal system from the top, one
 * sub-layer at a time, while the mode stages of the next sub-layers run on the plan's other
 * workspace slots and their streams, forked from and joined back into `stream`) with the
 * plan's synthesis; requires a plan created with VRTE_FLAG_SLAB (else VRTE_ERR_STATE).
 * Asynchronous; no allocation. */
vrte_status vrte_solve_slab_brdf(vrte_plan* plan, void* d_brdf, int out_dtype, void* stream);

/* Same solve as vrte_solve_brdf (same passages) with host buffers: copies h_coeffs (host
 * FP64, layout as d_coeffs
 * of vrte_set_layer) to the plan's staging buffer, solves, copies the table to
 * h_brdf (host, layout as d_brdf) and synchronizes `stream` before returning. The table
 * leaves a device staging buffer in blocks of incident cosines, each copied as soon as the
 * synthesis kernels that complete it have run, on four streams of the plan (several copy
 * engines) that wait on `stream` by events and are joined back into it. In the VRTE_MIXED
 * form a layer whose orders fit one batch, with no reflecting base and 2n + 4L <= 1024, is
 * also reconstructed block by block (the same values as vrte_solve_brdf, bit for bit), so
 * that the copies overlap the reconstruction; for that the first call allocates a second
 * device workspace (the homogeneous contraction's slices and the synthesis workspace, kept
 * by the plan and counted by vrte_workspace_bytes); if that allocation fails the layer is
 * reconstructed whole. The staging buffers are allocated by the first call (or a call with a
 * larger table); VRTE_ERR_OOM if they do not fit. Pinned host memory gives full copy
 * bandwidth. */
vrte_status vrte_solve_brdf_host(vrte_plan* plan, const double* h_coeffs, void* h_brdf,
                                 int out_dtype, void* stream);

/* Adjoint of the BRDF table (the paper has no adjoint; it is the differentiation target of
 * the inverse material-fitting use): given d_grad_brdf = dL/dF for a scalar loss L of the
 * table F that vrte_solve_brdf writes for the plan's current layers (device, layout as
 * d_brdf, FP32 or FP64 per grad_dtype), writes
 *   d_grad_params[n_layers][3 + 6 n_coef_max]  (device FP64, caller-owned)
 * = dL/d(omega, tau0, n_interface, coefficients), the coefficients in the order of
 * d_coeffs ((alpha1, alpha2, alpha3, alpha4, beta1, beta2) per l), zero beyond a layer's
 * n_coef. The interface entry is zero for a layer without interface (n_interface <= 1).
 * The derivative is that of the FP64 solution (the VRTE_FP64 table; a VRTE_MIXED table
 * agrees with it to the mixed form's accuracy). Every order batch is solved again in FP64
 * (eigen-decomposition, boundary system, particular solution) and then reversed: the
 * reverse of Secs. 2.D / 3.D (synthesis, reconstruction), Sec. 3.C (boundary system) and
 * Sec. 3.B (particular solution) with the eigenpairs held fixed, plus the dependence of the
 * homogeneous modes on F'E' (Sec. 3.A) through the adjoint two-point problem of the order,
 * whose mode integrals are closed-form divided differences (finite at degenerate and complex
 * eigenvalues). Requires a plan created with VRTE_FLAG_ADJOINT and vrte_set_layer, else
 * VRTE_ERR_STATE; VRTE_ERR_INVALID_ARG for NULL pointers or an unknown grad_dtype;
 * VRTE_ERR_UNSUPPORTED when a layer has a reflecting base (base_albedo > 0 or a nonzero
 * base_mueller).
 * Asynchronous on `stream`; no allocation; layers run on the plan's streams as in
 * vrte_solve_brdf. Accuracy: ~1e-8 relative in the gradient's largest entries (the FP64
 * solution's rounding, amplified near a resonance mu kappa_j ~ 1 as in the solve). */
vrte_status vrte_brdf_backward(vrte_plan* plan, const void* d_grad_brdf, int grad_dtype,
                               double* d_grad_params, void* stream);

/* The azimuth pairing the tensor-core synthesis uses (Eqs. 7, 12: the cosine class of the table
 * is even and the sine class odd in the azimuth difference, so the table at -phi follows from
 * the one at phi). Host only, no GPU needed. phi: n_phi azimuths (radians, any range);
 * map_out: 2 n_phi ints, caller-owned: map_out[0 .. n_rep) the azimuths computed, in
 * increasing index order, and map_out[n_phi + r] the index of the azimuth at -phi[map_out[r]]
 * (mod 2 pi, within 1e-12 rad) that is stored from it, or -1 (none on the grid, the azimuth
 * itself at 0 or pi, or already paired); the rest of map_out is -1. *n_rep_out receives
 * n_rep. VRTE_ERR_INVALID_ARG for NULL pointers, n_phi < 1 or a non-finite azimuth. */
vrte_status vrte_azimuth_mirrors(int n_phi, const double* phi, int* map_out, int* n_rep_out);

/* (Library bookkeeping; no passage.) Synchronizes the plan's last stream and returns the
 * device status word as a
 * vrte_status (VRTE_OK if no device-side error was recorded), then clears it. */
vrte_status vrte_plan_status(vrte_plan* plan);

/* (Measurement; the paper times its steps per stage, Sec. 4 Table 4.) Copies up to
 * max_stages stage statistics into out (host) and returns the number of
 * stages (or -1 for a NULL plan). Synchronizes the plan's last stream. */
int vrte_profile_stages(vrte_plan* plan, vrte_stage_stat* out, int max_stages);

/* (Measurement.) Clears the stage statistics and the recorded events. */
void vrte_profile_reset(vrte_plan* plan);

/* (Testing; the buffers are the quantities of Secs. 2.C and 3.A-3.D.) Diagnostic read of
 * one internal buffer of the most recent order batch, for
 * stage-level checks: copies min(bytes, buffer size) bytes into host_dst and returns
 * the buffer's full size in *size_out (may be NULL). Synchronizes. Names: "pts",
 * "nodes", "weights", "E", "F", "FE", "schur", "X", "Y", "lam_re", "lam_im", "K",
 * "Kinv", "Xinv", "beam_p", "beam_r", "SD", "RHS", "C", "Upm", "Hhat", "T1", "Isyn",
 * "mode_res" (per-order mode residual of the reduced eigen-decomposition),
 * "status" (the raw device status bits as one double, not cleared) and "refined"
 * (mixed form: number of (order, incident) column blocks of the last solve whose
 * reconstruction was recomputed in FP64, as one double).
 * Unknown names return VRTE_ERR_INVALID_ARG; calling before a solve returns
 * VRTE_ERR_STATE. */
vrte_status vrte_debug_copy(vrte_plan* plan, const char* name, void* host_dst, size_t bytes,
                            size_t* size_out);

/* Batched eigen-decomposition of `batch` real n x n matrices (row-major, device
 * d_A[batch][n][n], read only) without allocating any device memory, for callers that
 * cannot call cudaMalloc: code whose device memory is owned by another allocator or a
 * fixed pool, and code where an allocation would synchronize the device or is not
 * allowed. The paper has
 * no counterpart; this is the library's homogeneous-step eigensolver (balancing,
 * Hessenberg, Francis double-shift QR, back-substitution) run on scratch space taken
 * from a file-scope device array of 2^21 doubles (16 MiB) that every GPU loading the
 * library holds until the process exits.
 *   Outputs (device, caller-owned): d_lam_re, d_lam_im [batch][n]; d_X [batch][n][n]
 *   row-major eigenvectors, a complex pair (j, j+1) with d_lam_im[j] > 0 stored as
 *   real part in column j and imaginary part in column j+1, each vector or pair scaled
 *   to a largest component modulus of one.
 *   d_status: optional device word (caller zeroes it) that receives the device-detected
 *   error bits (1 = no convergence, 4 = non-finite); NULL discards them.
 * Limits: 1 <= n <= 768, 1 <= batch <= 65535 and (3 n^2 + n) * batch <= 2^21 - 8, else
 * VRTE_ERR_INVALID_ARG before any launch. A launch error pending from earlier work on the
 * calling thread is cleared on entry, so VRTE_ERR_CUDA reports this call's launches only.
 * The first call on each device resolves the scratch array's device address (with that
 * device current); make that first call before any stream capture.
 * All calls share the one array and it keeps the previous call's contents (the kernels
 * initialise what they read): calls that overlap on the GPU, on any streams, race.
 * Asynchronous on `stream`. */
vrte_status vrte_eigen_noalloc(const double* d_A, int n, int batch, double* d_lam_re,
                               double* d_lam_im, double* d_X, unsigned* d_status, void* stream);

/* The dense contractions of Secs. 3.B-3.D (particular solution, boundary system,
 * reconstruction) as used by the VRTE_MIXED form, on caller buffers:
 * batched C = A B in FP64 on the tcgen05 tensor cores by exact fixed-point slicing:
 * every row of A and column of B is scaled by a power of two and cut into `slices`
 * signed 7-bit integer slices (each times a power of two) held in BF16; each slice
 * product is exact, products of equal scale are accumulated exactly in FP32 for K <= 1024,
 * so the error is the slices dropped (relative to max|A_i| max|B_j| per term, measured:
 * 4 -> 9e-10, 5 -> 8e-12, 6 -> 7e-14, 7 -> 6e-16, 8 -> 1.4e-16).
 * A [batch][M][K] (row stride lda, unit stride stride_a), B [batch][K][N] (ldb,
 * stride_b), C [batch][M][N] (ldc, stride_c): device FP64, row-major, caller-owned.
 * d_workspace: device buffer of vrte_gemm_sliced_workspace() bytes. d_status: device word
 * (caller zeroes it) receiving device error bits (16 = a bounded wait timed out).
 * Limits: 1 <= slices <= 8, 1 <= K <= 1024, else VRTE_ERR_INVALID_ARG. Asynchronous on
 * `stream`; not thread-safe against other calls sharing the workspace. */
size_t vrte_gemm_sliced_workspace(int M, int N, int K, int batch, int slices);
vrte_status vrte_gemm_sliced(int M, int N, int K, const double* d_A, int lda, long long stride_a,
                             const double* d_B, int ldb, long long stride_b, double* d_C, int ldc,
                             long long stride_c, int batch, int slices, void* d_workspace,
                             size_t workspace_bytes, unsigned* d_status, void* stream);

/* (Library bookkeeping.) Bytes of device workspace the plan currently holds. */
size_t vrte_workspace_bytes(const vrte_plan* plan);

/* (Library bookkeeping.) Frees the plan and its workspace. Accepts NULL. */
void vrte_destroy(vrte_plan* plan);

/* (Library bookkeeping.) Static string for a status code. */
const char* vrte_status_string(vrte_status status);

#ifdef __cplusplus
}
#endif

#endif /* VRTE_H */
