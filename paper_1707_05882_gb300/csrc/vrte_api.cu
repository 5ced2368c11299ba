// C ABI of the VRTE BRDF solver: plan lifetime, workspace, and the per-order pipeline.
//
// Pipeline for each layer and each batch of Fourier orders (all on one stream):
//   a0 tables      Gauss nodes, Fresnel data, generalized spherical functions
//   a1 assembly    E', F' (Eq. 41), beam vectors p, r (Eq. 47), reconstruction operators
//   a2 homogeneous F'E' -> eigenpairs (Eqs. 43-45), Y = E'X / kappa
//   a3 boundary    K (Eqs. 49-56) and its inverse
//   a4/a5 particular  (F'E' - 1/mu0^2) s = F'p - r/mu0 solved in the eigenbasis (Eq. 47),
//                  d = mu0 (p - E's) (Eq. 48)
//   a6 boundary solve  C = K^-1 [-(Z-(0) - R_F Z+(0)); -Z+(tau0) e^{-tau0/mu0}]
//   a7 reconstruction  I^m(0, mu_out) = [Hhat | U+-] [C ; s ; d] with depth integrals (Eqs. 36, 38)
//   a8 synthesis   sum over orders with the Fourier factors (Eqs. 7, 12)
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "vrte_internal.cuh"

using namespace vrte;

namespace {
enum Stage {
  ST_TABLES, ST_ASSEMBLE, ST_EIGEN, ST_MODES, ST_PARTICULAR, ST_BC_SOLVE, ST_RECON_OPS,
  ST_RECON_HOM, ST_RECON_PART, ST_REFINE, ST_SYNTHESIS, ST_ADJOINT, ST_SIDE_OPS, kStages
};
// mixed form: BF16 slices per FP64 operand (exact products, ~6e-16 relative per term) and
// incident cosines per tensor-core synthesis block
constexpr int kSlices = 7;
constexpr int kSlicesSynth = 5;
constexpr int kSynthBlock = 64;
// per-term error of the 7-slice product relative to max|A_i| max|B_j| (measured 6e-16),
// and the bound, relative to the order-0 I_00 of the same (incident, outgoing) pair,
// above which a column block is recomputed in FP64
constexpr double kSliceEps = 2e-15;
constexpr double kRefineTol = 1e-7;
// mixed form: Newton-Schulz steps after the FP32 starting inverse of K and X, and the final
// max|I - A X| above which a matrix is inverted again in FP64
constexpr int kNewtonSteps = 2;
// idle SMs that the eigen-decomposition must leave for the side stream to be used
constexpr int kSideMinSMs = 16;
constexpr double kNewtonTol = 1e-11;

const char* kStageNames[kStages] = {"tables",     "assemble",   "eigen",
                                    "modes_bc_inverse", "particular", "bc_solve",
                                    "recon_ops",  "recon_hom",  "recon_part",
                                    "refine",     "synthesis", "adjoint",
                                    "side_ops"};
}  // namespace

// Buffers of one order batch of one layer. A plan holds up to kMaxSlots of them so that
// the layers of a multi-layer solve run on concurrent streams (a layer's orders occupy
// only as many SMs as it has orders in the FP64 stages).
struct Work {
  // per-layer tables (sized for N_max)
  double *d_mu_nodes = nullptr, *d_w_nodes = nullptr, *d_pts = nullptr, *d_min4 = nullptr,
         *d_mout4 = nullptr, *d_rtop4 = nullptr;
  // order-batch workspace (sized for the largest layer)
  double *gp = nullptr, *gr = nullptr, *gt = nullptr;
  double *E = nullptr, *F = nullptr, *FE = nullptr, *X = nullptr, *EX = nullptr, *Y = nullptr,
         *Xinv = nullptr, *Hs = nullptr, *Zs = nullptr, *Vs = nullptr;
  double *lam_re = nullptr, *lam_im = nullptr, *bal = nullptr;
  double *K = nullptr, *Kinv = nullptr;
  double *Pb = nullptr, *Rb = nullptr, *Wv = nullptr, *Yv = nullptr, *Es = nullptr;
  double *SD = nullptr, *RHS = nullptr, *C = nullptr;
  double *Upm = nullptr, *P1 = nullptr, *P2 = nullptr, *Hhat = nullptr, *T1 = nullptr;
  // block-form eigen fallback (2n x 2n per order)
  double *FY = nullptr, *mode_res = nullptr, *Bm = nullptr, *Hb = nullptr, *Zb = nullptr,
         *Vb = nullptr, *Xb = nullptr, *kb_re = nullptr, *kb_im = nullptr, *balb = nullptr;
  int* mode_flag = nullptr;
  // mixed form: slice workspace of the tensor-core GEMMs (shared with the synthesis)
  void* tcw = nullptr;
  // mixed form: FP64 refinement of ill-conditioned columns (maxima, counters, work list)
  double* rscratch = nullptr;
  // mixed form: factors of the (l, component) contractions for U+- and the beam vectors
  double *Ln = nullptr, *RU = nullptr, *Rbp = nullptr, *Rbm = nullptr;
  int* rcount = nullptr;  // [flagged in this batch, flagged in this solve, FP64 re-inverses]
  int* nfflag = nullptr;  // mixed form: column blocks (unit, incident) to refine, [U][n_in]
  void* nscratch = nullptr;              // mixed form: Newton inverse scratch
  // mixed form, one layer in flight: the eigen-independent operators and beams run on `side`
  // (least priority) on the SMs the eigen-decomposition leaves idle, with their own GEMM
  // workspace; fork and join events order them against the slot's stream
  cudaStream_t side = nullptr;
  cudaEvent_t side_fork = nullptr, side_join = nullptr;
  void* tcw_side = nullptr;
  unsigned long long* nerr = nullptr;    // mixed form: final residuals [K, X][U]
  int2* rlist = nullptr;
  double* Isyn = nullptr;   // [M_max][n_in][n_out][16]; the adjoint keeps Ibar here
  // adjoint (VRTE_FLAG_ADJOINT): per-unit workspace carved per layer, and per-layer data
  double* bw = nullptr;
  // transmission (VRTE_FLAG_TRANSMISSION): [U][Ro][R] each, and the top reflection at mu_out
  double *Qp = nullptr, *Qb = nullptr, *Tbot = nullptr, *Tup = nullptr, *rout4 = nullptr;
  double* Isyn2 = nullptr;  // upward order radiances when both radiance tables are solved
  // Lambertian base: column sums of the bottom radiance [2n] and the reflected source [R]
  double* basebuf = nullptr;
  double *dpts = nullptr, *dmin4 = nullptr, *dmout4 = nullptr, *drtop4 = nullptr,
         *acc = nullptr;
  double* g0tab = nullptr;  // [n_out][n_in] depth factors of the layer
  // slab (VRTE_FLAG_SLAB), per sub-layer [S][U]: D'^-1 (2n x 2n), y then c (2n x R), Uup
  // (n x 2n), Hhat (Ro x 2n); shared: Ldn and Pd of the previous and current sub-layer,
  // Zt, Ldn W, a contraction and the slab's top radiance (Ro x R), Uup c (n x R)
  double *sDinv = nullptr, *sY = nullptr, *sUup = nullptr, *sH = nullptr, *sL[2] = {},
         *sPd[2] = {}, *sZt = nullptr, *sTnn = nullptr, *sTq = nullptr, *sAcc = nullptr,
         *sV = nullptr;
  cudaStream_t stream = nullptr;  // own stream when the plan runs several slots
  cudaEvent_t done = nullptr;
  // slab on several slots: the slot's modes are ready / the slot may be reused
  cudaEvent_t ready = nullptr, freed = nullptr;
};
constexpr int kMaxSlots = 4;

struct vrte_plan {
  vrte_plan_desc desc{};
  int n_in = 0, n_out = 0, n_phi = 0;
  double *d_mu_in = nullptr, *d_mu_out = nullptr, *d_phi = nullptr;
  double *d_wc = nullptr, *d_ws = nullptr;  // [M_max][n_phi]
  // azimuth mirror pairs of the grid (see azimuth_mirrors): [0, n_rep) the computed
  // azimuths, [n_phi, n_phi + n_rep) their mirrors (-1: none)
  int* d_syn_map = nullptr;
  int n_rep = 0;
  unsigned* d_status = nullptr;
  cudaStream_t last_stream = nullptr;
  // layers
  std::vector<vrte_layer> layers;
  const double* d_coeffs = nullptr;
  int n_layers = 0;
  // order-batch workspaces, one per concurrent layer slot
  Work ws[kMaxSlots];
  int nslots = 1;
  int chunk = 0;
  size_t tcw_bytes = 0;
  int kdir = 0;  // extra K of the direct term in the mixed form (4 L_max)
  cudaEvent_t fork = nullptr;
  // host-API output copy: blocks of incident cosines on four streams (several copy engines)
  cudaStream_t cstream[4] = {};
  cudaEvent_t cdone[4] = {}, cready[4] = {};
  cudaEvent_t solved = nullptr;
  // host-API staging
  double* d_coef_stage = nullptr;
  size_t coef_stage_bytes = 0;
  void* d_out_stage = nullptr;
  size_t out_stage_bytes = 0;
  // host-API block-wise reconstruction: the homogeneous contraction's slices and the synthesis
  // workspace (allocated by the first host-buffer solve that can use it; none if that fails)
  void* d_chunk_ws = nullptr;
  size_t chunk_ws_bytes = 0;
  std::vector<void*> allocs;
  std::vector<size_t> alloc_bytes;
  // stage statistics: launches always, event pairs when VRTE_FLAG_PROFILE is set
  vrte_stage_stat stats[kStages];
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> events;
  bool profile = false;
  // geometry of the most recent order batch (for vrte_debug_copy)
  int last_n = 0, last_U = 0, last_P = 0, last_Meff = 0, last_ldU = 0, last_slot = 0;
};

namespace {

vrte_status alloc(vrte_plan* p, void** ptr, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(ptr, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return VRTE_ERR_OOM;
  }
  p->allocs.push_back(*ptr);
  p->alloc_bytes.push_back(bytes);
  return VRTE_OK;
}

template <typename T>
vrte_status allocd(vrte_plan* p, T** ptr, size_t count) {
  return alloc(p, (void**)ptr, count * sizeof(T));
}

void free_workspace(vrte_plan* p, size_t keep) {
  // frees allocations made after index `keep`
  while (p->allocs.size() > keep) {
    cudaFree(p->allocs.back());
    p->allocs.pop_back();
    p->alloc_bytes.pop_back();
  }
}

// Stage bracket: counts launches, adds algorithmic work, records events if profiling.
struct StageScope {
  vrte_plan* p;
  int st;
  cudaStream_t s;
  cudaEvent_t e0 = nullptr;
  StageScope(vrte_plan* p_, int st_, cudaStream_t s_, int launches, double flops, double bytes)
      : p(p_), st(st_), s(s_) {
    p->stats[st].launches += launches;
    p->stats[st].flops += flops;
    p->stats[st].bytes += bytes;
    if (p->profile && cudaEventCreate(&e0) == cudaSuccess) cudaEventRecord(e0, s);
  }
  void tensor_flops(double f) { p->stats[st].tc_flops += f; }
  ~StageScope() {
    if (!e0) return;
    cudaEvent_t e1;
    if (cudaEventCreate(&e1) == cudaSuccess) {
      cudaEventRecord(e1, s);
      p->events.push_back({st, {e0, e1}});
    } else {
      cudaEventDestroy(e0);
    }
  }
};

void reset_stats(vrte_plan* p) {
  for (auto& e : p->events) {
    cudaEventDestroy(e.second.first);
    cudaEventDestroy(e.second.second);
  }
  p->events.clear();
  for (int i = 0; i < kStages; ++i) {
    memset(&p->stats[i], 0, sizeof(vrte_stage_stat));
    strncpy(p->stats[i].name, kStageNames[i], sizeof(p->stats[i].name) - 1);
  }
}

// buffers allocated by vrte_plan_create (kept by vrte_set_layer)
constexpr size_t kPlanAllocs = 7;

// Adjoint workspace of one order batch: consecutive [U][size] arrays for the layer's n.
struct BwBufs {
  double *Tb, *G0, *Qp, *Tdir, *SOI, *Cb, *nu, *SDb, *pb, *rb, *ysb, *wb, *ptmp, *rtmp, *Hb, *Ub,
      *Utmp, *P1b, *P2b, *Kb, *E2, *F2, *Eb, *Fb, *Xc, *Yc, *Xic, *Zc, *Pmc, *Gtc, *Tc, *OmF,
      *OmE, *Om, *kap, *D, *Ch, *zeta, *Dp2, *Ta, *Tz, *PsiT1, *PsiT2, *Ah, *SNN, *SNI, *SON,
      *PYn, *PYi, *QNN, *QNI, *QON, *QOI, *mix[6];
};

// Doubles of the carved workspace (and the pointers when base is given).
size_t bw_carve(double* base, size_t U, size_t n, size_t R, size_t Ro, size_t L, size_t P,
                BwBufs* b) {
  size_t off = 0;
  auto take = [&](double** ptr, size_t per_unit) {
    if (base) *ptr = base + off;
    off += U * per_unit;
  };
  BwBufs d{};
  BwBufs* t = b ? b : &d;
  const size_t RoR = Ro * R, nR = n * R, nn = n * n, Ro2n = Ro * 2 * n, L4 = 4 * L;
  take(&t->Tb, RoR); take(&t->G0, RoR); take(&t->Qp, RoR); take(&t->Tdir, RoR); take(&t->SOI, RoR);
  take(&t->Cb, 2 * nR); take(&t->nu, 2 * nR); take(&t->SDb, 2 * nR);
  take(&t->pb, nR); take(&t->rb, nR); take(&t->ysb, nR); take(&t->wb, nR); take(&t->ptmp, nR);
  take(&t->rtmp, nR);
  take(&t->Hb, Ro2n); take(&t->Ub, Ro2n); take(&t->Utmp, Ro2n);
  take(&t->P1b, Ro * n); take(&t->P2b, Ro * n);
  take(&t->Kb, 4 * nn); take(&t->E2, nn); take(&t->F2, nn); take(&t->Eb, nn); take(&t->Fb, nn);
  take(&t->Xc, 2 * nn); take(&t->Yc, 2 * nn); take(&t->Xic, 2 * nn); take(&t->Zc, 2 * nn);
  take(&t->Pmc, 2 * nn); take(&t->Gtc, 2 * nn); take(&t->Tc, 2 * nn);
  take(&t->OmF, 2 * nn); take(&t->OmE, 2 * nn); take(&t->Om, 8 * nn); take(&t->kap, 2 * n);
  take(&t->D, 4 * nR); take(&t->Ch, 4 * nR); take(&t->zeta, 4 * nR); take(&t->Dp2, 4 * nR);
  take(&t->Ta, 2 * nR); take(&t->Tz, 2 * nR);
  take(&t->PsiT1, 2 * Ro2n); take(&t->PsiT2, 2 * Ro2n); take(&t->Ah, 2 * Ro2n);
  take(&t->SNN, 2 * nn); take(&t->SNI, 2 * nR); take(&t->SON, 2 * Ro * n);
  take(&t->PYn, n * L4); take(&t->PYi, R * L4);
  take(&t->QNN, 2 * n * L4); take(&t->QNI, 2 * n * L4); take(&t->QON, 2 * Ro * L4);
  take(&t->QOI, Ro * L4);
  for (int q = 0; q < 6; ++q) take(&t->mix[q], L * P);
  return off;
}

}  // namespace

extern "C" {

const char* vrte_status_string(vrte_status st) {
  switch (st) {
    case VRTE_OK: return "ok";
    case VRTE_ERR_INVALID_ARG: return "invalid argument";
    case VRTE_ERR_STATE: return "call order violated";
    case VRTE_ERR_CUDA: return "CUDA runtime error";
    case VRTE_ERR_OOM: return "device allocation failed";
    case VRTE_ERR_NO_CONVERGENCE: return "eigen iteration did not converge";
    case VRTE_ERR_SINGULAR: return "singular pivot";
    case VRTE_ERR_NONFINITE: return "non-finite value";
    case VRTE_ERR_UNSUPPORTED: return "unsupported request";
  }
  return "unknown status";
}

static int device_sm_count() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        sms < 1)
      sms = 1;
  }
  return sms;
}

// Mirror pairs of the azimuth grid for the tensor-core synthesis: the cosine class of the
// table is even in the azimuth difference and the sine class odd (Eqs. 7, 12), so the table at
// -phi follows from the one at phi. Returns [rep (n_phi) | mirror (n_phi)] with the computed
// azimuths rep[0 .. n_rep) in increasing order and mirror[r] the index of the azimuth at
// -phi_rep[r] (mod 2 pi, within 1e-12 rad), or -1 when it is not on the grid, is rep[r]
// itself (0, pi) or was already paired.
static std::vector<int> azimuth_mirrors(int n, const double* phi, int* n_rep) {
  const double two_pi = 6.283185307179586476925286766559;
  auto wrap = [&](double a) {
    a = std::fmod(a, two_pi);
    if (a < 0.0) a += two_pi;
    return a;
  };
  std::vector<std::pair<double, int>> key(n);
  for (int j = 0; j < n; ++j) key[j] = {wrap(phi[j]), j};
  std::sort(key.begin(), key.end());
  // the indices whose wrapped angle lies within 1e-12 of a (also across 0 = 2 pi)
  auto candidates = [&](double a, std::vector<int>& out) {
    out.clear();
    for (double c : {a, a - two_pi, a + two_pi}) {
      auto it = std::lower_bound(key.begin(), key.end(), std::make_pair(c - 1e-12, -1));
      for (; it != key.end() && it->first <= c + 1e-12; ++it) out.push_back(it->second);
    }
  };
  std::vector<int> map(2 * (size_t)n, -1), used(n, 0), cand;
  int r = 0;
  for (int j = 0; j < n; ++j) {
    if (used[j]) continue;
    used[j] = 1;
    int m = -1;
    candidates(wrap(-phi[j]), cand);
    for (int c : cand)
      if (!used[c]) {
        m = c;
        break;
      }
    if (m >= 0) used[m] = 1;
    map[r] = j;
    map[n + r] = m;
    ++r;
  }
  *n_rep = r;
  return map;
}

vrte_status vrte_azimuth_mirrors(int n_phi, const double* phi, int* map_out, int* n_rep_out) {
  if (n_phi < 1 || !phi || !map_out || !n_rep_out) return VRTE_ERR_INVALID_ARG;
  for (int j = 0; j < n_phi; ++j)
    if (!std::isfinite(phi[j])) return VRTE_ERR_INVALID_ARG;
  std::vector<int> map = azimuth_mirrors(n_phi, phi, n_rep_out);
  std::copy(map.begin(), map.end(), map_out);
  return VRTE_OK;
}

vrte_status vrte_plan_create(const vrte_plan_desc* d, vrte_plan** out) {
  if (!d || !out) return VRTE_ERR_INVALID_ARG;
  *out = nullptr;
  // size limits keep every launch inside the grid and shared-memory limits
  if (d->n_nodes_max < 1 || d->n_nodes_max > 96 || d->n_orders_max < 1 ||
      d->n_orders_max > 1024 || d->n_coef_max < 1 || d->n_coef_max > 1024 ||
      d->n_layers_max < 1 || d->n_mu_in < 1 || d->n_mu_in > 16384 || d->n_mu_out < 1 ||
      d->n_mu_out > 16384 || d->n_phi < 1 || !d->mu_in || !d->mu_out || !d->phi ||
      (d->flags & ~(VRTE_FLAG_PROFILE | VRTE_FLAG_ADJOINT | VRTE_FLAG_TRANSMISSION |
                    VRTE_FLAG_SLAB)) != 0)
    return VRTE_ERR_INVALID_ARG;
  if (d->precision != VRTE_FP64 && d->precision != VRTE_MIXED) return VRTE_ERR_INVALID_ARG;
  for (int i = 0; i < d->n_mu_in; ++i)
    if (!(d->mu_in[i] > 0.0 && d->mu_in[i] <= 1.0)) return VRTE_ERR_INVALID_ARG;
  for (int i = 0; i < d->n_mu_out; ++i)
    if (!(d->mu_out[i] > 0.0 && d->mu_out[i] <= 1.0)) return VRTE_ERR_INVALID_ARG;
  for (int i = 0; i < d->n_phi; ++i)
    if (!(d->phi[i] == d->phi[i])) return VRTE_ERR_INVALID_ARG;
  vrte_plan* p = new vrte_plan();
  p->desc = *d;
  p->desc.mu_in = p->desc.mu_out = p->desc.phi = nullptr;
  p->n_in = d->n_mu_in;
  p->n_out = d->n_mu_out;
  p->n_phi = d->n_phi;
  p->profile = (d->flags & VRTE_FLAG_PROFILE) != 0;
  reset_stats(p);
  vrte_status st = VRTE_OK;
  int Mx = d->n_orders_max;
  if ((st = allocd(p, &p->d_mu_in, p->n_in)) || (st = allocd(p, &p->d_mu_out, p->n_out)) ||
      (st = allocd(p, &p->d_phi, p->n_phi)) || (st = allocd(p, &p->d_wc, (size_t)Mx * p->n_phi)) ||
      (st = allocd(p, &p->d_ws, (size_t)Mx * p->n_phi)) || (st = allocd(p, &p->d_status, 1)) ||
      (st = allocd(p, &p->d_syn_map, 2 * (size_t)p->n_phi))) {
    vrte_destroy(p);
    return st;
  }
  if (cudaMemcpy(p->d_mu_in, d->mu_in, p->n_in * sizeof(double), cudaMemcpyHostToDevice) ||
      cudaMemcpy(p->d_mu_out, d->mu_out, p->n_out * sizeof(double), cudaMemcpyHostToDevice) ||
      cudaMemcpy(p->d_phi, d->phi, p->n_phi * sizeof(double), cudaMemcpyHostToDevice) ||
      cudaMemset(p->d_status, 0, sizeof(unsigned))) {
    vrte_destroy(p);
    return VRTE_ERR_CUDA;
  }
  {
    std::vector<int> map = azimuth_mirrors(p->n_phi, d->phi, &p->n_rep);
    if (cudaMemcpy(p->d_syn_map, map.data(), map.size() * sizeof(int), cudaMemcpyHostToDevice)) {
      vrte_destroy(p);
      return VRTE_ERR_CUDA;
    }
  }
  launch_trig_table(Mx, p->n_phi, p->d_phi, p->d_wc, p->d_ws, 0);
  if (cudaDeviceSynchronize() != cudaSuccess) {
    vrte_destroy(p);
    return VRTE_ERR_CUDA;
  }
  *out = p;
  return VRTE_OK;
}

// A reflecting base's matrix: finite, no (I, Q) x (U, V) coupling (order 0 cannot carry one),
// and a total R_00 (with the Lambertian 2 rho) in [0, 2] (the bare base reflects at most the
// unpolarized flux it receives).
static bool base_valid(const vrte_layer& l) {
  BaseR b;
  layer_base(l, &b);
  for (int i = 0; i < 16; ++i) {
    if (!std::isfinite(b.r[i])) return false;
    const int r = i / 4, c = i % 4;
    if ((r < 2) != (c < 2) && b.r[i] != 0.0) return false;
  }
  return b.r[0] >= 0.0 && b.r[0] <= 2.0;
}

vrte_status vrte_set_layer(vrte_plan* p, int n_layers, const vrte_layer* hp, const double* d_coeffs) {
  if (!p || !hp || !d_coeffs || n_layers < 1 || n_layers > p->desc.n_layers_max)
    return VRTE_ERR_INVALID_ARG;
  for (int b = 0; b < n_layers; ++b) {
    const vrte_layer& l = hp[b];
    if (!(l.tau > 0.0) || !(l.omega >= 0.0 && l.omega < 1.0) || !(l.n_interface <= 3.0) ||
        !(l.base_albedo >= 0.0 && l.base_albedo <= 1.0) || !base_valid(l) ||
        l.n_nodes < 1 || l.n_nodes > p->desc.n_nodes_max || l.n_orders < 1 ||
        l.n_orders > p->desc.n_orders_max || l.n_coef < 1 || l.n_coef > p->desc.n_coef_max)
      return VRTE_ERR_INVALID_ARG;
    // the mixed form contracts over the 4L (l, component) pairs with the sliced
    // tensor-core GEMM, whose exact accumulation holds for K <= 1024
    if (p->desc.precision == VRTE_MIXED && 4 * l.n_coef > 1024) return VRTE_ERR_UNSUPPORTED;
  }
  cudaDeviceSynchronize();
  free_workspace(p, kPlanAllocs);
  for (Work& x : p->ws) {
    cudaStream_t st_ = x.stream, sd_ = x.side;
    cudaEvent_t ev_ = x.done, er_ = x.ready, ef_ = x.freed, sf_ = x.side_fork, sj_ = x.side_join;
    x = Work();
    x.stream = st_;
    x.side = sd_;
    x.side_fork = sf_;
    x.side_join = sj_;
    x.done = ev_;
    x.ready = er_;
    x.freed = ef_;
  }
  p->last_U = 0;
  p->layers.assign(hp, hp + n_layers);
  p->n_layers = n_layers;
  p->d_coeffs = d_coeffs;
  int Nx = 0, Lx = 0, Mx = 0;
  for (auto& l : p->layers) {
    Nx = std::max(Nx, l.n_nodes);
    Lx = std::max(Lx, l.n_coef);
    Mx = std::max(Mx, std::min(l.n_orders, l.n_coef));
  }
  size_t n = 4 * (size_t)Nx, R = 4 * (size_t)p->n_in, Ro = 4 * (size_t)p->n_out;
  size_t P = Nx + p->n_in + p->n_out;
  const bool mixed = p->desc.precision == VRTE_MIXED;
  p->kdir = mixed ? 4 * Lx : 0;
  size_t kd = p->kdir;
  const int S = kSlices;
  size_t tc_unit = 0, tc_side_unit = 0;
  const bool adjoint_tc = (p->desc.flags & VRTE_FLAG_ADJOINT) != 0;
  if (adjoint_tc) {
    // the adjoint's contractions (op(A) op(B): the workspace depends on M, N, K only)
    const int nn2 = (int)(2 * n), ni = (int)n, Ri = (int)R, Roi = (int)Ro;
    const int sh[9][3] = {{Roi, Ri, nn2}, {nn2, Ri, Roi}, {Roi, nn2, Ri}, {nn2, Ri, nn2},
                          {nn2, nn2, Ri}, {Roi, ni, ni}, {ni, Ri, ni}, {ni, ni, ni},
                          {nn2, nn2, Roi}};
    for (const auto& q : sh)
      if (tc_shape_ok(q[2], S))
        tc_unit = std::max(tc_unit, tc_workspace_bytes(q[0], q[1], q[2], 1, S) - tc_scratch_bytes());
  }
  if (mixed) {
    size_t c[9] = {tc_workspace_bytes((int)(2 * n), (int)(2 * n), (int)(2 * n), 1, S),
                   tc_workspace_bytes((int)n, (int)R, (int)n, 1, S),
                   tc_workspace_bytes((int)n, (int)n, (int)n, 1, S),
                   tc_workspace_bytes((int)n, (int)R, (int)kd, 1, S),
                   tc_workspace_bytes((int)Ro, (int)(2 * n), (int)kd, 1, S),
                   tc_workspace_bytes((int)Ro, (int)n, (int)n, 1, S),
                   tc_workspace_bytes((int)(2 * n), (int)R, (int)(2 * n), 1, S),
                   tc_workspace_bytes((int)Ro, (int)R, (int)(2 * n), 1, S),
                   tc_workspace_bytes((int)Ro, (int)R, (int)(2 * n + kd), 1, S)};
    for (size_t v : c) tc_unit = std::max(tc_unit, v - tc_scratch_bytes());
    size_t cs[3] = {tc_workspace_bytes((int)n, (int)R, (int)kd, 1, S),
                    tc_workspace_bytes((int)n, (int)R, (int)n, 1, S),
                    tc_workspace_bytes((int)Ro, (int)(2 * n), (int)kd, 1, S)};
    for (size_t v : cs) tc_side_unit = std::max(tc_side_unit, v - tc_scratch_bytes());
  }
  size_t per_unit = 3 * (size_t)Lx * P + 10 * n * n + 3 * n + 8 * n * n + 5 * n * R +
                    (4 * n + kd) * R + 2 * n * R + 4 * Ro * n + Ro * (2 * n + kd) + Ro * R + n * n +
                    1 + 5 * 4 * n * n + 3 * 2 * n + 1 + (tc_unit + 7) / 8 +
                    (mixed ? refine_scratch_doubles(1, p->n_in, p->n_out) + p->n_in : 0) +
                    (mixed ? 7 * n * n + 3 : 0) +  // Newton inverse scratch and residuals
                    (tc_side_unit + 7) / 8 +         // GEMM workspace of the side stream
                    n * kd + kd * 2 * n + 2 * kd * R;
  const bool adjoint = (p->desc.flags & VRTE_FLAG_ADJOINT) != 0;
  if (adjoint) per_unit += bw_carve(nullptr, 1, n, R, Ro, Lx, P, nullptr);
  const bool transmission = (p->desc.flags & VRTE_FLAG_TRANSMISSION) != 0;
  if (transmission) per_unit += 4 * Ro * R;
  const bool slab = (p->desc.flags & VRTE_FLAG_SLAB) != 0;
  const size_t S_sub = (size_t)n_layers;
  // a slab's elimination buffers, once per plan (slot 0): per sub-layer and order D'^-1, y,
  // Uup, Hhat; shared Ldn x 2, Pd x 2, Zt, Ldn W, a contraction, the top radiance, Uup c
  const size_t slab_unit =
      slab ? S_sub * (4 * n * n + 2 * n * R + 2 * n * n + Ro * 2 * n) + 2 * 2 * n * n +
                 2 * n * R + n * R + n * n + 2 * Ro * R + n * R
           : 0;
  size_t isyn = (size_t)Mx * p->n_in * p->n_out * 16;
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  // Several layers run in up to kMaxSlots concurrent slots, each with its own order
  // radiances and workspace, as long as every slot still takes all of a layer's orders in
  // one batch. The order radiances must fit; the per-order workspace takes at most 35% of
  // what is left (capped at 96 GiB) so that the caller's output table still fits beside it.
  const size_t fixed_slot =
      ((transmission ? 2 : 1) * isyn + (size_t)p->n_in * p->n_out) * sizeof(double);
  int nslots = std::max(1, std::min(n_layers, kMaxSlots));
  size_t U = 0;
  for (;; --nslots) {
    size_t need_fixed = nslots * fixed_slot + ((size_t)64 << 20);
    if (need_fixed >= free_b) {
      if (nslots == 1) return VRTE_ERR_OOM;
      continue;
    }
    size_t budget = std::min((size_t)(0.35 * (double)(free_b - need_fixed)), (size_t)96 << 30);
    size_t units = budget / ((nslots * per_unit + slab_unit) * sizeof(double));
    units = std::max<size_t>(1, std::min<size_t>(units, (size_t)Mx));
    U = units;
    if (nslots == 1 || units == (size_t)Mx) break;
  }
  p->nslots = nslots;
  p->chunk = (int)U;
  vrte_status st = VRTE_OK;
  Work* w = nullptr;
#define VRTE_ALLOC(ptr, cnt)                        \
  if ((st = allocd(p, &w->ptr, (cnt))) != VRTE_OK) { \
    free_workspace(p, kPlanAllocs);                  \
    for (Work& x : p->ws) x.Isyn = nullptr;          \
    return st;                                       \
  }
  for (int slot = 0; slot < nslots; ++slot) {
  w = &p->ws[slot];
  VRTE_ALLOC(d_mu_nodes, Nx) VRTE_ALLOC(d_w_nodes, Nx) VRTE_ALLOC(d_pts, P) VRTE_ALLOC(d_min4, 4 * (size_t)p->n_in)
  VRTE_ALLOC(d_mout4, 4 * (size_t)p->n_out) VRTE_ALLOC(d_rtop4, 4 * (size_t)Nx)
  VRTE_ALLOC(gp, U * Lx * P) VRTE_ALLOC(gr, U * Lx * P) VRTE_ALLOC(gt, U * Lx * P)
  VRTE_ALLOC(E, U * n * n) VRTE_ALLOC(F, U * n * n) VRTE_ALLOC(FE, U * n * n) VRTE_ALLOC(X, U * n * n) VRTE_ALLOC(EX, U * n * n)
  VRTE_ALLOC(Y, U * n * n) VRTE_ALLOC(Xinv, U * n * n) VRTE_ALLOC(Hs, U * n * n) VRTE_ALLOC(Zs, U * n * n) VRTE_ALLOC(Vs, U * n * n)
  VRTE_ALLOC(lam_re, U * n) VRTE_ALLOC(lam_im, U * n) VRTE_ALLOC(bal, U * n)
  VRTE_ALLOC(K, U * 4 * n * n) VRTE_ALLOC(Kinv, U * 4 * n * n)
  VRTE_ALLOC(Pb, U * n * R) VRTE_ALLOC(Rb, U * n * R) VRTE_ALLOC(Wv, U * n * R) VRTE_ALLOC(Yv, U * n * R) VRTE_ALLOC(Es, U * n * R)
  VRTE_ALLOC(SD, U * (2 * n + kd) * R) VRTE_ALLOC(RHS, U * 2 * n * R) VRTE_ALLOC(C, U * 2 * n * R)
  VRTE_ALLOC(Upm, U * Ro * (2 * n + kd)) VRTE_ALLOC(P1, U * Ro * n) VRTE_ALLOC(P2, U * Ro * n) VRTE_ALLOC(Hhat, U * Ro * 2 * n)
  VRTE_ALLOC(T1, U * Ro * R) VRTE_ALLOC(g0tab, (size_t)p->n_in * p->n_out + 2 * (size_t)p->n_in)
  VRTE_ALLOC(FY, U * n * n) VRTE_ALLOC(mode_res, U) VRTE_ALLOC(mode_flag, U)
  VRTE_ALLOC(Bm, U * 4 * n * n) VRTE_ALLOC(Hb, U * 4 * n * n) VRTE_ALLOC(Zb, U * 4 * n * n)
  VRTE_ALLOC(Vb, U * 4 * n * n) VRTE_ALLOC(Xb, U * 4 * n * n)
  VRTE_ALLOC(kb_re, U * 2 * n) VRTE_ALLOC(kb_im, U * 2 * n) VRTE_ALLOC(balb, U * 2 * n)
  if (mixed) {
    VRTE_ALLOC(Ln, U * n * kd) VRTE_ALLOC(RU, U * kd * 2 * n)
    VRTE_ALLOC(Rbp, U * kd * R) VRTE_ALLOC(Rbm, U * kd * R)
  }
  if (!mixed && adjoint_tc) {
    p->tcw_bytes = tc_unit * U + tc_scratch_bytes();
    if ((st = alloc(p, &w->tcw, p->tcw_bytes)) != VRTE_OK) {
      free_workspace(p, kPlanAllocs);
      for (Work& x : p->ws) x.Isyn = nullptr;
      return st;
    }
  }
  if (mixed) {
    size_t synth = tc_synthesis_workspace(Mx, p->n_in, p->n_out, p->n_phi, kSynthBlock);
    p->tcw_bytes = std::max(tc_unit * U + tc_scratch_bytes(), synth);
    if ((st = alloc(p, &w->tcw, p->tcw_bytes)) != VRTE_OK ||
        (st = allocd(p, &w->rscratch, refine_scratch_doubles((int)U, p->n_in, p->n_out))) !=
            VRTE_OK ||
        (st = allocd(p, &w->rcount, 3)) != VRTE_OK ||
        (st = alloc(p, &w->nscratch, newton_inverse_scratch_bytes(2 * (int)n, (int)n, (int)U))) !=
            VRTE_OK ||
        (st = allocd(p, &w->nerr, 2 * U)) != VRTE_OK ||
        (nslots == 1 &&
         (st = alloc(p, &w->tcw_side, tc_side_unit * U + tc_scratch_bytes())) != VRTE_OK) ||
        (st = allocd(p, &w->rlist, U * p->n_in)) != VRTE_OK ||
        (st = allocd(p, &w->nfflag, U * p->n_in)) != VRTE_OK) {
      free_workspace(p, kPlanAllocs);
      for (Work& x : p->ws) x.Isyn = nullptr;
      return st;
    }
  }
  VRTE_ALLOC(Isyn, isyn)
  VRTE_ALLOC(basebuf, base_buffer_doubles(n, R))
  if (slab && slot == 0) {
    VRTE_ALLOC(sDinv, S_sub * U * 4 * n * n) VRTE_ALLOC(sY, S_sub * U * 2 * n * R)
    VRTE_ALLOC(sUup, S_sub * U * 2 * n * n) VRTE_ALLOC(sH, S_sub * U * Ro * 2 * n)
    VRTE_ALLOC(sL[0], U * 2 * n * n) VRTE_ALLOC(sL[1], U * 2 * n * n)
    VRTE_ALLOC(sPd[0], U * n * R) VRTE_ALLOC(sPd[1], U * n * R) VRTE_ALLOC(sZt, U * n * R)
    VRTE_ALLOC(sTnn, U * n * n) VRTE_ALLOC(sTq, U * Ro * R) VRTE_ALLOC(sAcc, U * Ro * R)
    VRTE_ALLOC(sV, U * n * R)
  }
  if (transmission) {
    VRTE_ALLOC(Qp, U * Ro * R) VRTE_ALLOC(Qb, U * Ro * R) VRTE_ALLOC(Tbot, U * Ro * R)
    VRTE_ALLOC(Tup, U * Ro * R) VRTE_ALLOC(rout4, 4 * (size_t)p->n_out) VRTE_ALLOC(Isyn2, isyn)
  }
  if (adjoint) {
    VRTE_ALLOC(bw, bw_carve(nullptr, U, n, R, Ro, Lx, P, nullptr))
    VRTE_ALLOC(dpts, P) VRTE_ALLOC(dmin4, 4 * (size_t)p->n_in) VRTE_ALLOC(dmout4, 4 * (size_t)p->n_out)
    VRTE_ALLOC(drtop4, 4 * (size_t)Nx) VRTE_ALLOC(acc, 3 + 6 * (size_t)p->desc.n_coef_max)
  }
  if (mixed && nslots == 1) {
    int least = 0, greatest = 0;
    cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if ((!w->side &&
         cudaStreamCreateWithPriority(&w->side, cudaStreamNonBlocking, least) != cudaSuccess) ||
        (!w->side_fork &&
         cudaEventCreateWithFlags(&w->side_fork, cudaEventDisableTiming) != cudaSuccess) ||
        (!w->side_join &&
         cudaEventCreateWithFlags(&w->side_join, cudaEventDisableTiming) != cudaSuccess))
      return VRTE_ERR_CUDA;
  }
  if (nslots > 1) {
    if (!w->stream && cudaStreamCreateWithFlags(&w->stream, cudaStreamNonBlocking) != cudaSuccess)
      return VRTE_ERR_CUDA;
    if (!w->done && cudaEventCreateWithFlags(&w->done, cudaEventDisableTiming) != cudaSuccess)
      return VRTE_ERR_CUDA;
    if (slab && ((!w->ready && cudaEventCreateWithFlags(&w->ready, cudaEventDisableTiming) !=
                                   cudaSuccess) ||
                 (!w->freed && cudaEventCreateWithFlags(&w->freed, cudaEventDisableTiming) !=
                                   cudaSuccess)))
      return VRTE_ERR_CUDA;
  }
  }
#undef VRTE_ALLOC
  if (nslots > 1 && !p->fork &&
      cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming) != cudaSuccess)
    return VRTE_ERR_CUDA;
  return VRTE_OK;
}

// One batch of U Fourier orders m0 .. m0+U-1 of layer `ly` through steps a0 (tables)
// to a7 on stream s: the plan's precision when `mixed` follows it, else the FP64 form.
// With `reconstruct` false the batch stops after the reconstruction operators (U+-, P1,
// P2, Hhat and, in the FP64 form, the direct term in T1): what the adjoint needs. With
// `boundary` false it also leaves out the layer's own boundary system (K, its inverse, the
// right-hand side and C): a slab solves one system for all of its sub-layers.
// The host-buffer solve's second workspace for a layer of n = 4N and U orders: the homogeneous
// contraction's slices (kept while the particular contraction's stay in the slot's workspace),
// then the synthesis workspace.
static size_t chunk_hom_bytes(const vrte_plan* p, int n, int U) {
  return (tc_workspace_bytes(4 * p->n_out, 4 * p->n_in, 2 * n, U, kSlices) + 1023) / 1024 * 1024;
}
static size_t chunk_ws_need(const vrte_plan* p, int n, int U) {
  return chunk_hom_bytes(p, n, U) +
         tc_synthesis_workspace(U, p->n_in, p->n_out, p->n_phi, kSynthBlock);
}

// Reconstruction and synthesis in blocks of incident cosines (host-buffer solve): the layer's
// table, its element type, the hook that starts the copy of each finished block, the second
// workspace; `done` is set when the batch has synthesized the table.
struct ChunkSynth {
  void* out;
  int out_dtype;
  const SynthHook* hook;
  void* ws;
  size_t ws_bytes;
  bool done;
};

static void run_order_batch(vrte_plan* p, Work* w, const vrte_layer& ly, const double* coef,
                          int m0, int U, bool mixed, bool reconstruct, cudaStream_t s,
                          bool boundary = true, ChunkSynth* cs = nullptr) {
  const int N = ly.n_nodes, n = 4 * N, L = ly.n_coef;
  const int P = N + p->n_in + p->n_out;
  const int R = 4 * p->n_in, Ro = 4 * p->n_out;
  const int Meff = std::min(ly.n_orders, ly.n_coef);
  // operator rows [U+ | U- | direct] and beams [s; d; direct] carry 4 L extra entries
  // in the mixed form, where the direct term rides on the particular contraction
  const int kdir = mixed ? 4 * L : 0;
  const int ldU = 2 * n + (mixed ? p->kdir : 0);
  OrderBatch ob{N, n, L, m0, U, p->n_in, p->n_out, P, ly.tau, ly.omega, coef, p->d_status,
                ldU, (long long)ldU * R};
  BaseR Rg;
  const bool has_base = layer_base(ly, &Rg);
  // the layer's beam table (e^{-tau0/mu0}, 1/mu0), written with its depth factors
  const double* btab = w->g0tab + (size_t)p->n_in * p->n_out;
  p->last_n = n;
  p->last_U = U;
  p->last_ldU = ldU;
  p->last_P = P;
  p->last_Meff = Meff;
  const long long nn = (long long)n * n, nR = (long long)n * R, Ron = (long long)Ro * n;
  const long long sU_part = (long long)Ro * ldU;
  const int gl = mixed ? 3 : 1;  // launches per contraction
  // BF16 FLOPs issued per FP64 multiply-add by the sliced product
  const double tcf = mixed ? 2.0 * kSlices * (kSlices + 1) / 2 : 0.0;
  // boundary solve and reconstruction contractions: FP64 on the CUDA cores, or the
  // sliced BF16 product on the tensor cores in the mixed form
  auto gemm = [&](int M_, int N_, int K_, const double* A_, int lda_, long long sA_,
                  const double* B_, int ldb_, long long sB_, double beta_, double* C_,
                  int ldc_, long long sC_, TcKSkip z_ = TcKSkip{}) {
    if (mixed)
      tc_gemm_store(M_, N_, K_, A_, lda_, sA_, B_, ldb_, sB_, beta_, C_, ldc_, sC_, U,
                    kSlices, w->tcw, p->d_status, s, z_);
    else
      dgemm_batched(M_, N_, K_, 1.0, A_, lda_, sA_, B_, ldb_, sB_, beta_, C_, ldc_, sC_, U,
                    s);
  };
  const double dn = n, dR = R, dRo = Ro, dU = U;
  double lsum = 0.0;  // sum over the batch of (L - m)
  for (int u = 0; u < U; ++u) lsum += std::max(0, L - (m0 + u));
  // the (l, component) contractions of order m0 + u have no terms with l < m0 + u: K
  // [4 (m0 + u), 4 L) of the direct operators and beams, skipped block-wise by the sliced
  // product; kdsum = their summed depth over the batch (the algorithmic work)
  const TcKSkip zdir{0, 4 * m0, 4};
  const TcKSkip zpart{2 * n, 4 * m0, 4};
  const double kdsum = 4.0 * lsum;
  // One layer in flight (mixed form): the eigen-decomposition holds one SM per order, and
  // the operators and beams that do not depend on it run meanwhile on the SMs it leaves
  // idle, on the slot's side stream (least priority; GEMMs capped at the idle SM count).
  const int idle_sms = device_sm_count() - U;
  const bool overlap = mixed && reconstruct && boundary && w->side && p->nslots == 1 &&
                       idle_sms >= kSideMinSMs;
  {
    StageScope sc(p, ST_TABLES, s, 1, 30.0 * P * lsum, 24.0 * P * lsum);
    launch_gsf_tables(ob, w->d_pts, w->gp, w->gr, w->gt, s);
  }
  {
    StageScope sc(p, ST_ASSEMBLE, s, 2, 72.0 * N * N * lsum + 2.0 * dn * dn * dn * dU,
                  8.0 * 3 * dn * dn * dU);
    launch_assemble_EF(ob, w->gp, w->gr, w->gt, w->d_mu_nodes, w->d_w_nodes, w->E, w->F, s);
    dgemm_batched(n, n, n, 1.0, w->F, n, nn, w->E, n, nn, 0.0, w->FE, n, nn, U, s);
  }
  if (overlap) {
    const cudaStream_t ss = w->side;
    cudaEventRecord(w->side_fork, s);
    cudaStreamWaitEvent(ss, w->side_fork, 0);
    auto gemm_side = [&](int M_, int N_, int K_, const double* A_, int lda_, long long sA_,
                         const double* B_, int ldb_, long long sB_, double* C_, int ldc_,
                         long long sC_, TcKSkip z_) {
      tc_gemm_store(M_, N_, K_, A_, lda_, sA_, B_, ldb_, sB_, 0.0, C_, ldc_, sC_, U, kSlices,
                    w->tcw_side, p->d_status, ss, z_, idle_sms);
    };
    StageScope sc(p, ST_SIDE_OPS, ss, 3 + 3 * gl + 1 + 2 + gl,
                  72.0 * N * p->n_in * lsum + 2.0 * dn * dn * dR * dU +
                      72.0 * N * p->n_out * lsum + 72.0 * p->n_in * p->n_out * lsum,
                  8.0 * (4 * dn * dR + 2 * dRo * dn + dRo * dR) * dU);
    sc.tensor_flops(tcf * (dn * dU + 2.0 * kdsum) * dn * dR + tcf * 2.0 * dRo * dn * kdsum);
    // beam vectors (Eq. 47) as contractions over (l, component), F'p - r / mu0 (Eq. 46)
    launch_mixed_operators(ob, w->gp, w->gr, w->gt, w->d_mu_nodes, w->d_w_nodes, w->d_min4,
                           w->Ln, w->RU, w->Rbp, w->Rbm, ss);
    const long long sL = (long long)n * kdir, sB = (long long)kdir * R;
    gemm_side(n, R, kdir, w->Ln, kdir, sL, w->Rbp, R, sB, w->Pb, R, nR, zdir);
    gemm_side(n, R, kdir, w->Ln, kdir, sL, w->Rbm, R, sB, w->Rb, R, nR, zdir);
    gemm_side(n, R, n, w->F, n, nn, w->Pb, R, nR, w->Wv, R, nR, TcKSkip{});
    launch_particular_rhs(ob, w->Wv, w->Rb, btab, w->Wv, ss);
    // the direct operators and U+- = [M_out P(mu_o) B] x RU+- (reconstruction, Eq. 38)
    launch_direct_operators(ob, w->gp, w->gr, w->gt, w->d_min4, w->d_mout4, w->Upm, w->SD, ss);
    gemm_side(Ro, 2 * n, kdir, w->Upm + 2 * n, ldU, sU_part, w->RU, 2 * n,
              (long long)kdir * 2 * n, w->Upm, ldU, sU_part, zdir);
    cudaEventRecord(w->side_join, ss);
  }
  {
    // algorithmic work counted: the nominal 25 n^3 of a real Schur decomposition with
    // eigenvectors, the stage's dominant kernel. E'X, Y = E'X / kappa and the mode
    // residual F'Y - X kappa (4 n^3 more; on the tensor cores in the mixed form) are
    // not counted, so the stage's FP64 rate is that of the eigen-decomposition.
    StageScope sc(p, ST_EIGEN, s, mixed ? 10 + 2 * (gl - 1) : 10, 25.0 * dn * dn * dn * dU,
                  8.0 * 6 * dn * dn * dU);
    batched_eigen(n, w->FE, w->Hs, w->Zs, w->Vs, w->X, w->lam_re, w->lam_im, w->bal, U,
                  p->d_status, s);
    gemm(n, n, n, w->E, n, nn, w->X, n, nn, 0.0, w->EX, n, nn);
    launch_pack_Y(ob, w->EX, w->lam_re, w->lam_im, w->Y, s);
    gemm(n, n, n, w->F, n, nn, w->Y, n, nn, 0.0, w->FY, n, nn);
    // the FP64 form re-solves order 0 (diffusion mode) and any order with a poor mode
    // residual in the 2n block form; the mixed form only catastrophic ones
    const bool fp64 = p->desc.precision == VRTE_FP64;
    eigen_block_fallback(n, m0, w->E, w->F, w->FY, w->X, w->Y, w->lam_re, w->lam_im,
                         fp64 ? 1e-4 : 1e-1, fp64 ? 1 : 0, w->mode_res, w->mode_flag, w->Bm,
                         w->Hb, w->Zb, w->Vb, w->Xb, w->kb_re, w->kb_im, w->balb, U,
                         p->d_status, s);
  }
  {
    // algorithmic work: the inverses' nominal 2 m^3 each (K: m = 2n, X: m = n); the mixed
    // form does it as an FP32 elimination and Newton-Schulz products on the tensor cores
    // (2 per step and one residual check, each m^3 multiply-adds)
    StageScope sc(p, ST_MODES, s, boundary ? 3 : 1,
                  (boundary ? 18.0 : 2.0) * dn * dn * dn * dU,
                  8.0 * (boundary ? 12 : 2) * dn * dn * dU);
    if (mixed)
      sc.tensor_flops(tcf * (2 * kNewtonSteps + 1) * (boundary ? 9.0 : 1.0) * dn * dn * dn * dU);
    if (boundary) {
      launch_build_K(ob, w->X, w->Y, w->lam_re, w->lam_im, w->d_rtop4, w->K, s);
      if (has_base && m0 == 0)
        launch_base_K(N, n, ly.tau, Rg, w->X, w->Y, w->lam_re, w->lam_im,
                      w->d_mu_nodes, w->d_w_nodes, w->K, w->basebuf, s);
      if (!mixed) batched_inverse(2 * n, w->K, w->Kinv, U, p->d_status, s);
    }
    if (mixed)  // K^-1 (with the boundary system) and X^-1, the eliminations in one launch
      newton_inverse(boundary ? 2 * n : n, boundary ? w->K : w->X, boundary ? w->Kinv : w->Xinv,
                     boundary ? n : 0, w->X, w->Xinv, U, kNewtonSteps, kNewtonTol, w->nscratch,
                     w->nerr, w->rcount + 2, w->tcw, kSlices, p->d_status, s);
    else
      batched_inverse(n, w->X, w->Xinv, U, p->d_status, s);
  }
  {
    StageScope sc(p, ST_PARTICULAR, s,
                  (overlap ? 4 + 3 * gl : (mixed ? 7 + 6 * gl : 9)) - (boundary ? 0 : 1),
                  (overlap ? 0.0 : 72.0 * N * p->n_in * lsum + 2.0 * dn * dn * dR * dU) +
                      6.0 * dn * dn * dR * dU,
                  8.0 * 10 * dn * dR * dU);
    sc.tensor_flops(overlap ? tcf * 3.0 * dn * dU * dn * dR
                            : tcf * (4.0 * dn * dU + 2.0 * kdsum) * dn * dR);
    if (overlap) {
      cudaStreamWaitEvent(s, w->side_join, 0);  // beams, F'p - r / mu0, U+- from the side
    } else {
      if (mixed) {
        // beam vectors as contractions over (l, component) on the tensor cores
        launch_mixed_operators(ob, w->gp, w->gr, w->gt, w->d_mu_nodes, w->d_w_nodes,
                               w->d_min4, w->Ln, w->RU, w->Rbp, w->Rbm, s);
        const long long sL = (long long)n * kdir, sB = (long long)kdir * R;
        gemm(n, R, kdir, w->Ln, kdir, sL, w->Rbp, R, sB, 0.0, w->Pb, R, nR, zdir);
        gemm(n, R, kdir, w->Ln, kdir, sL, w->Rbm, R, sB, 0.0, w->Rb, R, nR, zdir);
      } else {
        launch_assemble_beam(ob, w->gp, w->gr, w->gt, w->d_mu_nodes, w->d_min4, w->Pb, w->Rb,
                             s);
      }
      gemm(n, R, n, w->F, n, nn, w->Pb, R, nR, 0.0, w->Wv, R, nR);
      launch_particular_rhs(ob, w->Wv, w->Rb, btab, w->Wv, s);
    }
    // near a resonance mu0 ~ 1/kappa_j the eigenbasis solve amplifies rounding by
    // 1/(kappa_j^2 - mu0^-2) and the homogeneous part cancels it: the mixed form
    // keeps FP64-level products here (7 slices, ~2e-15 per term)
    gemm(n, R, n, w->Xinv, n, nn, w->Wv, R, nR, 0.0, w->Yv, R, nR);
    launch_eigen_scale(ob, w->lam_re, w->lam_im, btab, w->Yv, s);
    gemm(n, R, n, w->X, n, nn, w->Yv, R, nR, 0.0, w->SD, R, ob.sSD);
    gemm(n, R, n, w->E, n, nn, w->SD, R, ob.sSD, 0.0, w->Es, R, nR);
    launch_particular_sd(ob, w->Pb, w->Es, w->d_pts, w->SD, s);
    if (boundary) {
      launch_bc_rhs(ob, w->SD, nullptr, w->d_rtop4, btab, w->RHS, s);
      if (has_base && m0 == 0)
        launch_base_rhs(N, n, R, ob.sSD, ly.tau, Rg, w->SD, w->d_pts, w->d_min4,
                        w->d_mu_nodes, w->d_w_nodes, w->RHS, w->basebuf + 8 * n, 1, s);
    }
  }
  if (boundary) {
    StageScope sc(p, ST_BC_SOLVE, s, gl, 2.0 * 4 * dn * dn * dR * dU,
                  8.0 * (4 * dn * dn + 4 * dn * dR) * dU);
    sc.tensor_flops(tcf * 4.0 * dn * dn * dR * dU);
    gemm(2 * n, R, 2 * n, w->Kinv, 2 * n, 4 * nn, w->RHS, R, 2 * nR, 0.0, w->C, R, 2 * nR);
  }
  {
    StageScope sc(p, ST_RECON_OPS, s, overlap ? 1 + 2 * gl : (mixed ? 3 + 3 * gl : 5),
                  (overlap ? 0.0 : 72.0 * N * p->n_out * lsum + 72.0 * p->n_in * p->n_out * lsum) +
                      4.0 * dRo * dn * dn * dU,
                  8.0 * (6 * dRo * dn + dRo * dR) * dU);
    sc.tensor_flops(tcf * 2.0 * dRo * dn * (dn * dU + (overlap ? 0.0 : kdsum)));
    if (overlap) {
      // the direct operators and U+- came from the side stream (joined before the
      // particular stage)
    } else if (mixed) {
      // U+- = [M_out P(mu_o) B] x RU+-: the direct operator's columns are the left factor
      launch_direct_operators(ob, w->gp, w->gr, w->gt, w->d_min4, w->d_mout4, w->Upm, w->SD,
                              s);
      gemm(Ro, 2 * n, kdir, w->Upm + 2 * n, ldU, sU_part, w->RU, 2 * n,
           (long long)kdir * 2 * n, 0.0, w->Upm, ldU, sU_part, zdir);
    } else {
      launch_assemble_U(ob, w->gp, w->gr, w->gt, w->d_w_nodes, w->d_mout4, w->Upm, s);
    }
    gemm(Ro, n, n, w->Upm, ldU, sU_part, w->X, n, nn, 0.0, w->P1, n, Ron);
    gemm(Ro, n, n, w->Upm + n, ldU, sU_part, w->Y, n, nn, 0.0, w->P2, n, Ron);
    launch_build_Hhat(ob, w->P1, w->P2, w->lam_re, w->lam_im, w->d_pts, w->Hhat, s);
    if (!mixed)
      launch_assemble_direct(ob, w->gp, w->gr, w->gt, w->d_pts, w->d_min4, w->d_mout4, w->T1,
                             s);
  }
  if (!reconstruct) return;
  const bool chunked = cs && cs->ws && mixed && boundary && m0 == 0 && U == Meff && !has_base &&
                       2 * n + kdir <= 1024 && cs->ws_bytes >= chunk_ws_need(p, n, U);
  if (chunked) {
    // The reconstruction, its FP64 column fixes and the synthesis per block of kSynthBlock
    // incident cosines, so that each block's table rows leave for the host while the next
    // block is computed. Both contractions are sliced once (the homogeneous one into the second
    // workspace) and then run on the column tiles of each block; the operand maxima of the
    // error bound are taken once.
    static_assert(kSynthBlock % (kTcTileCols / 4) == 0, "blocks start on a column tile");
    const int Kp = 2 * n + kdir;
    void* hom_ws = cs->ws;
    void* syn_ws = (char*)cs->ws + chunk_hom_bytes(p, n, U);
    const long long RoR = (long long)Ro * R;
    const double kpsum = 2.0 * dn * dU + kdsum;
    {
      StageScope sc(p, ST_RECON_HOM, s, 2, 0.0, 8.0 * (dRo * 2 * dn + 2 * dn * dR) * dU);
      tc_gemm_store(Ro, R, 2 * n, w->Hhat, 2 * n, 2 * Ron, w->C, R, 2 * nR, 0.0, w->T1, R, RoR,
                    U, kSlices, hom_ws, p->d_status, s, TcKSkip{}, 0, TcRange{true, false});
    }
    {
      StageScope sc(p, ST_RECON_PART, s, 2, 0.0, 8.0 * ((double)Kp * (dRo + dR)) * dU);
      cudaMemsetAsync(w->nfflag, 0, (size_t)U * p->n_in * sizeof(int), s);
      tc_gemm_part(ob, Kp, w->Upm, ldU, sU_part, w->SD, ob.sSD, w->T1, w->g0tab, w->Isyn,
                   kSlices, w->tcw, s, zpart, w->nfflag, TcRange{true, false});
    }
    {
      StageScope sc(p, ST_REFINE, s, 4, 0.0, 0.0);
      refine_maxima(ob, Kp, w->C, w->Hhat, w->Upm, w->SD, w->rscratch, s);
    }
    const double table = (double)p->n_in * p->n_out * p->n_phi * 16;
    const double esz = cs->out_dtype == VRTE_OUT_F64 ? 8.0 : 4.0;
    for (int k0 = 0; k0 < p->n_in; k0 += kSynthBlock) {
      const int k1 = std::min(p->n_in, k0 + kSynthBlock);
      const double f = double(k1 - k0) / p->n_in;  // the block's share of the work
      const TcRange run{false, true, 4 * k0 / kTcTileCols,
                        (4 * (k1 - k0) + kTcTileCols - 1) / kTcTileCols};
      {
        StageScope sc(p, ST_RECON_HOM, s, 1, f * 2.0 * dRo * dR * 2 * dn * dU,
                      f * 8.0 * 2 * dRo * dR * dU);
        sc.tensor_flops(f * tcf * dRo * dR * 2.0 * dn * dU);
        tc_gemm_store(Ro, R, 2 * n, w->Hhat, 2 * n, 2 * Ron, w->C, R, 2 * nR, 0.0, w->T1, R,
                      RoR, U, kSlices, hom_ws, p->d_status, s, TcKSkip{}, 0, run);
      }
      {
        StageScope sc(p, ST_RECON_PART, s, 1, f * 2.0 * dRo * dR * kpsum,
                      f * 8.0 * 2 * dRo * dR * dU);
        sc.tensor_flops(f * tcf * dRo * dR * kpsum);
        tc_gemm_part(ob, Kp, w->Upm, ldU, sU_part, w->SD, ob.sSD, w->T1, w->g0tab, w->Isyn,
                     kSlices, w->tcw, s, zpart, w->nfflag, run);
      }
      {
        StageScope sc(p, ST_REFINE, s, 4, 0.0, 0.0);
        refine_range(ob, Kp, w->Kinv, w->RHS, w->C, w->Hhat, w->Upm, w->SD, w->g0tab,
                     kSliceEps, kRefineTol, w->rscratch, w->rcount, w->rlist, U * p->n_in,
                     w->Isyn, w->nfflag, k0, k1, s);
      }
      {
        StageScope sc(p, ST_SYNTHESIS, s, (k0 == 0 ? 1 : 0) + 2, f * 2.0 * table * Meff,
                      f * (table * esz + (double)Meff * p->n_in * p->n_out * 16 * 8));
        const int Ss = kSlicesSynth;
        sc.tensor_flops(f * 2.0 * Ss * (Ss + 1) / 2 * 16.0 * p->n_in * p->n_out * p->n_rep *
                        Meff);
        tc_synthesis(Meff, p->n_in, p->n_out, p->n_phi, p->n_rep, p->d_syn_map, w->Isyn,
                     p->d_wc, p->d_ws, cs->out, cs->out_dtype, kSynthBlock, syn_ws,
                     p->d_status, s, cs->hook, k0, k1, k0 == 0);
      }
    }
    cs->done = true;
    return;
  }
  {
    // homogeneous part: [4 n_out x 2n] x [2n x 4 n_in] per order. FP64: T1 holds the
    // direct term and gains the homogeneous part; mixed: T1 is the homogeneous part and
    // the direct term is the tail of the particular contraction
    StageScope sc(p, ST_RECON_HOM, s, gl, 2.0 * dRo * dR * 2 * dn * dU,
                  8.0 * (dRo * 2 * dn + 2 * dn * dR + 2 * dRo * dR) * dU);
    sc.tensor_flops(tcf * dRo * dR * 2.0 * dn * dU);
    gemm(Ro, R, 2 * n, w->Hhat, 2 * n, 2 * Ron, w->C, R, 2 * nR, mixed ? 0.0 : 1.0, w->T1, R,
         (long long)Ro * R);
  }
  {
    // particular (+ direct, mixed) part with the depth factor, into I^m
    // summed contraction depth over the batch: 2n per order plus, mixed, the direct term's
    // 4 (L - m)
    const double kpsum = 2.0 * dn * dU + (mixed ? kdsum : 0.0);
    const double kp = 2.0 * dn + kdir;
    StageScope sc(p, ST_RECON_PART, s, mixed ? (2 * n + kdir <= 1024 ? 1 : 2) * gl : 1,
                  2.0 * dRo * dR * kpsum, 8.0 * (dRo * kp + kp * dR + 2 * dRo * dR) * dU);
    sc.tensor_flops(tcf * dRo * dR * kpsum);
    if (mixed) {
      cudaMemsetAsync(w->nfflag, 0, (size_t)U * p->n_in * sizeof(int), s);
      if (2 * n + kdir <= 1024) {
        tc_gemm_part(ob, 2 * n + kdir, w->Upm, ldU, sU_part, w->SD, ob.sSD, w->T1,
                     w->g0tab, w->Isyn, kSlices, w->tcw, s, zpart, w->nfflag);
      } else {
        // too deep for one exact accumulation: [U+ U-][s; d] into T1, then the direct part
        tc_gemm_part_accum(ob, 2 * n, w->Upm, ldU, sU_part, w->SD, ob.sSD, w->T1, w->g0tab,
                           kSlices, w->tcw, s);
        tc_gemm_part(ob, kdir, w->Upm + 2 * n, ldU, sU_part, w->SD + (size_t)2 * n * R,
                     ob.sSD, w->T1, w->g0tab, w->Isyn, kSlices, w->tcw, s, zdir, w->nfflag);
      }
    } else {
      dgemm_part_epilogue(ob, w->Upm, w->SD, w->T1, w->g0tab, w->Isyn, s);
    }
  }
  if (mixed) {
    StageScope sc(p, ST_REFINE, s, 8, 0.0, 0.0);
    refine_columns(ob, 2 * n + kdir, w->Kinv, w->RHS, w->C, w->Hhat, w->Upm, w->SD,
                   w->g0tab, kSliceEps, kRefineTol, w->rscratch, w->rcount, w->rlist,
                   U * p->n_in, w->Isyn, w->nfflag, s);
  }
  // reflecting base: its radiance at the bottom (the same in every upward direction),
  // attenuated to the top (order 0)
  if (has_base && m0 == 0)
    launch_base_recon(n, N, p->n_in, p->n_out, ly.tau, Rg, w->C, w->basebuf, w->d_pts,
                      w->d_mout4, w->Isyn, 1, s);
}

// Adjoint of one order batch (forward factors of the batch already in the slot's buffers,
// Ibar of the layer in w->Isyn): adds the batch's contributions to w->acc. Steps in the
// order of the header of k_adjoint.cu: reconstruction and boundary reverse, particular
// reverse, mode space, parameter chain.
static void backward_batch(vrte_plan* p, Work* w, const vrte_layer& ly, const double* coef,
                           int m0, int U, cudaStream_t s) {
  const int N = ly.n_nodes, n = 4 * N, L = ly.n_coef;
  const int P = N + p->n_in + p->n_out;
  const int R = 4 * p->n_in, Ro = 4 * p->n_out;
  OrderBatch ob{N, n, L, m0, U, p->n_in, p->n_out, P, ly.tau, ly.omega, coef, p->d_status,
                2 * n, 2LL * n * R};
  BwBufs b;
  bw_carve(w->bw, U, n, R, Ro, L, P, &b);
  const long long nn = (long long)n * n, nR = (long long)n * R, RoR = (long long)Ro * R,
                  Ro2n = (long long)Ro * 2 * n, L4 = 4LL * L;
  double* acc = w->acc;
  const double* pts = w->d_pts;
  const double* dpts = w->dpts;
  // the adjoint's contractions: sliced FP64-accurate products on the tensor cores (7 slices,
  // ~1e-15 relative per term, as the mixed form's) where the depth allows, else FP64
  auto gm = [&](bool tA, bool tB, int M_, int N_, int K_, double al, const double* A_, int lda,
                long long sA, const double* B_, int ldb, long long sB, double be, double* C_,
                int ldc, long long sC) {
    if (w->tcw && tc_shape_ok(K_, kSlices))
      tc_gemm_store_t(tA, tB, M_, N_, K_, al, A_, lda, sA, B_, ldb, sB, be, C_, ldc, sC, U,
                      kSlices, w->tcw, p->d_status, s);
    else
      dgemm_batched_t(tA, tB, M_, N_, K_, al, A_, lda, sA, B_, ldb, sB, be, C_, ldc, sC, U, s);
  };
  const double dU = U, dn = n, dR = R, dRo = Ro;
  StageScope sc(p, ST_ADJOINT, s, 120,
                2.0 * dU * (6 * dRo * dR * dn + 8 * dn * dn * dR + 24 * dn * dn * dR + 16 * dn * dn * dn),
                8.0 * dU * (6 * dRo * dR + 20 * dn * dR));
  // ---- reconstruction reverse
  bw_tb(ob, w->Isyn, w->g0tab, b.Tb, b.G0, s);
  gm(false, false, Ro, R, 2 * n, 1.0, w->Upm, 2 * n, Ro2n, w->SD, R, 2 * nR, 0.0, b.Qp, R, RoR);
  bw_g0(ob, b.Tb, b.Qp, w->T1, pts, dpts, acc, s);
  gm(true, false, 2 * n, R, Ro, 1.0, w->Hhat, 2 * n, Ro2n, b.Tb, R, RoR, 0.0, b.Cb, R, 2 * nR);
  gm(false, true, Ro, 2 * n, R, 1.0, b.Tb, R, RoR, w->C, R, 2 * nR, 0.0, b.Hb, 2 * n, Ro2n);
  gm(false, true, Ro, 2 * n, R, 1.0, b.G0, R, RoR, w->SD, R, 2 * nR, 0.0, b.Ub, 2 * n, Ro2n);
  gm(true, false, 2 * n, R, Ro, 1.0, w->Upm, 2 * n, Ro2n, b.G0, R, RoR, 0.0, b.SDb, R, 2 * nR);
  // ---- boundary system: nu = K^-T Cbar, Kbar = -nu C^T
  gm(true, false, 2 * n, R, 2 * n, 1.0, w->Kinv, 2 * n, 4 * nn, b.Cb, R, 2 * nR, 0.0, b.nu, R,
     2 * nR);
  gm(false, true, 2 * n, 2 * n, R, -1.0, b.nu, R, 2 * nR, w->C, R, 2 * nR, 0.0, b.Kb, 2 * n, 4 * nn);
  bw_kappa(ob, w->lam_re, w->lam_im, b.kap, s);
  bw_hhat(ob, b.Hb, w->P1, w->P2, b.kap, pts, dpts, b.P1b, b.P2b, acc, s);
  gm(false, true, Ro, n, n, 1.0, b.P1b, n, (long long)Ro * n, w->X, n, nn, 1.0, b.Ub, 2 * n, Ro2n);
  gm(false, true, Ro, n, n, 1.0, b.P2b, n, (long long)Ro * n, w->Y, n, nn, 1.0, b.Ub + n, 2 * n,
     Ro2n);
  bw_K(ob, b.Kb, w->X, w->Y, b.kap, w->d_rtop4, w->drtop4, acc, s);
  bw_rhs(ob, b.nu, w->SD, b.SDb, w->d_rtop4, w->drtop4, pts, dpts, acc, s);
  // ---- particular solution reverse (E', F', X, lambda fixed)
  bw_part_d(ob, w->SD, b.SDb, pts, dpts, b.pb, acc, s);
  gm(true, false, n, R, n, -1.0, w->E, n, nn, b.pb, R, nR, 1.0, b.SDb, R, 2 * nR);
  gm(true, false, n, R, n, 1.0, w->X, n, nn, b.SDb, R, 2 * nR, 0.0, b.ysb, R, nR);
  bw_scale(ob, w->lam_re, w->lam_im, w->Yv, b.ysb, pts, dpts, acc, s);
  gm(true, false, n, R, n, 1.0, w->Xinv, n, nn, b.ysb, R, nR, 0.0, b.wb, R, nR);
  gm(true, false, n, R, n, 1.0, w->F, n, nn, b.wb, R, nR, 1.0, b.pb, R, nR);
  bw_part_w(ob, b.wb, w->Rb, pts, dpts, b.rb, acc, s);
  // ---- mode space: dL/dF', dL/dE' through the adjoint two-point problem
  bw_cplx_cols(ob, w->X, w->Y, b.kap, w->d_rtop4, b.Xc, b.Yc, b.Pmc, b.Gtc, s);
  bw_cplx_rows(n, n, n, nn, w->Xinv, b.kap, b.Xic, U, s);
  gm(false, false, n, n, n, 1.0, b.Xic, n, 2 * nn, w->F, n, nn, 0.0, b.Zc, n, 2 * nn);
  gm(false, false, n, n, n, 1.0, b.Xic + nn, n, 2 * nn, w->F, n, nn, 0.0, b.Zc + nn, n, 2 * nn);
  bw_rowdiv(n, n, b.kap, b.Zc, U, s);
  // D = [-phi-^T nu_bottom; (D phi- - R phi+)^T nu_top] (adjoint mode amplitudes)
  for (int q = 0; q < 2; ++q) {
    gm(true, false, n, R, n, -1.0, b.Pmc + q * nn, n, 2 * nn, b.nu + nR, R, 2 * nR, 0.0,
       b.D + q * 2 * nR, R, 4 * nR);
    gm(true, false, n, R, n, 1.0, b.Gtc + q * nn, n, 2 * nn, b.nu, R, 2 * nR, 0.0,
       b.D + q * 2 * nR + nR, R, 4 * nR);
  }
  bw_cplx_rows(n, 2 * n, R, 2 * nR, w->C, b.kap, b.Ch, U, s);
  for (int q = 0; q < 2; ++q) {
    gm(false, false, n, R, n, 1.0, b.Xic + q * nn, n, 2 * nn, w->SD, R, 2 * nR, 0.0, b.Ta + q * nR,
       R, 2 * nR);
    gm(false, false, n, R, n, 1.0, b.Zc + q * nn, n, 2 * nn, w->SD + nR, R, 2 * nR, 0.0,
       b.Tz + q * nR, R, 2 * nR);
  }
  bw_zeta(n, R, b.Ta, b.Tz, b.zeta, U, s);
  bw_psi(ob, w->P1, w->P2, b.kap, pts, b.PsiT1, b.PsiT2, s);
  for (int q = 0; q < 2; ++q) {
    // D' = D - Psi2 Tb
    gm(true, false, 2 * n, R, Ro, -1.0, b.PsiT2 + q * Ro2n, 2 * n, 2 * Ro2n, b.Tb, R, RoR, 1.0,
       b.D + q * 2 * nR, R, 4 * nR);
    // Ahat = (Tb Ch^T) o gf + G0 zeta^T
    gm(false, true, Ro, 2 * n, R, 1.0, b.Tb, R, RoR, b.Ch + q * 2 * nR, R, 4 * nR, 0.0,
       b.Ah + q * Ro2n, 2 * n, 2 * Ro2n);
  }
  bw_gf(ob, b.kap, pts, b.Ah, s);
  for (int q = 0; q < 2; ++q)
    gm(false, true, Ro, 2 * n, R, 1.0, b.G0, R, RoR, b.zeta + q * 2 * nR, R, 4 * nR, 1.0,
       b.Ah + q * Ro2n, 2 * n, 2 * Ro2n);
  // complex products C (+)= A op(B): re = Ar Br - Ai Bi, im = Ar Bi + Ai Br
  auto zgm = [&](bool tA, bool tB, int M_, int N_, int K_, const double* A_, int lda, long long pA,
                 long long sA, const double* B_, int ldb, long long pB, long long sB, double be,
                 double* C_, int ldc, long long pC, long long sC) {
    gm(tA, tB, M_, N_, K_, 1.0, A_, lda, sA, B_, ldb, sB, be, C_, ldc, sC);
    gm(tA, tB, M_, N_, K_, -1.0, A_ + pA, lda, sA, B_ + pB, ldb, sB, 1.0, C_, ldc, sC);
    gm(tA, tB, M_, N_, K_, 1.0, A_, lda, sA, B_ + pB, ldb, sB, be, C_ + pC, ldc, sC);
    gm(tA, tB, M_, N_, K_, 1.0, A_ + pA, lda, sA, B_, ldb, sB, 1.0, C_ + pC, ldc, sC);
  };
  // Omega = I1 o (D' Ch^T) + (D' o I2) zeta^T + Psi1 Ahat
  zgm(false, true, 2 * n, 2 * n, R, b.D, R, 2 * nR, 4 * nR, b.Ch, R, 2 * nR, 4 * nR, 0.0, b.Om,
      2 * n, 4 * nn, 8 * nn);
  bw_i1(n, ly.tau, b.kap, b.Om, U, s);
  bw_i2(ob, b.kap, pts, b.D, b.Dp2, s);
  zgm(false, true, 2 * n, 2 * n, R, b.Dp2, R, 2 * nR, 4 * nR, b.zeta, R, 2 * nR, 4 * nR, 1.0, b.Om,
      2 * n, 4 * nn, 8 * nn);
  zgm(true, false, 2 * n, 2 * n, Ro, b.PsiT1, 2 * n, Ro2n, 2 * Ro2n, b.Ah, 2 * n, Ro2n, 2 * Ro2n,
      1.0, b.Om, 2 * n, 4 * nn, 8 * nn);
  bw_omblk(n, b.Om, b.OmF, b.OmE, U, s);
  // F'bar = Re(Xc^-T OmF Yc^T) / 2, E'bar = Re(Zc^T OmE Xc^T) / 2 (Zc = Yc^-1)
  zgm(false, true, n, n, n, b.OmF, n, nn, 2 * nn, b.Yc, n, nn, 2 * nn, 0.0, b.Tc, n, nn, 2 * nn);
  gm(true, false, n, n, n, 0.5, b.Xic, n, 2 * nn, b.Tc, n, 2 * nn, 0.0, b.Fb, n, nn);
  gm(true, false, n, n, n, -0.5, b.Xic + nn, n, 2 * nn, b.Tc + nn, n, 2 * nn, 1.0, b.Fb, n, nn);
  zgm(false, true, n, n, n, b.OmE, n, nn, 2 * nn, b.Xc, n, nn, 2 * nn, 0.0, b.Tc, n, nn, 2 * nn);
  gm(true, false, n, n, n, 0.5, b.Zc, n, 2 * nn, b.Tc, n, 2 * nn, 0.0, b.Eb, n, nn);
  gm(true, false, n, n, n, -0.5, b.Zc + nn, n, 2 * nn, b.Tc + nn, n, 2 * nn, 1.0, b.Eb, n, nn);
  // ---- parameter chain: omega (every operator is linear in omega at fixed tables)
  OrderBatch o2 = ob, o2pi = ob, o4 = ob;
  o2.omega = 2.0;
  o2pi.omega = 2.0 * kPi;
  o4.omega = 4.0;
  launch_assemble_EF(o2, w->gp, w->gr, w->gt, w->d_mu_nodes, w->d_w_nodes, b.E2, b.F2, s);
  bw_dot_ef(n, N, b.Eb, b.E2, b.Fb, b.F2, w->d_mu_nodes, acc, U, s);
  launch_assemble_beam(o2pi, w->gp, w->gr, w->gt, w->d_mu_nodes, w->d_min4, b.ptmp, b.rtmp, s);
  bw_dot(nR, b.pb, nR, b.ptmp, nR, 1.0 / (2.0 * kPi), acc, U, s);
  bw_dot(nR, b.rb, nR, b.rtmp, nR, 1.0 / (2.0 * kPi), acc, U, s);
  launch_assemble_U(o4, w->gp, w->gr, w->gt, w->d_w_nodes, w->d_mout4, b.Utmp, s);
  bw_dot(Ro2n, b.Ub, Ro2n, b.Utmp, Ro2n, 0.25, acc, U, s);
  launch_assemble_direct(o2pi, w->gp, w->gr, w->gt, pts, w->d_min4, w->d_mout4, b.Tdir, s);
  bw_dot(RoR, b.Tb, RoR, b.Tdir, RoR, 1.0 / (2.0 * kPi), acc, U, s);
  // ---- interface index: tangent operators (tables at the incident / outgoing points and the
  // transmission blocks replaced by their n-derivatives)
  if (ly.n_interface > 1.0) {
    double** mx = b.mix;
    launch_gsf_tables_dn(ob, pts, dpts, mx[0], mx[1], mx[2], mx[3], mx[4], mx[5], s);
    launch_assemble_beam(ob, mx[0], mx[1], mx[2], w->d_mu_nodes, w->d_min4, b.ptmp, b.rtmp, s);
    bw_dot(nR, b.pb, nR, b.ptmp, nR, 1.0, acc + 2, U, s);
    bw_dot(nR, b.rb, nR, b.rtmp, nR, 1.0, acc + 2, U, s);
    launch_assemble_beam(ob, w->gp, w->gr, w->gt, w->d_mu_nodes, w->dmin4, b.ptmp, b.rtmp, s);
    bw_dot(nR, b.pb, nR, b.ptmp, nR, 1.0, acc + 2, U, s);
    bw_dot(nR, b.rb, nR, b.rtmp, nR, 1.0, acc + 2, U, s);
    launch_assemble_U(ob, mx[3], mx[4], mx[5], w->d_w_nodes, w->d_mout4, b.Utmp, s);
    bw_dot(Ro2n, b.Ub, Ro2n, b.Utmp, Ro2n, 1.0, acc + 2, U, s);
    launch_assemble_U(ob, w->gp, w->gr, w->gt, w->d_w_nodes, w->dmout4, b.Utmp, s);
    bw_dot(Ro2n, b.Ub, Ro2n, b.Utmp, Ro2n, 1.0, acc + 2, U, s);
    launch_assemble_direct(ob, mx[0], mx[1], mx[2], pts, w->d_min4, w->d_mout4, b.Tdir, s);
    bw_dot(RoR, b.Tb, RoR, b.Tdir, RoR, 1.0, acc + 2, U, s);
    launch_assemble_direct(ob, mx[3], mx[4], mx[5], pts, w->d_min4, w->d_mout4, b.Tdir, s);
    bw_dot(RoR, b.Tb, RoR, b.Tdir, RoR, 1.0, acc + 2, U, s);
    launch_assemble_direct(ob, w->gp, w->gr, w->gt, pts, w->dmin4, w->d_mout4, b.Tdir, s);
    bw_dot(RoR, b.Tb, RoR, b.Tdir, RoR, 1.0, acc + 2, U, s);
    launch_assemble_direct(ob, w->gp, w->gr, w->gt, pts, w->d_min4, w->dmout4, b.Tdir, s);
    bw_dot(RoR, b.Tb, RoR, b.Tdir, RoR, 1.0, acc + 2, U, s);
  }
  // ---- expansion coefficients: Sbar of the four point families, contracted with the tables
  bw_sbar_nn(ob, b.Eb, b.Fb, w->d_mu_nodes, w->d_w_nodes, b.SNN, s);
  bw_sbar_ni(ob, b.pb, b.rb, w->d_mu_nodes, w->d_min4, b.SNI, s);
  bw_sbar_on(ob, b.Ub, w->d_w_nodes, w->d_mout4, b.SON, s);
  bw_sbar_oi(ob, b.G0, w->d_min4, w->d_mout4, b.SOI, s);
  bw_pstack(ob, 0, N, w->gp, w->gr, w->gt, b.PYn, s);
  bw_pstack(ob, N, p->n_in, w->gp, w->gr, w->gt, b.PYi, s);
  gm(false, false, 2 * n, 4 * L, n, 1.0, b.SNN, n, 2 * nn, b.PYn, 4 * L, n * L4, 0.0, b.QNN,
     4 * L, 2 * n * L4);
  gm(false, false, 2 * n, 4 * L, R, 1.0, b.SNI, R, 2 * nR, b.PYi, 4 * L, R * L4, 0.0, b.QNI,
     4 * L, 2 * n * L4);
  gm(false, false, 2 * Ro, 4 * L, n, 1.0, b.SON, n, 2LL * Ro * n, b.PYn, 4 * L, n * L4, 0.0,
     b.QON, 4 * L, 2 * Ro * L4);
  gm(false, false, Ro, 4 * L, R, 1.0, b.SOI, R, RoR, b.PYi, 4 * L, R * L4, 0.0, b.QOI, 4 * L,
     Ro * L4);
  bw_bbar(ob, 0, N, b.QNN, b.QNN + n * L4, 2 * n * L4, w->gp, w->gr, w->gt, acc, s);
  bw_bbar(ob, 0, N, b.QNI, b.QNI + n * L4, 2 * n * L4, w->gp, w->gr, w->gt, acc, s);
  bw_bbar(ob, N + p->n_in, p->n_out, b.QON, b.QON + Ro * L4, 2 * Ro * L4, w->gp, w->gr, w->gt,
          acc, s);
  bw_bbar(ob, N + p->n_in, p->n_out, nullptr, b.QOI, Ro * L4, w->gp, w->gr, w->gt, acc, s);
}

static vrte_status run_solve(vrte_plan* p, const double* coeffs, void* d_brdf, int out_dtype,
                             cudaStream_t s0, void (*hook_fn)(void*, int, int, int, cudaStream_t) = nullptr,
                             void* hook_user = nullptr) {
  const size_t table = (size_t)p->n_in * p->n_out * p->n_phi * 16;
  const size_t esz = out_dtype == VRTE_OUT_F64 ? sizeof(double) : sizeof(float);
  const int R = 4 * p->n_in, Ro = 4 * p->n_out;
  // layer lb runs on slot lb % nslots; with several slots each has its own stream, forked
  // from and joined back into the caller's stream
  const int ns = p->nslots;
  if (ns > 1) {
    if (cudaEventRecord(p->fork, s0) != cudaSuccess) return VRTE_ERR_CUDA;
    for (int k = 0; k < ns; ++k)
      if (cudaStreamWaitEvent(p->ws[k].stream, p->fork, 0) != cudaSuccess) return VRTE_ERR_CUDA;
  }
  vrte_status result = VRTE_OK;
  for (int k = 0; k < ns && result == VRTE_OK; ++k)
    if (p->desc.precision == VRTE_MIXED &&
        cudaMemsetAsync(p->ws[k].rcount, 0, 3 * sizeof(int), ns > 1 ? p->ws[k].stream : s0))
      result = VRTE_ERR_CUDA;
  for (int lb = 0; lb < p->n_layers && result == VRTE_OK; ++lb) {
    Work* w = &p->ws[lb % ns];
    cudaStream_t s = ns > 1 ? w->stream : s0;
    p->last_slot = lb % ns;
    const vrte_layer& ly = p->layers[lb];
    const int N = ly.n_nodes, n = 4 * N, L = ly.n_coef;
    const int Meff = std::min(ly.n_orders, ly.n_coef);
    const int P = N + p->n_in + p->n_out;
    const double* coef = coeffs + (size_t)lb * p->desc.n_coef_max * 6;
    {
      StageScope sc(p, ST_TABLES, s, 3, 0.0, 0.0);
      launch_gauss_nodes(N, w->d_mu_nodes, w->d_w_nodes, p->d_status, s);
      launch_interface(N, p->n_in, p->n_out, ly.n_interface, w->d_mu_nodes, p->d_mu_in,
                       p->d_mu_out, w->d_pts, w->d_min4, w->d_mout4, w->d_rtop4, s);
      launch_depth_table(N, p->n_in, p->n_out, ly.tau, w->d_pts, w->g0tab, s);
    }
    char* outb = (char*)d_brdf + (size_t)lb * table * esz;
    SynthHook hook{hook_fn, hook_user, lb};
    // with a hook (host-buffer solve), a layer of one order batch reconstructs and synthesizes
    // block by block when the second workspace is there
    ChunkSynth cs{outb, out_dtype, &hook, p->d_chunk_ws, p->chunk_ws_bytes, false};
    for (int m0 = 0; m0 < Meff; m0 += p->chunk)
      run_order_batch(p, w, ly, coef, m0, std::min(p->chunk, Meff - m0),
                      p->desc.precision == VRTE_MIXED, true, s, true,
                      hook_fn && ns == 1 ? &cs : nullptr);
    // a launch that could not start (resources, configuration) fails the solve here
    if (cudaPeekAtLastError() != cudaSuccess) {
      cudaGetLastError();
      result = VRTE_ERR_CUDA;
      break;
    }
    if (!cs.done) {
      const bool mixed = p->desc.precision == VRTE_MIXED;
      StageScope sc(p, ST_SYNTHESIS, s,
                    mixed ? 1 + 2 * ((p->n_in + kSynthBlock - 1) / kSynthBlock) : 1,
                    2.0 * table * Meff,
                    (double)table * esz + (double)Meff * p->n_in * p->n_out * 16 * 8);
      if (mixed) {
        const int Ss = kSlicesSynth;
        sc.tensor_flops(2.0 * Ss * (Ss + 1) / 2 * 16.0 * p->n_in * p->n_out * p->n_rep * Meff);
      }
      if (mixed) {
        tc_synthesis(Meff, p->n_in, p->n_out, p->n_phi, p->n_rep, p->d_syn_map, w->Isyn, p->d_wc,
                     p->d_ws, outb, out_dtype, kSynthBlock, w->tcw, p->d_status, s,
                     hook_fn ? &hook : nullptr);
      } else {
        launch_synthesis_fp64(Meff, p->n_in, p->n_out, p->n_phi, w->Isyn, p->d_wc, p->d_ws, outb,
                              out_dtype, p->d_status, s);
        if (hook_fn) hook_fn(hook_user, lb, 0, p->n_in, s);
      }
    }
  }
  // join: the caller's stream waits for every slot, also after a failed launch
  if (ns > 1)
    for (int k = 0; k < ns; ++k)
      if (cudaEventRecord(p->ws[k].done, p->ws[k].stream) != cudaSuccess ||
          cudaStreamWaitEvent(s0, p->ws[k].done, 0) != cudaSuccess)
        result = VRTE_ERR_CUDA;
  if (cudaGetLastError() != cudaSuccess) return VRTE_ERR_CUDA;
  return result;
}

vrte_status vrte_solve_brdf(vrte_plan* p, void* d_brdf, int out_dtype, void* stream) {
  if (!p || !d_brdf) return VRTE_ERR_INVALID_ARG;
  if (out_dtype != VRTE_OUT_F32 && out_dtype != VRTE_OUT_F64) return VRTE_ERR_INVALID_ARG;
  if (p->n_layers < 1 || !p->d_coeffs || !p->ws[0].Isyn) return VRTE_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  p->last_stream = s;
  return run_solve(p, p->d_coeffs, d_brdf, out_dtype, s);
}

// Radiance tables at depth taus[lb] of every layer (upward into d_up, downward into d_down;
// either may be null): the FP64 form of the order batches, then the reconstruction at that
// depth (k_modes.cu) and the plan's synthesis.
static vrte_status solve_depth(vrte_plan* p, const double* taus, void* d_up, void* d_down,
                               int out_dtype, cudaStream_t s0) {
  const int ns = p->nslots;
  if (ns > 1) {
    if (cudaEventRecord(p->fork, s0) != cudaSuccess) return VRTE_ERR_CUDA;
    for (int k = 0; k < ns; ++k)
      if (cudaStreamWaitEvent(p->ws[k].stream, p->fork, 0) != cudaSuccess) return VRTE_ERR_CUDA;
  }
  const size_t table = (size_t)p->n_in * p->n_out * p->n_phi * 16;
  const size_t esz = out_dtype == VRTE_OUT_F64 ? sizeof(double) : sizeof(float);
  const int R = 4 * p->n_in, Ro = 4 * p->n_out;
  const bool mixed = p->desc.precision == VRTE_MIXED;
  vrte_status result = VRTE_OK;
  for (int lb = 0; lb < p->n_layers && result == VRTE_OK; ++lb) {
    Work* w = &p->ws[lb % ns];
    cudaStream_t s = ns > 1 ? w->stream : s0;
    p->last_slot = lb % ns;
    const vrte_layer& ly = p->layers[lb];
    const int N = ly.n_nodes, n = 4 * N, L = ly.n_coef;
    const int Meff = std::min(ly.n_orders, ly.n_coef);
    const int P = N + p->n_in + p->n_out;
    const double tau = taus[lb];
    const double* coef = p->d_coeffs + (size_t)lb * p->desc.n_coef_max * 6;
    // upward orders go to Isyn2 when both tables are wanted
    double* Iup = d_down ? w->Isyn2 : w->Isyn;
    {
      StageScope sc(p, ST_TABLES, s, 4, 0.0, 0.0);
      launch_gauss_nodes(N, w->d_mu_nodes, w->d_w_nodes, p->d_status, s);
      launch_interface(N, p->n_in, p->n_out, ly.n_interface, w->d_mu_nodes, p->d_mu_in,
                       p->d_mu_out, w->d_pts, w->d_min4, w->d_mout4, w->d_rtop4, s);
      launch_btdf_points(N, p->n_in, p->n_out, ly.n_interface, p->d_mu_out, w->d_pts, w->d_mout4,
                         w->rout4, s);
      launch_depth_table(N, p->n_in, p->n_out, ly.tau, w->d_pts, w->g0tab, s);
    }
    for (int m0 = 0; m0 < Meff; m0 += p->chunk) {
      const int U = std::min(p->chunk, Meff - m0);
      run_order_batch(p, w, ly, coef, m0, U, false, false, s);
      OrderBatch ob{N, n, L, m0, U, p->n_in, p->n_out, P, ly.tau, ly.omega, coef, p->d_status,
                    2 * n, 2LL * n * R};
      const long long nR = (long long)n * R, RoR = (long long)Ro * R, Ro2n = (long long)Ro * 2 * n;
      BaseR Rg;
      const bool base = layer_base(ly, &Rg) && m0 == 0;
      StageScope sc(p, ST_RECON_HOM, s, 12, 2.0 * U * (double)Ro * R * 2 * n * 5,
                    8.0 * U * 8.0 * Ro * R);
      // upward radiance at the top (identity exit): T1 = direct + Hhat C (+ the base's
      // radiance), and Qp = U+ s + U- d
      dgemm_batched(Ro, R, 2 * n, 1.0, w->Hhat, 2 * n, Ro2n, w->C, R, 2 * nR, 1.0, w->T1, R, RoR, U,
                    s);
      if (base)
        launch_base_recon(n, N, p->n_in, p->n_out, ly.tau, Rg, w->C, w->basebuf, w->d_pts,
                          nullptr, w->T1, 0, s);
      dgemm_batched(Ro, R, 2 * n, 1.0, w->Upm, 2 * n, Ro2n, w->SD, R, 2 * nR, 0.0, w->Qp, R, RoR,
                    U, s);
      if (d_up) {
        launch_assemble_direct_depth(ob, tau, 0, w->gp, w->gr, w->gt, w->d_pts, w->d_min4, w->Tup,
                                     s);
        launch_build_Hdepth(ob, tau, 0, w->P1, w->P2, w->lam_re, w->lam_im, w->d_pts, w->Hhat, s);
        dgemm_batched(Ro, R, 2 * n, 1.0, w->Hhat, 2 * n, Ro2n, w->C, R, 2 * nR, 1.0, w->Tup, R, RoR,
                      U, s);
        launch_depth_combine(ob, tau, 0, w->Tup, w->Qp, w->T1, w->Qp, w->d_pts, w->rout4, Iup, s);
        if (base)
          launch_base_recon(n, N, p->n_in, p->n_out, ly.tau - tau, Rg, w->C, w->basebuf,
                            w->d_pts, nullptr, Iup, 1, s);
      }
      if (d_down) {
        // Qb = U+ s - U- d; Tbot = direct + Hdepth C at depth tau, downward
        dgemm_batched(Ro, R, n, 1.0, w->Upm, 2 * n, Ro2n, w->SD, R, 2 * nR, 0.0, w->Qb, R, RoR, U,
                      s);
        dgemm_batched(Ro, R, n, -1.0, w->Upm + n, 2 * n, Ro2n, w->SD + nR, R, 2 * nR, 1.0, w->Qb, R,
                      RoR, U, s);
        launch_assemble_direct_depth(ob, tau, 1, w->gp, w->gr, w->gt, w->d_pts, w->d_min4, w->Tbot,
                                     s);
        launch_build_Hdepth(ob, tau, 1, w->P1, w->P2, w->lam_re, w->lam_im, w->d_pts, w->Hhat, s);
        dgemm_batched(Ro, R, 2 * n, 1.0, w->Hhat, 2 * n, Ro2n, w->C, R, 2 * nR, 1.0, w->Tbot, R,
                      RoR, U, s);
        launch_depth_combine(ob, tau, 1, w->Tbot, w->Qb, w->T1, w->Qp, w->d_pts, w->rout4, w->Isyn,
                             s);
      }
    }
    if (cudaPeekAtLastError() != cudaSuccess) {
      cudaGetLastError();
      result = VRTE_ERR_CUDA;
      break;
    }
    for (int q = 0; q < 2; ++q) {
      void* dst = q == 0 ? d_up : d_down;
      if (!dst) continue;
      const double* src = q == 0 ? Iup : w->Isyn;
      char* outb = (char*)dst + (size_t)lb * table * esz;
      StageScope sc(p, ST_SYNTHESIS, s, 1, 2.0 * table * Meff, (double)table * esz);
      if (mixed)
        tc_synthesis(Meff, p->n_in, p->n_out, p->n_phi, p->n_rep, p->d_syn_map, src, p->d_wc,
                     p->d_ws, outb, out_dtype, kSynthBlock, w->tcw, p->d_status, s);
      else
        launch_synthesis_fp64(Meff, p->n_in, p->n_out, p->n_phi, src, p->d_wc, p->d_ws, outb,
                              out_dtype, p->d_status, s);
    }
  }
  if (ns > 1)
    for (int k = 0; k < ns; ++k)
      if (cudaEventRecord(p->ws[k].done, p->ws[k].stream) != cudaSuccess ||
          cudaStreamWaitEvent(s0, p->ws[k].done, 0) != cudaSuccess)
        result = VRTE_ERR_CUDA;
  if (cudaGetLastError() != cudaSuccess) return VRTE_ERR_CUDA;
  return result;
}

vrte_status vrte_solve_radiance(vrte_plan* p, const double* h_tau, void* d_up, void* d_down,
                                int out_dtype, void* stream) {
  if (!p || !h_tau || (!d_up && !d_down)) return VRTE_ERR_INVALID_ARG;
  if (out_dtype != VRTE_OUT_F32 && out_dtype != VRTE_OUT_F64) return VRTE_ERR_INVALID_ARG;
  if (!(p->desc.flags & VRTE_FLAG_TRANSMISSION) || p->n_layers < 1 || !p->d_coeffs ||
      !p->ws[0].Tbot)
    return VRTE_ERR_STATE;
  for (int lb = 0; lb < p->n_layers; ++lb)
    if (!(h_tau[lb] >= 0.0 && h_tau[lb] <= p->layers[lb].tau)) return VRTE_ERR_INVALID_ARG;
  std::vector<double> taus(h_tau, h_tau + p->n_layers);
  p->last_stream = (cudaStream_t)stream;
  return solve_depth(p, taus.data(), d_up, d_down, out_dtype, (cudaStream_t)stream);
}

vrte_status vrte_solve_btdf(vrte_plan* p, void* d_btdf, int out_dtype, void* stream) {
  if (!p || !d_btdf) return VRTE_ERR_INVALID_ARG;
  if (out_dtype != VRTE_OUT_F32 && out_dtype != VRTE_OUT_F64) return VRTE_ERR_INVALID_ARG;
  if (!(p->desc.flags & VRTE_FLAG_TRANSMISSION) || p->n_layers < 1 || !p->d_coeffs ||
      !p->ws[0].Tbot)
    return VRTE_ERR_STATE;
  std::vector<double> taus(p->n_layers);
  for (int lb = 0; lb < p->n_layers; ++lb) taus[lb] = p->layers[lb].tau;
  p->last_stream = (cudaStream_t)stream;
  return solve_depth(p, taus.data(), nullptr, d_btdf, out_dtype, (cudaStream_t)stream);
}

// One slab made of the set layers, top first (Sec. 2.C, multi-layer materials): per order
// batch the sub-layers' modes, particular solutions and reconstruction operators in turn
// (FP64 form), each sub-layer's row block entering the block elimination of k_slab.cu as it
// arrives; then back-substitution from the bottom, the sub-layers' top radiances summed with
// the attenuation through the sub-layers above, the base's radiance, and the plan's synthesis.
static vrte_status solve_slab(vrte_plan* p, void* d_brdf, int out_dtype, cudaStream_t s) {
  // slot 0 holds the elimination buffers; sub-layer k computes its modes on slot k mod ns,
  // on the slot's own stream when the plan has several, so that the mode stages (eigen-
  // decompositions first of all) of consecutive sub-layers run concurrently while the
  // caller's stream carries the elimination, one sub-layer after the other. Each slot's
  // `ready` event hands its modes to the elimination, its `freed` event hands the slot back.
  Work* w = &p->ws[0];
  const int ns = p->nslots;
  p->last_slot = 0;
  const int S = p->n_layers;
  const vrte_layer& top = p->layers[0];
  const vrte_layer& bot = p->layers[S - 1];
  Work* wl = &p->ws[(S - 1) % ns];  // the last sub-layer's slot (the base's buffers)
  const int N = top.n_nodes, n = 4 * N, n2 = 2 * n;
  const int R = 4 * p->n_in, Ro = 4 * p->n_out;
  const int P = N + p->n_in + p->n_out;
  const bool mixed = p->desc.precision == VRTE_MIXED;
  int Meff = 0;
  for (const auto& l : p->layers) Meff = std::max(Meff, std::min(l.n_orders, l.n_coef));
  std::vector<double> t_top(S);
  double ttot = 0.0;
  for (int k = 0; k < S; ++k) {
    t_top[k] = ttot;
    ttot += p->layers[k].tau;
  }
  const int U0 = p->chunk;
  const long long nn = (long long)n * n, nR = (long long)n * R, RoR = (long long)Ro * R;
  const long long sD = 4 * nn, sYk = 2 * nR, sUk = 2 * nn, sHk = (long long)Ro * n2;
  auto slot_stream = [&](int j) { return ns > 1 ? p->ws[j].stream : s; };
  if (ns > 1) {
    if (cudaEventRecord(p->fork, s) != cudaSuccess) return VRTE_ERR_CUDA;
    for (int j = 0; j < ns; ++j)
      if (cudaStreamWaitEvent(p->ws[j].stream, p->fork, 0) != cudaSuccess) return VRTE_ERR_CUDA;
  }
  for (int j = 0; j < std::min(ns, S); ++j) {
    Work* wj = &p->ws[j];
    StageScope sc(p, ST_TABLES, slot_stream(j), 2, 0.0, 0.0);
    launch_gauss_nodes(N, wj->d_mu_nodes, wj->d_w_nodes, p->d_status, slot_stream(j));
    launch_interface(N, p->n_in, p->n_out, top.n_interface, wj->d_mu_nodes, p->d_mu_in,
                     p->d_mu_out, wj->d_pts, wj->d_min4, wj->d_mout4, wj->d_rtop4,
                     slot_stream(j));
  }
  for (int m0 = 0; m0 < Meff; m0 += U0) {
    const int U = std::min(U0, Meff - m0);
    const double dn = n, dR = R, dRo = Ro, dU = U;
    double* Lprev = w->sL[0];
    double* Lcur = w->sL[1];
    double* Pprev = w->sPd[0];
    double* Pcur = w->sPd[1];
    OrderBatch ob{};
    for (int k = 0; k < S; ++k) {
      const vrte_layer& ly = p->layers[k];
      const double* coef = p->d_coeffs + (size_t)k * p->desc.n_coef_max * 6;
      const bool first = k == 0, last = k == S - 1;
      BaseR Rg;
      const bool base = last && layer_base(ly, &Rg) && m0 == 0;
      Work* wk = &p->ws[k % ns];
      const cudaStream_t sk = slot_stream(k % ns);
      if (ns > 1 && cudaStreamWaitEvent(sk, wk->freed, 0) != cudaSuccess) return VRTE_ERR_CUDA;
      {
        StageScope sc(p, ST_TABLES, sk, 1, 0.0, 0.0);
        launch_depth_table(N, p->n_in, p->n_out, ly.tau, wk->d_pts, wk->g0tab, sk);
      }
      run_order_batch(p, wk, ly, coef, m0, U, false, false, sk, false);
      if (ns > 1 && (cudaEventRecord(wk->ready, sk) != cudaSuccess ||
                     cudaStreamWaitEvent(s, wk->ready, 0) != cudaSuccess))
        return VRTE_ERR_CUDA;
      ob = OrderBatch{N, n, ly.n_coef, m0, U, p->n_in, p->n_out, P, ly.tau, ly.omega, coef,
                      p->d_status, n2, 2 * nR};
      double* Dk = w->sDinv + (size_t)k * U0 * sD;
      double* Yk = w->sY + (size_t)k * U0 * sYk;
      double* Uk = w->sUup + (size_t)k * U0 * sUk;
      double* Hk = w->sH + (size_t)k * U0 * sHk;
      {
        // the sub-layer's particular and direct parts at the slab's top
        StageScope sc(p, ST_RECON_PART, s, first ? 2 : 3, 2.0 * dRo * dR * 2 * dn * dU,
                      8.0 * (dRo * 2 * dn + 2 * dn * dR + 3 * dRo * dR) * dU);
        if (!first) launch_slab_scale_sd(ob, t_top[k], wk->d_pts, wk->SD, s);
        dgemm_batched(Ro, R, n2, 1.0, wk->Upm, n2, sHk, wk->SD, R, 2 * nR, 0.0, w->sTq, R, RoR,
                      U, s);
        launch_slab_accum(ob, t_top[k], wk->d_pts, wk->T1, w->sTq, wk->g0tab, w->sAcc, first, s);
        cudaMemcpyAsync(Hk, wk->Hhat, (size_t)U * sHk * sizeof(double), cudaMemcpyDeviceToDevice,
                        s);
      }
      StageScope sc(p, ST_BC_SOLVE, s, 4 + (base ? 2 : 0) + (first ? 0 : 4),
                    (first ? 0.0 : 2.0 * dn * dR * dn + 2.0 * dn * dn * 2 * dn * 2 +
                                       2.0 * dn * dR * 2 * dn) * dU +
                        (16.0 * dn * dn * dn + 2.0 * 4 * dn * dn * dR) * dU,
                    8.0 * (12 * dn * dn + 6 * dn * dR) * dU);
      launch_slab_blocks(ob, first, wk->X, wk->Y, wk->lam_re, wk->lam_im, wk->d_rtop4, wk->K, Uk,
                         Lcur, s);
      launch_slab_rhs(ob, first, wk->SD, wk->d_rtop4, wk->d_pts, Pprev, wk->RHS, Pcur, w->sZt, s);
      if (base) {
        launch_base_K(N, n, ly.tau, Rg, wk->X, wk->Y, wk->lam_re, wk->lam_im,
                      wk->d_mu_nodes, wk->d_w_nodes, wk->K, wk->basebuf, s);
        launch_base_rhs(N, n, R, 2 * nR, ly.tau, Rg, wk->SD, wk->d_pts, wk->d_min4,
                        wk->d_mu_nodes, wk->d_w_nodes, wk->RHS, wk->basebuf + 8 * n, 1, s,
                        t_top[k]);
      }
      if (!first) {
        const double* Dp = w->sDinv + (size_t)(k - 1) * U0 * sD;  // D'_{k-1}^-1
        double* Yp = w->sY + (size_t)(k - 1) * U0 * sYk;
        // the upward particular radiance at the top of k completes row block k-1
        dgemm_batched(n2, R, n, 1.0, Dp + n, n2, sD, w->sZt, R, nR, 1.0, Yp, R, sYk, U, s);
        // D'_k = D_k - [Ldn_{k-1} W_{k-1} Uup_k; 0],  b'_k = b_k - [Ldn_{k-1} y_{k-1}; 0]
        dgemm_batched(n, n, n2, 1.0, Lprev, n2, sUk, Dp + n, n2, sD, 0.0, w->sTnn, n, nn, U, s);
        dgemm_batched(n, n2, n, -1.0, w->sTnn, n, nn, Uk, n2, sUk, 1.0, wk->K, n2, sD, U, s);
        dgemm_batched(n, R, n2, -1.0, Lprev, n2, sUk, Yp, R, sYk, 1.0, wk->RHS, R, sYk, U, s);
      }
      batched_inverse(n2, wk->K, Dk, U, p->d_status, s);
      dgemm_batched(n2, R, n2, 1.0, Dk, n2, sD, wk->RHS, R, sYk, 0.0, Yk, R, sYk, U, s);
      std::swap(Lprev, Lcur);
      std::swap(Pprev, Pcur);
      if (ns > 1 && cudaEventRecord(wk->freed, s) != cudaSuccess) return VRTE_ERR_CUDA;
    }
    {
      // back-substitution from the bottom, c_k = y_k - W_k (Uup_{k+1} c_{k+1}), then the
      // homogeneous parts of the sub-layers' top radiances
      BaseR Rbot;
      const bool bot_base = layer_base(bot, &Rbot) && m0 == 0;
      StageScope sc(p, ST_RECON_HOM, s, 2 * (S - 1) + 2 * S + 1 + 2 * bot_base,
                    (S - 1) * 2.0 * (2 * dn * dR * 2 * dn) * dU + S * 2.0 * dRo * dR * 2 * dn * dU,
                    8.0 * ((S - 1) * (6 * dn * dn + 6 * dn * dR) + S * (2 * dRo * dn + 2 * dn * dR +
                                                                    2 * dRo * dR)) * dU);
      for (int k = S - 2; k >= 0; --k) {
        const double* Un = w->sUup + (size_t)(k + 1) * U0 * sUk;
        const double* Yn = w->sY + (size_t)(k + 1) * U0 * sYk;
        const double* Dc = w->sDinv + (size_t)k * U0 * sD;
        double* Yc = w->sY + (size_t)k * U0 * sYk;
        dgemm_batched(n, R, n2, 1.0, Un, n2, sUk, Yn, R, sYk, 0.0, w->sV, R, nR, U, s);
        dgemm_batched(n2, R, n, -1.0, Dc + n, n2, sD, w->sV, R, nR, 1.0, Yc, R, sYk, U, s);
      }
      for (int k = 0; k < S; ++k) {
        dgemm_batched(Ro, R, n2, 1.0, w->sH + (size_t)k * U0 * sHk, n2, sHk,
                      w->sY + (size_t)k * U0 * sYk, R, sYk, 0.0, w->sTq, R, RoR, U, s);
        launch_slab_accum(ob, t_top[k], w->d_pts, nullptr, w->sTq, nullptr, w->sAcc, 0, s);
      }
      launch_slab_store(ob, w->sAcc, w->Isyn, s);
      // reflecting base: its radiance at the bottom, attenuated through the slab
      if (bot_base)
        launch_base_recon(n, N, p->n_in, p->n_out, ttot, Rbot,
                          w->sY + (size_t)(S - 1) * U0 * sYk, wl->basebuf, w->d_pts, w->d_mout4,
                          w->Isyn, 1, s);
    }
  }
  // join: every slot stream's work is already behind a `ready` the caller's stream waited on;
  // the join keeps the slot streams ordered before any later use of the plan
  if (ns > 1)
    for (int j = 0; j < ns; ++j)
      if (cudaEventRecord(p->ws[j].done, p->ws[j].stream) != cudaSuccess ||
          cudaStreamWaitEvent(s, p->ws[j].done, 0) != cudaSuccess)
        return VRTE_ERR_CUDA;
  if (cudaPeekAtLastError() != cudaSuccess) {
    cudaGetLastError();
    return VRTE_ERR_CUDA;
  }
  const size_t table = (size_t)p->n_in * p->n_out * p->n_phi * 16;
  const size_t esz = out_dtype == VRTE_OUT_F64 ? sizeof(double) : sizeof(float);
  {
    StageScope sc(p, ST_SYNTHESIS, s, 1, 2.0 * table * Meff, (double)table * esz);
    if (mixed)
      tc_synthesis(Meff, p->n_in, p->n_out, p->n_phi, p->n_rep, p->d_syn_map, w->Isyn, p->d_wc,
                   p->d_ws, d_brdf, out_dtype, kSynthBlock, w->tcw, p->d_status, s);
    else
      launch_synthesis_fp64(Meff, p->n_in, p->n_out, p->n_phi, w->Isyn, p->d_wc, p->d_ws,
                            d_brdf, out_dtype, p->d_status, s);
  }
  if (cudaGetLastError() != cudaSuccess) return VRTE_ERR_CUDA;
  return VRTE_OK;
}

vrte_status vrte_solve_slab_brdf(vrte_plan* p, void* d_brdf, int out_dtype, void* stream) {
  if (!p || !d_brdf) return VRTE_ERR_INVALID_ARG;
  if (out_dtype != VRTE_OUT_F32 && out_dtype != VRTE_OUT_F64) return VRTE_ERR_INVALID_ARG;
  if (!(p->desc.flags & VRTE_FLAG_SLAB) || p->n_layers < 1 || !p->d_coeffs || !p->ws[0].sDinv)
    return VRTE_ERR_STATE;
  const vrte_layer& top = p->layers[0];
  for (int k = 0; k < p->n_layers; ++k) {
    const vrte_layer& l = p->layers[k];
    // one quadrature and one order range for the whole slab; a smooth top only above the
    // first sub-layer and a Lambertian base only under the last
    if (l.n_nodes != top.n_nodes || l.n_orders != top.n_orders) return VRTE_ERR_INVALID_ARG;
    if (k > 0 && l.n_interface > 1.0) return VRTE_ERR_INVALID_ARG;
    if (k < p->n_layers - 1 && layer_base(l, nullptr)) return VRTE_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  p->last_stream = s;
  return solve_slab(p, d_brdf, out_dtype, s);
}

vrte_status vrte_solve_brdf_host(vrte_plan* p, const double* h_coeffs, void* h_brdf,
                                 int out_dtype, void* stream) {
  if (!p || !h_coeffs || !h_brdf) return VRTE_ERR_INVALID_ARG;
  if (out_dtype != VRTE_OUT_F32 && out_dtype != VRTE_OUT_F64) return VRTE_ERR_INVALID_ARG;
  if (p->n_layers < 1 || !p->ws[0].Isyn) return VRTE_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  size_t cbytes = (size_t)p->n_layers * p->desc.n_coef_max * 6 * sizeof(double);
  size_t obytes = (size_t)p->n_layers * p->n_in * p->n_out * p->n_phi * 16 *
                  (out_dtype == VRTE_OUT_F64 ? sizeof(double) : sizeof(float));
  // staging buffers persist across calls; the first call (or a larger request) allocates
  if (cbytes > p->coef_stage_bytes) {
    if (p->d_coef_stage) cudaFree(p->d_coef_stage);
    p->d_coef_stage = nullptr;
    if (cudaMalloc(&p->d_coef_stage, cbytes) != cudaSuccess) { cudaGetLastError(); return VRTE_ERR_OOM; }
    p->coef_stage_bytes = cbytes;
  }
  if (obytes > p->out_stage_bytes) {
    if (p->d_out_stage) cudaFree(p->d_out_stage);
    p->d_out_stage = nullptr;
    if (cudaMalloc(&p->d_out_stage, obytes) != cudaSuccess) { cudaGetLastError(); return VRTE_ERR_OOM; }
    p->out_stage_bytes = obytes;
  }
  // the block-wise reconstruction's workspace, for the largest layer that can use it (one
  // order batch, no base, one particular contraction); optional: without it the layer is
  // reconstructed whole and the copies start with its synthesis
  if (p->desc.precision == VRTE_MIXED && p->nslots == 1) {
    size_t need = 0;
    for (int lb = 0; lb < p->n_layers; ++lb) {
      const vrte_layer& l = p->layers[lb];
      const int Meff = std::min(l.n_orders, l.n_coef), n = 4 * l.n_nodes;
      if (Meff <= p->chunk && !layer_base(l, nullptr) && 2 * n + 4 * l.n_coef <= 1024)
        need = std::max(need, chunk_ws_need(p, n, Meff));
    }
    if (need > p->chunk_ws_bytes) {
      if (p->d_chunk_ws) cudaFree(p->d_chunk_ws);
      p->d_chunk_ws = nullptr;
      p->chunk_ws_bytes = 0;
      if (cudaMalloc(&p->d_chunk_ws, need) == cudaSuccess) {
        p->chunk_ws_bytes = need;
      } else {
        cudaGetLastError();
        p->d_chunk_ws = nullptr;
      }
    }
  }
  if (cudaMemcpyAsync(p->d_coef_stage, h_coeffs, cbytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return VRTE_ERR_CUDA;
  p->last_stream = s;
  // The table leaves in blocks of incident cosines, each as soon as the synthesis kernels that
  // complete it have run: the solve stream records an event after them and one of four copy
  // streams (several copy engines) waits on it and copies the block, so the copies overlap
  // the rest of the solve. The copy streams join back into the caller's stream at the end.
  constexpr int kCopyStreams = 4;
  if (!p->solved) {
    if (cudaEventCreateWithFlags(&p->solved, cudaEventDisableTiming) != cudaSuccess)
      return VRTE_ERR_CUDA;
    for (int c = 0; c < kCopyStreams; ++c)
      if (cudaStreamCreateWithFlags(&p->cstream[c], cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&p->cdone[c], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&p->cready[c], cudaEventDisableTiming) != cudaSuccess)
        return VRTE_ERR_CUDA;
  }
  struct CopyCtx {
    vrte_plan* p;
    char* h;
    size_t row_bytes, layer_bytes;
    int next;
    bool failed;
  } ctx{p, (char*)h_brdf,
        (size_t)p->n_out * p->n_phi * 16 * (out_dtype == VRTE_OUT_F64 ? sizeof(double) : sizeof(float)),
        0, 0, false};
  ctx.layer_bytes = ctx.row_bytes * p->n_in;
  auto copy_block = [](void* user, int layer, int k0, int k1, cudaStream_t sl) {
    CopyCtx* c = (CopyCtx*)user;
    const int q = c->next++ % kCopyStreams;
    const size_t off = (size_t)layer * c->layer_bytes + (size_t)k0 * c->row_bytes;
    const size_t len = (size_t)(k1 - k0) * c->row_bytes;
    if (cudaEventRecord(c->p->cready[q], sl) != cudaSuccess ||
        cudaStreamWaitEvent(c->p->cstream[q], c->p->cready[q], 0) != cudaSuccess ||
        cudaMemcpyAsync(c->h + off, (const char*)c->p->d_out_stage + off, len,
                        cudaMemcpyDeviceToHost, c->p->cstream[q]) != cudaSuccess)
      c->failed = true;
  };
  vrte_status st = run_solve(p, p->d_coef_stage, p->d_out_stage, out_dtype, s, copy_block, &ctx);
  // join the copy streams (also after a failure, so that no copy outlives the call)
  for (int c = 0; c < kCopyStreams; ++c)
    if (cudaEventRecord(p->cdone[c], p->cstream[c]) != cudaSuccess ||
        cudaStreamWaitEvent(s, p->cdone[c], 0) != cudaSuccess)
      st = st == VRTE_OK ? VRTE_ERR_CUDA : st;
  if (cudaStreamSynchronize(s) != cudaSuccess) return VRTE_ERR_CUDA;
  if (st != VRTE_OK) return st;
  return ctx.failed ? VRTE_ERR_CUDA : VRTE_OK;
}

vrte_status vrte_brdf_backward(vrte_plan* p, const void* g, int gd, double* d_grad, void* stream) {
  if (!p || !g || !d_grad) return VRTE_ERR_INVALID_ARG;
  if (gd != VRTE_OUT_F32 && gd != VRTE_OUT_F64) return VRTE_ERR_INVALID_ARG;
  if (!(p->desc.flags & VRTE_FLAG_ADJOINT) || p->n_layers < 1 || !p->ws[0].bw)
    return VRTE_ERR_STATE;
  for (const vrte_layer& l : p->layers)
    if (layer_base(l, nullptr)) return VRTE_ERR_UNSUPPORTED;
  cudaStream_t s0 = (cudaStream_t)stream;
  p->last_stream = s0;
  const int ns = p->nslots;
  if (ns > 1) {
    if (cudaEventRecord(p->fork, s0) != cudaSuccess) return VRTE_ERR_CUDA;
    for (int k = 0; k < ns; ++k)
      if (cudaStreamWaitEvent(p->ws[k].stream, p->fork, 0) != cudaSuccess) return VRTE_ERR_CUDA;
  }
  const size_t table = (size_t)p->n_in * p->n_out * p->n_phi * 16;
  const size_t esz = gd == VRTE_OUT_F64 ? sizeof(double) : sizeof(float);
  const int Lmax = p->desc.n_coef_max;
  vrte_status result = VRTE_OK;
  for (int lb = 0; lb < p->n_layers && result == VRTE_OK; ++lb) {
    Work* w = &p->ws[lb % ns];
    cudaStream_t s = ns > 1 ? w->stream : s0;
    p->last_slot = lb % ns;
    const vrte_layer& ly = p->layers[lb];
    const int N = ly.n_nodes, L = ly.n_coef;
    const int Meff = std::min(ly.n_orders, ly.n_coef);
    const double* coef = p->d_coeffs + (size_t)lb * Lmax * 6;
    {
      StageScope sc(p, ST_TABLES, s, 4, 0.0, 0.0);
      launch_gauss_nodes(N, w->d_mu_nodes, w->d_w_nodes, p->d_status, s);
      launch_interface(N, p->n_in, p->n_out, ly.n_interface, w->d_mu_nodes, p->d_mu_in,
                       p->d_mu_out, w->d_pts, w->d_min4, w->d_mout4, w->d_rtop4, s);
      launch_interface_dn(N, p->n_in, p->n_out, ly.n_interface, w->d_mu_nodes, p->d_mu_in,
                          p->d_mu_out, w->dpts, w->dmin4, w->dmout4, w->drtop4, s);
      launch_depth_table(N, p->n_in, p->n_out, ly.tau, w->d_pts, w->g0tab, s);
    }
    {
      StageScope sc(p, ST_ADJOINT, s, 2, 2.0 * table * Meff, (double)table * esz);
      cudaMemsetAsync(w->acc, 0, (3 + 6 * (size_t)Lmax) * sizeof(double), s);
      launch_synth_transpose(Meff, p->n_in, p->n_out, p->n_phi,
                             (const char*)g + (size_t)lb * table * esz, gd, p->d_wc, p->d_ws,
                             w->Isyn, s);
    }
    for (int m0 = 0; m0 < Meff; m0 += p->chunk) {
      const int U = std::min(p->chunk, Meff - m0);
      run_order_batch(p, w, ly, coef, m0, U, false, false, s);
      backward_batch(p, w, ly, coef, m0, U, s);
    }
    bw_finish(L, Lmax, ly.n_interface, w->acc, d_grad + (size_t)lb * (3 + 6 * Lmax), s);
    if (cudaPeekAtLastError() != cudaSuccess) {
      cudaGetLastError();
      result = VRTE_ERR_CUDA;
    }
  }
  if (ns > 1)
    for (int k = 0; k < ns; ++k)
      if (cudaEventRecord(p->ws[k].done, p->ws[k].stream) != cudaSuccess ||
          cudaStreamWaitEvent(s0, p->ws[k].done, 0) != cudaSuccess)
        result = VRTE_ERR_CUDA;
  if (cudaGetLastError() != cudaSuccess) return VRTE_ERR_CUDA;
  return result;
}

vrte_status vrte_plan_status(vrte_plan* p) {
  if (!p) return VRTE_ERR_INVALID_ARG;
  if (cudaStreamSynchronize(p->last_stream) != cudaSuccess) return VRTE_ERR_CUDA;
  unsigned h = 0;
  if (cudaMemcpy(&h, p->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess)
    return VRTE_ERR_CUDA;
  cudaMemset(p->d_status, 0, sizeof(unsigned));
  if (h & ST_NONFINITE) return VRTE_ERR_NONFINITE;
  if (h & ST_NO_CONVERGENCE) return VRTE_ERR_NO_CONVERGENCE;
  if (h & ST_SINGULAR) return VRTE_ERR_SINGULAR;
  if (h) return VRTE_ERR_CUDA;  // ST_TIMEOUT: a bounded device wait gave up
  return VRTE_OK;
}

vrte_status vrte_debug_copy(vrte_plan* p, const char* name, void* dst, size_t bytes,
                            size_t* size_out) {
  if (!p || !name) return VRTE_ERR_INVALID_ARG;
  if (strcmp(name, "status") == 0) {  // raw device status bits, as one double
    unsigned h = 0;
    if (cudaStreamSynchronize(p->last_stream) != cudaSuccess ||
        cudaMemcpy(&h, p->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess)
      return VRTE_ERR_CUDA;
    double v = (double)h;
    if (size_out) *size_out = sizeof(double);
    if (dst && bytes >= sizeof(double)) memcpy(dst, &v, sizeof(double));
    return VRTE_OK;
  }
  if (strcmp(name, "newton_fallbacks") == 0 || strcmp(name, "newton_residual") == 0) {
    // mixed form: matrices inverted again in FP64 in the last solve, summed over the slots;
    // or the final Newton residuals max|I - A X| of the last order batch, [K, X][U]
    if (cudaStreamSynchronize(p->last_stream) != cudaSuccess) return VRTE_ERR_CUDA;
    std::vector<double> v;
    if (name[7] == 'f') {
      double c = 0.0;
      for (const Work& x : p->ws) {
        int h = 0;
        if (x.rcount &&
            cudaMemcpy(&h, x.rcount + 2, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
          return VRTE_ERR_CUDA;
        c += h;
      }
      v.push_back(c);
    } else {
      const Work& x = p->ws[p->last_slot];
      if (!x.nerr || p->last_U == 0) return VRTE_ERR_STATE;
      std::vector<unsigned long long> h(2 * (size_t)p->last_U);
      for (int k = 0; k < 2; ++k)
        if (cudaMemcpy(h.data() + (size_t)k * p->last_U, x.nerr + (size_t)k * p->last_U,
                       p->last_U * sizeof(unsigned long long), cudaMemcpyDeviceToHost) !=
            cudaSuccess)
          return VRTE_ERR_CUDA;
      for (unsigned long long b : h) {
        double d;
        memcpy(&d, &b, sizeof(d));
        v.push_back(d);
      }
    }
    if (size_out) *size_out = v.size() * sizeof(double);
    if (dst && bytes >= v.size() * sizeof(double)) memcpy(dst, v.data(), v.size() * sizeof(double));
    return VRTE_OK;
  }
  if (strcmp(name, "refined") == 0) {  // mixed form: column blocks recomputed in FP64
    if (cudaStreamSynchronize(p->last_stream) != cudaSuccess) return VRTE_ERR_CUDA;
    double v = 0.0;
    for (const Work& x : p->ws) {
      int h = 0;
      if (x.rcount &&
          cudaMemcpy(&h, x.rcount + 1, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return VRTE_ERR_CUDA;
      v += h;
    }
    if (size_out) *size_out = sizeof(double);
    if (dst && bytes >= sizeof(double)) memcpy(dst, &v, sizeof(double));
    return VRTE_OK;
  }
  if (p->last_U == 0) return VRTE_ERR_STATE;
  const Work* w = &p->ws[p->last_slot];  // the slot of the last layer solved
  size_t n = p->last_n, U = p->last_U, R = 4 * (size_t)p->n_in, Ro = 4 * (size_t)p->n_out;
  const void* src = nullptr;
  size_t cnt = 0;
  struct Entry { const char* nm; const double* ptr; size_t count; };
  const Entry tab[] = {
      {"pts", w->d_pts, (size_t)p->last_P},
      {"nodes", w->d_mu_nodes, n / 4},
      {"weights", w->d_w_nodes, n / 4},
      {"E", w->E, U * n * n},
      {"F", w->F, U * n * n},
      {"FE", w->FE, U * n * n},
      {"schur", w->Hs, U * n * n},
      {"X", w->X, U * n * n},
      {"Y", w->Y, U * n * n},
      {"lam_re", w->lam_re, U * n},
      {"lam_im", w->lam_im, U * n},
      {"K", w->K, U * 4 * n * n},
      {"Kinv", w->Kinv, U * 4 * n * n},
      {"Xinv", w->Xinv, U * n * n},
      {"beam_p", w->Pb, U * n * R},
      {"beam_r", w->Rb, U * n * R},
      {"SD", w->SD, U * (size_t)p->last_ldU * R},
      {"RHS", w->RHS, U * 2 * n * R},
      {"C", w->C, U * 2 * n * R},
      {"Upm", w->Upm, U * Ro * (size_t)p->last_ldU},
      {"Hhat", w->Hhat, U * Ro * 2 * n},
      {"T1", w->T1, U * Ro * R},
      {"Isyn", w->Isyn, (size_t)p->last_Meff * p->n_in * p->n_out * 16},
      {"mode_res", w->mode_res, U},
  };
  for (const Entry& e : tab)
    if (strcmp(e.nm, name) == 0) { src = e.ptr; cnt = e.count; }
  if (!src) return VRTE_ERR_INVALID_ARG;
  size_t full = cnt * sizeof(double);
  if (size_out) *size_out = full;
  if (cudaStreamSynchronize(p->last_stream) != cudaSuccess) return VRTE_ERR_CUDA;
  if (dst && bytes)
    if (cudaMemcpy(dst, src, std::min(bytes, full), cudaMemcpyDeviceToHost) != cudaSuccess)
      return VRTE_ERR_CUDA;
  return VRTE_OK;
}

int vrte_profile_stages(vrte_plan* p, vrte_stage_stat* out, int max_stages) {
  if (!p) return -1;
  cudaStreamSynchronize(p->last_stream);
  for (auto& e : p->events) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, e.second.first, e.second.second) == cudaSuccess)
      p->stats[e.first].ms += ms;
    cudaEventDestroy(e.second.first);
    cudaEventDestroy(e.second.second);
  }
  p->events.clear();
  cudaGetLastError();
  int n = std::min(max_stages, (int)kStages);
  for (int i = 0; out && i < n; ++i) out[i] = p->stats[i];
  return kStages;
}

void vrte_profile_reset(vrte_plan* p) {
  if (!p) return;
  cudaStreamSynchronize(p->last_stream);
  reset_stats(p);
}

size_t vrte_workspace_bytes(const vrte_plan* p) {
  if (!p) return 0;
  size_t t = p->coef_stage_bytes + p->out_stage_bytes + p->chunk_ws_bytes;
  for (size_t b : p->alloc_bytes) t += b;
  return t;
}

void vrte_destroy(vrte_plan* p) {
  if (!p) return;
  cudaDeviceSynchronize();
  reset_stats(p);
  free_workspace(p, 0);
  for (Work& x : p->ws) {
    if (x.stream) cudaStreamDestroy(x.stream);
    if (x.done) cudaEventDestroy(x.done);
    if (x.ready) cudaEventDestroy(x.ready);
    if (x.freed) cudaEventDestroy(x.freed);
    if (x.side) cudaStreamDestroy(x.side);
    if (x.side_fork) cudaEventDestroy(x.side_fork);
    if (x.side_join) cudaEventDestroy(x.side_join);
  }
  if (p->fork) cudaEventDestroy(p->fork);
  for (int c = 0; c < 4; ++c) {
    if (p->cstream[c]) cudaStreamDestroy(p->cstream[c]);
    if (p->cdone[c]) cudaEventDestroy(p->cdone[c]);
    if (p->cready[c]) cudaEventDestroy(p->cready[c]);
  }
  if (p->solved) cudaEventDestroy(p->solved);
  if (p->d_coef_stage) cudaFree(p->d_coef_stage);
  if (p->d_out_stage) cudaFree(p->d_out_stage);
  if (p->d_chunk_ws) cudaFree(p->d_chunk_ws);
  delete p;
}

}  // extern "C"
