// Multi-layer slabs (Sec. 2.C): every sub-layer has its own modes and particular solution, and
// the 8N mode coefficients of all sub-layers solve one block-banded system, the top and bottom
// conditions of the slab plus the continuity of all 8N radiances at each inner boundary.
//
// Rows and unknowns are grouped per sub-layer k (2n = 8N each, n = 4N). Row block k holds
//   a-rows (n): k = 0 the top condition, else the downward continuity at the boundary above k;
//   b-rows (n): the upward continuity at the boundary below k, or the bottom condition (last).
// Block k then touches the coefficients of k-1 (a-rows only), k and k+1 (b-rows only): a
// block-tridiagonal system whose off-diagonal blocks have half of their rows zero,
//   L_k = [Ldn_{k-1}; 0],  U_k = [0; Uup_{k+1}],
// with Ldn_k the downward radiance at the bottom of k and Uup_k minus the upward radiance at
// the top of k, as functions of c_k. Block elimination from the top,
//   D'_k = D_k - L_k D'_{k-1}^-1 U_{k-1},  y_k = D'_k^-1 (b_k - L_k y_{k-1}),
// needs only W_{k-1} = the b-columns of D'_{k-1}^-1, and back-substitution from the bottom is
//   c_k = y_k - W_k (Uup_{k+1} c_{k+1}).
// The elimination is the adding of the sub-layers from the top: D'_k is sub-layer k's own
// boundary matrix with the stack above folded into its top condition, so its conditioning is
// that of a single layer under a reflecting top.
//
// The mode columns follow the boundary matrix of one layer (k_build_K): decaying modes first,
// a complex pair as its real and imaginary columns; Phi+- = (X +- Y)/2, E = exp(-kappa tau_k).

#include "vrte_internal.cuh"

namespace vrte {

// Boundary blocks of sub-layer k for every unit: D (2n x 2n), Uup and Ldn (n x 2n each).
__global__ void k_slab_blocks(int N, int n, double tau, int first, const double* X,
                              const double* Y, const double* lam_re, const double* lam_im,
                              const double* rtop4, double* D, double* Uup, double* Ldn) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y, u = blockIdx.z;
  if (j >= n) return;
  const double* lr = lam_re + (size_t)u * n;
  const double* li = lam_im + (size_t)u * n;
  if (li[j] < 0.0) return;
  const bool cplx = li[j] > 0.0;
  const cd kap = kappa_of(lr, li, j);
  const cd E = cexpv(cd{-kap.r * tau, -kap.i * tau});
  const double* Xb = X + (size_t)u * n * n;
  const double* Yb = Y + (size_t)u * n * n;
  const int n2 = 2 * n;
  double* Db = D + (size_t)u * n2 * n2;
  double* Ub = Uup + (size_t)u * n * n2;
  double* Lb = Ldn + (size_t)u * n * n2;
  const double* Rm = rtop4 + 4 * i;
  cd pp[4], pm[4];
  for (int a = 0; a < 4; ++a) {
    const size_t idx = (size_t)(4 * i + a) * n + j;
    const cd x{Xb[idx], cplx ? Xb[idx + 1] : 0.0};
    const cd y{Yb[idx], cplx ? Yb[idx + 1] : 0.0};
    pp[a] = cd{0.5 * (x.r + y.r), 0.5 * (x.i + y.i)};
    pm[a] = cd{0.5 * (x.r - y.r), 0.5 * (x.i - y.i)};
  }
  // (R_F v)_a of the top's internal reflection (the first sub-layer only)
  auto rmul = [&](const cd* v, int a) -> cd {
    if (a == 0) return cd{Rm[0] * v[0].r + Rm[1] * v[1].r, Rm[0] * v[0].i + Rm[1] * v[1].i};
    if (a == 1) return cd{Rm[1] * v[0].r + Rm[0] * v[1].r, Rm[1] * v[0].i + Rm[0] * v[1].i};
    if (a == 2) return cd{Rm[2] * v[2].r + Rm[3] * v[3].r, Rm[2] * v[2].i + Rm[3] * v[3].i};
    return cd{-Rm[3] * v[2].r + Rm[2] * v[3].r, -Rm[3] * v[2].i + Rm[2] * v[3].i};
  };
  auto put = [&](double* row, int col, cd v) {
    row[col] = v.r;
    if (cplx) row[col + 1] = v.i;
  };
  for (int a = 0; a < 4; ++a) {
    const double sgn = a < 2 ? 1.0 : -1.0;
    const cd dpp{sgn * pp[a].r, sgn * pp[a].i}, dpm{sgn * pm[a].r, sgn * pm[a].i};
    double* ra = Db + (size_t)(4 * i + a) * n2;
    double* rb = Db + (size_t)(n + 4 * i + a) * n2;
    if (first) {
      // top condition: I(0, -mu) - R_F I(0, +mu) = 0
      const cd rm = rmul(pm, a), rp = rmul(pp, a);
      put(ra, j, cd{dpp.r - rm.r, dpp.i - rm.i});
      put(ra, n + j, cmul(cd{dpm.r - rp.r, dpm.i - rp.i}, E));
    } else {
      // minus the downward radiance at the top of k
      put(ra, j, cd{-dpp.r, -dpp.i});
      put(ra, n + j, cmul(cd{-dpm.r, -dpm.i}, E));
    }
    // upward radiance at the bottom of k
    put(rb, j, cmul(pm[a], E));
    put(rb, n + j, pp[a]);
    // minus the upward radiance at the top of k
    double* ru = Ub + (size_t)(4 * i + a) * n2;
    put(ru, j, cd{-pm[a].r, -pm[a].i});
    put(ru, n + j, cmul(cd{-pp[a].r, -pp[a].i}, E));
    // downward radiance at the bottom of k
    double* rl = Lb + (size_t)(4 * i + a) * n2;
    put(rl, j, cmul(dpp, E));
    put(rl, n + j, dpm);
  }
}

// Right-hand side of row block k from the particular solution SD = [s; d] of sub-layer k
// (already scaled by the beam's attenuation to its top): with z+ = (s + d)/2 and
// z- = D (s - d)/2 the upward and downward radiances at the top of k,
//   a-rows: k = 0: -(z- - R_F z+); else z- - Pd_prev (the particular downward radiance at the
//           bottom of k-1);
//   b-rows: -z+ e^{-tau_k/mu0} (the upward particular radiance at the bottom of k; the term
//           +z+ of sub-layer k+1 at its top is added to y_k once k+1 is known).
// Writes Pd_cur = z- e^{-tau_k/mu0} and Zt = z+ for the neighbours.
__global__ void k_slab_rhs(int N, int n, int R, long long sSD, double tau, int first,
                           const double* SD, const double* rtop4, const double* pts,
                           const double* Pd_prev, double* rhs, double* Pd_cur, double* Zt) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y, u = blockIdx.z;
  if (c >= R) return;
  const double* sv = SD + (size_t)u * sSD;
  const double* dv = sv + (size_t)n * R;
  double zp[4], zm[4];
  for (int a = 0; a < 4; ++a) {
    const size_t idx = (size_t)(4 * i + a) * R + c;
    const double s = sv[idx], d = dv[idx];
    zp[a] = 0.5 * (s + d);
    zm[a] = (a < 2 ? 0.5 : -0.5) * (s - d);
  }
  const double* Rm = rtop4 + 4 * i;
  const double rz[4] = {Rm[0] * zp[0] + Rm[1] * zp[1], Rm[1] * zp[0] + Rm[0] * zp[1],
                        Rm[2] * zp[2] + Rm[3] * zp[3], -Rm[3] * zp[2] + Rm[2] * zp[3]};
  const double att = exp(-tau / pts[N + (c >> 2)]);
  const size_t nR = (size_t)n * R;
  double* rb = rhs + (size_t)u * 2 * nR;
  for (int a = 0; a < 4; ++a) {
    const size_t idx = (size_t)(4 * i + a) * R + c;
    rb[idx] = first ? -(zm[a] - rz[a]) : zm[a] - Pd_prev[(size_t)u * nR + idx];
    rb[nR + idx] = -zp[a] * att;
    Pd_cur[(size_t)u * nR + idx] = zm[a] * att;
    Zt[(size_t)u * nR + idx] = zp[a];
  }
}

// SD[u][r][c] *= e^{-t/mu0(c)} for the 2n rows of the particular solution: the beam reaches
// a sub-layer whose top lies at depth t attenuated by that factor.
__global__ void k_slab_scale_sd(int N, int n, int R, long long sSD, double t, const double* pts,
                                double* SD) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y, u = blockIdx.z;
  if (c >= R) return;
  SD[(size_t)u * sSD + (size_t)r * R + c] *= exp(-t / pts[N + (c >> 2)]);
}

// Acc[u][i][c] (+)= e^{-t/mu_o} (e^{-t/mu0} T1 + g0 Tq): a sub-layer's contribution to the
// upward radiance at the slab's top, attenuated along the exit path through the sub-layers
// above. T1 (the direct part, beam not yet attenuated) and g0tab may be null.
__global__ void k_slab_accum(int N, int n_in, int n_out, double t, const double* pts,
                             const double* T1, const double* Tq, const double* g0tab,
                             double* Acc, int first) {
  const int R = 4 * n_in, Ro = 4 * n_out;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int o = blockIdx.y, u = blockIdx.z;
  if (c >= R) return;
  const int k = c >> 2;
  const double g = g0tab ? g0tab[(size_t)o * n_in + k] : 1.0;
  const double ain = T1 ? exp(-t / pts[N + k]) : 0.0;
  const double aout = exp(-t / pts[N + n_in + o]);
  for (int a = 0; a < 4; ++a) {
    const size_t idx = ((size_t)u * Ro + 4 * o + a) * R + c;
    double v = g * Tq[idx];
    if (T1) v += ain * T1[idx];
    v *= aout;
    Acc[idx] = first ? v : Acc[idx] + v;
  }
}

// Isyn[m0 + u][k][o][a][s] = Acc[u][4o + a][4k + s].
__global__ void k_slab_store(int n_in, int n_out, int m0, const double* Acc, double* Isyn) {
  const int R = 4 * n_in, Ro = 4 * n_out;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int o = blockIdx.y, u = blockIdx.z;
  if (c >= R) return;
  const int k = c >> 2, s = c & 3;
  for (int a = 0; a < 4; ++a)
    Isyn[(((size_t)(m0 + u) * n_in + k) * n_out + o) * 16 + 4 * a + s] =
        Acc[((size_t)u * Ro + 4 * o + a) * R + c];
}

void launch_slab_blocks(const OrderBatch& b, int first, const double* X, const double* Y,
                        const double* lam_re, const double* lam_im, const double* rtop4,
                        double* D, double* Uup, double* Ldn, cudaStream_t s) {
  dim3 grid((b.n + 127) / 128, b.N, b.n_units);
  k_slab_blocks<<<grid, 128, 0, s>>>(b.N, b.n, b.tau, first, X, Y, lam_re, lam_im, rtop4, D, Uup,
                                     Ldn);
}

void launch_slab_rhs(const OrderBatch& b, int first, const double* SD, const double* rtop4,
                     const double* pts, const double* Pd_prev, double* rhs, double* Pd_cur,
                     double* Zt, cudaStream_t s) {
  const int R = 4 * b.n_in;
  dim3 grid((R + 127) / 128, b.N, b.n_units);
  k_slab_rhs<<<grid, 128, 0, s>>>(b.N, b.n, R, b.sSD, b.tau, first, SD, rtop4, pts, Pd_prev, rhs,
                                  Pd_cur, Zt);
}

void launch_slab_scale_sd(const OrderBatch& b, double t, const double* pts, double* SD,
                          cudaStream_t s) {
  const int R = 4 * b.n_in;
  dim3 grid((R + 127) / 128, 2 * b.n, b.n_units);
  k_slab_scale_sd<<<grid, 128, 0, s>>>(b.N, b.n, R, b.sSD, t, pts, SD);
}

void launch_slab_accum(const OrderBatch& b, double t, const double* pts, const double* T1,
                       const double* Tq, const double* g0tab, double* Acc, int first,
                       cudaStream_t s) {
  dim3 grid((4 * b.n_in + 127) / 128, b.n_out, b.n_units);
  k_slab_accum<<<grid, 128, 0, s>>>(b.N, b.n_in, b.n_out, t, pts, T1, Tq, g0tab, Acc, first);
}

void launch_slab_store(const OrderBatch& b, const double* Acc, double* Isyn, cudaStream_t s) {
  dim3 grid((4 * b.n_in + 127) / 128, b.n_out, b.n_units);
  k_slab_store<<<grid, 128, 0, s>>>(b.n_in, b.n_out, b.m0, Acc, Isyn);
}

}  // namespace vrte
