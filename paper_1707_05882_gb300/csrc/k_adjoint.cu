// Step a9: adjoint of the BRDF table with respect to the layer parameters (albedo omega,
// optical thickness tau0, interface index n and the expansion coefficients of every l).
//
// Given G = dL/dF for the table F of one layer, every order m contributes
//   dL/dp = sum over the order's radiances  Ibar^m . dI^m/dp,  Ibar^m = synthesis^T G.
// Within one order the exiting radiance of Sec. 2.C depends on p through
//   (i)  the reduced operator B = [[0, F'], [E', 0]] of the transfer equation w' = B w + g,
//        w = [s; d] (Eqs. 41-45), whose eigen-decomposition carries the homogeneous modes;
//   (ii) everything after that decomposition: the beam source g = -[r; p] (Eq. 47), the
//        boundary conditions (Eqs. 49-56, with the dielectric top), the depth integrals of
//        the reconstruction (Eqs. 36, 38), the operators U+- and the direct term.
// Part (ii) is differentiated in plain reverse mode with the eigenpairs held fixed.
// Part (i) is not differentiated through the eigenvectors, whose derivative divides by
// eigenvalue gaps (the operators here have many exactly degenerate and complex eigenvalues):
// with the adjoint field lam(t) of the order's two-point problem,
//   -lam' = B^T lam + h(t),   h = the reconstruction weight exp(-t/mu_o)/mu_o [U+ U-]^T Ibar,
// lam(0) = P0^T nu0, lam(tau0) = -P1^T nu1 (nu = K^-T C-bar, the multipliers of the top and
// bottom conditions P0 w(0) = 0, P1 w(tau0) = 0), the gradient is
//   dL/dB = sum over columns of int_0^tau0 lam(t) w(t)^T dt = V^-T Omega V^T,
// where V holds the 2n eigenvectors of B ([x; -y] for -kappa, [x; y] for +kappa) and
// Omega_KJ integrates products of mode exponentials in closed form: divided differences
// (exp(-a tau0) - exp(-b tau0)) / (b - a) that stay finite when a = b. Mode space is complex
// (pairs of complex eigenvalues), stored in split real / imaginary planes.
//
// Interface derivatives come from dual-number versions of the table kernels (k_tables.cu);
// the albedo and interface derivatives of the assembled operators are taken by running the
// assembly kernels again on scaled or tangent inputs (each operator is linear in omega, in
// the beam and exit blocks, and bilinear in the tables at its two points).
#include <algorithm>

#include "vrte_internal.cuh"

namespace vrte {

// ----------------------------------------------------------------- small helpers
__device__ inline double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Adds the block-wide sums of a and b to *pa and *pb (one atomic each per block). Every
// thread of the block must call it; blockDim.x * blockDim.y is a multiple of 32.
__device__ inline void block_add2(double a, double b, double* pa, double* pb) {
  __shared__ double sa[32], sb[32];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int nw = (blockDim.x * blockDim.y) >> 5;
  a = warp_sum(a);
  b = warp_sum(b);
  if ((tid & 31) == 0) { sa[tid >> 5] = a; sb[tid >> 5] = b; }
  __syncthreads();
  if (tid < 32) {
    a = tid < nw ? sa[tid] : 0.0;
    b = tid < nw ? sb[tid] : 0.0;
    a = warp_sum(a);
    b = warp_sum(b);
    if (tid == 0) {
      if (pa && a != 0.0) atomicAdd(pa, a);
      if (pb && b != 0.0) atomicAdd(pb, b);
    }
  }
}

__device__ inline cd cadd(cd a, cd b) { return cd{a.r + b.r, a.i + b.i}; }
__device__ inline cd csub(cd a, cd b) { return cd{a.r - b.r, a.i - b.i}; }
__device__ inline cd cconj(cd a) { return cd{a.r, -a.i}; }
__device__ inline cd cscale(cd a, double f) { return cd{a.r * f, a.i * f}; }
// Re(conj(a) b)
__device__ inline double cdotr(cd a, cd b) { return a.r * b.r + a.i * b.i; }

// Phi1(z) = (1 - exp(-z tau)) / z = int_0^tau exp(-z t) dt and its z-derivative, by their
// Taylor series where |z tau| is small (no cancellation there).
__device__ inline void phi1_real(double z, double tau, double& ph, double& dph) {
  const double zt = z * tau;
  if (fabs(zt) < 1e-3) {
    ph = tau * (1.0 - zt * (1.0 / 2 - zt * (1.0 / 6 - zt * (1.0 / 24 - zt / 120))));
    dph = tau * tau * (-0.5 + zt * (1.0 / 3 - zt * (1.0 / 8 - zt * (1.0 / 30 - zt / 144))));
  } else {
    ph = -expm1(-zt) / z;
    dph = (tau * exp(-zt) - ph) / z;
  }
}

__device__ inline void phi1_cplx(cd z, double tau, cd& ph, cd& dph) {
  const cd zt{z.r * tau, z.i * tau};
  if (fabs(zt.r) + fabs(zt.i) < 1e-2) {
    // sum_k (-zt)^k / (k+1)!  and  sum_k k (-1)^k zt^(k-1) / (k+1)!
    cd s{0.0, 0.0}, ds{0.0, 0.0}, pw{1.0, 0.0}, pwm{1.0, 0.0};  // pw = (-zt)^k, pwm = (-zt)^(k-1)
    double fact = 1.0;                                            // (k+1)!
    for (int k = 0; k < 12; ++k) {
      fact *= (k + 1);
      s = cadd(s, cscale(pw, 1.0 / fact));
      if (k >= 1) {
        ds = cadd(ds, cscale(pwm, -(double)k / fact));  // k (-1)^k zt^(k-1) = -k (-zt)^(k-1)
        pwm = cmul(pwm, cd{-zt.r, -zt.i});
      }
      pw = cmul(pw, cd{-zt.r, -zt.i});
    }
    ph = cscale(s, tau);
    dph = cscale(ds, tau * tau);
  } else {
    const cd em = cexpm1v(cd{-zt.r, -zt.i});
    ph = cdivv(cd{-em.r, -em.i}, z);
    const cd e = cexpv(cd{-zt.r, -zt.i});
    dph = cdivv(csub(cscale(e, tau), ph), z);
  }
}

// Depth factors of the reconstruction (Eqs. 36, 38; same values as k_build_Hhat) and their
// derivatives with respect to tau0 and x = 1/mu_o:
//   gD = x Phi1(x + kappa)  (decaying mode),  gG = x exp(-x tau0) Phi1(kappa - x)  (growing).
struct DepthD {
  cd gD, gG, dD_dt, dD_dx, dG_dt, dG_dx;
};
__device__ inline DepthD depth_factors(cd kap, double x, double tau) {
  DepthD r;
  cd ph, dph;
  const cd a{x + kap.r, kap.i};
  phi1_cplx(a, tau, ph, dph);
  r.gD = cscale(ph, x);
  r.dD_dt = cscale(cexpv(cd{-a.r * tau, -a.i * tau}), x);
  r.dD_dx = cadd(ph, cscale(dph, x));
  // h = (e^{-x tau0} - e^{-kappa tau0}) / (kappa - x), taken as e^{-x tau0} Phi1(kappa - x)
  // when Re(kappa - x) >= 0 and as e^{-kappa tau0} Phi1(x - kappa) otherwise: Phi1 of an
  // argument with a negative real part overflows for thick layers (and the product with the
  // vanishing exponential is then NaN)
  const cd ek = cexpv(cd{-kap.r * tau, -kap.i * tau});
  const double ex = exp(-x * tau);
  cd h, dh_dx;
  if (kap.r - x >= 0.0) {
    phi1_cplx(cd{kap.r - x, kap.i}, tau, ph, dph);
    h = cscale(ph, ex);
    dh_dx = csub(cscale(h, -tau), cscale(dph, ex));
  } else {
    phi1_cplx(cd{x - kap.r, -kap.i}, tau, ph, dph);
    h = cmul(ph, ek);
    dh_dx = cmul(dph, ek);
  }
  r.gG = cscale(h, x);
  r.dG_dt = cscale(cadd(cscale(h, -x), ek), x);
  r.dG_dx = cadd(h, cscale(dh_dx, x));
  return r;
}

// Mode kappa_J of the 2n-mode list (J < n: decaying block, else growing; the second member
// of a complex pair holds the conjugate): from the planar kappa table kap[u][2][n].
__device__ inline cd kap_at(const double* kap, int n, int j) {
  return cd{kap[j], kap[n + j]};
}

// Reverse-mode 2x2 block of R_F: [[a, b], [b, a]] on (I, Q), [[c, d], [-d, c]] on (U, V).
__device__ inline double blkR(const double* q, int i, int j) {
  if (i < 2 && j < 2) return i == j ? q[0] : q[1];
  if (i >= 2 && j >= 2) return i == j ? q[2] : (i == 2 ? q[3] : -q[3]);
  return 0.0;
}

// ----------------------------------------------------------------- a8^T: synthesis transpose
// Ibar[m][k][o][a][s] = sum_j w_as(m, j) G[k][o][j][a][s] with the weights of the forward
// synthesis (cos on the (IQ, IQ) and (UV, UV) blocks, -sin on IQ rows / UV columns, +sin on
// UV rows / IQ columns). One CTA per (incident, outgoing) pair.
template <typename T>
__global__ void __launch_bounds__(128) k_synth_transpose(int M, int n_in, int n_out, int n_phi,
                                                         const T* __restrict__ G,
                                                         const double* __restrict__ wc,
                                                         const double* __restrict__ ws,
                                                         double* Ibar) {
  extern __shared__ double Gs[];  // [n_phi][16]
  const int pair = blockIdx.x;
  const int k = pair / n_out, o = pair - k * n_out;
  const T* src = G + (size_t)pair * n_phi * 16;
  for (int e = threadIdx.x; e < n_phi * 16; e += blockDim.x) Gs[e] = (double)src[e];
  __syncthreads();
  for (int e = threadIdx.x; e < M * 16; e += blockDim.x) {
    const int m = e >> 4, q = e & 15, a = q >> 2, b = q & 3;
    const bool same = (a < 2) == (b < 2);
    const double sg = a < 2 ? -1.0 : 1.0;
    const double* c = wc + (size_t)m * n_phi;
    const double* s = ws + (size_t)m * n_phi;
    double acc = 0.0;
    for (int j = 0; j < n_phi; ++j) acc = fma(same ? c[j] : sg * s[j], Gs[j * 16 + q], acc);
    Ibar[(((size_t)m * n_in + k) * n_out + o) * 16 + q] = acc;
  }
}

void launch_synth_transpose(int M, int n_in, int n_out, int n_phi, const void* G, int g_dtype,
                            const double* wc, const double* ws, double* Ibar, cudaStream_t s) {
  const size_t smem = (size_t)n_phi * 16 * sizeof(double);
  const unsigned pairs = (unsigned)((long long)n_in * n_out);
  if (g_dtype == VRTE_OUT_F64) {
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(k_synth_transpose<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
    k_synth_transpose<double><<<pairs, 128, smem, s>>>(M, n_in, n_out, n_phi, (const double*)G,
                                                       wc, ws, Ibar);
  } else {
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(k_synth_transpose<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
    k_synth_transpose<float><<<pairs, 128, smem, s>>>(M, n_in, n_out, n_phi, (const float*)G, wc,
                                                      ws, Ibar);
  }
}

// ----------------------------------------------------------------- reconstruction reverse
// Tb[u][4o+a][4k+s] = Ibar of order m0+u as the order's [4 n_out x 4 n_in] matrix, and
// G0 = Tb scaled by the direct/particular depth factor g0(o, k).
__global__ void k_bw_tb(OrderBatch b, const double* Ibar, const double* g0tab, double* Tb,
                        double* G0) {
  const int R = 4 * b.n_in, Ro = 4 * b.n_out;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y, u = blockIdx.z;
  if (c >= R) return;
  const int o = i >> 2, a = i & 3, k = c >> 2, s = c & 3;
  const double v = Ibar[(((size_t)(b.m0 + u) * b.n_in + k) * b.n_out + o) * 16 + 4 * a + s];
  const size_t idx = (size_t)u * Ro * R + (size_t)i * R + c;
  Tb[idx] = v;
  G0[idx] = v * g0tab[(size_t)o * b.n_in + k];
}

// Depth factor g0(o, k) = x Phi1(x + y), x = 1/mu_o, y = 1/mu0, multiplies the particular and
// direct parts. gbar = sum over the 4x4 block of Tb (Qp + T1 / g0), with Qp = [U+ U-][s; d]
// and T1 = g0 x direct term; contributes to tau0 and, through x and y, to n.
__global__ void k_bw_g0(OrderBatch b, const double* Tb, const double* Qp, const double* T1,
                        const double* pts, const double* dpts, double* acc) {
  const int R = 4 * b.n_in, Ro = 4 * b.n_out;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int o = blockIdx.y, u = blockIdx.z;
  double dt = 0.0, dn = 0.0;
  if (k < b.n_in) {
    const double muo = pts[b.N + b.n_in + o], mu0 = pts[b.N + k];
    const double x = 1.0 / muo, y = 1.0 / mu0, z = x + y;
    double ph, dph;
    phi1_real(z, b.tau, ph, dph);
    const double g0 = x * ph;
    double gb = 0.0;
    for (int a = 0; a < 4; ++a)
      for (int s = 0; s < 4; ++s) {
        const size_t idx = (size_t)u * Ro * R + (size_t)(4 * o + a) * R + 4 * k + s;
        gb += Tb[idx] * (Qp[idx] + T1[idx] / g0);
      }
    dt = gb * x * exp(-z * b.tau);
    const double gx = gb * (ph + x * dph), gy = gb * x * dph;
    dn = gx * (-dpts[b.N + b.n_in + o] * x * x) + gy * (-dpts[b.N + k] * y * y);
  }
  block_add2(dt, dn, acc + 1, acc + 2);
}

// Hhat = [(P1 - P2) gD | (P1 + P2) gG] in real form (k_build_Hhat). From Hb = dL/dHhat:
// P1b, P2b (real form) and the tau0 and mu_o (-> n) parts through the depth factors.
__global__ void k_bw_hhat(OrderBatch b, const double* Hb, const double* P1, const double* P2,
                          const double* kap, const double* pts, const double* dpts, double* P1b,
                          double* P2b, double* acc) {
  const int n = b.n, Ro = 4 * b.n_out;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int o = blockIdx.y, u = blockIdx.z;
  double dt = 0.0, dn = 0.0;
  const double* kp = kap + (size_t)u * 2 * n;
  // first member of a pair (Im kappa > 0) or a real mode; the conjugate member is skipped
  if (j < n && kp[n + j] >= 0.0) {
    const bool cplx = kp[n + j] > 0.0;
    const cd kj = kap_at(kp, n, j);
    const double muo = pts[b.N + b.n_in + o], x = 1.0 / muo;
    const DepthD g = depth_factors(kj, x, b.tau);
    double gx = 0.0;
    for (int ar = 0; ar < 4; ++ar) {
      const size_t row = (size_t)u * Ro + 4 * o + ar;
      const double* h = Hb + row * 2 * n;
      const cd vD{h[j], cplx ? h[j + 1] : 0.0}, vG{h[n + j], cplx ? h[n + j + 1] : 0.0};
      const cd p1{P1[row * n + j], cplx ? P1[row * n + j + 1] : 0.0};
      const cd p2{P2[row * n + j], cplx ? P2[row * n + j + 1] : 0.0};
      const cd hD = csub(p1, p2), hG = cadd(p1, p2);
      const cd hDb = cmul(vD, cconj(g.gD)), hGb = cmul(vG, cconj(g.gG));
      const cd p1b = cadd(hDb, hGb), p2b = csub(hGb, hDb);
      P1b[row * n + j] = p1b.r;
      P2b[row * n + j] = p2b.r;
      if (cplx) {
        P1b[row * n + j + 1] = p1b.i;
        P2b[row * n + j + 1] = p2b.i;
      }
      const cd gDb = cmul(vD, cconj(hD)), gGb = cmul(vG, cconj(hG));
      dt += cdotr(gDb, g.dD_dt) + cdotr(gGb, g.dG_dt);
      gx += cdotr(gDb, g.dD_dx) + cdotr(gGb, g.dG_dx);
    }
    dn = gx * (-dpts[b.N + b.n_in + o] * x * x);
  }
  block_add2(dt, dn, acc + 1, acc + 2);
}

// Boundary matrix (k_build_K): tau0 enters through exp(-kappa tau0) on the growing columns
// of the top rows and the decaying columns of the bottom rows, n through R_F in the top rows.
__global__ void k_bw_K(OrderBatch b, const double* Kb, const double* X, const double* Y,
                       const double* kap, const double* rtop4, const double* drtop4,
                       double* acc) {
  const int n = b.n, n2 = 2 * n;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y, u = blockIdx.z;
  double dt = 0.0, dn = 0.0;
  const double* kp = kap + (size_t)u * 2 * n;
  if (j < n && kp[n + j] >= 0.0) {
    const bool cplx = kp[n + j] > 0.0;
    const cd kj = kap_at(kp, n, j);
    const cd E = cexpv(cd{-kj.r * b.tau, -kj.i * b.tau});
    const double* Xb = X + (size_t)u * n * n;
    const double* Yb = Y + (size_t)u * n * n;
    cd pp[4], pm[4];
    for (int a = 0; a < 4; ++a) {
      const size_t idx = (size_t)(4 * i + a) * n + j;
      const cd xv{Xb[idx], cplx ? Xb[idx + 1] : 0.0}, yv{Yb[idx], cplx ? Yb[idx + 1] : 0.0};
      pp[a] = cscale(cadd(xv, yv), 0.5);
      pm[a] = cscale(csub(xv, yv), 0.5);
    }
    const double* R = rtop4 + 4 * i;
    const double* dR = drtop4 + 4 * i;
    const double* Kbu = Kb + (size_t)u * n2 * n2;
    const cd mk{-kj.r, -kj.i};
    for (int a = 0; a < 4; ++a) {
      const double sgn = a < 2 ? 1.0 : -1.0;
      cd rp{0.0, 0.0};
      for (int c = 0; c < 4; ++c) rp = cadd(rp, cscale(pp[c], blkR(R, a, c)));
      const cd topG = cmul(csub(cscale(pm[a], sgn), rp), E);
      const cd botD = cmul(pm[a], E);
      const size_t rt = (size_t)(4 * i + a) * n2, rb = (size_t)(n + 4 * i + a) * n2;
      const cd qTA{Kbu[rt + j], cplx ? Kbu[rt + j + 1] : 0.0};
      const cd qTB{Kbu[rt + n + j], cplx ? Kbu[rt + n + j + 1] : 0.0};
      const cd qBA{Kbu[rb + j], cplx ? Kbu[rb + j + 1] : 0.0};
      dt += cdotr(qTB, cmul(mk, topG)) + cdotr(qBA, cmul(mk, botD));
      // dK_top/dR_ab = -(phi-)_b on decaying columns, -(phi+ E)_b on growing columns
      for (int c = 0; c < 4; ++c) {
        const double d = blkR(dR, a, c);
        if (d != 0.0) dn -= d * (cdotr(qTA, pm[c]) + cdotr(qTB, cmul(pp[c], E)));
      }
    }
  }
  block_add2(dt, dn, acc + 1, acc + 2);
}

// Right-hand side of the boundary system (k_bc_rhs) reversed: nu = dL/drhs gives
// SDb += d[s; d], and the tau0, mu0 and R_F (-> n) parts.
__global__ void k_bw_rhs(OrderBatch b, const double* nu, const double* SD, double* SDb,
                         const double* rtop4, const double* drtop4, const double* pts,
                         const double* dpts, double* acc) {
  const int n = b.n, R = 4 * b.n_in;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y, u = blockIdx.z;
  double dt = 0.0, dn = 0.0;
  if (c < R) {
    const double* sv = SD + (size_t)u * b.sSD;
    const double* dv = sv + (size_t)n * R;
    const double* nt = nu + (size_t)u * 2 * n * R;
    const double* nb = nt + (size_t)n * R;
    double* sb = SDb + (size_t)u * 2 * n * R;
    double* dbp = sb + (size_t)n * R;
    double zp[4], vt[4], vb[4];
    for (int a = 0; a < 4; ++a) {
      const size_t idx = (size_t)(4 * i + a) * R + c;
      zp[a] = 0.5 * (sv[idx] + dv[idx]);
      vt[a] = nt[idx];
      vb[a] = nb[idx];
    }
    const double* Rm = rtop4 + 4 * i;
    const double* dR = drtop4 + 4 * i;
    const double mu0 = pts[b.N + (c >> 2)];
    const double att = exp(-b.tau / mu0);
    double attb = 0.0;
    for (int a = 0; a < 4; ++a) {
      const double dl = a < 2 ? 1.0 : -1.0;
      double rtv = 0.0;  // (R^T nu_top)_a
      for (int e = 0; e < 4; ++e) rtv += blkR(Rm, e, a) * vt[e];
      const double zpb = rtv - vb[a] * att, zmb = -vt[a];
      const size_t idx = (size_t)(4 * i + a) * R + c;
      sb[idx] += 0.5 * zpb + 0.5 * dl * zmb;
      dbp[idx] += 0.5 * zpb - 0.5 * dl * zmb;
      attb -= vb[a] * zp[a];
      for (int e = 0; e < 4; ++e) dn += vt[a] * zp[e] * blkR(dR, a, e);
    }
    dt = attb * (-att / mu0);
    dn += attb * att * b.tau / (mu0 * mu0) * dpts[b.N + (c >> 2)];
  }
  block_add2(dt, dn, acc + 1, acc + 2);
}

// d = mu0 (p - E's): pb = mu0 dbar, and the mu0 part sum dbar d / mu0.
__global__ void k_bw_part_d(OrderBatch b, const double* SD, const double* SDb, const double* pts,
                            const double* dpts, double* pb, double* acc) {
  const int n = b.n, R = 4 * b.n_in;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y, u = blockIdx.z;
  double dn = 0.0;
  if (c < R) {
    const size_t idx = (size_t)(n + i) * R + c;
    const double db = SDb[(size_t)u * 2 * n * R + idx], d = SD[(size_t)u * b.sSD + idx];
    const double mu0 = pts[b.N + (c >> 2)];
    pb[(size_t)u * n * R + (size_t)i * R + c] = mu0 * db;
    dn = db * d / mu0 * dpts[b.N + (c >> 2)];
  }
  block_add2(0.0, dn, nullptr, acc + 2);
}

// ys = (Lambda - 1/mu0^2)^-1 y (k_eigen_scale) reversed in place on ysb, with the mu0 part
// through c = 1/mu0^2 (ys: the forward's scaled values).
__global__ void k_bw_scale(OrderBatch b, const double* lam_re, const double* lam_im,
                           const double* ys, double* ysb, const double* pts, const double* dpts,
                           double* acc) {
  const int n = b.n, R = 4 * b.n_in;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y, u = blockIdx.z;
  double dn = 0.0;
  const double* lr = lam_re + (size_t)u * n;
  const double* li = lam_im + (size_t)u * n;
  if (c < R && li[j] >= 0.0) {
    const double mu0 = pts[b.N + (c >> 2)];
    const double cc = 1.0 / (mu0 * mu0);
    const size_t idx = (size_t)u * n * R + (size_t)j * R + c;
    double cb;
    if (li[j] == 0.0) {
      const double den = lr[j] - cc;
      cb = ysb[idx] * ys[idx] / den;
      ysb[idx] /= den;
    } else {
      const double a = lr[j] - cc, bb = li[j], den = a * a + bb * bb;
      const double y0 = ysb[idx], y1 = ysb[idx + R];
      // d ys / dc = ys / (a - i b) for the pair's complex value ys_j + i ys_{j+1}
      const cd q = cdivv(cd{ys[idx], ys[idx + R]}, cd{a, -bb});
      cb = y0 * q.r + y1 * q.i;
      ysb[idx] = (a * y0 + bb * y1) / den;
      ysb[idx + R] = (-bb * y0 + a * y1) / den;
    }
    dn = cb * (-2.0 * cc / mu0) * dpts[b.N + (c >> 2)];
  }
  block_add2(0.0, dn, nullptr, acc + 2);
}

// w = F'p - r/mu0: rb = -wb/mu0 and the mu0 part sum wb r / mu0^2.
__global__ void k_bw_part_w(OrderBatch b, const double* wb, const double* r, const double* pts,
                            const double* dpts, double* rb, double* acc) {
  const int n = b.n, R = 4 * b.n_in;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y, u = blockIdx.z;
  double dn = 0.0;
  if (c < R) {
    const size_t idx = (size_t)u * n * R + (size_t)i * R + c;
    const double mu0 = pts[b.N + (c >> 2)];
    rb[idx] = -wb[idx] / mu0;
    dn = wb[idx] * r[idx] / (mu0 * mu0) * dpts[b.N + (c >> 2)];
  }
  block_add2(0.0, dn, nullptr, acc + 2);
}

// ----------------------------------------------------------------- mode space (complex)
// kap[u][2][n] (planar) from the eigenvalues of F'E': kappa = sqrt(lambda), the second
// member of a pair the conjugate.
__global__ void k_bw_kappa(int n, int U, const double* lam_re, const double* lam_im,
                           double* kap) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int u = blockIdx.y;
  if (j >= n || u >= U) return;
  const double* lr = lam_re + (size_t)u * n;
  const double* li = lam_im + (size_t)u * n;
  cd k;
  if (li[j] >= 0.0) k = kappa_of(lr, li, j);
  else k = cconj(kappa_of(lr, li, j - 1));
  kap[(size_t)u * 2 * n + j] = k.r;
  kap[(size_t)u * 2 * n + n + j] = k.i;
}

// Complex eigenvector matrices from their real form, per node block of rows:
//   Xc, Yc; Pmc = (Xc - Yc)/2 = phi-; Gtc = D phi- - R_F phi+ (the growing modes' top rows).
// Planar: real plane at u * 2 n^2, imaginary plane n^2 further.
__global__ void k_bw_cplx_cols(OrderBatch b, const double* X, const double* Y, const double* kap,
                               const double* rtop4, double* Xc, double* Yc, double* Pmc,
                               double* Gtc) {
  const int n = b.n;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y, u = blockIdx.z;
  const double* kp = kap + (size_t)u * 2 * n;
  if (j >= n || kp[n + j] < 0.0) return;
  const bool cplx = kp[n + j] > 0.0;
  const size_t nn = (size_t)n * n, pl = (size_t)u * 2 * nn;
  cd xv[4], yv[4], pp[4], pm[4];
  for (int a = 0; a < 4; ++a) {
    const size_t idx = (size_t)u * nn + (size_t)(4 * i + a) * n + j;
    xv[a] = cd{X[idx], cplx ? X[idx + 1] : 0.0};
    yv[a] = cd{Y[idx], cplx ? Y[idx + 1] : 0.0};
    pp[a] = cscale(cadd(xv[a], yv[a]), 0.5);
    pm[a] = cscale(csub(xv[a], yv[a]), 0.5);
  }
  const double* R = rtop4 + 4 * i;
  for (int a = 0; a < 4; ++a) {
    cd rp{0.0, 0.0};
    for (int c = 0; c < 4; ++c) rp = cadd(rp, cscale(pp[c], blkR(R, a, c)));
    const cd gt = csub(cscale(pm[a], a < 2 ? 1.0 : -1.0), rp);
    const cd v[4] = {xv[a], yv[a], pm[a], gt};
    double* dst[4] = {Xc, Yc, Pmc, Gtc};
    const size_t e = pl + (size_t)(4 * i + a) * n + j;
    for (int q = 0; q < 4; ++q) {
      dst[q][e] = v[q].r;
      dst[q][e + nn] = v[q].i;
      if (cplx) {
        dst[q][e + 1] = v[q].r;
        dst[q][e + 1 + nn] = -v[q].i;
      }
    }
  }
}

// Rows of a mode-indexed real-form matrix A [rows][cols] (rows = blocks of n modes) to
// complex amplitudes: a pair (j, j+1) becomes ((A_j - i A_{j+1})/2, (A_j + i A_{j+1})/2),
// a real mode stays. Used for X^-1 (-> Xc^-1) and the boundary coefficients C.
__global__ void k_bw_cplx_rows(int n, int rows, int cols, long long sA, const double* A,
                               const double* kap, double* Z) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y, u = blockIdx.z;
  if (c >= cols) return;
  const int j = r % n;
  const double* kp = kap + (size_t)u * 2 * n;
  const double* Au = A + (size_t)u * sA;
  const size_t plane = (size_t)rows * cols;
  double* Zu = Z + (size_t)u * 2 * plane;
  const size_t e = (size_t)r * cols + c;
  const double im = kp[n + j];
  if (im == 0.0) {
    Zu[e] = Au[e];
    Zu[e + plane] = 0.0;
  } else if (im > 0.0) {
    Zu[e] = 0.5 * Au[e];
    Zu[e + plane] = -0.5 * Au[e + cols];
  } else {
    Zu[e] = 0.5 * Au[e - cols];
    Zu[e + plane] = 0.5 * Au[e];
  }
}

// Z <- diag(1/kappa) Z for a complex [n][cols] matrix (rows = modes).
__global__ void k_bw_rowdiv(int n, int cols, const double* kap, double* Z) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y, u = blockIdx.z;
  if (c >= cols) return;
  const size_t plane = (size_t)n * cols;
  double* Zu = Z + (size_t)u * 2 * plane;
  const cd k = kap_at(kap + (size_t)u * 2 * n, n, j);
  const size_t e = (size_t)j * cols + c;
  const cd v = cdivv(cd{Zu[e], Zu[e + plane]}, k);
  Zu[e] = v.r;
  Zu[e + plane] = v.i;
}

// zeta = V^-1 [s; d] = [(Ta - Tz)/2; (Ta + Tz)/2] with Ta = Xc^-1 s, Tz = Zc d ([n][R] each).
__global__ void k_bw_zeta(int n, int R, const double* Ta, const double* Tz, double* zeta) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y, u = blockIdx.z;
  if (c >= R) return;
  const size_t pl = (size_t)n * R, e = (size_t)j * R + c;
  const double* a = Ta + (size_t)u * 2 * pl;
  const double* z = Tz + (size_t)u * 2 * pl;
  double* zt = zeta + (size_t)u * 4 * pl;
  const size_t pz = 2 * pl;  // planes of zeta: [2n][R]
  zt[e] = 0.5 * (a[e] - z[e]);
  zt[e + pz] = 0.5 * (a[e + pl] - z[e + pl]);
  zt[pl + e] = 0.5 * (a[e] + z[e]);
  zt[pl + e + pz] = 0.5 * (a[e + pl] + z[e + pl]);
}

// Psi^T = U V ([Ro][2n], complex): decaying block P1c - P2c, growing block P1c + P2c, times
// alpha1 = 1/(x + kappa) (decaying) or 1/(x - kappa) (growing), x = 1/mu_o; PsiT2 carries
// alpha2 / mu_o with alpha2 = alpha1 exp(-x tau0) (decaying) or alpha1 (growing).
__global__ void k_bw_psi(OrderBatch b, const double* P1, const double* P2, const double* kap,
                         const double* pts, double* PsiT1, double* PsiT2) {
  const int n = b.n, Ro = 4 * b.n_out;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int row = blockIdx.y, u = blockIdx.z;
  const double* kp = kap + (size_t)u * 2 * n;
  if (j >= n || kp[n + j] < 0.0) return;
  const bool cplx = kp[n + j] > 0.0;
  const size_t r = (size_t)u * Ro + row;
  const cd p1{P1[r * n + j], cplx ? P1[r * n + j + 1] : 0.0};
  const cd p2{P2[r * n + j], cplx ? P2[r * n + j + 1] : 0.0};
  const cd kj = kap_at(kp, n, j);
  const double muo = pts[b.N + b.n_in + (row >> 2)], x = 1.0 / muo;
  const cd a1A = cdivv(cd{1.0, 0.0}, cd{x + kj.r, kj.i});
  const cd a1B = cdivv(cd{1.0, 0.0}, cd{x - kj.r, -kj.i});
  const cd pA = csub(p1, p2), pB = cadd(p1, p2);
  const cd v1A = cmul(pA, a1A), v1B = cmul(pB, a1B);
  const cd v2A = cscale(v1A, exp(-x * b.tau) * x), v2B = cscale(v1B, x);
  const size_t plane = (size_t)Ro * 2 * n;
  const size_t e = (size_t)u * 2 * plane + (size_t)row * 2 * n + j;
  const cd vals[4] = {v1A, v1B, v2A, v2B};
  double* dst[4] = {PsiT1, PsiT1 + n, PsiT2, PsiT2 + n};
  for (int q = 0; q < 4; ++q) {
    dst[q][e] = vals[q].r;
    dst[q][e + plane] = vals[q].i;
    if (cplx) {
      dst[q][e + 1] = vals[q].r;
      dst[q][e + 1 + plane] = -vals[q].i;
    }
  }
}

// Ahat[(o,a)][J] *= gf(o, J): the forward depth factor of mode J at outgoing o (gD for the
// decaying block, gG for the growing block).
__global__ void k_bw_gf(OrderBatch b, const double* kap, const double* pts, double* Ah) {
  const int n = b.n, Ro = 4 * b.n_out;
  const int J = blockIdx.x * blockDim.x + threadIdx.x;
  const int o = blockIdx.y, u = blockIdx.z;
  if (J >= 2 * n) return;
  const int j = J < n ? J : J - n;
  const cd kj = kap_at(kap + (size_t)u * 2 * n, n, j);
  const double x = 1.0 / pts[b.N + b.n_in + o];
  const DepthD g = depth_factors(kj, x, b.tau);
  const cd f = J < n ? g.gD : g.gG;
  const size_t plane = (size_t)Ro * 2 * n;
  double* A = Ah + (size_t)u * 2 * plane;
  for (int a = 0; a < 4; ++a) {
    const size_t e = (size_t)(4 * o + a) * 2 * n + J;
    const cd v = cmul(cd{A[e], A[e + plane]}, f);
    A[e] = v.r;
    A[e + plane] = v.i;
  }
}

// Integral over [0, tau0] of the adjoint mode function of K times the forward mode function of
// J (I1), for the 2n x 2n complex matrix Om (in place, Om *= I1):
//   same block:      (exp(-kK tau0) - exp(-kJ tau0)) / (kJ - kK) = exp(-kK tau0) Phi1(kJ - kK)
//                    (= exp(-kJ tau0) Phi1(kK - kJ), the form taken when Re(kJ - kK) < 0, so
//                    that Phi1 never sees an argument with a negative real part: it would
//                    overflow for thick layers, and its product with the vanishing
//                    exponential be NaN)
//   different block: Phi1(kK + kJ).
__global__ void k_bw_i1(int n, double tau, const double* kap, double* Om) {
  const int J = blockIdx.x * blockDim.x + threadIdx.x;
  const int K = blockIdx.y, u = blockIdx.z;
  if (J >= 2 * n) return;
  const double* kp = kap + (size_t)u * 2 * n;
  const cd kK = kap_at(kp, n, K < n ? K : K - n), kJ = kap_at(kp, n, J < n ? J : J - n);
  cd f, dph;
  if ((K < n) == (J < n)) {
    if (kJ.r - kK.r >= 0.0) {
      phi1_cplx(csub(kJ, kK), tau, f, dph);
      f = cmul(f, cexpv(cd{-kK.r * tau, -kK.i * tau}));
    } else {
      phi1_cplx(csub(kK, kJ), tau, f, dph);
      f = cmul(f, cexpv(cd{-kJ.r * tau, -kJ.i * tau}));
    }
  } else {
    phi1_cplx(cadd(kK, kJ), tau, f, dph);
  }
  const size_t plane = (size_t)4 * n * n;
  double* O = Om + (size_t)u * 2 * plane;
  const size_t e = (size_t)K * 2 * n + J;
  const cd v = cmul(cd{O[e], O[e + plane]}, f);
  O[e] = v.r;
  O[e + plane] = v.i;
}

// Dp2 = Dp * I2 with I2(K, c) = int_0^tau0 (adjoint mode function of K) exp(-t/mu0_c) dt:
//   decaying block exp(-y tau0) Phi1(kK - y) (= exp(-kK tau0) Phi1(y - kK), taken when
//   Re kK < y), growing block Phi1(kK + y), y = 1/mu0.
__global__ void k_bw_i2(OrderBatch b, const double* kap, const double* pts, const double* Dp,
                        double* Dp2) {
  const int n = b.n, R = 4 * b.n_in;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int K = blockIdx.y, u = blockIdx.z;
  if (c >= R) return;
  const cd kK = kap_at(kap + (size_t)u * 2 * n, n, K < n ? K : K - n);
  const double y = 1.0 / pts[b.N + (c >> 2)];
  cd f, dph;
  if (K < n) {
    if (kK.r - y >= 0.0) {
      phi1_cplx(cd{kK.r - y, kK.i}, b.tau, f, dph);
      f = cscale(f, exp(-y * b.tau));
    } else {
      phi1_cplx(cd{y - kK.r, -kK.i}, b.tau, f, dph);
      f = cmul(f, cexpv(cd{-kK.r * b.tau, -kK.i * b.tau}));
    }
  } else {
    phi1_cplx(cd{kK.r + y, kK.i}, b.tau, f, dph);
  }
  const size_t plane = (size_t)2 * n * R;
  const size_t e = (size_t)u * 2 * plane + (size_t)K * R + c;
  const cd v = cmul(cd{Dp[e], Dp[e + plane]}, f);
  Dp2[e] = v.r;
  Dp2[e + plane] = v.i;
}

// Blocks of Omega (decaying A, growing B) that the gradients of F' and E' need:
//   OmF = Om_AB + Om_BB - Om_AA - Om_BA,  OmE = Om_BA + Om_BB - Om_AA - Om_AB.
__global__ void k_bw_omblk(int n, const double* Om, double* OmF, double* OmE) {
  const int jj = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y, u = blockIdx.z;
  if (jj >= n) return;
  const size_t pO = (size_t)4 * n * n, pS = (size_t)n * n;
  const double* O = Om + (size_t)u * 2 * pO;
  double* F = OmF + (size_t)u * 2 * pS;
  double* E = OmE + (size_t)u * 2 * pS;
  const size_t n2 = 2 * n;
  for (int q = 0; q < 2; ++q) {
    const double* Oq = O + q * pO;
    const double aa = Oq[(size_t)i * n2 + jj], ab = Oq[(size_t)i * n2 + n + jj];
    const double ba = Oq[(size_t)(n + i) * n2 + jj], bb = Oq[(size_t)(n + i) * n2 + n + jj];
    F[q * pS + (size_t)i * n + jj] = ab + bb - aa - ba;
    E[q * pS + (size_t)i * n + jj] = ba + bb - aa - ab;
  }
}

// ----------------------------------------------------------------- parameter chain
// sum over the batch of scale * <A, B> (contiguous [count] per unit, unit strides sA, sB)
// into *dst.
__global__ void k_bw_dot(long long count, const double* A, long long sA, const double* B,
                         long long sB, double scale, double* dst) {
  const int u = blockIdx.y;
  double v = 0.0;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x)
    v += A[(size_t)u * sA + e] * B[(size_t)u * sB + e];
  block_add2(scale * v, 0.0, dst, nullptr);
}

// <Eb, dE'/domega> with dE'/domega = -(1/2)(I/mu_i - E2) and E2 = E' at omega = 2 (likewise F').
__global__ void k_bw_dot_ef(int n, int N, const double* Eb, const double* E2, const double* Fb,
                            const double* F2, const double* mu_nodes, double* acc) {
  const int u = blockIdx.y;
  const size_t nn = (size_t)n * n;
  double v = 0.0;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < nn;
       e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), jj = (int)(e % n);
    const double id = i == jj ? 1.0 / mu_nodes[i >> 2] : 0.0;
    v += -0.5 * (Eb[u * nn + e] * (id - E2[u * nn + e]) + Fb[u * nn + e] * (id - F2[u * nn + e]));
  }
  block_add2(v, 0.0, acc, nullptr);
}

// Gradients of the parity-split sums S+- at the four point-pair families, as the sum and the
// difference (Sg = S+bar + S-bar, Sd = S+bar - S-bar), each [4 nx][4 ny] per unit:
//   nodes x nodes   from E'bar, F'bar:  S+bar = -(omega/2) alpha_j E'bar / mu_i, S- with F'bar
__global__ void k_bw_sbar_nn(OrderBatch b, const double* Eb, const double* Fb,
                             const double* mu_nodes, const double* w_nodes, double* S) {
  const int n = b.n;
  const int jj = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y, u = blockIdx.z;
  if (jj >= n) return;
  const size_t nn = (size_t)n * n, e = (size_t)i * n + jj;
  const double f = -0.5 * b.omega * w_nodes[jj >> 2] / mu_nodes[i >> 2];
  const double sp = f * Eb[u * nn + e], sm = f * Fb[u * nn + e];
  S[u * 2 * nn + e] = sp + sm;
  S[u * 2 * nn + nn + e] = sp - sm;
}

//   nodes x incident from pb, rb:  S+bar(i,k) = (c/mu_i) pb(i,k) (D M_k)^T, S-bar = -(c/mu_i) rb ...
__global__ void k_bw_sbar_ni(OrderBatch b, const double* pb, const double* rb,
                             const double* mu_nodes, const double* min4, double* S) {
  const int n = b.n, R = 4 * b.n_in;
  const int cidx = blockIdx.x * blockDim.x + threadIdx.x;  // column (k, bb)
  const int row = blockIdx.y, u = blockIdx.z;             // row (i, a)
  if (cidx >= R) return;
  const int k = cidx >> 2, bb = cidx & 3;
  const double cq = b.omega / (2.0 * kPi) / mu_nodes[row >> 2];
  const double* q = min4 + 4 * k;
  const double dl = bb < 2 ? 1.0 : -1.0;
  const size_t base = (size_t)u * n * R + (size_t)row * R + 4 * k;
  double sp = 0.0, sm = 0.0;
  for (int s = 0; s < 4; ++s) {
    const double dm = dl * blkR(q, bb, s);
    sp += pb[base + s] * dm;
    sm -= rb[base + s] * dm;
  }
  const size_t nR = (size_t)n * R, e = (size_t)row * R + cidx;
  S[u * 2 * nR + e] = cq * (sp + sm);
  S[u * 2 * nR + nR + e] = cq * (sp - sm);
}

//   outgoing x nodes from Ub = [U+bar | U-bar]:  S+-bar(o,j) = (omega/4) alpha_j M_o^T U+-bar(o,j)
__global__ void k_bw_sbar_on(OrderBatch b, const double* Ub, const double* w_nodes,
                             const double* mout4, double* S) {
  const int n = b.n, Ro = 4 * b.n_out;
  const int col = blockIdx.x * blockDim.x + threadIdx.x;  // (j, c)
  const int row = blockIdx.y, u = blockIdx.z;            // (o, a)
  if (col >= n) return;
  const int o = row >> 2, a = row & 3;
  const double f = 0.25 * b.omega * w_nodes[col >> 2];
  const double* q = mout4 + 4 * o;
  double sp = 0.0, sm = 0.0;
  for (int e = 0; e < 4; ++e) {
    const size_t r = (size_t)u * Ro * 2 * n + (size_t)(4 * o + e) * 2 * n;
    const double mo = blkR(q, e, a);
    sp += mo * Ub[r + col];
    sm += mo * Ub[r + n + col];
  }
  const size_t pl = (size_t)Ro * n, idx = (size_t)row * n + col;
  S[u * 2 * pl + idx] = f * (sp + sm);
  S[u * 2 * pl + pl + idx] = f * (sp - sm);
}

//   outgoing x incident from G0 (the direct term, S+bar = -S-bar): only the difference,
//   Sd(o,k) = (omega/2pi) M_o^T G0(o,k) (D M_k)^T.
__global__ void k_bw_sbar_oi(OrderBatch b, const double* G0, const double* min4,
                             const double* mout4, double* S) {
  const int R = 4 * b.n_in, Ro = 4 * b.n_out;
  const int cidx = blockIdx.x * blockDim.x + threadIdx.x;  // (k, bb)
  const int row = blockIdx.y, u = blockIdx.z;             // (o, a)
  if (cidx >= R) return;
  const int o = row >> 2, a = row & 3, k = cidx >> 2, bb = cidx & 3;
  const double cq = b.omega / (2.0 * kPi);
  const double* qi = min4 + 4 * k;
  const double* qo = mout4 + 4 * o;
  const double dl = bb < 2 ? 1.0 : -1.0;
  double v = 0.0;
  for (int e = 0; e < 4; ++e) {
    const double mo = blkR(qo, e, a);
    if (mo == 0.0) continue;
    const size_t r = (size_t)u * Ro * R + (size_t)(4 * o + e) * R + 4 * k;
    double t = 0.0;
    for (int s = 0; s < 4; ++s) t += G0[r + s] * dl * blkR(qi, bb, s);
    v += mo * t;
  }
  S[(size_t)u * Ro * R + (size_t)row * R + cidx] = cq * v;
}

// PY[u][(y, b)][(l, d)] = P_l(y)_bd for the points y0 .. y0+ny-1 of the tables (zero for l < m),
// P = [[p, 0, 0, 0], [0, r, -t, 0], [0, -t, r, 0], [0, 0, 0, p]].
__global__ void k_bw_pstack(OrderBatch b, int y0, int ny, const double* pt, const double* rt,
                            const double* tt, double* PY) {
  const int L = b.L, L4 = 4 * L;
  const int col = blockIdx.x * blockDim.x + threadIdx.x;  // (l, d)
  const int row = blockIdx.y, u = blockIdx.z;            // (y, bb)
  if (col >= L4) return;
  const int l = col >> 2, d = col & 3, y = row >> 2, bb = row & 3;
  double v = 0.0;
  if (l >= b.m0 + u) {
    const size_t t = ((size_t)u * L + l) * b.P + y0 + y;
    const double p = pt[t], r = rt[t], tv = tt[t];
    if (bb == d) v = (bb == 0 || bb == 3) ? p : r;
    else if ((bb == 1 && d == 2) || (bb == 2 && d == 1)) v = -tv;
  }
  PY[(size_t)u * 4 * ny * L4 + (size_t)row * L4 + col] = v;
}

// B_l bar = sum_x P_l(x)^T (Qg(x) + (-1)^(l-m) Qd(x) D), Q = Sbar . PY of one point family
// (Qg the sum rows, Qd the difference rows, each [4 nx][4L]); converted to the coefficient
// gradient (alpha1..alpha4, beta1, beta2) of B_l = [[a1, b1, 0, 0], [b1, a2, 0, 0],
// [0, 0, a3, b2], [0, 0, -b2, a4]] and added to acc[3 + 6 l + q].
__global__ void k_bw_bbar(OrderBatch b, int x0, int nx, const double* Qg, const double* Qd,
                          long long sQ, const double* pt, const double* rt, const double* tt,
                          double* acc) {
  const int L = b.L, L4 = 4 * L;
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  const int u = blockIdx.y;
  const int m = b.m0 + u;
  if (l >= L || l < m) return;
  const double par = ((l - m) & 1) ? -1.0 : 1.0;
  double B[4][4] = {};
  const double* qg = Qg ? Qg + (size_t)u * sQ : nullptr;
  const double* qd = Qd ? Qd + (size_t)u * sQ : nullptr;
  for (int x = 0; x < nx; ++x) {
    const size_t t = ((size_t)u * L + l) * b.P + x0 + x;
    const double p = pt[t], r = rt[t], tv = tt[t];
    const double P[4][4] = {{p, 0, 0, 0}, {0, r, -tv, 0}, {0, -tv, r, 0}, {0, 0, 0, p}};
    for (int a = 0; a < 4; ++a) {
      const size_t row = (size_t)(4 * x + a) * L4 + 4 * l;
      double q[4];
      for (int d = 0; d < 4; ++d)
        q[d] = (qg ? qg[row + d] : 0.0) + (qd ? par * (d < 2 ? 1.0 : -1.0) * qd[row + d] : 0.0);
      for (int ap = 0; ap < 4; ++ap) {
        const double pa = P[a][ap];
        if (pa == 0.0) continue;
        for (int d = 0; d < 4; ++d) B[ap][d] += pa * q[d];
      }
    }
  }
  double* g = acc + 3 + 6 * l;
  atomicAdd(g + 0, B[0][0]);
  atomicAdd(g + 1, B[1][1]);
  atomicAdd(g + 2, B[2][2]);
  atomicAdd(g + 3, B[3][3]);
  atomicAdd(g + 4, B[0][1] + B[1][0]);
  atomicAdd(g + 5, B[2][3] - B[3][2]);
}

// Writes one layer's gradient row [3 + 6 Lmax]: (omega, tau0, n, coefficients), the interface
// entry zero without an interface and the coefficients beyond the layer's L zero.
__global__ void k_bw_finish(int L, int Lmax, double nif, const double* acc, double* grad) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 3 + 6 * Lmax) return;
  double v = 0.0;
  if (e < 3) v = (e == 2 && !(nif > 1.0)) ? 0.0 : acc[e];
  else if (e < 3 + 6 * L) v = acc[e];
  grad[e] = v;
}

// ----------------------------------------------------------------- launchers
namespace {
inline dim3 g3(long long x, int y, int z, int bx = 128) {
  return dim3((unsigned)((x + bx - 1) / bx), (unsigned)y, (unsigned)z);
}
}  // namespace

void bw_tb(const OrderBatch& b, const double* Ibar, const double* g0tab, double* Tb, double* G0,
           cudaStream_t s) {
  k_bw_tb<<<g3(4 * b.n_in, 4 * b.n_out, b.n_units), 128, 0, s>>>(b, Ibar, g0tab, Tb, G0);
}
void bw_g0(const OrderBatch& b, const double* Tb, const double* Qp, const double* T1,
           const double* pts, const double* dpts, double* acc, cudaStream_t s) {
  k_bw_g0<<<g3(b.n_in, b.n_out, b.n_units), 128, 0, s>>>(b, Tb, Qp, T1, pts, dpts, acc);
}
void bw_kappa(const OrderBatch& b, const double* lam_re, const double* lam_im, double* kap,
              cudaStream_t s) {
  k_bw_kappa<<<dim3((b.n + 127) / 128, b.n_units), 128, 0, s>>>(b.n, b.n_units, lam_re, lam_im,
                                                                 kap);
}
void bw_hhat(const OrderBatch& b, const double* Hb, const double* P1, const double* P2,
             const double* kap, const double* pts, const double* dpts, double* P1b, double* P2b,
             double* acc, cudaStream_t s) {
  k_bw_hhat<<<g3(b.n, b.n_out, b.n_units), 128, 0, s>>>(b, Hb, P1, P2, kap, pts, dpts, P1b, P2b,
                                                        acc);
}
void bw_K(const OrderBatch& b, const double* Kb, const double* X, const double* Y,
          const double* kap, const double* rtop4, const double* drtop4, double* acc,
          cudaStream_t s) {
  k_bw_K<<<g3(b.n, b.N, b.n_units), 128, 0, s>>>(b, Kb, X, Y, kap, rtop4, drtop4, acc);
}
void bw_rhs(const OrderBatch& b, const double* nu, const double* SD, double* SDb,
            const double* rtop4, const double* drtop4, const double* pts, const double* dpts,
            double* acc, cudaStream_t s) {
  k_bw_rhs<<<g3(4 * b.n_in, b.N, b.n_units), 128, 0, s>>>(b, nu, SD, SDb, rtop4, drtop4, pts, dpts,
                                                          acc);
}
void bw_part_d(const OrderBatch& b, const double* SD, const double* SDb, const double* pts,
               const double* dpts, double* pb, double* acc, cudaStream_t s) {
  k_bw_part_d<<<g3(4 * b.n_in, b.n, b.n_units), 128, 0, s>>>(b, SD, SDb, pts, dpts, pb, acc);
}
void bw_scale(const OrderBatch& b, const double* lam_re, const double* lam_im, const double* ys,
              double* ysb, const double* pts, const double* dpts, double* acc, cudaStream_t s) {
  k_bw_scale<<<g3(4 * b.n_in, b.n, b.n_units), 128, 0, s>>>(b, lam_re, lam_im, ys, ysb, pts, dpts,
                                                            acc);
}
void bw_part_w(const OrderBatch& b, const double* wb, const double* r, const double* pts,
               const double* dpts, double* rb, double* acc, cudaStream_t s) {
  k_bw_part_w<<<g3(4 * b.n_in, b.n, b.n_units), 128, 0, s>>>(b, wb, r, pts, dpts, rb, acc);
}
void bw_cplx_cols(const OrderBatch& b, const double* X, const double* Y, const double* kap,
                  const double* rtop4, double* Xc, double* Yc, double* Pmc, double* Gtc,
                  cudaStream_t s) {
  k_bw_cplx_cols<<<g3(b.n, b.N, b.n_units), 128, 0, s>>>(b, X, Y, kap, rtop4, Xc, Yc, Pmc, Gtc);
}
void bw_cplx_rows(int n, int rows, int cols, long long sA, const double* A, const double* kap,
                  double* Z, int units, cudaStream_t s) {
  k_bw_cplx_rows<<<g3(cols, rows, units), 128, 0, s>>>(n, rows, cols, sA, A, kap, Z);
}
void bw_rowdiv(int n, int cols, const double* kap, double* Z, int units, cudaStream_t s) {
  k_bw_rowdiv<<<g3(cols, n, units), 128, 0, s>>>(n, cols, kap, Z);
}
void bw_zeta(int n, int R, const double* Ta, const double* Tz, double* zeta, int units,
             cudaStream_t s) {
  k_bw_zeta<<<g3(R, n, units), 128, 0, s>>>(n, R, Ta, Tz, zeta);
}
void bw_psi(const OrderBatch& b, const double* P1, const double* P2, const double* kap,
            const double* pts, double* PsiT1, double* PsiT2, cudaStream_t s) {
  k_bw_psi<<<g3(b.n, 4 * b.n_out, b.n_units), 128, 0, s>>>(b, P1, P2, kap, pts, PsiT1, PsiT2);
}
void bw_gf(const OrderBatch& b, const double* kap, const double* pts, double* Ah, cudaStream_t s) {
  k_bw_gf<<<g3(2 * b.n, b.n_out, b.n_units), 128, 0, s>>>(b, kap, pts, Ah);
}
void bw_i1(int n, double tau, const double* kap, double* Om, int units, cudaStream_t s) {
  k_bw_i1<<<g3(2 * n, 2 * n, units), 128, 0, s>>>(n, tau, kap, Om);
}
void bw_i2(const OrderBatch& b, const double* kap, const double* pts, const double* Dp,
           double* Dp2, cudaStream_t s) {
  k_bw_i2<<<g3(4 * b.n_in, 2 * b.n, b.n_units), 128, 0, s>>>(b, kap, pts, Dp, Dp2);
}
void bw_omblk(int n, const double* Om, double* OmF, double* OmE, int units, cudaStream_t s) {
  k_bw_omblk<<<g3(n, n, units), 128, 0, s>>>(n, Om, OmF, OmE);
}
void bw_dot(long long count, const double* A, long long sA, const double* B, long long sB,
            double scale, double* dst, int units, cudaStream_t s) {
  const int blocks = (int)std::min<long long>((count + 255) / 256, 256);
  k_bw_dot<<<dim3(blocks, units), 256, 0, s>>>(count, A, sA, B, sB, scale, dst);
}
void bw_dot_ef(int n, int N, const double* Eb, const double* E2, const double* Fb,
               const double* F2, const double* mu_nodes, double* acc, int units, cudaStream_t s) {
  const int blocks = (int)std::min<long long>(((long long)n * n + 255) / 256, 128);
  k_bw_dot_ef<<<dim3(blocks, units), 256, 0, s>>>(n, N, Eb, E2, Fb, F2, mu_nodes, acc);
}
void bw_sbar_nn(const OrderBatch& b, const double* Eb, const double* Fb, const double* mu_nodes,
                const double* w_nodes, double* S, cudaStream_t s) {
  k_bw_sbar_nn<<<g3(b.n, b.n, b.n_units), 128, 0, s>>>(b, Eb, Fb, mu_nodes, w_nodes, S);
}
void bw_sbar_ni(const OrderBatch& b, const double* pb, const double* rb, const double* mu_nodes,
                const double* min4, double* S, cudaStream_t s) {
  k_bw_sbar_ni<<<g3(4 * b.n_in, b.n, b.n_units), 128, 0, s>>>(b, pb, rb, mu_nodes, min4, S);
}
void bw_sbar_on(const OrderBatch& b, const double* Ub, const double* w_nodes, const double* mout4,
                double* S, cudaStream_t s) {
  k_bw_sbar_on<<<g3(b.n, 4 * b.n_out, b.n_units), 128, 0, s>>>(b, Ub, w_nodes, mout4, S);
}
void bw_sbar_oi(const OrderBatch& b, const double* G0, const double* min4, const double* mout4,
                double* S, cudaStream_t s) {
  k_bw_sbar_oi<<<g3(4 * b.n_in, 4 * b.n_out, b.n_units), 128, 0, s>>>(b, G0, min4, mout4, S);
}
void bw_pstack(const OrderBatch& b, int y0, int ny, const double* pt, const double* rt,
               const double* tt, double* PY, cudaStream_t s) {
  k_bw_pstack<<<g3(4 * b.L, 4 * ny, b.n_units), 128, 0, s>>>(b, y0, ny, pt, rt, tt, PY);
}
void bw_bbar(const OrderBatch& b, int x0, int nx, const double* Qg, const double* Qd,
             long long sQ, const double* pt, const double* rt, const double* tt, double* acc,
             cudaStream_t s) {
  k_bw_bbar<<<dim3((b.L + 63) / 64, b.n_units), 64, 0, s>>>(b, x0, nx, Qg, Qd, sQ, pt, rt, tt,
                                                            acc);
}
void bw_finish(int L, int Lmax, double nif, const double* acc, double* grad, cudaStream_t s) {
  const int cnt = 3 + 6 * Lmax;
  k_bw_finish<<<(cnt + 127) / 128, 128, 0, s>>>(L, Lmax, nif, acc, grad);
}

}  // namespace vrte
