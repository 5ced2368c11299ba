// Elementwise mode algebra between the dense stages (steps a2-a7).
//
// Reduced form used throughout (tau downward, mu > 0 upward; a = I(+mu), b = D I(-mu)):
//   s = a + b, d = a - b satisfy d' = E' s, s' = F' d, so s'' = F'E' s (Sec. 3.A, Eq. 43).
// For an eigenpair (lambda, x) of F'E' with kappa = sqrt(lambda) (principal branch) and
// y = E' x / kappa, phi+- = (x +- y)/2 (Eq. 45):
//   decaying mode (coefficient A_j, basis exp(-kappa tau)):       I(+mu) = phi-, I(-mu) = D phi+
//   growing mode  (coefficient B_j, basis exp(-kappa (tau0-tau))): I(+mu) = phi+, I(-mu) = D phi-
// which is the scaled homogeneous solution of Eqs. 24-25. A complex pair (j, j+1) is
// stored in real form: column j holds the real part, column j+1 the imaginary part of
// the complex mode of lambda_j (Im lambda_j > 0).
#include "vrte_internal.cuh"

namespace vrte {

// ------------------------------------------------------------------ Y = E'X / kappa
__global__ void k_pack_Y(int n, const double* EX, const double* lam_re, const double* lam_im,
                         double* Y, unsigned* status) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  int i = blockIdx.y, u = blockIdx.z;
  if (j >= n) return;
  const double* lr = lam_re + (size_t)u * n;
  const double* li = lam_im + (size_t)u * n;
  if (li[j] < 0.0) return;
  size_t row = (size_t)u * n * n + (size_t)i * n;
  if (li[j] == 0.0) {
    if (!(lr[j] > 0.0)) {
      if (i == 0) atomicOr(status, ST_NONFINITE);
      Y[row + j] = 0.0;
      return;
    }
    Y[row + j] = EX[row + j] / sqrt(lr[j]);
  } else {
    cd k = kappa_of(lr, li, j);
    cd y = cdivv(cd{EX[row + j], EX[row + j + 1]}, k);
    Y[row + j] = y.r;
    Y[row + j + 1] = y.i;
  }
}

void launch_pack_Y(const OrderBatch& b, const double* EX, const double* lam_re,
                   const double* lam_im, double* Y, cudaStream_t s) {
  dim3 grid((b.n + 127) / 128, b.n, b.n_units);
  k_pack_Y<<<grid, 128, 0, s>>>(b.n, EX, lam_re, lam_im, Y, b.status);
}

// ------------------------------------------------------------------ boundary matrix
// Rows 0..n-1: top condition I(0, -mu_i) - R_F(mu_i) I(0, +mu_i) = 0 (Eq. 49; R_F = 0
// without an interface). Rows n..2n-1: black base I(tau0, +mu_i) = 0 (Eq. 50).
// Columns 0..n-1: decaying modes, n..2n-1: growing modes (Eqs. 51-56).
__global__ void k_build_K(int N, int n, double tau, const double* X, const double* Y,
                          const double* lam_re, const double* lam_im, const double* rtop4,
                          double* K) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  int i = blockIdx.y, u = blockIdx.z;
  if (j >= n) return;
  const double* lr = lam_re + (size_t)u * n;
  const double* li = lam_im + (size_t)u * n;
  if (li[j] < 0.0) return;
  bool cplx = li[j] > 0.0;
  cd kap = kappa_of(lr, li, j);
  cd E = cexpv(cd{-kap.r * tau, -kap.i * tau});
  const double* Xb = X + (size_t)u * n * n;
  const double* Yb = Y + (size_t)u * n * n;
  cd pp[4], pm[4];
  for (int a = 0; a < 4; ++a) {
    size_t idx = (size_t)(4 * i + a) * n + j;
    cd x{Xb[idx], cplx ? Xb[idx + 1] : 0.0};
    cd y{Yb[idx], cplx ? Yb[idx + 1] : 0.0};
    pp[a] = cd{0.5 * (x.r + y.r), 0.5 * (x.i + y.i)};
    pm[a] = cd{0.5 * (x.r - y.r), 0.5 * (x.i - y.i)};
  }
  const double* R = rtop4 + 4 * i;
  auto rmul = [&](const cd* v, int a) -> cd {
    // (R_F v)_a with R_F = [[ra, rb, 0, 0], [rb, ra, 0, 0], [0, 0, rc, rd], [0, 0, -rd, rc]]
    if (a == 0) return cd{R[0] * v[0].r + R[1] * v[1].r, R[0] * v[0].i + R[1] * v[1].i};
    if (a == 1) return cd{R[1] * v[0].r + R[0] * v[1].r, R[1] * v[0].i + R[0] * v[1].i};
    if (a == 2) return cd{R[2] * v[2].r + R[3] * v[3].r, R[2] * v[2].i + R[3] * v[3].i};
    return cd{-R[3] * v[2].r + R[2] * v[3].r, -R[3] * v[2].i + R[2] * v[3].i};
  };
  double* Kb = K + (size_t)u * (2 * n) * (2 * n);
  int n2 = 2 * n;
  for (int a = 0; a < 4; ++a) {
    double sgn = a < 2 ? 1.0 : -1.0;
    cd rm = rmul(pm, a), rp = rmul(pp, a);
    cd topD{sgn * pp[a].r - rm.r, sgn * pp[a].i - rm.i};
    cd topG = cmul(cd{sgn * pm[a].r - rp.r, sgn * pm[a].i - rp.i}, E);
    cd botD = cmul(pm[a], E);
    cd botG = pp[a];
    size_t rt = (size_t)(4 * i + a) * n2, rb = (size_t)(n + 4 * i + a) * n2;
    Kb[rt + j] = topD.r;
    Kb[rt + n + j] = topG.r;
    Kb[rb + j] = botD.r;
    Kb[rb + n + j] = botG.r;
    if (cplx) {
      Kb[rt + j + 1] = topD.i;
      Kb[rt + n + j + 1] = topG.i;
      Kb[rb + j + 1] = botD.i;
      Kb[rb + n + j + 1] = botG.i;
    }
  }
}

void launch_build_K(const OrderBatch& b, const double* X, const double* Y, const double* lam_re,
                    const double* lam_im, const double* rtop4, double* K, cudaStream_t s) {
  dim3 grid((b.n + 127) / 128, b.N, b.n_units);
  k_build_K<<<grid, 128, 0, s>>>(b.N, b.n, b.tau, X, Y, lam_re, lam_im, rtop4, K);
}

// ------------------------------------------------------------------ particular solution
// Reduced particular problem (Sec. 3.B, Eqs. 46-48) for beam column c = 4k + s with
// internal cosine mu0 = pts[N + k]:  (F'E' - 1/mu0^2) s = F' p - r / mu0,
// d = mu0 (p - E' s), Z+ = (s + d)/2, Z- = D (s - d)/2.
// (btab: the layer's beam table, 1/mu0 per incident cosine at btab[n_in + k])
__global__ void k_particular_rhs(int n, int R, int n_in, const double* r, const double* btab,
                                 double* w) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  int i = blockIdx.y, u = blockIdx.z;
  if (c >= R) return;
  size_t idx = (size_t)u * n * R + (size_t)i * R + c;
  w[idx] = fma(-r[idx], btab[n_in + (c >> 2)], w[idx]);
}

void launch_particular_rhs(const OrderBatch& b, const double* w_in, const double* r,
                           const double* btab, double* w_out, cudaStream_t s) {
  (void)w_in;
  int R = 4 * b.n_in;
  dim3 grid((R + 127) / 128, b.n, b.n_units);
  k_particular_rhs<<<grid, 128, 0, s>>>(b.n, R, b.n_in, r, btab, w_out);
}

// y <- (Lambda - 1/mu0^2)^-1 y in the eigenbasis; a pair uses the real 2x2 block
// [[a, b], [-b, a]] of lambda = a + ib. One thread per (u, j, incident k): the factor is
// formed once (one FP64 division) for the four Stokes columns of k (btab: 1/mu0 at
// btab[n_in + k]).
__global__ void k_eigen_scale(int n, int R, int n_in, const double* lam_re, const double* lam_im,
                              const double* btab, double* y) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y, u = blockIdx.z;
  if (k >= n_in) return;
  const double* lr = lam_re + (size_t)u * n;
  const double* li = lam_im + (size_t)u * n;
  if (li[j] < 0.0) return;
  const double rm = btab[n_in + k];
  const double cc = rm * rm;
  double* yr = y + (size_t)u * n * R + (size_t)j * R + 4 * k;
  if (li[j] == 0.0) {
    const double f = 1.0 / (lr[j] - cc);
    for (int s = 0; s < 4; ++s) yr[s] *= f;
  } else {
    const double a = lr[j] - cc, bb = li[j];
    const double inv = 1.0 / fma(a, a, bb * bb);
    const double fa = a * inv, fb = bb * inv;
    for (int s = 0; s < 4; ++s) {
      const double y0 = yr[s], y1 = yr[R + s];
      yr[s] = fma(fa, y0, -fb * y1);
      yr[R + s] = fma(fb, y0, fa * y1);
    }
  }
}

void launch_eigen_scale(const OrderBatch& b, const double* lam_re, const double* lam_im,
                        const double* btab, double* y, cudaStream_t s) {
  int R = 4 * b.n_in;
  dim3 grid((b.n_in + 127) / 128, b.n, b.n_units);
  k_eigen_scale<<<grid, 128, 0, s>>>(b.n, R, b.n_in, lam_re, lam_im, btab, y);
}

// d = mu0 (p - E's), written into the second half of SD = [s; d].
__global__ void k_particular_sd(int n, int R, int N, long long sSD, const double* pbeam,
                                const double* Es, const double* pts, double* SD) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  int i = blockIdx.y, u = blockIdx.z;
  if (c >= R) return;
  size_t idx = (size_t)u * n * R + (size_t)i * R + c;
  double mu0 = pts[N + (c >> 2)];
  SD[(size_t)u * sSD + (size_t)(n + i) * R + c] = mu0 * (pbeam[idx] - Es[idx]);
}

void launch_particular_sd(const OrderBatch& b, const double* pbeam, const double* Es,
                          const double* pts, double* SD, cudaStream_t s) {
  int R = 4 * b.n_in;
  dim3 grid((R + 127) / 128, b.n, b.n_units);
  k_particular_sd<<<grid, 128, 0, s>>>(b.n, R, b.N, b.sSD, pbeam, Es, pts, SD);
}

// Right-hand side of the boundary system (Eq. 54 with the dielectric top):
//   top:    -(Z-(mu_i) - R_F Z+(mu_i))
//   bottom: -Z+(mu_i) exp(-tau0 / mu0)
__global__ void k_bc_rhs(int N, int n, int R, long long sSD, const double* SD,
                         const double* rtop4, const double* btab, double* rhs) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  int i = blockIdx.y, u = blockIdx.z;
  if (c >= R) return;
  const double* sv = SD + (size_t)u * sSD;
  const double* dv = sv + (size_t)n * R;
  double zp[4], zm[4];
  for (int a = 0; a < 4; ++a) {
    size_t idx = (size_t)(4 * i + a) * R + c;
    double s = sv[idx], d = dv[idx];
    zp[a] = 0.5 * (s + d);
    zm[a] = (a < 2 ? 0.5 : -0.5) * (s - d);
  }
  const double* Rm = rtop4 + 4 * i;
  double rz[4] = {Rm[0] * zp[0] + Rm[1] * zp[1], Rm[1] * zp[0] + Rm[0] * zp[1],
                  Rm[2] * zp[2] + Rm[3] * zp[3], -Rm[3] * zp[2] + Rm[2] * zp[3]};
  const double att = btab[c >> 2];  // e^{-tau0/mu0}
  double* rb = rhs + (size_t)u * 2 * n * R;
  for (int a = 0; a < 4; ++a) {
    rb[(size_t)(4 * i + a) * R + c] = -(zm[a] - rz[a]);
    rb[(size_t)(n + 4 * i + a) * R + c] = -zp[a] * att;
  }
}

void launch_bc_rhs(const OrderBatch& b, const double* SD, const double* d, const double* rtop4,
                   const double* btab, double* rhs, cudaStream_t s) {
  (void)d;
  int R = 4 * b.n_in;
  dim3 grid((R + 127) / 128, b.N, b.n_units);
  k_bc_rhs<<<grid, 128, 0, s>>>(b.N, b.n, R, b.sSD, SD, rtop4, btab, rhs);
}

// ------------------------------------------------------------------ reconstruction operator
// For outgoing mu (row 4o + a) the homogeneous modes contribute (Eqs. 36, 38)
//   H_mode(mu) g_mode(mu) with H_D = U+ x - U- y, H_G = U+ x + U- y (P1 = U+ X, P2 = U- Y),
//   g_D = int_0^tau0 exp(-kappa t) exp(-t/mu) dt / mu = (1 - e^{-a tau0}) / (mu a), a = 1/mu + kappa
//   g_G = int_0^tau0 exp(-kappa (tau0 - t)) exp(-t/mu) dt / mu
//       = e^{-tau0/mu} (1 - e^{-b tau0}) / (mu b), b = kappa - 1/mu (limit tau0 e^{-tau0/mu}/mu).
constexpr int HHAT_OB = 16;  // outgoing cosines per block of k_build_Hhat

__global__ void k_build_Hhat(int N, int n, int n_in, int n_out, double tau, const double* P1,
                             const double* P2, const double* lam_re, const double* lam_im,
                             const double* pts, double* Hhat) {
  // one thread per mode j for HHAT_OB outgoing cosines o: the depth factors depend on (o, j)
  // only and are applied to the four rows 4o .. 4o+3. The exponentials factor,
  // e^{-a tau0} = e^{-tau0/mu} e^{-kappa tau0}: e^{-kappa tau0} once per thread and
  // e^{-tau0/mu} once per block (FP64 transcendentals are expensive on this part); the
  // expm1 forms stay where 1 - e^{-x} would cancel.
  __shared__ double s_mu[HHAT_OB], s_x[HHAT_OB], s_ex[HHAT_OB];
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int o0 = blockIdx.y * HHAT_OB, u = blockIdx.z;
  if (threadIdx.x < HHAT_OB && o0 + (int)threadIdx.x < n_out) {
    const double mu = pts[N + n_in + o0 + threadIdx.x];
    s_mu[threadIdx.x] = mu;
    s_x[threadIdx.x] = 1.0 / mu;
    s_ex[threadIdx.x] = exp(-tau / mu);
  }
  __syncthreads();
  if (j >= n) return;
  const double* lr = lam_re + (size_t)u * n;
  const double* li = lam_im + (size_t)u * n;
  if (li[j] < 0.0) return;
  const bool cplx = li[j] > 0.0;
  const int Ro = 4 * n_out;
  const cd kap = kappa_of(lr, li, j);
  const cd ek = cexpv(cd{-kap.r * tau, -kap.i * tau});
  for (int oo = 0; oo < HHAT_OB; ++oo) {
    const int o = o0 + oo;
    if (o >= n_out) break;
    const double mu = s_mu[oo], x = s_x[oo], ex = s_ex[oo];
    // decaying: 1 - e^{-a tau0} = 1 - e^{-tau0/mu} e^{-kappa tau0} without cancellation once
    // Re(a) tau0 > 1/2 (|e^{-a tau0}| < 0.61)
    const cd a{x + kap.r, kap.i};
    cd one_m;
    if (a.r * tau > 0.5) {
      one_m = cd{1.0 - ex * ek.r, -ex * ek.i};
    } else {
      cd em = cexpm1v(cd{-a.r * tau, -a.i * tau});
      one_m = cd{-em.r, -em.i};
    }
    const cd gD = cdivv(one_m, cd{mu * a.r, mu * a.i});
    // growing
    const cd bb{kap.r - x, kap.i};
    cd gG;
    if (bb.r == 0.0 && bb.i == 0.0) {
      gG = cd{tau * ex / mu, 0.0};
    } else if (fabs(bb.r * tau) + fabs(bb.i * tau) < 1e-2) {
      cd e2 = cexpm1v(cd{-bb.r * tau, -bb.i * tau});
      gG = cdivv(cd{-e2.r * ex, -e2.i * ex}, cd{mu * bb.r, mu * bb.i});
    } else {
      gG = cdivv(cd{ex - ek.r, -ek.i}, cd{mu * bb.r, mu * bb.i});
    }
    for (int ar = 0; ar < 4; ++ar) {
      const int ro = 4 * o + ar;
      size_t rowp = (size_t)u * Ro * n + (size_t)ro * n;
      double* Hb = Hhat + (size_t)u * Ro * 2 * n + (size_t)ro * 2 * n;
      cd p1{P1[rowp + j], cplx ? P1[rowp + j + 1] : 0.0};
      cd p2{P2[rowp + j], cplx ? P2[rowp + j + 1] : 0.0};
      cd hD{p1.r - p2.r, p1.i - p2.i};
      cd hG{p1.r + p2.r, p1.i + p2.i};
      cd vD = cmul(hD, gD), vG = cmul(hG, gG);
      Hb[j] = vD.r;
      Hb[n + j] = vG.r;
      if (cplx) {
        Hb[j + 1] = vD.i;
        Hb[n + j + 1] = vG.i;
      }
    }
  }
}

void launch_build_Hhat(const OrderBatch& b, const double* P1, const double* P2,
                       const double* lam_re, const double* lam_im, const double* pts,
                       double* Hhat, cudaStream_t s) {
  dim3 grid((b.n + 127) / 128, (b.n_out + HHAT_OB - 1) / HHAT_OB, b.n_units);
  k_build_Hhat<<<grid, 128, 0, s>>>(b.N, b.n, b.n_in, b.n_out, b.tau, P1, P2, lam_re, lam_im, pts,
                                    Hhat);
}

// ------------------------------------------------------------------ radiance at depth tau
// Reconstruction of Sec. 2.C inside the layer (0 <= tau <= tau0), for internal cosines mu
// (row 4o + a), x = 1/mu:
//   upward:   I(tau, +mu) = I(tau0, +mu) e^{-(tau0-tau)/mu} + int_tau^tau0 S(t, mu) e^{-(t-tau)/mu} dt/mu
//   downward: I(tau, -mu) = I(0, -mu) e^{-tau/mu} + int_0^tau S(t, -mu) e^{-(tau-t)/mu} dt/mu
// With A^m(-mu, s mu_n) = D A^m(mu, -s mu_n) D the downward scattering part on the reduced
// field is D (U+ s - U- d), the upward one U+ s + U- d (U+- with the identity exit). The modes
// then contribute, with D(a, b; T) = (e^{-aT} - e^{-bT})/(b - a):
//   upward:   decaying (P1 - P2) x e^{-kappa tau} D(0, x + kappa; tau0 - tau),
//             growing  (P1 + P2) x D(x, kappa; tau0 - tau)
//   downward: decaying D (P1 + P2) x D(x, kappa; tau),
//             growing  D (P1 - P2) x e^{-kappa (tau0 - tau)} D(0, kappa + x; tau)
// (at tau = 0 upward these are the top's factors of k_build_Hhat, at tau = tau0 downward the
// same two factors swapped).
__device__ inline cd dd_exp(cd a, cd b, double T) {
  const cd d{b.r - a.r, b.i - a.i};
  const cd ea = cexpv(cd{-a.r * T, -a.i * T});
  if (d.r == 0.0 && d.i == 0.0) return cd{T * ea.r, T * ea.i};
  if (fabs(d.r * T) + fabs(d.i * T) < 1e-2) {
    const cd em = cexpm1v(cd{-d.r * T, -d.i * T});
    return cdivv(cmul(ea, cd{-em.r, -em.i}), d);
  }
  const cd eb = cexpv(cd{-b.r * T, -b.i * T});
  return cdivv(cd{ea.r - eb.r, ea.i - eb.i}, d);
}

__global__ void k_build_Hdepth(int N, int n, int n_in, int n_out, double tau0, double tau,
                               int down, const double* P1, const double* P2, const double* lam_re,
                               const double* lam_im, const double* pts, double* H) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int o = blockIdx.y, u = blockIdx.z;
  if (j >= n) return;
  const double* lr = lam_re + (size_t)u * n;
  const double* li = lam_im + (size_t)u * n;
  if (li[j] < 0.0) return;
  const bool cplx = li[j] > 0.0;
  const int Ro = 4 * n_out;
  const cd kap = kappa_of(lr, li, j);
  const double x = 1.0 / pts[N + n_in + o];
  const cd X{x, 0.0}, Z{0.0, 0.0};
  cd gA, gB;
  if (!down) {
    gA = cmul(cexpv(cd{-kap.r * tau, -kap.i * tau}), dd_exp(Z, cd{x + kap.r, kap.i}, tau0 - tau));
    gB = dd_exp(X, kap, tau0 - tau);
  } else {
    gA = dd_exp(X, kap, tau);
    gB = cmul(cexpv(cd{-kap.r * (tau0 - tau), -kap.i * (tau0 - tau)}),
              dd_exp(Z, cd{kap.r + x, kap.i}, tau));
  }
  gA = cd{x * gA.r, x * gA.i};
  gB = cd{x * gB.r, x * gB.i};
  const double sA = down ? 1.0 : -1.0;  // decaying: P1 + P2 downward, P1 - P2 upward
  for (int ar = 0; ar < 4; ++ar) {
    const int ro = 4 * o + ar;
    const double dl = down ? (ar < 2 ? 1.0 : -1.0) : 1.0;
    const size_t rowp = (size_t)u * Ro * n + (size_t)ro * n;
    double* Hr = H + (size_t)u * Ro * 2 * n + (size_t)ro * 2 * n;
    const cd p1{P1[rowp + j], cplx ? P1[rowp + j + 1] : 0.0};
    const cd p2{P2[rowp + j], cplx ? P2[rowp + j + 1] : 0.0};
    const cd vA = cmul(cd{dl * (p1.r + sA * p2.r), dl * (p1.i + sA * p2.i)}, gA);
    const cd vB = cmul(cd{dl * (p1.r - sA * p2.r), dl * (p1.i - sA * p2.i)}, gB);
    Hr[j] = vA.r;
    Hr[n + j] = vB.r;
    if (cplx) {
      Hr[j + 1] = vA.i;
      Hr[n + j + 1] = vB.i;
    }
  }
}

void launch_build_Hdepth(const OrderBatch& b, double tau, int down, const double* P1,
                         const double* P2, const double* lam_re, const double* lam_im,
                         const double* pts, double* H, cudaStream_t s) {
  dim3 grid((b.n + 127) / 128, b.n_out, b.n_units);
  k_build_Hdepth<<<grid, 128, 0, s>>>(b.N, b.n, b.n_in, b.n_out, b.tau, tau, down, P1, P2, lam_re,
                                      lam_im, pts, H);
}

// Depth factor of the particular and direct parts (e^{-t/mu0} sources), y = 1/mu0:
//   upward x e^{-y tau} D(0, x + y; tau0 - tau),  downward x D(y, x; tau).
__device__ inline double g0_depth(double x, double y, double tau0, double tau, int down) {
  auto dd = [](double a, double b, double T) {
    const double d = b - a;
    if (d == 0.0) return T * exp(-a * T);
    if (fabs(d * T) < 1e-2) return exp(-a * T) * -expm1(-d * T) / d;
    return (exp(-a * T) - exp(-b * T)) / d;
  };
  return down ? x * dd(y, x, tau) : x * exp(-y * tau) * dd(0.0, x + y, tau0 - tau);
}

// Order radiance at depth tau into Isyn[m][k][o][a][s]:
//   upward:   Tdep + g0u (U+ s + U- d)      (+ the base's radiance, added by k_base_recon)
//   downward: Tdep + g0d D (U+ s - U- d) + e^{-tau/mu_o} R_F(mu_o) I(0, +mu_o),
// Tdep = [homogeneous part + direct part] at depth tau, Q = U+ s + U- d or U+ s - U- d, and
// I(0, +mu_o) = T1 + g0(tau = 0) Qp the upward radiance at the top (T1: its homogeneous and
// direct parts).
__global__ void k_depth_combine(OrderBatch b, double tau, int down, const double* Tdep,
                                const double* Q, const double* T1, const double* Qp,
                                const double* pts, const double* rout4, double* Isyn) {
  const int R = 4 * b.n_in, Ro = 4 * b.n_out;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int o = blockIdx.y, u = blockIdx.z;
  if (c >= R) return;
  const int k = c >> 2, s = c & 3;
  const double x = 1.0 / pts[b.N + b.n_in + o], y = 1.0 / pts[b.N + k];
  const double g = g0_depth(x, y, b.tau, tau, down);
  const size_t base = (size_t)u * Ro * R;
  double top[4] = {0.0, 0.0, 0.0, 0.0};
  if (down) {
    const double g0 = depth_factor(b.tau, 1.0 / x, 1.0 / y);
    for (int e = 0; e < 4; ++e) {
      const size_t idx = base + (size_t)(4 * o + e) * R + c;
      top[e] = T1[idx] + g0 * Qp[idx];
    }
  }
  const double att = exp(-x * tau);
  const double* Rm = rout4 + 4 * o;
  for (int a = 0; a < 4; ++a) {
    const size_t idx = base + (size_t)(4 * o + a) * R + c;
    double v = Tdep[idx];
    if (down) {
      double refl = 0.0;
      for (int e = 0; e < 4; ++e) {
        double r;
        if (a < 2 && e < 2) r = a == e ? Rm[0] : Rm[1];
        else if (a >= 2 && e >= 2) r = a == e ? Rm[2] : (a == 2 ? Rm[3] : -Rm[3]);
        else r = 0.0;
        refl += r * top[e];
      }
      v += g * (a < 2 ? 1.0 : -1.0) * Q[idx] + att * refl;
    } else {
      v += g * Q[idx];
    }
    Isyn[(((size_t)(b.m0 + u) * b.n_in + k) * b.n_out + o) * 16 + 4 * a + s] = v;
  }
}

void launch_depth_combine(const OrderBatch& b, double tau, int down, const double* Tdep,
                          const double* Q, const double* T1, const double* Qp, const double* pts,
                          const double* rout4, double* Isyn, cudaStream_t s) {
  dim3 grid((4 * b.n_in + 127) / 128, b.n_out, b.n_units);
  k_depth_combine<<<grid, 128, 0, s>>>(b, tau, down, Tdep, Q, T1, Qp, pts, rout4, Isyn);
}

// ------------------------------------------------------------------ reflecting base
// Base reflection (Sec. 3.C, Eqs. 57-66) for a base whose Mueller BRDF matrix R does not
// depend on the directions (the depolarizing Lambertian base of albedo rho is R_00 = 2 rho):
// only order 0 sees it, and the upward radiance at the bottom is the same at every node,
//   I^0(tau0, +mu) = R sum_j alpha_j mu_j I^0(tau0, -mu_j) + (1/pi) mu0 R b e^{-tau0/mu0}
// (b the beam column, whose order-0 Fourier part is b/pi in the Fourier convention of Eq. 12).
// R's (I, Q) x (U, V) blocks are zero (the host rejects others): an azimuth-independent base
// cannot couple them at order 0. In the reduced form the downward radiance at the bottom of
// component e is sgn_e (decaying modes: phi+ e^{-kappa tau0}, growing ones: phi-), sgn = D.
// basev[e][col] = sum_j alpha_j mu_j I_e(tau0, -mu_j) of boundary-matrix column col (real
// form; layout [4][2n]); the bottom rows n + 4i + a of K lose sum_e R_ae basev[e] (the
// reflected radiance moves to the left side, Eq. 66).
__global__ void k_base_K(int N, int n, double tau, BaseR Rg, const double* X, const double* Y,
                         const double* lam_re, const double* lam_im, const double* mu_nodes,
                         const double* w_nodes, double* K, double* basev) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n || lam_im[j] < 0.0) return;
  const bool cplx = lam_im[j] > 0.0;
  const cd kap = kappa_of(lam_re, lam_im, j);
  const cd E = cexpv(cd{-kap.r * tau, -kap.i * tau});
  cd vA[4], vB[4];
  for (int e = 0; e < 4; ++e) vA[e] = vB[e] = cd{0.0, 0.0};
  for (int q = 0; q < N; ++q) {
    const double f = w_nodes[q] * mu_nodes[q];
    for (int e = 0; e < 4; ++e) {
      const size_t idx = (size_t)(4 * q + e) * n + j;
      const cd x{X[idx], cplx ? X[idx + 1] : 0.0}, y{Y[idx], cplx ? Y[idx + 1] : 0.0};
      const double fs = e < 2 ? 0.5 * f : -0.5 * f;
      const cd pp = cmul(cd{fs * (x.r + y.r), fs * (x.i + y.i)}, E);
      vA[e] = cd{vA[e].r + pp.r, vA[e].i + pp.i};
      vB[e] = cd{vB[e].r + fs * (x.r - y.r), vB[e].i + fs * (x.i - y.i)};
    }
  }
  const int n2 = 2 * n;
  for (int e = 0; e < 4; ++e) {
    basev[e * n2 + j] = vA[e].r;
    basev[e * n2 + n + j] = vB[e].r;
    if (cplx) {
      basev[e * n2 + j + 1] = vA[e].i;
      basev[e * n2 + n + j + 1] = vB[e].i;
    }
  }
  for (int a = 0; a < 4; ++a) {
    cd rA{0.0, 0.0}, rB{0.0, 0.0};
    for (int e = 0; e < 4; ++e) {
      const double r = Rg.r[4 * a + e];
      rA = cd{rA.r + r * vA[e].r, rA.i + r * vA[e].i};
      rB = cd{rB.r + r * vB[e].r, rB.i + r * vB[e].i};
    }
    for (int i = 0; i < N; ++i) {
      double* row = K + (size_t)(n + 4 * i + a) * n2;
      row[j] -= rA.r;
      row[n + j] -= rB.r;
      if (cplx) {
        row[j + 1] -= rA.i;
        row[n + j + 1] -= rB.i;
      }
    }
  }
}

// The reflected particular radiance and the reflected attenuated beam, for column c = 4k + s:
//   zb[a][c] = sum_e R_ae [ (sum_j alpha_j mu_j zm_e(j)[c]) e^{-tau0/mu0}
//                           + (mu0 / pi) b_e[c] e^{-(t + tau0)/mu0} ]
// (zm = D (s - d)/2 the particular solution's downward radiance at tau = 0; t = t_above, the
// depth of the layer's top in a slab: the beam reaches the base through it; b_e[c] entry
// (e, s) of the beam block of incident k), added to the bottom rows n + 4i + a of the
// right-hand side when add_rhs (Eqs. 62-63).
__global__ void k_base_rhs(int N, int n, int R, long long sSD, double tau, BaseR Rg,
                           const double* SD, const double* pts, const double* min4,
                           const double* mu_nodes, const double* w_nodes, double* RHS,
                           double* zb, int add_rhs, double t_above) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= R) return;
  const double* sv = SD;
  const double* dv = SD + (size_t)n * R;
  double z[4] = {0.0, 0.0, 0.0, 0.0};
  for (int q = 0; q < N; ++q) {
    const double f = 0.5 * w_nodes[q] * mu_nodes[q];
    for (int e = 0; e < 4; ++e) {
      const size_t idx = (size_t)(4 * q + e) * R + c;
      z[e] += (e < 2 ? f : -f) * (sv[idx] - dv[idx]);
    }
  }
  const int k = c >> 2, s = c & 3;
  const double mu0 = pts[N + k], att = exp(-tau / mu0);
  const double fb = mu0 / kPi * exp(-(t_above + tau) / mu0);
  const double* q4 = min4 + 4 * k;
  double ze[4];
  for (int e = 0; e < 4; ++e) {
    double b = 0.0;  // entry (e, s) of the beam block [[qa, qb, 0, 0], [qb, qa, 0, 0], [0, 0, qc, qd], [0, 0, -qd, qc]]
    if (e < 2 && s < 2) b = e == s ? q4[0] : q4[1];
    else if (e >= 2 && s >= 2) b = e == s ? q4[2] : (e == 2 ? q4[3] : -q4[3]);
    ze[e] = z[e] * att + fb * b;
  }
  for (int a = 0; a < 4; ++a) {
    double v = 0.0;
    for (int e = 0; e < 4; ++e) v += Rg.r[4 * a + e] * ze[e];
    zb[(size_t)a * R + c] = v;
    if (add_rhs)
      for (int i = 0; i < N; ++i) RHS[(size_t)(n + 4 * i + a) * R + c] += v;
  }
}

// The base's radiance at the bottom for column c (the same at every upward direction):
//   vb[a][c] = sum_e R_ae (basev[e] . C[:, c]) + zb[a][c].
__global__ void k_base_value(int n, int R, BaseR Rg, const double* C, const double* basev,
                             const double* zb, double* vb) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= R) return;
  const int n2 = 2 * n;
  double d[4] = {0.0, 0.0, 0.0, 0.0};
  for (int col = 0; col < n2; ++col) {
    const double cv = C[(size_t)col * R + c];
    for (int e = 0; e < 4; ++e) d[e] += basev[e * n2 + col] * cv;
  }
  for (int a = 0; a < 4; ++a) {
    double v = zb[(size_t)a * R + c];
    for (int e = 0; e < 4; ++e) v += Rg.r[4 * a + e] * d[e];
    vb[(size_t)a * R + c] = v;
  }
}

// The base's radiance attenuated along the exit path and added to the order-0 upward radiance:
// out[(o, a)][c] += e^{-tau/mu_o} (M_out(o) vb[:, c])_a (M_out = identity when mout4 is null,
// else the exit block [[m0, m1, 0, 0], [m1, m0, 0, 0], [0, 0, m2, m3], [0, 0, -m3, m2]]).
// `isyn` selects the order-radiance layout Isyn[0][k][o][a][s] for out.
__global__ void k_base_add(int N, int n_in, int n_out, double tau, const double* vb,
                           const double* pts, const double* mout4, double* out, int isyn) {
  const int R = 4 * n_in;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int o = blockIdx.y;
  if (c >= R) return;
  const double att = exp(-tau / pts[N + n_in + o]);
  double v[4];
  for (int e = 0; e < 4; ++e) v[e] = att * vb[(size_t)e * R + c];
  double w[4];
  if (mout4) {
    const double* q = mout4 + 4 * o;
    w[0] = q[0] * v[0] + q[1] * v[1];
    w[1] = q[1] * v[0] + q[0] * v[1];
    w[2] = q[2] * v[2] + q[3] * v[3];
    w[3] = -q[3] * v[2] + q[2] * v[3];
  } else {
    for (int e = 0; e < 4; ++e) w[e] = v[e];
  }
  const int k = c >> 2, s = c & 3;
  for (int a = 0; a < 4; ++a) {
    if (isyn)
      out[((size_t)k * n_out + o) * 16 + 4 * a + s] += w[a];
    else
      out[(size_t)(4 * o + a) * R + c] += w[a];
  }
}

void launch_base_K(int N, int n, double tau, const BaseR& Rg, const double* X, const double* Y,
                   const double* lam_re, const double* lam_im, const double* mu_nodes,
                   const double* w_nodes, double* K, double* basev, cudaStream_t s) {
  k_base_K<<<(n + 127) / 128, 128, 0, s>>>(N, n, tau, Rg, X, Y, lam_re, lam_im, mu_nodes, w_nodes,
                                           K, basev);
}
void launch_base_rhs(int N, int n, int R, long long sSD, double tau, const BaseR& Rg,
                     const double* SD, const double* pts, const double* min4,
                     const double* mu_nodes, const double* w_nodes, double* RHS, double* zb,
                     int add_rhs, cudaStream_t s, double t_above) {
  k_base_rhs<<<(R + 127) / 128, 128, 0, s>>>(N, n, R, sSD, tau, Rg, SD, pts, min4, mu_nodes,
                                             w_nodes, RHS, zb, add_rhs, t_above);
}
void launch_base_recon(int n, int N, int n_in, int n_out, double tau, const BaseR& Rg,
                       const double* C, double* basebuf, const double* pts,
                       const double* mout4, double* out, int isyn, cudaStream_t s) {
  const int R = 4 * n_in;
  const double* basev = basebuf;
  const double* zb = basebuf + 8 * n;
  double* vb = basebuf + 8 * n + 4 * (size_t)R;
  k_base_value<<<(R + 127) / 128, 128, 0, s>>>(n, R, Rg, C, basev, zb, vb);
  dim3 grid((R + 127) / 128, n_out);
  k_base_add<<<grid, 128, 0, s>>>(N, n_in, n_out, tau, vb, pts, mout4, out, isyn);
}

}  // namespace vrte
