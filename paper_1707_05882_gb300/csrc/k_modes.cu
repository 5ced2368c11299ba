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
__global__ void k_particular_rhs(int n, int R, int N, const double* r, const double* pts,
                                 double* w) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  int i = blockIdx.y, u = blockIdx.z;
  if (c >= R) return;
  size_t idx = (size_t)u * n * R + (size_t)i * R + c;
  w[idx] -= r[idx] / pts[N + (c >> 2)];
}

void launch_particular_rhs(const OrderBatch& b, const double* w_in, const double* r,
                           const double* pts, double* w_out, cudaStream_t s) {
  (void)w_in;
  int R = 4 * b.n_in;
  dim3 grid((R + 127) / 128, b.n, b.n_units);
  k_particular_rhs<<<grid, 128, 0, s>>>(b.n, R, b.N, r, pts, w_out);
}

// y <- (Lambda - 1/mu0^2)^-1 y in the eigenbasis; a pair uses the real 2x2 block
// [[a, b], [-b, a]] of lambda = a + ib.
__global__ void k_eigen_scale(int n, int R, int N, const double* lam_re, const double* lam_im,
                              const double* pts, double* y) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y, u = blockIdx.z;
  if (c >= R) return;
  const double* lr = lam_re + (size_t)u * n;
  const double* li = lam_im + (size_t)u * n;
  if (li[j] < 0.0) return;
  double mu0 = pts[N + (c >> 2)];
  double cc = 1.0 / (mu0 * mu0);
  size_t idx = (size_t)u * n * R + (size_t)j * R + c;
  if (li[j] == 0.0) {
    y[idx] /= (lr[j] - cc);
  } else {
    double a = lr[j] - cc, bb = li[j];
    double den = a * a + bb * bb;
    double y0 = y[idx], y1 = y[idx + R];
    y[idx] = (a * y0 - bb * y1) / den;
    y[idx + R] = (bb * y0 + a * y1) / den;
  }
}

void launch_eigen_scale(const OrderBatch& b, const double* lam_re, const double* lam_im,
                        const double* pts, double* y, cudaStream_t s) {
  int R = 4 * b.n_in;
  dim3 grid((R + 127) / 128, b.n, b.n_units);
  k_eigen_scale<<<grid, 128, 0, s>>>(b.n, R, b.N, lam_re, lam_im, pts, y);
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
__global__ void k_bc_rhs(int N, int n, int R, long long sSD, double tau, const double* SD,
                         const double* rtop4, const double* pts, double* rhs) {
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
  double att = exp(-tau / pts[N + (c >> 2)]);
  double* rb = rhs + (size_t)u * 2 * n * R;
  for (int a = 0; a < 4; ++a) {
    rb[(size_t)(4 * i + a) * R + c] = -(zm[a] - rz[a]);
    rb[(size_t)(n + 4 * i + a) * R + c] = -zp[a] * att;
  }
}

void launch_bc_rhs(const OrderBatch& b, const double* SD, const double* d, const double* rtop4,
                   const double* pts, double* rhs, cudaStream_t s) {
  (void)d;
  int R = 4 * b.n_in;
  dim3 grid((R + 127) / 128, b.N, b.n_units);
  k_bc_rhs<<<grid, 128, 0, s>>>(b.N, b.n, R, b.sSD, b.tau, SD, rtop4, pts, rhs);
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

}  // namespace vrte
