// Tables of the hot path (step a0): double-Gauss nodes (Sec. 2.B, Eq. 15),
// smooth-interface Fresnel data, generalized spherical functions of Eqs. 9-10 at
// every table point, and the azimuthal synthesis weights of Eqs. 7 and 12.
#include "vrte_internal.cuh"

namespace vrte {

// One thread per node: Newton iteration on P_N from the Tricomi guess, at most 100
// steps; nodes and weights mapped to [0, 1] (weights sum to one per hemisphere).
__global__ void k_gauss_nodes(int N, double* mu, double* w, unsigned* status) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double z = cos(kPi * (i + 0.75) / (N + 0.5));
  double p0 = 1.0, p1 = z, dp = 1.0;
  bool ok = false;
  for (int it = 0; it < 100; ++it) {
    p0 = 1.0;
    p1 = z;
    for (int k = 2; k <= N; ++k) {
      double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    dp = N * (z * p1 - p0) / (z * z - 1.0);
    double dz = p1 / dp;
    z -= dz;
    if (fabs(dz) < 1e-16) { ok = true; break; }
  }
  p0 = 1.0;
  p1 = z;
  for (int k = 2; k <= N; ++k) {
    double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
    p0 = p1;
    p1 = p2;
  }
  dp = N * (z * p1 - p0) / (z * z - 1.0);
  if (!ok && N > 1) atomicOr(status, ST_NO_CONVERGENCE);
  // root i counted from x = 1 downward; store ascending on [0, 1]
  int slot = N - 1 - i;
  mu[slot] = 0.5 * (1.0 + z);
  w[slot] = 1.0 / ((1.0 - z * z) * dp * dp);
}

void launch_gauss_nodes(int N, double* mu, double* w, unsigned* status, cudaStream_t s) {
  k_gauss_nodes<<<(N + 127) / 128, 128, 0, s>>>(N, mu, w, status);
}

// Mueller block (a, b, c, d) of a diagonal Jones matrix diag(jp, js) on meridian frames:
// [[a, b, 0, 0], [b, a, 0, 0], [0, 0, c, d], [0, 0, -d, c]].
struct Blk4 { double a, b, c, d; };

__device__ inline Blk4 jones_block(double jpr, double jpi, double jsr, double jsi) {
  double p2 = jpr * jpr + jpi * jpi, s2 = jsr * jsr + jsi * jsi;
  // z = jp * conj(js)
  double zr = jpr * jsr + jpi * jsi, zi = jpi * jsr - jpr * jsi;
  return Blk4{0.5 * (p2 + s2), 0.5 * (p2 - s2), zr, zi};
}

// Table points and interface matrices of one layer.
//   pts  = [mu_nodes (N) | mu0 internal (n_in) | mu_out internal (n_out)]
//   min4[k]  = beam transmission block divided by mu_in[k] (folds the 1/mu_in of F_r)
//   mout4[o] = radiance exit block; rtop4[i] = internal reflection block at node i.
__global__ void k_interface(int N, int n_in, int n_out, double nif, const double* mu_nodes,
                            const double* mu_in, const double* mu_out, double* pts, double* min4,
                            double* mout4, double* rtop4) {
  int tid = blockIdx.x * blockDim.x + threadIdx.x;
  int total = N + n_in + n_out;
  if (tid >= total) return;
  bool iface = nif > 1.0;
  if (tid < N) {
    double c1 = mu_nodes[tid];
    pts[tid] = c1;
    Blk4 r{0.0, 0.0, 0.0, 0.0};
    if (iface) {
      // inside (index nif) towards outside (index 1)
      double s2sq = nif * nif * (1.0 - c1 * c1);
      if (s2sq <= 1.0) {
        double c2 = sqrt(1.0 - s2sq);
        double rs = (nif * c1 - c2) / (nif * c1 + c2);
        double rp = (c1 - nif * c2) / (c1 + nif * c2);
        r = jones_block(rp, 0.0, rs, 0.0);
      } else {
        // total internal reflection, c2 = i beta
        double beta = sqrt(s2sq - 1.0);
        double A = nif * c1, B = beta;      // rs = (A - iB) / (A + iB)
        double C = c1, Dd = nif * beta;     // rp = (C - iD) / (C + iD)
        double nA = A * A + B * B, nC = C * C + Dd * Dd;
        double rsr = (A * A - B * B) / nA, rsi = -2.0 * A * B / nA;
        double rpr = (C * C - Dd * Dd) / nC, rpi = -2.0 * C * Dd / nC;
        r = jones_block(rpr, rpi, rsr, rsi);
      }
    }
    rtop4[4 * tid + 0] = r.a;
    rtop4[4 * tid + 1] = r.b;
    rtop4[4 * tid + 2] = r.c;
    rtop4[4 * tid + 3] = r.d;
  } else if (tid < N + n_in) {
    int k = tid - N;
    double me = mu_in[k];
    Blk4 t{1.0, 0.0, 1.0, 0.0};
    double mi = me;
    if (iface) {
      mi = sqrt(1.0 - (1.0 - me * me) / (nif * nif));
      double ts = 2.0 * me / (me + nif * mi);
      double tp = 2.0 * me / (nif * me + mi);
      t = jones_block(tp, 0.0, ts, 0.0);
      t.a *= nif; t.b *= nif; t.c *= nif; t.d *= nif;
    }
    pts[tid] = mi;
    double inv = 1.0 / me;
    min4[4 * k + 0] = t.a * inv;
    min4[4 * k + 1] = t.b * inv;
    min4[4 * k + 2] = t.c * inv;
    min4[4 * k + 3] = t.d * inv;
  } else {
    int o = tid - N - n_in;
    double me = mu_out[o];
    Blk4 t{1.0, 0.0, 1.0, 0.0};
    double mi = me;
    if (iface) {
      mi = sqrt(1.0 - (1.0 - me * me) / (nif * nif));
      // inside -> outside amplitudes, radiance factor me / (nif^3 mi)
      double ts = 2.0 * nif * mi / (nif * mi + me);
      double tp = 2.0 * nif * mi / (mi + nif * me);
      t = jones_block(tp, 0.0, ts, 0.0);
      double f = me / (nif * nif * nif * mi);
      t.a *= f; t.b *= f; t.c *= f; t.d *= f;
    }
    pts[tid] = mi;
    mout4[4 * o + 0] = t.a;
    mout4[4 * o + 1] = t.b;
    mout4[4 * o + 2] = t.c;
    mout4[4 * o + 3] = t.d;
  }
}

void launch_interface(int N, int n_in, int n_out, double nif, const double* mu_nodes,
                      const double* mu_in, const double* mu_out, double* pts, double* min4,
                      double* mout4, double* rtop4, cudaStream_t s) {
  int total = N + n_in + n_out;
  k_interface<<<(total + 255) / 256, 256, 0, s>>>(N, n_in, n_out, nif, mu_nodes, mu_in, mu_out,
                                                   pts, min4, mout4, rtop4);
}

// Wigner d^l_{m n}(x) seed at l0 = max(|m|, |n|):
//   xi 2^-l0 sqrt((2 l0)! / (|m-n|! |m+n|!)) (1-x)^{|m-n|/2} (1+x)^{|m+n|/2},
//   xi = 1 if n >= m else (-1)^(m-n), evaluated in logarithms.
__device__ inline double wigner_seed(int m, int n, double x) {
  int l0 = max(abs(m), abs(n));
  int a = abs(m - n), b = abs(m + n);
  double lg = -l0 * 0.69314718055994530942 +
              0.5 * (lgamma(2.0 * l0 + 1.0) - lgamma(a + 1.0) - lgamma(b + 1.0));
  if (a > 0) {
    double u = 1.0 - x;
    if (u <= 0.0) return 0.0;
    lg += 0.5 * a * log(u);
  }
  if (b > 0) {
    double u = 1.0 + x;
    if (u <= 0.0) return 0.0;
    lg += 0.5 * b * log(u);
  }
  double v = exp(lg);
  if (n < m && ((m - n) & 1)) v = -v;
  return v;
}

// One thread per (order, point): p = d^l_{m0}, r = -(d^l_{m2} + d^l_{m,-2})/2,
// t = -(d^l_{m2} - d^l_{m,-2})/2 for l = m..L-1 by the three-term recurrence
//   l sqrt((l+1)^2-m^2) sqrt((l+1)^2-n^2) d^{l+1}
//     = (2l+1)(l(l+1)x - m n) d^l - (l+1) sqrt(l^2-m^2) sqrt(l^2-n^2) d^{l-1}.
// Layout: tab[(u * L + l) * P + k].
__global__ void k_gsf(int L, int m0, int n_units, int P, const double* pts, double* pt, double* rt,
                      double* tt) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  int u = blockIdx.y;
  if (k >= P || u >= n_units) return;
  int m = m0 + u;
  double x = pts[k];
  size_t base = (size_t)u * L * P + k;
  // family n = 0
  {
    double dm1 = 0.0, d0 = 0.0;
    int l0 = m;
    for (int l = l0; l < L; ++l) {
      double d;
      if (l == l0) {
        d = (m == 0) ? 1.0 : wigner_seed(m, 0, x);
      } else if (m == 0) {
        int lp = l - 1;  // Legendre
        d = ((2 * lp + 1) * x * d0 - lp * dm1) / (lp + 1);
      } else {
        int lp = l - 1;
        double den = lp * sqrt((double)(l * l - m * m)) * (double)l;
        double num = (2 * lp + 1) * (lp * (double)l * x) * d0;
        if (lp > l0) num -= l * sqrt((double)(lp * lp - m * m)) * (double)lp * dm1;
        d = num / den;
      }
      pt[base + (size_t)l * P] = d;
      dm1 = d0;
      d0 = d;
    }
  }
  // families n = +2 and n = -2
  {
    int l0 = max(m, 2);
    double ap = 0.0, bp = 0.0, am = 0.0, bm = 0.0;  // d^{l-1}, d^l for n = +2 and -2
    for (int l = m; l < L; ++l) {
      double dp2 = 0.0, dm2 = 0.0;
      if (l >= l0) {
        if (l == l0) {
          dp2 = wigner_seed(m, 2, x);
          dm2 = wigner_seed(m, -2, x);
        } else {
          int lp = l - 1;
          double s1 = sqrt((double)(l * l - m * m)) * sqrt((double)(l * l - 4));
          double den = lp * s1;
          double c0 = (2 * lp + 1) * (lp * (double)l * x - 2.0 * m);
          double c0m = (2 * lp + 1) * (lp * (double)l * x + 2.0 * m);
          double cpre = 0.0;
          if (lp > l0) cpre = l * sqrt((double)(lp * lp - m * m)) * sqrt((double)(lp * lp - 4));
          dp2 = (c0 * bp - cpre * ap) / den;
          dm2 = (c0m * bm - cpre * am) / den;
        }
        ap = bp; bp = dp2;
        am = bm; bm = dm2;
      }
      rt[base + (size_t)l * P] = -0.5 * (dp2 + dm2);
      tt[base + (size_t)l * P] = -0.5 * (dp2 - dm2);
    }
  }
}

void launch_gsf_tables(const OrderBatch& b, const double* pts, double* p, double* r, double* t,
                       cudaStream_t s) {
  dim3 grid((b.P + 127) / 128, b.n_units);
  k_gsf<<<grid, 128, 0, s>>>(b.L, b.m0, b.n_units, b.P, pts, p, r, t);
}

// wc[m][j] = (2 - delta_m0)/2 (-1)^m cos(m dphi_j), ws likewise with sin: the Fourier
// factors of Eq. 7 with the 1/2 of Eq. 12 and the half-turn between the beam's
// propagation azimuth and the source azimuth.
__global__ void k_trig(int M, int n_phi, const double* phi, double* wc, double* ws) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  int m = blockIdx.y;
  if (j >= n_phi || m >= M) return;
  double f = (m == 0 ? 0.5 : 1.0) * ((m & 1) ? -1.0 : 1.0);
  double sn, cs;
  sincos(m * phi[j], &sn, &cs);
  wc[(size_t)m * n_phi + j] = f * cs;
  ws[(size_t)m * n_phi + j] = f * sn;
}

void launch_trig_table(int M, int n_phi, const double* phi, double* wc, double* ws, cudaStream_t s) {
  dim3 grid((n_phi + 127) / 128, M);
  k_trig<<<grid, 128, 0, s>>>(M, n_phi, phi, wc, ws);
}

}  // namespace vrte
