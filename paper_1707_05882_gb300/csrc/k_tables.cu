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
// [[a, b, 0, 0], [b, a, 0, 0], [0, 0, c, d], [0, 0, -d, c]]. T is double, or a dual number
// carrying the derivative with respect to the interface index n.
template <class T>
struct Blk4 { T a, b, c, d; };

template <class T>
__device__ inline Blk4<T> jones_block(T jpr, T jpi, T jsr, T jsi) {
  T p2 = jpr * jpr + jpi * jpi, s2 = jsr * jsr + jsi * jsi;
  // z = jp * conj(js)
  T zr = jpr * jsr + jpi * jsi, zi = jpi * jsr - jpr * jsi;
  return Blk4<T>{0.5 * (p2 + s2), 0.5 * (p2 - s2), zr, zi};
}

template <class T>
__device__ inline Blk4<T> scale_blk(Blk4<T> t, T f) {
  return Blk4<T>{t.a * f, t.b * f, t.c * f, t.d * f};
}

// Interface data of table point tid for relative index nif (see k_interface); returns the
// point's internal cosine and writes its block (reflection, transmission in or out).
template <class T>
__device__ inline T interface_point(int tid, int N, int n_in, T nif, bool iface,
                                    const double* mu_nodes, const double* mu_in,
                                    const double* mu_out, Blk4<T>& blk) {
  const T zero = nif * 0.0;
  if (tid < N) {
    double c1 = mu_nodes[tid];
    blk = Blk4<T>{zero, zero, zero, zero};
    if (iface) {
      // inside (index nif) towards outside (index 1)
      T s2sq = nif * nif * (1.0 - c1 * c1);
      if (val(s2sq) <= 1.0) {
        T c2 = dsqrt(1.0 - s2sq);
        T rs = (nif * c1 - c2) / (nif * c1 + c2);
        T rp = (c1 - nif * c2) / (c1 + nif * c2);
        blk = jones_block<T>(rp, zero, rs, zero);
      } else {
        // total internal reflection, c2 = i beta
        T beta = dsqrt(s2sq - 1.0);
        T A = nif * c1, B = beta;      // rs = (A - iB) / (A + iB)
        T C = zero + c1, Dd = nif * beta;  // rp = (C - iD) / (C + iD)
        T nA = A * A + B * B, nC = C * C + Dd * Dd;
        T rsr = (A * A - B * B) / nA, rsi = -2.0 * A * B / nA;
        T rpr = (C * C - Dd * Dd) / nC, rpi = -2.0 * C * Dd / nC;
        blk = jones_block<T>(rpr, rpi, rsr, rsi);
      }
    }
    return zero + c1;
  }
  if (tid < N + n_in) {
    double me = mu_in[tid - N];
    Blk4<T> t{zero + 1.0, zero, zero + 1.0, zero};
    T mi = zero + me;
    if (iface) {
      mi = dsqrt(1.0 - (1.0 - me * me) / (nif * nif));
      T ts = 2.0 * me / (me + nif * mi);
      T tp = 2.0 * me / (nif * me + mi);
      t = scale_blk<T>(jones_block<T>(tp, zero, ts, zero), nif);
    }
    blk = scale_blk<T>(t, zero + 1.0 / me);
    return mi;
  }
  double me = mu_out[tid - N - n_in];
  Blk4<T> t{zero + 1.0, zero, zero + 1.0, zero};
  T mi = zero + me;
  if (iface) {
    mi = dsqrt(1.0 - (1.0 - me * me) / (nif * nif));
    // inside -> outside amplitudes, radiance factor me / (nif^3 mi)
    T ts = 2.0 * nif * mi / (nif * mi + me);
    T tp = 2.0 * nif * mi / (mi + nif * me);
    t = scale_blk<T>(jones_block<T>(tp, zero, ts, zero), me / (nif * nif * nif * mi));
  }
  blk = t;
  return mi;
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
  Blk4<double> b;
  pts[tid] = interface_point<double>(tid, N, n_in, nif, nif > 1.0, mu_nodes, mu_in, mu_out, b);
  double* dst = tid < N ? rtop4 + 4 * tid
                        : (tid < N + n_in ? min4 + 4 * (tid - N) : mout4 + 4 * (tid - N - n_in));
  dst[0] = b.a;
  dst[1] = b.b;
  dst[2] = b.c;
  dst[3] = b.d;
}

// Derivatives of the same data with respect to the interface index n (forward mode): dpts
// (zero at the nodes), dmin4, dmout4, drtop4. All zero without an interface.
__global__ void k_interface_dn(int N, int n_in, int n_out, double nif, const double* mu_nodes,
                               const double* mu_in, const double* mu_out, double* dpts,
                               double* dmin4, double* dmout4, double* drtop4) {
  int tid = blockIdx.x * blockDim.x + threadIdx.x;
  int total = N + n_in + n_out;
  if (tid >= total) return;
  Blk4<dual> b;
  dual mi = interface_point<dual>(tid, N, n_in, dual{nif, 1.0}, nif > 1.0, mu_nodes, mu_in,
                                  mu_out, b);
  dpts[tid] = mi.d;
  double* dst = tid < N ? drtop4 + 4 * tid
                        : (tid < N + n_in ? dmin4 + 4 * (tid - N) : dmout4 + 4 * (tid - N - n_in));
  dst[0] = b.a.d;
  dst[1] = b.b.d;
  dst[2] = b.c.d;
  dst[3] = b.d.d;
}

// Transmission table (radiance leaving the bottom downward, no interface there): the outgoing
// points are the internal cosines as given, their exit block is the identity, and rout4[o]
// is the internal specular reflection at the top at that cosine (zero for a bare top), which
// sends the upward radiance at mu_out back down through the layer.
__global__ void k_btdf_points(int N, int n_in, int n_out, double nif, const double* mu_out,
                              double* pts, double* mout4, double* rout4) {
  int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n_out) return;
  Blk4<double> r;
  pts[N + n_in + o] = interface_point<double>(o, n_out, 0, nif, nif > 1.0, mu_out, nullptr,
                                              nullptr, r);
  mout4[4 * o + 0] = 1.0;
  mout4[4 * o + 1] = 0.0;
  mout4[4 * o + 2] = 1.0;
  mout4[4 * o + 3] = 0.0;
  rout4[4 * o + 0] = r.a;
  rout4[4 * o + 1] = r.b;
  rout4[4 * o + 2] = r.c;
  rout4[4 * o + 3] = r.d;
}

void launch_btdf_points(int N, int n_in, int n_out, double nif, const double* mu_out, double* pts,
                        double* mout4, double* rout4, cudaStream_t s) {
  k_btdf_points<<<(n_out + 127) / 128, 128, 0, s>>>(N, n_in, n_out, nif, mu_out, pts, mout4,
                                                    rout4);
}

void launch_interface(int N, int n_in, int n_out, double nif, const double* mu_nodes,
                      const double* mu_in, const double* mu_out, double* pts, double* min4,
                      double* mout4, double* rtop4, cudaStream_t s) {
  int total = N + n_in + n_out;
  k_interface<<<(total + 255) / 256, 256, 0, s>>>(N, n_in, n_out, nif, mu_nodes, mu_in, mu_out,
                                                   pts, min4, mout4, rtop4);
}

void launch_interface_dn(int N, int n_in, int n_out, double nif, const double* mu_nodes,
                         const double* mu_in, const double* mu_out, double* dpts, double* dmin4,
                         double* dmout4, double* drtop4, cudaStream_t s) {
  int total = N + n_in + n_out;
  k_interface_dn<<<(total + 255) / 256, 256, 0, s>>>(N, n_in, n_out, nif, mu_nodes, mu_in, mu_out,
                                                      dpts, dmin4, dmout4, drtop4);
}

// Wigner d^l_{m n}(x) seed at l0 = max(|m|, |n|):
//   xi 2^-l0 sqrt((2 l0)! / (|m-n|! |m+n|!)) (1-x)^{|m-n|/2} (1+x)^{|m+n|/2},
//   xi = 1 if n >= m else (-1)^(m-n), evaluated in logarithms.
template <class T>
__device__ inline T wigner_seed(int m, int n, T x) {
  int l0 = max(abs(m), abs(n));
  int a = abs(m - n), b = abs(m + n);
  T lg = x * 0.0 + (-l0 * 0.69314718055994530942 +
                    0.5 * (lgamma(2.0 * l0 + 1.0) - lgamma(a + 1.0) - lgamma(b + 1.0)));
  if (a > 0) {
    T u = 1.0 - x;
    if (val(u) <= 0.0) return x * 0.0;
    lg = lg + 0.5 * a * dlog(u);
  }
  if (b > 0) {
    T u = 1.0 + x;
    if (val(u) <= 0.0) return x * 0.0;
    lg = lg + 0.5 * b * dlog(u);
  }
  T v = dexp(lg);
  if (n < m && ((m - n) & 1)) v = -v;
  return v;
}

// p = d^l_{m0}, r = -(d^l_{m2} + d^l_{m,-2})/2, t = -(d^l_{m2} - d^l_{m,-2})/2 at cosine x for
// l = m..L-1 by the three-term recurrence
//   l sqrt((l+1)^2-m^2) sqrt((l+1)^2-n^2) d^{l+1}
//     = (2l+1)(l(l+1)x - m n) d^l - (l+1) sqrt(l^2-m^2) sqrt(l^2-n^2) d^{l-1},
// handed to put(l, p, r, t).
template <class T, class PutP, class PutRT>
__device__ inline void gsf_point(int m, int L, T x, PutP put_p, PutRT put_rt) {
  // family n = 0
  {
    T dm1 = x * 0.0, d0 = x * 0.0;
    int l0 = m;
    for (int l = l0; l < L; ++l) {
      T d;
      if (l == l0) {
        d = (m == 0) ? x * 0.0 + 1.0 : wigner_seed<T>(m, 0, x);
      } else if (m == 0) {
        int lp = l - 1;  // Legendre
        d = ((2 * lp + 1) * x * d0 - lp * dm1) / (double)(lp + 1);
      } else {
        int lp = l - 1;
        double den = lp * sqrt((double)(l * l - m * m)) * (double)l;
        T num = (2 * lp + 1) * (lp * (double)l) * x * d0;
        if (lp > l0) num = num - l * sqrt((double)(lp * lp - m * m)) * (double)lp * dm1;
        d = num / den;
      }
      put_p(l, d, d);
      dm1 = d0;
      d0 = d;
    }
  }
  // families n = +2 and n = -2
  {
    int l0 = max(m, 2);
    T ap = x * 0.0, bp = x * 0.0, am = x * 0.0, bm = x * 0.0;  // d^{l-1}, d^l for n = +2 and -2
    for (int l = m; l < L; ++l) {
      T dp2 = x * 0.0, dm2 = x * 0.0;
      if (l >= l0) {
        if (l == l0) {
          dp2 = wigner_seed<T>(m, 2, x);
          dm2 = wigner_seed<T>(m, -2, x);
        } else {
          int lp = l - 1;
          double s1 = sqrt((double)(l * l - m * m)) * sqrt((double)(l * l - 4));
          double den = lp * s1;
          T c0 = (2 * lp + 1) * ((lp * (double)l) * x - 2.0 * m);
          T c0m = (2 * lp + 1) * ((lp * (double)l) * x + 2.0 * m);
          double cpre = 0.0;
          if (lp > l0) cpre = l * sqrt((double)(lp * lp - m * m)) * sqrt((double)(lp * lp - 4));
          dp2 = (c0 * bp - cpre * ap) / den;
          dm2 = (c0m * bm - cpre * am) / den;
        }
        ap = bp; bp = dp2;
        am = bm; bm = dm2;
      }
      put_rt(l, -0.5 * (dp2 + dm2), -0.5 * (dp2 - dm2));
    }
  }
}

// One thread per (order, point). Layout: tab[(u * L + l) * P + k].
__global__ void k_gsf(int L, int m0, int n_units, int P, const double* pts, double* pt, double* rt,
                      double* tt) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  int u = blockIdx.y;
  if (k >= P || u >= n_units) return;
  size_t base = (size_t)u * L * P + k;
  auto put_p = [&](int l, double d, double) { pt[base + (size_t)l * P] = d; };
  auto put_rt = [&](int l, double r, double t) {
    rt[base + (size_t)l * P] = r;
    tt[base + (size_t)l * P] = t;
  };
  gsf_point<double>(m0 + u, L, pts[k], put_p, put_rt);
}

// Tangent tables for the interface-index derivative: the functions at x(n) in dual
// arithmetic (x' = dpts = dmu_int/dn). Table 1 holds d/dn of the values at the incident
// points and the values themselves elsewhere; table 2 the same for the outgoing points.
// Since each assembled operator S+-(x, y) is bilinear in the tables at x and at y, an
// assembly kernel run on table 1 (2) gives the n-derivative through the incident
// (outgoing) cosines.
__global__ void k_gsf_dn(int L, int m0, int n_units, int N, int n_in, int P, const double* pts,
                         const double* dpts, double* p1, double* r1, double* t1, double* p2,
                         double* r2, double* t2) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  int u = blockIdx.y;
  if (k >= P || u >= n_units) return;
  const bool inc = k >= N && k < N + n_in, out = k >= N + n_in;
  size_t base = (size_t)u * L * P + k;
  auto put_p = [&](int l, dual d, dual) {
    p1[base + (size_t)l * P] = inc ? d.d : d.v;
    p2[base + (size_t)l * P] = out ? d.d : d.v;
  };
  auto put_rt = [&](int l, dual r, dual t) {
    r1[base + (size_t)l * P] = inc ? r.d : r.v;
    t1[base + (size_t)l * P] = inc ? t.d : t.v;
    r2[base + (size_t)l * P] = out ? r.d : r.v;
    t2[base + (size_t)l * P] = out ? t.d : t.v;
  };
  gsf_point<dual>(m0 + u, L, dual{pts[k], dpts[k]}, put_p, put_rt);
}

void launch_gsf_tables(const OrderBatch& b, const double* pts, double* p, double* r, double* t,
                       cudaStream_t s) {
  dim3 grid((b.P + 127) / 128, b.n_units);
  k_gsf<<<grid, 128, 0, s>>>(b.L, b.m0, b.n_units, b.P, pts, p, r, t);
}

void launch_gsf_tables_dn(const OrderBatch& b, const double* pts, const double* dpts, double* p1,
                          double* r1, double* t1, double* p2, double* r2, double* t2,
                          cudaStream_t s) {
  dim3 grid((b.P + 127) / 128, b.n_units);
  k_gsf_dn<<<grid, 128, 0, s>>>(b.L, b.m0, b.n_units, b.N, b.n_in, b.P, pts, dpts, p1, r1, t1, p2,
                                r2, t2);
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
