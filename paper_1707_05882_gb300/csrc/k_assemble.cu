// Step a1: assembly of the order-m operators from the expansion coefficients.
//
// Every operator the path needs is built from the parity-split sums
//   S+-(x, y) = sum_{l=m}^{L-1} P_l^m(x) B_l (I +- (-1)^(l-m) D) P_l^m(y)
// (Sec. 3.A, Eq. 41; P_l^m and B_l as in Eqs. 9-10), where
// (I + (-1)^(l-m) D) is 2 diag(1,1,0,0) for even l-m and 2 diag(0,0,1,1) for odd
// l-m. With p, r, t the entries of P_l^m (p on I and V, r/t on the Q-U block) the
// product P(x) B_l diag(1,1,0,0) P(y) has nine non-zero entries and
// P(x) B_l diag(0,0,1,1) P(y) nine more, so each l costs 18 multiply-adds per
// point pair instead of a dense 4x4x4x4 product.
#include "vrte_internal.cuh"

namespace vrte {

struct SPair {
  double sp[4][4];
  double sm[4][4];
};

// Accumulate S+ and S- for table points kx, ky of order unit u.
__device__ inline void accumulate_S(int m, int L, int P, const double* __restrict__ coef,
                                    const double* __restrict__ pt, const double* __restrict__ rt,
                                    const double* __restrict__ tt, size_t ubase, int kx, int ky,
                                    SPair& S) {
  // buckets: e1/o1 = T1 part for even/odd l-m, e2/o2 = T2 part
  double e1[9] = {0}, o1[9] = {0}, e2[9] = {0}, o2[9] = {0};
  for (int l = m; l < L; ++l) {
    size_t row = ubase + (size_t)l * P;
    double p = pt[row + kx], r = rt[row + kx], t = tt[row + kx];
    double pp = pt[row + ky], rp = rt[row + ky], tp = tt[row + ky];
    const double* c = coef + 6 * l;
    double a1 = c[0], a2 = c[1], a3 = c[2], a4 = c[3], b1 = c[4], b2 = c[5];
    double v1[9], v2[9];
    // T1 = P(x) B diag(1,1,0,0) P(y): rows 0..2, columns 0..2
    v1[0] = p * a1 * pp;  v1[1] = p * b1 * rp;  v1[2] = -p * b1 * tp;
    v1[3] = r * b1 * pp;  v1[4] = r * a2 * rp;  v1[5] = -r * a2 * tp;
    v1[6] = -t * b1 * pp; v1[7] = -t * a2 * rp; v1[8] = t * a2 * tp;
    // T2 = P(x) B diag(0,0,1,1) P(y): rows 1..3, columns 1..3
    v2[0] = t * a3 * tp;  v2[1] = -t * a3 * rp; v2[2] = -t * b2 * pp;
    v2[3] = -r * a3 * tp; v2[4] = r * a3 * rp;  v2[5] = r * b2 * pp;
    v2[6] = p * b2 * tp;  v2[7] = -p * b2 * rp; v2[8] = p * a4 * pp;
    if (((l - m) & 1) == 0) {
#pragma unroll
      for (int q = 0; q < 9; ++q) { e1[q] += v1[q]; e2[q] += v2[q]; }
    } else {
#pragma unroll
      for (int q = 0; q < 9; ++q) { o1[q] += v1[q]; o2[q] += v2[q]; }
    }
  }
  // S+ = 2 (e1 + o2), S- = 2 (o1 + e2), with T1 at (0..2, 0..2) and T2 at (1..3, 1..3)
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) { S.sp[a][b] = 0.0; S.sm[a][b] = 0.0; }
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      S.sp[a][b] += 2.0 * e1[3 * a + b];
      S.sm[a][b] += 2.0 * o1[3 * a + b];
      S.sp[a + 1][b + 1] += 2.0 * o2[3 * a + b];
      S.sm[a + 1][b + 1] += 2.0 * e2[3 * a + b];
    }
}

// Block matrix [[a, b, 0, 0], [b, a, 0, 0], [0, 0, c, d], [0, 0, -d, c]] entry (i, j).
__device__ inline double blk(const double* q, int i, int j) {
  if (i < 2 && j < 2) return i == j ? q[0] : q[1];
  if (i >= 2 && j >= 2) return i == j ? q[2] : (i == 2 ? q[3] : -q[3]);
  return 0.0;
}

// E'[4i+a][4j+b] = (delta - (omega/2) alpha_j S+_ab(i, j)) / mu_i, F' with S-  (Eq. 41,
// in the row-scaled form E' = M^-1 (...) whose product F'E' is similar to the paper's FE).
__global__ void k_assemble_EF(OrderBatch b, const double* pt, const double* rt, const double* tt,
                              const double* mu_nodes, const double* w_nodes, double* E, double* F) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  int i = blockIdx.y;
  int u = blockIdx.z;
  if (j >= b.N) return;
  int m = b.m0 + u;
  SPair S;
  accumulate_S(m, b.L, b.P, b.coef, pt, rt, tt, (size_t)u * b.L * b.P, i, j, S);
  double inv_mu = 1.0 / mu_nodes[i];
  double f = 0.5 * b.omega * w_nodes[j];
  size_t base = (size_t)u * b.n * b.n;
  for (int a = 0; a < 4; ++a)
    for (int c = 0; c < 4; ++c) {
      double delta = (i == j && a == c) ? 1.0 : 0.0;
      size_t idx = base + (size_t)(4 * i + a) * b.n + 4 * j + c;
      E[idx] = (delta - f * S.sp[a][c]) * inv_mu;
      F[idx] = (delta - f * S.sm[a][c]) * inv_mu;
    }
}

void launch_assemble_EF(const OrderBatch& b, const double* p, const double* r, const double* t,
                        const double* mu_nodes, const double* w_nodes, double* E, double* F,
                        cudaStream_t s) {
  dim3 grid((b.N + 63) / 64, b.N, b.n_units);
  k_assemble_EF<<<grid, 64, 0, s>>>(b, p, r, t, mu_nodes, w_nodes, E, F);
}

// Beam vectors of the reduced particular problem (Sec. 3.B, Eq. 47), for the
// collimated source q(+-mu_i) = (omega/2pi) A^m(+-mu_i, -mu0) b_k (Eq. 14):
//   p = M^-1 (q+ + D q-) = (omega/2pi) / mu_i  S+(mu_i, mu0) D b_k
//   r = M^-1 (q+ - D q-) = -(omega/2pi) / mu_i S-(mu_i, mu0) D b_k
// b_k = beam block of incident k (columns = incident Stokes basis vectors).
// Layout Pm[u][4i+a][4k+s].
__global__ void k_assemble_beam(OrderBatch b, const double* pt, const double* rt, const double* tt,
                                const double* mu_nodes, const double* min4, double* Pm,
                                double* Rm) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  int i = blockIdx.y;
  int u = blockIdx.z;
  if (k >= b.n_in) return;
  int m = b.m0 + u;
  SPair S;
  accumulate_S(m, b.L, b.P, b.coef, pt, rt, tt, (size_t)u * b.L * b.P, i, b.N + k, S);
  double cq = b.omega / (2.0 * kPi) / mu_nodes[i];
  const double* q = min4 + 4 * k;
  int R = 4 * b.n_in;
  size_t base = (size_t)u * b.n * R;
  for (int a = 0; a < 4; ++a)
    for (int s = 0; s < 4; ++s) {
      double vp = 0.0, vm = 0.0;
      for (int c = 0; c < 4; ++c) {
        double db = (c < 2 ? 1.0 : -1.0) * blk(q, c, s);
        vp += S.sp[a][c] * db;
        vm += S.sm[a][c] * db;
      }
      size_t idx = base + (size_t)(4 * i + a) * R + 4 * k + s;
      Pm[idx] = cq * vp;
      Rm[idx] = -cq * vm;
    }
}

void launch_assemble_beam(const OrderBatch& b, const double* p, const double* r, const double* t,
                          const double* mu_nodes, const double* min4, double* Pm, double* Rm,
                          cudaStream_t s) {
  dim3 grid((b.n_in + 63) / 64, b.N, b.n_units);
  k_assemble_beam<<<grid, 64, 0, s>>>(b, p, r, t, mu_nodes, min4, Pm, Rm);
}

// Reconstruction operators (Sec. 2.C, Eq. 38 and Sec. 3.D): the scattering part of the
// source at outgoing mu_o acting on a nodal field, split by the same parity sums:
//   U+-[4o+a][4j+c] = (omega/4) alpha_j (M_out[o] S+-(mu_o, mu_j))_ac.
// Stored as Upm[u][4o+a][0..2n) = [U+ | U-] (row stride b.ldU).
__global__ void k_assemble_U(OrderBatch b, const double* pt, const double* rt, const double* tt,
                             const double* w_nodes, const double* mout4, double* U) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  int o = blockIdx.y;
  int u = blockIdx.z;
  if (j >= b.N) return;
  int m = b.m0 + u;
  SPair S;
  accumulate_S(m, b.L, b.P, b.coef, pt, rt, tt, (size_t)u * b.L * b.P, b.N + b.n_in + o, j, S);
  double f = 0.25 * b.omega * w_nodes[j];
  const double* q = mout4 + 4 * o;
  size_t base = (size_t)u * (4 * b.n_out) * b.ldU;
  for (int a = 0; a < 4; ++a)
    for (int c = 0; c < 4; ++c) {
      double vp = 0.0, vm = 0.0;
      for (int e = 0; e < 4; ++e) {
        double mo = blk(q, a, e);
        vp += mo * S.sp[e][c];
        vm += mo * S.sm[e][c];
      }
      size_t row = base + (size_t)(4 * o + a) * b.ldU;
      U[row + 4 * j + c] = f * vp;
      U[row + b.n + 4 * j + c] = f * vm;
    }
}

void launch_assemble_U(const OrderBatch& b, const double* p, const double* r, const double* t,
                       const double* w_nodes, const double* mout4, double* U, cudaStream_t s) {
  dim3 grid((b.N + 63) / 64, b.n_out, b.n_units);
  k_assemble_U<<<grid, 64, 0, s>>>(b, p, r, t, w_nodes, mout4, U);
}

// Direct (once-scattered) source term of the reconstruction (Eq. 38, Q term), already
// multiplied by the depth integral g0 of exp(-t/mu0) along the exit path:
//   T1[u][4o+a][4k+s] = g0(o, k) (omega/2pi) (M_out[o] A^m(mu_o, -mu0_k) b_k)_as,
//   A^m(x, -y) = (S+(x, y) - S-(x, y)) D / 2,
//   g0 = (1 - exp(-tau0 (1/mu_o + 1/mu0))) / (mu_o (1/mu_o + 1/mu0)).
__global__ void k_assemble_direct(OrderBatch b, const double* pt, const double* rt,
                                  const double* tt, const double* pts, const double* min4,
                                  const double* mout4, double* T1) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  int o = blockIdx.y;
  int u = blockIdx.z;
  if (k >= b.n_in) return;
  int m = b.m0 + u;
  SPair S;
  accumulate_S(m, b.L, b.P, b.coef, pt, rt, tt, (size_t)u * b.L * b.P, b.N + b.n_in + o, b.N + k,
               S);
  double mu_o = pts[b.N + b.n_in + o], mu0 = pts[b.N + k];
  double xs = 1.0 / mu_o + 1.0 / mu0;
  double g0 = -expm1(-b.tau * xs) / (mu_o * xs);
  double f = g0 * b.omega / (2.0 * kPi) * 0.5;
  const double* qi = min4 + 4 * k;
  const double* qo = mout4 + 4 * o;
  int R = 4 * b.n_in;
  size_t base = (size_t)u * (4 * b.n_out) * R;
  double A[4][4];
  for (int a = 0; a < 4; ++a)
    for (int c = 0; c < 4; ++c) A[a][c] = (S.sp[a][c] - S.sm[a][c]) * (c < 2 ? 1.0 : -1.0);
  for (int a = 0; a < 4; ++a)
    for (int s = 0; s < 4; ++s) {
      double v = 0.0;
      for (int e = 0; e < 4; ++e) {
        double mo = blk(qo, a, e);
        if (mo == 0.0) continue;
        double w = 0.0;
        for (int c = 0; c < 4; ++c) w += A[e][c] * blk(qi, c, s);
        v += mo * w;
      }
      T1[base + (size_t)(4 * o + a) * R + 4 * k + s] = f * v;
    }
}

void launch_assemble_direct(const OrderBatch& b, const double* p, const double* r,
                            const double* t, const double* pts, const double* min4,
                            const double* mout4, double* T1, cudaStream_t s) {
  dim3 grid((b.n_in + 63) / 64, b.n_out, b.n_units);
  k_assemble_direct<<<grid, 64, 0, s>>>(b, p, r, t, pts, min4, mout4, T1);
}

// Direct (once-scattered) term of the radiance at depth tau (0 <= tau <= tau0) inside the
// layer, internal cosine mu_o (identity exit): the source (omega/2pi) A^m(+-mu_o, -mu0_k) b_k
// e^{-t/mu0} integrated along the path, upward (sign +) or downward (sign -):
//   A^m(x, -y) = (S+(x, y) - S-(x, y)) D / 2,  A^m(-x, -y) = D (S+(x, y) + S-(x, y)) D / 2,
// depth factors (x = 1/mu_o, y = 1/mu0, D(a, b; T) = (e^{-aT} - e^{-bT})/(b - a)):
//   upward x e^{-y tau} D(0, x + y; tau0 - tau),  downward x D(y, x; tau).
__global__ void k_assemble_direct_depth(OrderBatch b, double tau, int down, const double* pt,
                                        const double* rt, const double* tt, const double* pts,
                                        const double* min4, double* T) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  int o = blockIdx.y;
  int u = blockIdx.z;
  if (k >= b.n_in) return;
  int m = b.m0 + u;
  SPair S;
  accumulate_S(m, b.L, b.P, b.coef, pt, rt, tt, (size_t)u * b.L * b.P, b.N + b.n_in + o, b.N + k,
               S);
  const double x = 1.0 / pts[b.N + b.n_in + o], y = 1.0 / pts[b.N + k];
  auto dd = [](double a, double bb, double Tl) {
    const double d = bb - a;
    if (d == 0.0) return Tl * exp(-a * Tl);
    if (fabs(d * Tl) < 1e-2) return exp(-a * Tl) * -expm1(-d * Tl) / d;
    return (exp(-a * Tl) - exp(-bb * Tl)) / d;
  };
  const double g = down ? x * dd(y, x, tau) : x * exp(-y * tau) * dd(0.0, x + y, b.tau - tau);
  const double f = g * b.omega / (2.0 * kPi) * 0.5;
  const double* qi = min4 + 4 * k;
  const int R = 4 * b.n_in;
  const size_t base = (size_t)u * (4 * b.n_out) * R;
  for (int a = 0; a < 4; ++a)
    for (int s = 0; s < 4; ++s) {
      double v = 0.0;
      for (int c = 0; c < 4; ++c) {
        const double dc = c < 2 ? 1.0 : -1.0;
        v += (down ? (S.sp[a][c] + S.sm[a][c]) : (S.sp[a][c] - S.sm[a][c])) * dc * blk(qi, c, s);
      }
      T[base + (size_t)(4 * o + a) * R + 4 * k + s] = f * (down && a >= 2 ? -1.0 : 1.0) * v;
    }
}

void launch_assemble_direct_depth(const OrderBatch& b, double tau, int down, const double* p,
                                  const double* r, const double* t, const double* pts,
                                  const double* min4, double* T, cudaStream_t s) {
  dim3 grid((b.n_in + 63) / 64, b.n_out, b.n_units);
  k_assemble_direct_depth<<<grid, 64, 0, s>>>(b, tau, down, p, r, t, pts, min4, T);
}

// Direct-term operators for the mixed form (Eq. 38, Q term, as a contraction over the
// pairs (l, component c) so that the tensor cores can fold it into the particular
// contraction): with P = P_l^m and B = B_l,
//   Adir[(o, a), (l, c)] = (M_out[o] P(mu_o) B)_ac,
//   Bdir[(l, c), (k, s)] = (omega/2pi) (-1)^(l-m) (D P(mu0_k) D b_k)_cs,
// so that sum_{l,c} Adir Bdir = (omega/2pi) M_out A^m(mu_o, -mu0) b_k; zero for l < m.
__global__ void k_direct_A(OrderBatch b, const double* pt, const double* rt, const double* tt,
                           const double* mout4, double* Uext) {
  int l = blockIdx.x * blockDim.x + threadIdx.x;
  int o = blockIdx.y, u = blockIdx.z;
  if (l >= b.L) return;
  int m = b.m0 + u;
  double* row0 = Uext + (size_t)u * (4 * b.n_out) * b.ldU + (size_t)(4 * o) * b.ldU + 2 * b.n + 4 * l;
  double PB[4][4];
  for (int a = 0; a < 4; ++a)
    for (int c = 0; c < 4; ++c) PB[a][c] = 0.0;
  if (l >= m) {
    size_t idx = (size_t)u * b.L * b.P + (size_t)l * b.P + b.N + b.n_in + o;
    double p = pt[idx], r = rt[idx], t = tt[idx];
    const double* cf = b.coef + 6 * l;
    double Bm[4][4] = {{cf[0], cf[4], 0.0, 0.0}, {cf[4], cf[1], 0.0, 0.0},
                       {0.0, 0.0, cf[2], cf[5]}, {0.0, 0.0, -cf[5], cf[3]}};
    double P[4][4] = {{p, 0, 0, 0}, {0, r, -t, 0}, {0, -t, r, 0}, {0, 0, 0, p}};
    const double* q = mout4 + 4 * o;
    for (int a = 0; a < 4; ++a)
      for (int c = 0; c < 4; ++c) {
        double v = 0.0;
        for (int e = 0; e < 4; ++e) {
          double mp = 0.0;
          for (int f = 0; f < 4; ++f) mp += blk(q, a, f) * P[f][e];
          v += mp * Bm[e][c];
        }
        PB[a][c] = v;
      }
  }
  for (int a = 0; a < 4; ++a)
    for (int c = 0; c < 4; ++c) row0[(size_t)a * b.ldU + c] = PB[a][c];
}

__global__ void k_direct_B(OrderBatch b, const double* pt, const double* rt, const double* tt,
                           const double* min4, double* SDext) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  int l = blockIdx.y, u = blockIdx.z;
  if (k >= b.n_in) return;
  int m = b.m0 + u;
  int R = 4 * b.n_in;
  double* col0 = SDext + (size_t)u * b.sSD + (size_t)(2 * b.n + 4 * l) * R + 4 * k;
  double V[4][4];
  for (int c = 0; c < 4; ++c)
    for (int s = 0; s < 4; ++s) V[c][s] = 0.0;
  if (l >= m) {
    size_t idx = (size_t)u * b.L * b.P + (size_t)l * b.P + b.N + k;
    double p = pt[idx], r = rt[idx], t = tt[idx];
    // D P D flips the sign of the t entries
    double P[4][4] = {{p, 0, 0, 0}, {0, r, t, 0}, {0, t, r, 0}, {0, 0, 0, p}};
    double f = b.omega / (2.0 * kPi) * (((l - m) & 1) ? -1.0 : 1.0);
    const double* q = min4 + 4 * k;
    for (int c = 0; c < 4; ++c)
      for (int s = 0; s < 4; ++s) {
        double v = 0.0;
        for (int e = 0; e < 4; ++e) v += P[c][e] * blk(q, e, s);
        V[c][s] = f * v;
      }
  }
  for (int c = 0; c < 4; ++c)
    for (int s = 0; s < 4; ++s) col0[(size_t)c * R + s] = V[c][s];
}

void launch_direct_operators(const OrderBatch& b, const double* p, const double* r,
                             const double* t, const double* min4, const double* mout4,
                             double* Uext, double* SDext, cudaStream_t s) {
  dim3 ga((b.L + 63) / 64, b.n_out, b.n_units);
  k_direct_A<<<ga, 64, 0, s>>>(b, p, r, t, mout4, Uext);
  dim3 gb((b.n_in + 63) / 64, b.L, b.n_units);
  k_direct_B<<<gb, 64, 0, s>>>(b, p, r, t, min4, SDext);
}

__global__ void k_depth_table(int N, int n_in, int n_out, double tau, const double* pts,
                              double* g0tab) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  int o = blockIdx.y;
  if (k >= n_in) return;
  g0tab[(size_t)o * n_in + k] = depth_factor(tau, pts[N + n_in + o], pts[N + k]);
}

// The layer's beam table after the depth factors: e^{-tau0/mu0} and 1/mu0 per incident cosine.
__global__ void k_beam_table(int N, int n_in, double tau, const double* pts, double* btab) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_in) return;
  const double rm = 1.0 / pts[N + k];
  btab[k] = exp(-tau * rm);
  btab[n_in + k] = rm;
}

void launch_depth_table(int N, int n_in, int n_out, double tau, const double* pts, double* g0tab,
                        cudaStream_t s) {
  k_depth_table<<<dim3((n_in + 127) / 128, n_out), 128, 0, s>>>(N, n_in, n_out, tau, pts, g0tab);
  k_beam_table<<<(n_in + 127) / 128, 128, 0, s>>>(N, n_in, tau, pts,
                                                  g0tab + (size_t)n_in * n_out);
}

// ------------------------------------------------------------------ mixed-form operators
// S+-(x, y) = sum_l [P_l(x) B_l] [(I +- (-1)^(l-m) D) P_l(y)] is a contraction over the 4L
// pairs (l, component e). The mixed form builds the two factors and lets the sliced
// tensor-core GEMM do the sum (Sec. 3.A-3.D):
//   U+-            = Adir (M_out P(mu_o) B, from k_direct_A) x RU+-,
//   RU+-[(l,e)][(j,c)] = (omega/4) alpha_j ((I +- (-1)^(l-m) D) P_l(mu_j))_ec,
//   beam p = Ln x Rb+,  beam r = Ln x Rb-,
//   Ln[(i,a)][(l,e)]   = (omega/2pi) / mu_i (P_l(mu_i) B_l)_ae,
//   Rb+[(l,e)][(k,s)]  = ((I + (-1)^(l-m) D) P_l(mu0_k) D b_k)_es,
//   Rb-[(l,e)][(k,s)]  = -((I - (-1)^(l-m) D) P_l(mu0_k) D b_k)_es.
// All factors vanish for l < m.
__device__ inline void p_matrix(double p, double r, double t, double P[4][4]) {
  for (int a = 0; a < 4; ++a)
    for (int c = 0; c < 4; ++c) P[a][c] = 0.0;
  P[0][0] = p; P[1][1] = r; P[1][2] = -t; P[2][1] = -t; P[2][2] = r; P[3][3] = p;
}

__global__ void k_left_nodes(OrderBatch b, const double* pt, const double* rt, const double* tt,
                             const double* mu_nodes, double* Ln) {
  int l = blockIdx.x * blockDim.x + threadIdx.x;
  int i = blockIdx.y, u = blockIdx.z;
  if (l >= b.L) return;
  int m = b.m0 + u;
  const int ld = 4 * b.L;
  double* row0 = Ln + (size_t)u * b.n * ld + (size_t)(4 * i) * ld + 4 * l;
  double V[4][4];
  for (int a = 0; a < 4; ++a)
    for (int e = 0; e < 4; ++e) V[a][e] = 0.0;
  if (l >= m) {
    size_t idx = (size_t)u * b.L * b.P + (size_t)l * b.P + i;
    double P[4][4];
    p_matrix(pt[idx], rt[idx], tt[idx], P);
    const double* cf = b.coef + 6 * l;
    double Bm[4][4] = {{cf[0], cf[4], 0.0, 0.0}, {cf[4], cf[1], 0.0, 0.0},
                       {0.0, 0.0, cf[2], cf[5]}, {0.0, 0.0, -cf[5], cf[3]}};
    double f = b.omega / (2.0 * kPi) / mu_nodes[i];
    for (int a = 0; a < 4; ++a)
      for (int e = 0; e < 4; ++e) {
        double v = 0.0;
        for (int c = 0; c < 4; ++c) v += P[a][c] * Bm[c][e];
        V[a][e] = f * v;
      }
  }
  for (int a = 0; a < 4; ++a)
    for (int e = 0; e < 4; ++e) row0[(size_t)a * ld + e] = V[a][e];
}

__global__ void k_right_nodes(OrderBatch b, const double* pt, const double* rt, const double* tt,
                              const double* w_nodes, double* RU) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  int l = blockIdx.y, u = blockIdx.z;
  if (j >= b.N) return;
  int m = b.m0 + u;
  const int ld = 2 * b.n;
  double* base = RU + (size_t)u * (4 * b.L) * ld + (size_t)(4 * l) * ld;
  double Vp[4][4], Vm[4][4];
  for (int e = 0; e < 4; ++e)
    for (int c = 0; c < 4; ++c) Vp[e][c] = Vm[e][c] = 0.0;
  if (l >= m) {
    size_t idx = (size_t)u * b.L * b.P + (size_t)l * b.P + j;
    double P[4][4];
    p_matrix(pt[idx], rt[idx], tt[idx], P);
    double par = ((l - m) & 1) ? -1.0 : 1.0;
    double f = 0.25 * b.omega * w_nodes[j];
    for (int e = 0; e < 4; ++e) {
      double de = par * (e < 2 ? 1.0 : -1.0);  // (-1)^(l-m) D_ee
      for (int c = 0; c < 4; ++c) {
        Vp[e][c] = f * (1.0 + de) * P[e][c];
        Vm[e][c] = f * (1.0 - de) * P[e][c];
      }
    }
  }
  for (int e = 0; e < 4; ++e)
    for (int c = 0; c < 4; ++c) {
      base[(size_t)e * ld + 4 * j + c] = Vp[e][c];
      base[(size_t)e * ld + b.n + 4 * j + c] = Vm[e][c];
    }
}

__global__ void k_right_beam(OrderBatch b, const double* pt, const double* rt, const double* tt,
                             const double* min4, double* Rp, double* Rm) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  int l = blockIdx.y, u = blockIdx.z;
  if (k >= b.n_in) return;
  int m = b.m0 + u;
  const int R = 4 * b.n_in;
  size_t off = (size_t)u * (4 * b.L) * R + (size_t)(4 * l) * R + 4 * k;
  double Vp[4][4], Vm[4][4];
  for (int e = 0; e < 4; ++e)
    for (int s = 0; s < 4; ++s) Vp[e][s] = Vm[e][s] = 0.0;
  if (l >= m) {
    size_t idx = (size_t)u * b.L * b.P + (size_t)l * b.P + b.N + k;
    double P[4][4];
    p_matrix(pt[idx], rt[idx], tt[idx], P);
    double par = ((l - m) & 1) ? -1.0 : 1.0;
    const double* q = min4 + 4 * k;
    for (int e = 0; e < 4; ++e) {
      double de = par * (e < 2 ? 1.0 : -1.0);
      for (int s = 0; s < 4; ++s) {
        double v = 0.0;  // (P D b)_es
        for (int c = 0; c < 4; ++c) v += P[e][c] * (c < 2 ? 1.0 : -1.0) * blk(q, c, s);
        Vp[e][s] = (1.0 + de) * v;
        Vm[e][s] = -(1.0 - de) * v;
      }
    }
  }
  for (int e = 0; e < 4; ++e)
    for (int s = 0; s < 4; ++s) {
      Rp[off + (size_t)e * R + s] = Vp[e][s];
      Rm[off + (size_t)e * R + s] = Vm[e][s];
    }
}

void launch_mixed_operators(const OrderBatch& b, const double* p, const double* r,
                            const double* t, const double* mu_nodes, const double* w_nodes,
                            const double* min4, double* Ln, double* RU, double* Rp, double* Rm,
                            cudaStream_t s) {
  k_left_nodes<<<dim3((b.L + 63) / 64, b.N, b.n_units), 64, 0, s>>>(b, p, r, t, mu_nodes, Ln);
  k_right_nodes<<<dim3((b.N + 63) / 64, b.L, b.n_units), 64, 0, s>>>(b, p, r, t, w_nodes, RU);
  k_right_beam<<<dim3((b.n_in + 63) / 64, b.L, b.n_units), 64, 0, s>>>(b, p, r, t, min4, Rp, Rm);
}

}  // namespace vrte
