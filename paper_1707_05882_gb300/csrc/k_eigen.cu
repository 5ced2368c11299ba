// Step a2: batched FP64 eigen-decomposition of the reduced homogeneous matrix F'E'
// (Sec. 3.A, Eqs. 43-45), one CTA per Fourier order.
//
// The paper calls a CPU library (EIGEN) for this step, sequentially per order, and names
// it the bottleneck; here every order's matrix is decomposed concurrently. The
// algorithm is the textbook one (Golub & Van Loan, "Matrix Computations", 4th ed.,
// Sec. 7.4-7.6):
//   1. diagonal balancing by powers of two (Parlett-Reinsch), which keeps the small
//      eigenvalues of this strongly graded matrix accurate;
//   2. Householder reduction to upper Hessenberg form, accumulating Z;
//   3. Francis implicit double-shift QR sweeps with deflation on small
//      subdiagonals and the classical exceptional shifts after 10 and 20 stalled
//      sweeps (the shift strategy of the published QR algorithm as in EISPACK/LAPACK
//      hqr), applied to the full matrix so that H becomes the real Schur form T
//      and Z its Schur vectors; 2x2 blocks with real eigenvalues are split by a
//      rotation, so remaining 2x2 blocks hold complex-conjugate pairs;
//   4. eigenvectors of T by back-substitution (complex arithmetic for pairs), one warp
//      per eigenvector.
// Eigenvectors of the input are X = D Z V (finished by a GEMM and `finish_eigvec`).
// Output convention: for a pair (j, j+1), lam_im[j] > 0 and the eigenvector of
// lam_re[j] + i lam_im[j] is X[:, j] + i X[:, j+1].
// Storage: H row-major; Z and V column-major (column c at [c * n]).
#include <algorithm>

#include "vrte_internal.cuh"

namespace vrte {

constexpr int EIG_THREADS = 512;
constexpr double EPS = 2.220446049250313e-16;
constexpr double SAFMIN = 2.2250738585072014e-308;

// Householder reflector P = I - tau v v^T with v[0] = 1 mapping (x, y, z) to (beta, 0, 0),
// beta = -sign(x) |(x, y, z)|: tau = (beta - x) / beta = 1 + |x| / |(x, y, z)| and
// v = (y, z) / (x - beta) = sign(x) (y, z) / (|x| + |(x, y, z)|), from one reciprocal square
// root and one division (FP64 instructions are scarce on this part).
__device__ inline void house3(double x, double y, double z, double& tau, double& v1, double& v2) {
  const double s2 = fma(z, z, fma(y, y, x * x));
  if (s2 == 0.0 || (y == 0.0 && z == 0.0)) { tau = 0.0; v1 = 0.0; v2 = 0.0; return; }
  const double r = rsqrt(s2);
  const double nrm = s2 * r;
  tau = fma(fabs(x), r, 1.0);
  const double sc = copysign(1.0, x) / (fabs(x) + nrm);
  v1 = y * sc;
  v2 = z * sc;
}

// sum_i v[i] p[i s]: the loads of eight terms are issued before their multiply-adds, into two
// partial sums (a single running sum waited on each load in turn)
__device__ inline double dotv(int len, const double* v, const double* p, size_t s) {
  double w0 = 0.0, w1 = 0.0;
  int i = 0;
  for (; i + 8 <= len; i += 8, p += 8 * s) {
    double a[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) a[q] = p[q * s];
#pragma unroll
    for (int q = 0; q < 8; q += 2) {
      w0 = fma(v[i + q], a[q], w0);
      w1 = fma(v[i + q + 1], a[q + 1], w1);
    }
  }
  for (; i < len; ++i, p += s) w0 = fma(v[i], p[0], w0);
  return w0 + w1;
}

// p[i s] -= v[i] w, eight loads issued before their updates (a store and the next load are
// otherwise kept in order, the compiler not knowing that they never overlap)
__device__ inline void axpyv(int len, const double* v, double* p, size_t s, double w) {
  int i = 0;
  for (; i + 8 <= len; i += 8, p += 8 * s) {
    double a[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) a[q] = p[q * s];
#pragma unroll
    for (int q = 0; q < 8; ++q) p[q * s] = fma(-v[i + q], w, a[q]);
  }
  for (; i < len; ++i, p += s) p[0] = fma(-v[i], w, p[0]);
}

__global__ void __launch_bounds__(EIG_THREADS, 1) k_eigen(int n, const double* __restrict__ A,
                                                       double* Hbuf, double* Zbuf, double* Vbuf,
                                                       double* lam_re, double* lam_im,
                                                       double* scale, const int* mask,
                                                       unsigned* status) {
  extern __shared__ double vsh[];  // Householder vector of the Hessenberg step, n entries;
                                   // the balancing's norms and scalings, 3 n more
  __shared__ double red[32];
  __shared__ double hred[4];    // Hessenberg step: (|x|^2 below the subdiagonal, beta, tau, 1/(alpha - beta))
  __shared__ int ired[32];
  __shared__ double W[8][8];     // sweep: warp 0's window of H, element (r, c) at [r & 7][c & 7]
  __shared__ double refl[2][5];  // reflectors (tau, v1, v2, tau v1, tau v2) of the current
                                 // and the next sweep step
  int u = blockIdx.x;
  if (mask && !mask[u]) return;
  int tid = threadIdx.x, nt = blockDim.x;
  int lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
  double* H = Hbuf + (size_t)u * n * n;
  double* Z = Zbuf + (size_t)u * n * n;
  double* V = Vbuf + (size_t)u * n * n;
  double* wr = lam_re + (size_t)u * n;
  double* wi = lam_im + (size_t)u * n;
  double* dsc = scale + (size_t)u * n;
  const double* Ab = A + (size_t)u * n * n;

  for (size_t e = tid; e < (size_t)n * n; e += nt) {
    H[e] = Ab[e];
    int r = (int)(e / n), c = (int)(e - (size_t)r * n);
    Z[e] = (r == c) ? 1.0 : 0.0;  // column-major identity is the identity
  }
  for (int i = tid; i < n; i += nt) dsc[i] = 1.0;
  __syncthreads();

  // ---- 1. balancing: D^-1 H D with power-of-two entries (Parlett-Reinsch criterion). Each
  // sweep takes the off-diagonal row and column norms of every index at once and rescales,
  // together, every index whose scaling by 2^e, e = rint(log2(r / c) / 4), lowers c + r by
  // more than 5 %, until a sweep changes nothing. Deciding all indices from one set of norms
  // costs two passes over H per sweep instead of one barrier per index; the quarter (not
  // half) of log2(r / c) damps the simultaneous steps, which otherwise can oscillate between
  // two scalings, to the norm the one-index-at-a-time sweeps reach.
  {
    double* cn = vsh + n;   // column norms, then the inverse scalings
    double* rn = cn + n;    // row norms
    double* fs = rn + n;    // scaling of the sweep (1 = none)
    for (int sweep = 0; sweep < 32; ++sweep) {
      for (int j = tid; j < n; j += nt) {
        double c0 = 0.0, c1 = 0.0;
        for (int i = 0; i + 1 < n; i += 2) {
          c0 += (i == j) ? 0.0 : fabs(H[(size_t)i * n + j]);
          c1 += (i + 1 == j) ? 0.0 : fabs(H[(size_t)(i + 1) * n + j]);
        }
        if (n & 1) c0 += (n - 1 == j) ? 0.0 : fabs(H[(size_t)(n - 1) * n + j]);
        cn[j] = c0 + c1;
      }
      for (int i = warp; i < n; i += nwarps) {
        double r = 0.0;
        for (int j = lane; j < n; j += 32) r += (j == i) ? 0.0 : fabs(H[(size_t)i * n + j]);
        for (int off = 16; off > 0; off >>= 1) r += __shfl_xor_sync(0xffffffffu, r, off);
        if (lane == 0) rn[i] = r;
      }
      __syncthreads();
      int changed = 0;
      for (int i = tid; i < n; i += nt) {
        const double c = cn[i], r = rn[i];
        double f = 1.0, finv = 1.0;
        if (c > 0.0 && r > 0.0 && isfinite(c) && isfinite(r)) {
          const int e2 = (int)rint(0.25 * log2(r / c));
          if (e2 != 0) {
            const double ff = ldexp(1.0, e2);
            if (!(c * ff + r / ff >= 0.95 * (c + r))) { f = ff; finv = ldexp(1.0, -e2); }
          }
        }
        fs[i] = f;
        cn[i] = finv;  // this thread's own entry, read above
        if (f != 1.0) changed = 1;
      }
      if (!__syncthreads_or(changed)) break;
      // H[i][j] <- H[i][j] f_j / f_i (exact: powers of two)
      for (size_t e = tid; e < (size_t)n * n; e += nt) {
        const int i = (int)(e / n), j = (int)(e - (size_t)i * n);
        if (fs[i] != 1.0 || fs[j] != 1.0) H[e] = H[e] * fs[j] * cn[i];
      }
      for (int i = tid; i < n; i += nt) dsc[i] *= fs[i];
      __syncthreads();
    }
  }
  __syncthreads();

  // ---- 2. Householder reduction to Hessenberg form, Z <- Z (I - tau v v^T)
  // The reflector of each column comes from warp 0 alone; the right update runs a thread
  // per row (a sequential dot product, no shuffle reductions), like the Z update.
  for (int k = 0; k + 2 < n; ++k) {
    if (warp == 0) {
      double xs = 0.0;
      for (int i = k + 2 + lane; i < n; i += 32) {
        const double v = H[(size_t)i * n + k];
        xs = fma(v, v, xs);
      }
      for (int off = 16; off > 0; off >>= 1) xs += __shfl_xor_sync(0xffffffffu, xs, off);
      double beta = 0.0, tau = 0.0, sc = 0.0;
      if (xs != 0.0) {
        const double alpha = H[(size_t)(k + 1) * n + k];
        beta = -copysign(sqrt(fma(alpha, alpha, xs)), alpha);
        tau = (beta - alpha) / beta;
        sc = 1.0 / (alpha - beta);
      }
      if (lane == 0) { hred[0] = xs; hred[1] = beta; hred[2] = tau; hred[3] = sc; }
    }
    __syncthreads();
    if (hred[0] == 0.0) {  // uniform: the column is already reduced
      __syncthreads();     // hred is rewritten for the next column only after every read
      continue;
    }
    const double beta = hred[1], tau = hred[2], sc = hred[3];
    int len = n - k - 1;
    for (int i = tid; i < len; i += nt) vsh[i] = (i == 0) ? 1.0 : H[(size_t)(k + 1 + i) * n + k] * sc;
    __syncthreads();
    for (int i = tid; i < len; i += nt) H[(size_t)(k + 1 + i) * n + k] = (i == 0) ? beta : 0.0;
    // left: rows k+1.., columns k+1..
    for (int j = k + 1 + tid; j < n; j += nt) {
      double* Hj = H + (size_t)(k + 1) * n + j;
      const double w = dotv(len, vsh, Hj, n) * tau;
      axpyv(len, vsh, Hj, n, w);
    }
    __syncthreads();
    // right: every row of H and of Z (thread per row; Z column-major)
    for (int i = tid; i < n; i += nt) {
      double* Hi = H + (size_t)i * n + k + 1;
      const double w = dotv(len, vsh, Hi, 1) * tau;
      axpyv(len, vsh, Hi, 1, w);
    }
    for (int i = tid; i < n; i += nt) {
      double* Zi = Z + (size_t)(k + 1) * n + i;
      const double w = dotv(len, vsh, Zi, n) * tau;
      axpyv(len, vsh, Zi, n, w);
    }
    __syncthreads();
  }

  // norm estimate for deflation of zero diagonals
  double hn = 0.0;
  for (size_t e = tid; e < (size_t)n * n; e += nt) hn = fmax(hn, fabs(H[e]));
  for (int off = 16; off > 0; off >>= 1) hn = fmax(hn, __shfl_xor_sync(0xffffffffu, hn, off));
  __syncthreads();
  if (lane == 0) red[warp] = hn;
  __syncthreads();
  hn = 0.0;
  for (int i = 0; i < nwarps; ++i) hn = fmax(hn, red[i]);
  __syncthreads();
  const double smlnum = SAFMIN * (double)n / EPS;

  // ---- 3. Francis double-shift QR on the full matrix
  int hi = n - 1;
  int its = 0;
  long total = 0;
  const long max_total = 60L * n;
  while (hi >= 0) {
    // deflation scan: the largest l in [1, hi] with a negligible H[l][l-1] (0 if none),
    // every thread testing its own positions from the top, then a block max
    int lf = 0;
    for (int l2 = hi - tid; l2 > 0; l2 -= nt) {
      double sub = fabs(H[(size_t)l2 * n + l2 - 1]);
      double tst = fabs(H[(size_t)(l2 - 1) * n + l2 - 1]) + fabs(H[(size_t)l2 * n + l2]);
      if (tst == 0.0) tst = hn;
      if (sub <= fmax(smlnum, EPS * tst)) { lf = l2; break; }
    }
    lf = __reduce_max_sync(0xffffffffu, lf);
    if (lane == 0) ired[warp] = lf;
    __syncthreads();
    int l = 0;
    for (int i = 0; i < nwarps; ++i) l = max(l, ired[i]);
    __syncthreads();
    if (l > 0 && tid == 0) H[(size_t)l * n + l - 1] = 0.0;
    __syncthreads();
    if (l == hi) {  // 1x1 block
      if (tid == 0) { wr[hi] = H[(size_t)hi * n + hi]; wi[hi] = 0.0; }
      hi -= 1;
      its = 0;
      __syncthreads();
      continue;
    }
    if (l == hi - 1) {  // 2x2 block: split if real, record if complex
      int k = hi - 1;
      double a = H[(size_t)k * n + k], b = H[(size_t)k * n + hi];
      double c = H[(size_t)hi * n + k], d = H[(size_t)hi * n + hi];
      double p = 0.5 * (a - d);
      double disc = p * p + b * c;
      if (disc >= 0.0) {
        double z = p + copysign(sqrt(disc), p);
        double la = d + z;
        // eigenvector of la: (b, la - a) or (la - d, c)
        double v1 = b, v2 = la - a;
        double w1 = la - d, w2 = c;
        if (fabs(w1) + fabs(w2) > fabs(v1) + fabs(v2)) { v1 = w1; v2 = w2; }
        double nv = hypot(v1, v2);
        double cs = 1.0, sn = 0.0;
        if (nv > 0.0) { cs = v1 / nv; sn = v2 / nv; }
        __syncthreads();
        // rows k, hi (columns k..n-1): G^T
        for (int j = k + tid; j < n; j += nt) {
          double x1 = H[(size_t)k * n + j], x2 = H[(size_t)hi * n + j];
          H[(size_t)k * n + j] = cs * x1 + sn * x2;
          H[(size_t)hi * n + j] = -sn * x1 + cs * x2;
        }
        __syncthreads();
        // columns k, hi (rows 0..hi): G; Z columns k, hi
        for (int i = tid; i <= hi; i += nt) {
          double x1 = H[(size_t)i * n + k], x2 = H[(size_t)i * n + hi];
          H[(size_t)i * n + k] = cs * x1 + sn * x2;
          H[(size_t)i * n + hi] = -sn * x1 + cs * x2;
        }
        for (int i = tid; i < n; i += nt) {
          double x1 = Z[(size_t)k * n + i], x2 = Z[(size_t)hi * n + i];
          Z[(size_t)k * n + i] = cs * x1 + sn * x2;
          Z[(size_t)hi * n + i] = -sn * x1 + cs * x2;
        }
        __syncthreads();
        if (tid == 0) {
          H[(size_t)hi * n + k] = 0.0;
          wr[k] = H[(size_t)k * n + k];
          wi[k] = 0.0;
          wr[hi] = H[(size_t)hi * n + hi];
          wi[hi] = 0.0;
        }
      } else {
        if (tid == 0) {
          double im = sqrt(-disc);
          wr[k] = 0.5 * (a + d); wi[k] = im;
          wr[hi] = 0.5 * (a + d); wi[hi] = -im;
        }
      }
      hi -= 2;
      its = 0;
      __syncthreads();
      continue;
    }
    // Francis double-shift sweep on the active window [l, hi]
    ++its;
    ++total;
    if (total > max_total) {
      if (tid == 0) {
        atomicOr(status, ST_NO_CONVERGENCE);
        for (int i = 0; i <= hi; ++i) { wr[i] = H[(size_t)i * n + i]; wi[i] = 0.0; }
      }
      break;
    }
    // The reflectors of the sweep are computed by warp 0 alone (FP64 square roots and
    // divisions are scarce) and passed through shared memory, double-buffered by step
    // parity: refl[k & 1] = (tau, v1, v2) of step k.
    if (warp == 0) {
      double h11, h12, h21, h22;
      if (its % 20 == 10) {
        double s = fabs(H[(size_t)(l + 1) * n + l]) + fabs(H[(size_t)(l + 2) * n + l + 1]);
        h11 = 0.75 * s + H[(size_t)l * n + l]; h12 = -0.4375 * s; h21 = s; h22 = h11;
      } else if (its % 20 == 0) {
        double s = fabs(H[(size_t)hi * n + hi - 1]) + fabs(H[(size_t)(hi - 1) * n + hi - 2]);
        h11 = 0.75 * s + H[(size_t)hi * n + hi]; h12 = -0.4375 * s; h21 = s; h22 = h11;
      } else {
        h11 = H[(size_t)(hi - 1) * n + hi - 1]; h12 = H[(size_t)(hi - 1) * n + hi];
        h21 = H[(size_t)hi * n + hi - 1]; h22 = H[(size_t)hi * n + hi];
      }
      // Shifts: the eigenvalues of the 2x2 block (computed on a scaled copy). A complex
      // pair is used as a double shift; real shifts are replaced by the one closer to h22
      // taken twice. The first column of (H - s1)(H - s2) e1 is formed from differences
      // (h_ll - s1)(h_ll - s2) + h_{l,l+1} h_{l+1,l}, scaled by 1/s3: expanding it into
      // h_ll^2 - (s1 + s2) h_ll + s1 s2 cancels catastrophically when the shifts sit inside
      // a tight eigenvalue cluster and the sweeps then stall.
      double r1r, r1i, r2r, r2i;
      {
        double sc = fabs(h11) + fabs(h12) + fabs(h21) + fabs(h22);
        if (sc == 0.0) {
          r1r = r1i = r2r = r2i = 0.0;
        } else {
          double a11 = h11 / sc, a12 = h12 / sc, a21 = h21 / sc, a22 = h22 / sc;
          double tr = 0.5 * (a11 + a22);
          double det = (a11 - tr) * (a22 - tr) - a12 * a21;
          double rt = sqrt(fabs(det));
          if (det >= 0.0) {
            r1r = r2r = tr * sc;
            r1i = rt * sc;
            r2i = -r1i;
          } else {
            r1r = tr + rt;
            r2r = tr - rt;
            if (fabs(r1r - a22) <= fabs(r2r - a22)) { r1r *= sc; r2r = r1r; }
            else { r2r *= sc; r1r = r2r; }
            r1i = r2i = 0.0;
          }
        }
      }
      double hll = H[(size_t)l * n + l], hl1l = H[(size_t)(l + 1) * n + l];
      double s3 = fabs(hll - r2r) + fabs(r2i) + fabs(hl1l);
      double h21s = hl1l / s3;
      double x = h21s * H[(size_t)l * n + l + 1] + (hll - r1r) * ((hll - r2r) / s3) - r1i * (r2i / s3);
      double y = h21s * (hll + H[(size_t)(l + 1) * n + l + 1] - r1r - r2r);
      double z = h21s * H[(size_t)(l + 2) * n + l + 1];
      const int nr = (l < hi - 1) ? 3 : 2;
      double tau, v1, v2;
      house3(x, y, nr == 3 ? z : 0.0, tau, v1, v2);
      if (nr == 2) v2 = 0.0;
      if (lane == 0) {
        const double tv1 = tau * v1, tv2 = tau * v2;
        refl[l & 1][0] = tau; refl[l & 1][1] = v1; refl[l & 1][2] = v2;
        refl[l & 1][3] = tv1; refl[l & 1][4] = tv2;
      }
    }
    // the window of the first step: rows l .. l+3, columns l .. l+3 (column l+4 enters at step l)
    if (warp == 0) {
      for (int e = lane; e < 16; e += 32) {
        const int r = l + (e >> 2), c = l + (e & 3);
        if (r <= hi && c < n) W[r & 7][c & 7] = H[(size_t)r * n + c];
      }
    }
    __syncthreads();
    // Each step k applies P_k = I - tau v v^T, v = (1, v1, v2), to H from both sides and to
    // Z from the right; every element update is w = h0 + v1 h1 + v2 h2, then
    // h -= (tau, tau v1, tau v2) w (five FP64 operations). Dependent FP64 operations are
    // slow on this part, so the chain from one reflector to the next is kept short: the step
    // splits into three disjoint sets of elements done concurrently, with one barrier:
    //   warp 0 carries the bulge in a shared-memory window W of rows k .. k+3 and columns
    //   k-1 .. k+4: the left update of columns c0 .. k+2, the right update of rows
    //   k .. min(k+3, hi) (all that the next reflector reads), then that reflector;
    //   warp 1 brings column k+4 into the window (its rows k, k+1 hold the far update of
    //   step k-1) and applies the left update to columns k+3 and k+4, which steps k+1 and
    //   k+2 read first;
    //   warps 2.. apply the rest: the left update of columns k+5 .. n-1, the right update of
    //   rows 0 .. k-1, and Z <- Z P_k, issuing the loads of two tasks before their updates.
    // Row k leaves the window for H at the end of step k (columns c0 .. k+2 from warp 0,
    // k+3 .. k+4 from warp 1), with the two zeros of column k-1; row k+4 is read ahead by
    // warp 0 (nothing touches it before step k+1). Every element receives the same
    // operations in the same order as in a step done by all threads one update after the
    // other.
    const int ft = tid - 64, fn = nt - 64;
    for (int k = l; k <= hi - 1; ++k) {
      const int nr = (k < hi - 1) ? 3 : 2;
      const double tau = refl[k & 1][0], v1 = refl[k & 1][1], v2 = refl[k & 1][2];
      const double tv1 = refl[k & 1][3], tv2 = refl[k & 1][4];
      const int rmax = min(k + 3, hi);
      const int c0 = (k > l) ? k - 1 : l;
      if (warp == 0) {
        // row k+4 (lanes 8..12: columns k..k+4), read ahead
        double ent = 0.0;
        const bool row4 = lane >= 8 && lane < 13 && k + 4 <= hi && k + lane - 8 < n;
        if (row4) ent = H[(size_t)(k + 4) * n + k + lane - 8];
        double nb = 0.0;
        if (tau != 0.0) {
          // left: rows k..k+nr-1, columns c0 .. k+2 (what the right update reads)
          {
            const int j = c0 + lane;
            if (j <= min(k + 2, n - 1)) {
              const double h0 = W[k & 7][j & 7], h1 = W[(k + 1) & 7][j & 7];
              const double h2 = (nr == 3) ? W[(k + 2) & 7][j & 7] : 0.0;
              const double w = fma(v2, h2, fma(v1, h1, h0));
              W[k & 7][j & 7] = fma(-tau, w, h0);
              W[(k + 1) & 7][j & 7] = fma(-tv1, w, h1);
              if (nr == 3) W[(k + 2) & 7][j & 7] = fma(-tv2, w, h2);
            }
          }
          __syncwarp();
          if (k > l && lane == 0) {
            W[(k + 1) & 7][(k - 1) & 7] = 0.0;
            if (nr == 3) W[(k + 2) & 7][(k - 1) & 7] = 0.0;
          }
          // right: columns k..k+nr-1, rows k..rmax; row k + lane on lane `lane`, so rows
          // k+1 .. k+3 (the next bulge column) sit on lanes 1 .. 3
          {
            const int i = k + lane;
            if (i <= rmax) {
              const double h0 = W[i & 7][k & 7], h1 = W[i & 7][(k + 1) & 7];
              const double h2 = (nr == 3) ? W[i & 7][(k + 2) & 7] : 0.0;
              const double w = fma(v2, h2, fma(v1, h1, h0));
              const double g0 = fma(-tau, w, h0);
              W[i & 7][k & 7] = g0;
              nb = g0;
              W[i & 7][(k + 1) & 7] = fma(-tv1, w, h1);
              if (nr == 3) W[i & 7][(k + 2) & 7] = fma(-tv2, w, h2);
            }
          }
          __syncwarp();
        }
        // reflector of step k + 1 from column k of rows k+1 .. k+3
        if (k + 1 <= hi - 1) {
          const int nr1 = (k + 1 < hi - 1) ? 3 : 2;
          double x, y, z;
          if (tau != 0.0) {
            x = __shfl_sync(0xffffffffu, nb, 1);
            y = __shfl_sync(0xffffffffu, nb, 2);
            z = __shfl_sync(0xffffffffu, nb, 3);
          } else {
            x = W[(k + 1) & 7][k & 7];
            y = W[(k + 2) & 7][k & 7];
            z = (nr1 == 3) ? W[(k + 3) & 7][k & 7] : 0.0;
          }
          double t1, w1, w2;
          house3(x, y, nr1 == 3 ? z : 0.0, t1, w1, w2);
          if (nr1 == 2) w2 = 0.0;
          if (lane == 0) {
            const double tw1 = t1 * w1, tw2 = t1 * w2;
            refl[(k + 1) & 1][0] = t1; refl[(k + 1) & 1][1] = w1; refl[(k + 1) & 1][2] = w2;
            refl[(k + 1) & 1][3] = tw1; refl[(k + 1) & 1][4] = tw2;
          }
        }
        // row k+4 enters the window (its slot held row k-4); row k leaves (columns c0 .. k+2)
        if (row4) W[(k + 4) & 7][(k + lane - 8) & 7] = ent;
        {
          const int c = c0 + lane;
          if (c <= min(k + 2, n - 1)) H[(size_t)k * n + c] = W[k & 7][c & 7];
        }
        if (tau != 0.0 && k > l && lane == 0) {
          H[(size_t)(k + 1) * n + k - 1] = 0.0;
          if (nr == 3) H[(size_t)(k + 2) * n + k - 1] = 0.0;
        }
      } else if (warp == 1) {
        // column k+4 enters the window (lanes 0..3: rows k..rmax; its slot held column k-4)
        const int j4 = k + 4;
        const bool col4 = lane < 4 && j4 < n && k + lane <= rmax;
        if (col4) W[(k + lane) & 7][j4 & 7] = H[(size_t)(k + lane) * n + j4];
        __syncwarp();
        const int j = k + 3 + lane;
        if (tau != 0.0) {
          // left update of columns k+3, k+4 (read first at steps k+1 and k+2)
          if (lane < 2 && j < n) {
            const double h0 = W[k & 7][j & 7], h1 = W[(k + 1) & 7][j & 7];
            const double h2 = (nr == 3) ? W[(k + 2) & 7][j & 7] : 0.0;
            const double w = fma(v2, h2, fma(v1, h1, h0));
            W[k & 7][j & 7] = fma(-tau, w, h0);
            W[(k + 1) & 7][j & 7] = fma(-tv1, w, h1);
            if (nr == 3) W[(k + 2) & 7][j & 7] = fma(-tv2, w, h2);
          }
          __syncwarp();
        }
        // row k leaves the window (columns k+3, k+4)
        if (lane < 2 && j < n) H[(size_t)k * n + j] = W[k & 7][j & 7];
      } else if (tau != 0.0) {
        // tasks: far columns of the left update, far rows of the right update, rows of Z;
        // task t updates p[0], p[s], p[2 s]
        const int jf = k + 5;
        const int nA = max(0, n - jf), nAB = nA + k, nT = nAB + n;
        auto task = [&](int t, int& s) -> double* {
          if (t < nA) { s = n; return H + (size_t)k * n + jf + t; }
          if (t < nAB) { s = 1; return H + (size_t)(t - nA) * n + k; }
          s = n;
          return Z + (size_t)k * n + (t - nAB);
        };
        for (int t = ft; t < nT; t += 2 * fn) {
          int sa, sb = 0;
          double* pa = task(t, sa);
          const bool hb = t + fn < nT;
          double* pb = hb ? task(t + fn, sb) : pa;
          const double a0 = pa[0], a1 = pa[sa], a2 = (nr == 3) ? pa[2 * sa] : 0.0;
          double b0 = 0.0, b1 = 0.0, b2 = 0.0;
          if (hb) {
            b0 = pb[0];
            b1 = pb[sb];
            b2 = (nr == 3) ? pb[2 * sb] : 0.0;
          }
          const double wa = fma(v2, a2, fma(v1, a1, a0));
          pa[0] = fma(-tau, wa, a0);
          pa[sa] = fma(-tv1, wa, a1);
          if (nr == 3) pa[2 * sa] = fma(-tv2, wa, a2);
          if (hb) {
            const double wb = fma(v2, b2, fma(v1, b1, b0));
            pb[0] = fma(-tau, wb, b0);
            pb[sb] = fma(-tv1, wb, b1);
            if (nr == 3) pb[2 * sb] = fma(-tv2, wb, b2);
          }
        }
      }
      __syncthreads();
    }
    // the rows still in the window after the last step (k = hi - 1) go back to H
    if (warp == 0) {
      const int k = hi - 1, c0 = (k > l) ? k - 1 : l;
      const int r = k + 1 + (lane >> 3), c = c0 + (lane & 7);
      if (r <= hi && c <= min(k + 4, n - 1)) H[(size_t)r * n + c] = W[r & 7][c & 7];
    }
    __syncthreads();
  }
  __syncthreads();

  // ---- 4. eigenvectors of T by back-substitution, one warp per eigenvalue
  for (size_t e = tid; e < (size_t)n * n; e += nt) V[e] = 0.0;
  __syncthreads();
  for (int k = warp; k < n; k += nwarps) {
    double lr = wr[k], li = wi[k];
    if (li < 0.0) continue;  // second of a pair: handled with the first
    bool cplx = li > 0.0;
    double* vr = V + (size_t)k * n;
    double* vi = cplx ? V + (size_t)(k + 1) * n : nullptr;
    double smin = fmax(EPS * (fabs(lr) + fabs(li)), smlnum);
    int top;
    if (!cplx) {
      if (lane == 0) vr[k] = 1.0;
      top = k;
    } else {
      // block rows k, k+1: (a - lam) v_k + b v_{k+1} = 0 -> v = (b, lam - a)
      double a = H[(size_t)k * n + k], b = H[(size_t)k * n + k + 1];
      if (lane == 0) {
        vr[k] = b; vi[k] = 0.0;
        vr[k + 1] = lr - a; vi[k + 1] = li;
      }
      top = k + 1;
    }
    __syncwarp();
    int i = k - 1;
    while (i >= 0) {
      bool blk2 = (i > 0) && (H[(size_t)i * n + i - 1] != 0.0);
      int i0 = blk2 ? i - 1 : i;
      // right-hand sides r_row = sum_{j > i, j <= top} T[row][j] v_j
      double sr0 = 0.0, si0 = 0.0, sr1 = 0.0, si1 = 0.0;
      for (int j = i + 1 + lane; j <= top; j += 32) {
        double tr = H[(size_t)i * n + j];
        sr1 += tr * vr[j];
        if (cplx) si1 += tr * vi[j];
        if (blk2) {
          double t0 = H[(size_t)i0 * n + j];
          sr0 += t0 * vr[j];
          if (cplx) si0 += t0 * vi[j];
        }
      }
      // reduce only the sums this row needs (warp-uniform conditions)
      for (int off = 16; off > 0; off >>= 1) {
        sr1 += __shfl_xor_sync(0xffffffffu, sr1, off);
        if (cplx) si1 += __shfl_xor_sync(0xffffffffu, si1, off);
        if (blk2) {
          sr0 += __shfl_xor_sync(0xffffffffu, sr0, off);
          if (cplx) si0 += __shfl_xor_sync(0xffffffffu, si0, off);
        }
      }
      if (lane == 0) {
        if (!blk2) {
          // (T_ii - lam) v_i = -r
          double dr = H[(size_t)i * n + i] - lr, di = -li;
          if (fabs(dr) + fabs(di) < smin) { dr = smin; di = 0.0; }
          // v = -(sr + i si) / (dr + i di), with one division
          if (!cplx) {
            vr[i] = -sr1 / dr;
          } else {
            const double inv = 1.0 / (dr * dr + di * di);
            vr[i] = -(sr1 * dr + si1 * di) * inv;
            vi[i] = -(si1 * dr - sr1 * di) * inv;
          }
        } else {
          // [[a - lam, b], [c, d - lam]] [v0; v1] = -[r0; r1]
          double a = H[(size_t)i0 * n + i0] - lr, b = H[(size_t)i0 * n + i];
          double c = H[(size_t)i * n + i0], d = H[(size_t)i * n + i] - lr;
          // complex determinant (a - i li)(d - i li) - b c
          double ar = a, ai = -li, dr = d, di = -li;
          double detr = ar * dr - ai * di - b * c, deti = ar * di + ai * dr;
          if (fabs(detr) + fabs(deti) < smin) { detr = smin; deti = 0.0; }
          const double inv = 1.0 / (detr * detr + deti * deti);
          // Cramer with negated right-hand side: v0 = (b r1 - r0 d') / det, v1 = (c r0 - a' r1) / det
          double n0r = -(sr0 * dr - si0 * di) + b * sr1;
          double n0i = -(sr0 * di + si0 * dr) + b * si1;
          double n1r = c * sr0 - (ar * sr1 - ai * si1);
          double n1i = c * si0 - (ar * si1 + ai * sr1);
          double v0r = (n0r * detr + n0i * deti) * inv, v0i = (n0i * detr - n0r * deti) * inv;
          double v1r = (n1r * detr + n1i * deti) * inv, v1i = (n1i * detr - n1r * deti) * inv;
          vr[i0] = v0r; vr[i] = v1r;
          if (cplx) { vi[i0] = v0i; vi[i] = v1i; }
        }
      }
      __syncwarp();
      // rescale if the vector grows too large
      double big = fabs(vr[i0]) + (cplx ? fabs(vi[i0]) : 0.0) + fabs(vr[i]) + (cplx ? fabs(vi[i]) : 0.0);
      if (big > 1e100) {
        double f = 1.0 / big;
        for (int j = i0 + lane; j <= top; j += 32) {
          vr[j] *= f;
          if (cplx) vi[j] *= f;
        }
        __syncwarp();
      }
      i = i0 - 1;
    }
  }
  __syncthreads();
}

// X = D Z V has been formed by a GEMM into X (row-major). Scale each eigenvector (pair)
// so that its largest component modulus is one. One CTA per (order, column).
__global__ void k_finish_eigvec(int n, double* X, const double* lam_im, const double* scale,
                                const int* mask, unsigned* status) {
  __shared__ double red[32];
  int u = blockIdx.y, j = blockIdx.x;
  if (mask && !mask[u]) return;
  const double* wi = lam_im + (size_t)u * n;
  if (wi[j] < 0.0) return;
  bool cplx = wi[j] > 0.0;
  double* Xb = X + (size_t)u * n * n;
  const double* d = scale + (size_t)u * n;
  double mx = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double a = Xb[(size_t)i * n + j] * d[i];
    double b = cplx ? Xb[(size_t)i * n + j + 1] * d[i] : 0.0;
    Xb[(size_t)i * n + j] = a;
    if (cplx) Xb[(size_t)i * n + j + 1] = b;
    mx = fmax(mx, sqrt(a * a + b * b));
  }
  for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  mx = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) mx = fmax(mx, red[i]);
  if (!(mx > 0.0) || !isfinite(mx)) {
    if (threadIdx.x == 0) atomicOr(status, ST_NONFINITE);
    return;
  }
  double f = 1.0 / mx;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    Xb[(size_t)i * n + j] *= f;
    if (cplx) Xb[(size_t)i * n + j + 1] *= f;
  }
}

void dgemm_batched_mask(bool tA, bool tB, int M, int N, int K, double alpha, const double* A,
                        int lda, long long sA, const double* B, int ldb, long long sB, double beta,
                        double* C, int ldc, long long sC, int batch, const int* mask,
                        cudaStream_t s);

void batched_eigen(int n, const double* A, double* H, double* Z, double* V, double* X,
                   double* lam_re, double* lam_im, double* scale, int batch, unsigned* status,
                   cudaStream_t s, const int* mask) {
  size_t smem = 4 * (size_t)n * sizeof(double);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_eigen, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_eigen<<<batch, EIG_THREADS, smem, s>>>(n, A, H, Z, V, lam_re, lam_im, scale, mask, status);
  // X = Z V with Z, V column-major: in row-major terms X = Zc^T Vc^T
  dgemm_batched_mask(true, true, n, n, n, 1.0, Z, n, (long long)n * n, V, n, (long long)n * n, 0.0,
                     X, n, (long long)n * n, batch, mask, s);
  dim3 grid(n, batch);
  k_finish_eigvec<<<grid, 128, 0, s>>>(n, X, lam_im, scale, mask, status);
}

// ---------------------------------------------------------------- accuracy fallback
// The reduced problem squares the spread of the spectrum. For the order-0 diffusion
// mode (kappa -> 0 as omega -> 1) the eigenvector x of F'E' then carries errors that
// y = E'x / kappa amplifies (measured: up to 1e-9 relative in the BRDF at omega = 0.999).
// Such orders are re-solved with the 2n x 2n block form B = [[0, F'], [E', 0]]
// (B [x; y] = kappa [x; y], eigenvalues +-kappa, no squaring), whose eigenvectors give
// x and y directly. The mode residual |F'y - kappa x| / (|kappa| |x|) of the reduced
// solution decides, besides order 0 which the FP64 form always re-solves.

// res[u] = max over modes of |F'y - kappa x|_inf / (|kappa| |x|_inf); flag[u] set if
// res > tol or (order m0 + u == 0 and force0).
__global__ void k_mode_residual(int n, int m0, const double* FY, const double* X,
                                const double* lam_re, const double* lam_im, double tol,
                                int force0, double* res, int* flag) {
  __shared__ double red[32];
  int u = blockIdx.x;
  const double* lr = lam_re + (size_t)u * n;
  const double* li = lam_im + (size_t)u * n;
  const double* Fb = FY + (size_t)u * n * n;
  const double* Xb = X + (size_t)u * n * n;
  double worst = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    if (li[j] < 0.0) continue;
    bool cplx = li[j] > 0.0;
    // principal square root of lambda without cancellation
    double a = lr[j], b = li[j], kr, ki;
    if (b == 0.0) { kr = a > 0.0 ? sqrt(a) : 0.0; ki = 0.0; }
    else {
      double r = sqrt(0.5 * (fabs(a) + hypot(a, b)));
      if (a >= 0.0) { kr = r; ki = 0.5 * b / r; } else { kr = 0.5 * fabs(b) / r; ki = copysign(r, b); }
    }
    double num = 0.0, den = 0.0;
    for (int i = 0; i < n; ++i) {
      double xr = Xb[(size_t)i * n + j], xi = cplx ? Xb[(size_t)i * n + j + 1] : 0.0;
      double fr = Fb[(size_t)i * n + j], fi = cplx ? Fb[(size_t)i * n + j + 1] : 0.0;
      double rr = fr - (kr * xr - ki * xi), ri = fi - (kr * xi + ki * xr);
      num = fmax(num, hypot(rr, ri));
      den = fmax(den, hypot(xr, xi));
    }
    double kk = hypot(kr, ki);
    double rel = (kk > 0.0 && den > 0.0) ? num / (kk * den) : 1.0;
    if (!(rel == rel)) rel = 1.0;
    worst = fmax(worst, rel);
  }
  for (int off = 16; off > 0; off >>= 1) worst = fmax(worst, __shfl_xor_sync(0xffffffffu, worst, off));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = worst;
  __syncthreads();
  if (threadIdx.x == 0) {
    double w = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) w = fmax(w, red[i]);
    res[u] = w;
    flag[u] = (w > tol) || (force0 && m0 + u == 0);
  }
}

// B = [[0, F'], [E', 0]] for flagged orders.
__global__ void k_build_block(int n, const double* E, const double* F, const int* flag, double* B) {
  int u = blockIdx.y;
  if (!flag[u]) return;
  int n2 = 2 * n;
  size_t total = (size_t)n2 * n2;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    int r = (int)(e / n2), c = (int)(e - (size_t)r * n2);
    double v = 0.0;
    if (r < n && c >= n) v = F[(size_t)u * n * n + (size_t)r * n + (c - n)];
    else if (r >= n && c < n) v = E[(size_t)u * n * n + (size_t)(r - n) * n + c];
    B[(size_t)u * total + e] = v;
  }
}

// Keep the n eigenpairs of B with Re kappa > 0: x = first half, y = second half of the
// eigenvector, lambda = kappa^2 (a pair kappa = a +- ib, a > 0, becomes lambda with
// Im lambda = +-2ab, the first column keeping Im lambda > 0).
__global__ void k_select_modes(int n, const double* Xb, const double* kb_re, const double* kb_im,
                               const int* flag, double* X, double* Y, double* lam_re,
                               double* lam_im, unsigned* status) {
  extern __shared__ int src[];  // [n] source column per destination column
  __shared__ int count_sh;
  int u = blockIdx.x;
  if (!flag[u]) return;
  int n2 = 2 * n;
  const double* kr = kb_re + (size_t)u * n2;
  const double* ki = kb_im + (size_t)u * n2;
  if (threadIdx.x == 0) {
    int cnt = 0;
    for (int j = 0; j < n2 && cnt <= n; ++j) {
      if (ki[j] < 0.0) continue;
      if (kr[j] <= 0.0) { if (ki[j] > 0.0) ++j; continue; }
      if (ki[j] > 0.0) {
        if (cnt + 2 <= n) { src[cnt] = j; src[cnt + 1] = j + 1; }
        cnt += 2;
        ++j;
      } else {
        if (cnt + 1 <= n) src[cnt] = j;
        cnt += 1;
      }
    }
    count_sh = cnt;
    if (cnt != n) atomicOr(status, ST_NO_CONVERGENCE);
  }
  __syncthreads();
  if (count_sh != n) return;
  const double* W = Xb + (size_t)u * n2 * n2;
  double* Xo = X + (size_t)u * n * n;
  double* Yo = Y + (size_t)u * n * n;
  double* lr = lam_re + (size_t)u * n;
  double* li = lam_im + (size_t)u * n;
  for (int d = threadIdx.x; d < n; d += blockDim.x) {
    int j = src[d];
    double a = kr[j], b = ki[j];
    lr[d] = a * a - b * b;
    li[d] = 2.0 * a * b;
  }
  for (size_t e = threadIdx.x; e < (size_t)n * n; e += blockDim.x) {
    int i = (int)(e / n), d = (int)(e - (size_t)i * n);
    int j = src[d];
    Xo[e] = W[(size_t)i * n2 + j];
    Yo[e] = W[(size_t)(n + i) * n2 + j];
  }
}

void eigen_block_fallback(int n, int m0, const double* E, const double* F, const double* FY,
                          double* X, double* Y, double* lam_re, double* lam_im, double tol,
                          int force0, double* res, int* flag, double* B, double* Hb, double* Zb,
                          double* Vb, double* Xb, double* kb_re, double* kb_im, double* balb,
                          int batch, unsigned* status, cudaStream_t s) {
  k_mode_residual<<<batch, 128, 0, s>>>(n, m0, FY, X, lam_re, lam_im, tol, force0, res, flag);
  int n2 = 2 * n;
  dim3 g1((unsigned)std::min<size_t>(((size_t)n2 * n2 + 255) / 256, 4096), batch);
  k_build_block<<<g1, 256, 0, s>>>(n, E, F, flag, B);
  batched_eigen(n2, B, Hb, Zb, Vb, Xb, kb_re, kb_im, balb, batch, status, s, flag);
  k_select_modes<<<batch, 256, (size_t)n * sizeof(int), s>>>(n, Xb, kb_re, kb_im, flag, X, Y,
                                                               lam_re, lam_im, status);
}

}  // namespace vrte
