// Concentrated window on the GPU (Sec. III-D): the band-limited function of
// maximal energy concentration in the elliptical region R(theta_c, a)
// (Eq. region_def: the points whose great-circle distances to the foci
// (theta_c, 0) and (theta_c, pi) add up to at most 2a), i.e. the top
// eigenvector of the concentration matrix
//   D_{(l m),(l' m')} = int_R conj(Y_l^m) Y_l'^m' ds,   l, l' < L.
//
// The region is symmetric under phi -> -phi, and the most concentrated
// eigenfunction is even in phi and real, so the problem is solved in the real
// even basis u_{l0} = Ytilde_l^0, u_{lm} = sqrt(2) Ptilde_l^m(cos theta) cos(m phi)
// (m > 0): D becomes the real symmetric K_ab = int_R u_a u_b ds of order
// L(L+1)/2.  Quadrature over R, ring by ring: for each of n_phi longitudes the
// boundary colatitude theta_b(phi) by bisection on the focal-distance sum,
// Gauss-Legendre in theta on [0, theta_b], trapezoid in phi.  With
// A[pt][a] = sqrt(w_pt) u_a(pt), K = A^T A.  The top eigenpair by block
// subspace iteration (block larger than the Shannon number trace(K), where the
// eigenvalues cluster near 1): W = K V, V <- an orthonormal basis of W by
// shifted CholeskyQR3 (Fukaya, Kannan, Nakatsukasa, Yamamoto and Yanagisawa,
// "Shifted Cholesky QR for computing the QR factorization of ill-conditioned
// matrices", SIAM J. Sci. Comput. 2020: a shifted Cholesky QR, then Cholesky
// QR twice), and every few steps a Rayleigh-Ritz step (T = V^T W and its
// eigenpairs by cyclic Jacobi rotations).  Everything runs on the device in
// this file's FP64 kernels; the host only reads the Ritz value and residual
// norm of each Rayleigh-Ritz step and the final vector.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "common.cuh"

// ---------------------------------------------------------------- device
__device__ __forceinline__ double ang_dist(double t1, double p1, double t2, double p2) {
  double c = sin(t1) * sin(t2) * cos(p1 - p2) + cos(t1) * cos(t2);
  c = fmin(1.0, fmax(-1.0, c));
  return acos(c);
}

// One thread per longitude: theta_b by bisection, then the ring's n_theta
// nodes (cos theta, phi, sqrt of the weight).
__global__ void k_region_nodes(double theta_c, double a, int n_phi, int n_theta, const double* __restrict__ gl_t,
                               const double* __restrict__ gl_w, double* __restrict__ ct, double* __restrict__ ph,
                               double* __restrict__ sw) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_phi) return;
  const double pi = 3.14159265358979323846;
  const double phi = 2.0 * pi * j / n_phi;
  double lo = 0.0, hi = a;
  for (int it = 0; it < 80; ++it) {
    const double mid = 0.5 * (lo + hi);
    const double s = ang_dist(mid, phi, theta_c, 0.0) + ang_dist(mid, phi, theta_c, pi);
    if (s <= 2.0 * a) lo = mid; else hi = mid;
  }
  const double tb = 0.5 * (lo + hi);
  for (int i = 0; i < n_theta; ++i) {
    const double th = 0.5 * (gl_t[i] + 1.0) * tb;
    const double w = 0.5 * tb * gl_w[i] * sin(th) * (2.0 * pi / n_phi);
    const int pt = j * n_theta + i;
    ct[pt] = cos(th);
    ph[pt] = phi;
    sw[pt] = sqrt(w);
  }
}

// A[pt + col(l, m) * npts] = sqrt(w) u_{lm}(pt), col(l, m) = l(l+1)/2 + m, one
// thread per (point, m): the orthonormal Legendre recurrences in l.
__global__ void k_window_basis(const double* __restrict__ ct, const double* __restrict__ ph,
                               const double* __restrict__ sw, int npts, int L, double* __restrict__ A) {
  const int pt = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = blockIdx.y;
  if (pt >= npts) return;
  const double x = ct[pt], s = sqrt(fmax(0.0, 1.0 - x * x));
  double pmm = 1.0 / sqrt(4.0 * 3.14159265358979323846);
  for (int k = 1; k <= m; ++k) pmm *= -sqrt((2.0 * k + 1.0) / (2.0 * k)) * s;
  const double f = sw[pt] * (m == 0 ? 1.0 : sqrt(2.0) * cos(m * ph[pt]));
  double p2 = 0.0, p1 = pmm;
  A[pt + (size_t)(m * (m + 1) / 2 + m) * npts] = f * pmm;
  for (int l = m + 1; l < L; ++l) {
    double p;
    if (l == m + 1) {
      p = sqrt(2.0 * m + 3.0) * x * pmm;
    } else {
      const double aa = sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)m * m));
      const double bb = sqrt((((double)l - 1.0) * (l - 1.0) - (double)m * m) / (4.0 * ((double)l - 1.0) * (l - 1.0) - 1.0));
      p = aa * (x * p1 - bb * p2);
    }
    A[pt + (size_t)(l * (l + 1) / 2 + m) * npts] = f * p;
    p2 = p1;
    p1 = p;
  }
}

// ---------------------------------------------------------------- dense FP64 kernels
// C_s = op(A) B over the s-th of ksplit slices of the inner dimension (s =
// blockIdx.z), column-major: C_s[i + j ldc] = sum_k opA(i, k) B[k + j ldb],
// opA(i, k) = A[k + i lda] (TA) or A[i + k lda].  64 x 64 output tiles, 256
// threads of 4 x 4 outputs (rows ty + 16 r, columns tx + 16 c), the inner
// dimension staged 16 at a time in shared memory; FP64 fused multiply-adds
// in a fixed order.  sym: C is symmetric (op(A) B = B^T A): only the tiles on
// and below the diagonal run, each output written to both halves.
#define WG_T 64
#define WG_KC 16
template <bool TA>
__global__ void __launch_bounds__(256) k_wgemm(int m, int n, int kdim, int ksplit, const double* __restrict__ A,
                                               int lda, const double* __restrict__ B, int ldb, double* __restrict__ C,
                                               int ldc, size_t cstride, int sym) {
  if (sym && blockIdx.x < blockIdx.y) return;
  __shared__ double As[WG_KC][WG_T + 1];
  __shared__ double Bs[WG_KC][WG_T + 1];
  const int i0 = blockIdx.x * WG_T, j0 = blockIdx.y * WG_T;
  const int kper = (kdim + ksplit - 1) / ksplit;
  const int kb = blockIdx.z * kper, ke = min(kdim, kb + kper);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = 0.0;
  for (int k0 = kb; k0 < ke; k0 += WG_KC) {
    for (int e = threadIdx.x; e < WG_KC * WG_T; e += 256) {
      int kk, ii;
      if (TA) { kk = e & 15; ii = e >> 4; } else { ii = e & 63; kk = e >> 6; }
      const int k = k0 + kk, i = i0 + ii;
      double v = 0.0;
      if (k < ke && i < m) v = TA ? A[k + (size_t)i * lda] : A[i + (size_t)k * lda];
      As[kk][ii] = v;
    }
    for (int e = threadIdx.x; e < WG_KC * WG_T; e += 256) {
      const int kk = e & 15, jj = e >> 4;
      const int k = k0 + kk, j = j0 + jj;
      Bs[kk][jj] = (k < ke && j < n) ? B[k + (size_t)j * ldb] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < WG_KC; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[kk][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
  }
  double* Cs = C + (size_t)blockIdx.z * cstride;
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int i = i0 + ty + 16 * r, j = j0 + tx + 16 * c;
      if (i < m && j < n) {
        Cs[i + (size_t)j * ldc] = acc[r][c];
        if (sym && i != j) Cs[j + (size_t)i * ldc] = acc[r][c];
      }
    }
}

// C[i] = sum_s P[i + s stride], s in order (the split-K partials)
__global__ void k_wsum(const double* __restrict__ P, int ns, size_t stride, size_t n, double* __restrict__ C) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double v = 0.0;
  for (int s = 0; s < ns; ++s) v += P[i + (size_t)s * stride];
  C[i] = v;
}

// Upper Cholesky factor R (R^T R = G + shift I) of the b x b symmetric G
// (column-major, in place as R's storage), one block.  shift_on: shift =
// 11 (m b + b (b + 1)) 2^-53 trace(G), the shift of the shifted Cholesky QR
// (trace(G) = ||X||_F^2 bounds ||X||_2^2).  A non-positive pivot (columns
// dependent to working precision) is replaced by 2^-52 trace(G) and counted
// in *bad; the basis is then not quite orthonormal, which the caller's
// convergence test (the residual of a Ritz pair, valid for any basis) sees.
__global__ void k_wchol(double* __restrict__ G, int b, int m, int shift_on, int* __restrict__ bad) {
  extern __shared__ double sg[];          // b x b, column-major
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) sg[e] = G[e];
  __syncthreads();
  if (shift_on) {
    __shared__ double s_shift;
    if (threadIdx.x == 0) {
      double tr = 0.0;
      for (int i = 0; i < b; ++i) tr += sg[i + i * b];
      s_shift = 11.0 * ((double)m * b + (double)b * (b + 1)) * ldexp(1.0, -53) * tr;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < b; i += blockDim.x) sg[i + i * b] += s_shift;
    __syncthreads();
  }
  __shared__ double s_piv, s_floor;
  if (threadIdx.x == 0) {
    double tr = 0.0;
    for (int i = 0; i < b; ++i) tr += sg[i + i * b];
    s_floor = ldexp(fmax(tr, 1e-300), -52);
  }
  __syncthreads();
  for (int j = 0; j < b; ++j) {
    if (threadIdx.x == 0) {
      const double d = sg[j + j * b];
      if (!(d > s_floor)) { atomicAdd(bad, 1); s_piv = sqrt(s_floor); } else { s_piv = sqrt(d); }
      sg[j + j * b] = s_piv;
    }
    __syncthreads();
    for (int k = j + 1 + threadIdx.x; k < b; k += blockDim.x) sg[j + k * b] /= s_piv;   // row j of R
    __syncthreads();
    for (int e = threadIdx.x; e < (b - j - 1) * (b - j - 1); e += blockDim.x) {      // trailing update
      const int i = j + 1 + e % (b - j - 1), k = j + 1 + e / (b - j - 1);
      if (i <= k) sg[i + k * b] -= sg[j + i * b] * sg[j + k * b];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int i = e % b, k = e / b;
    G[e] = i <= k ? sg[e] : 0.0;
  }
}

// X <- X R^-1 (R upper b x b), one thread per row of X (m x b, ld m).
__global__ void k_wtrsm(double* __restrict__ X, int m, int b, const double* __restrict__ R) {
  extern __shared__ double sr[];
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) sr[e] = R[e];
  __syncthreads();
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= m) return;
  for (int j = 0; j < b; ++j) {
    double v = X[row + (size_t)j * m];
    for (int i = 0; i < j; ++i) v -= X[row + (size_t)i * m] * sr[i + j * b];
    X[row + (size_t)j * m] = v / sr[j + j * b];
  }
}

// Eigenpairs of the symmetric b x b T (column-major) by cyclic Jacobi
// rotations, one block: each rotation zeroes one off-diagonal pair and is
// applied to the columns, the rows and the accumulated Q by all threads;
// sweeps until the squared off-diagonal mass is below 1e-30 (T is a
// Rayleigh quotient of K, whose eigenvalues lie in [0, 1]).  Out: ev[i] and
// Q[:, i]; top[0] = the index of the largest eigenvalue.
__global__ void k_wjacobi(const double* __restrict__ Tin, int b, double* __restrict__ Qout, double* __restrict__ ev,
                          int* __restrict__ top) {
  extern __shared__ double sm[];
  double* T = sm;               // b x b
  double* Q = sm + b * b;       // b x b
  __shared__ double s_c, s_s, s_off;
  __shared__ int s_go;
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int i = e % b, k = e / b;
    T[e] = 0.5 * (Tin[e] + Tin[k + i * b]);   // symmetrised
    Q[e] = i == k ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int sweep = 0; sweep < 100; ++sweep) {
    if (threadIdx.x == 0) {
      double off = 0.0;
      for (int p = 0; p < b; ++p)
        for (int q = p + 1; q < b; ++q) off += T[p + q * b] * T[p + q * b];
      s_off = off;
    }
    __syncthreads();
    if (s_off < 1e-30) break;
    for (int p = 0; p < b; ++p) {
      for (int q = p + 1; q < b; ++q) {
        if (threadIdx.x == 0) {
          const double apq = T[p + q * b];
          s_go = fabs(apq) >= 1e-300;
          if (s_go) {
            const double app = T[p + p * b], aqq = T[q + q * b];
            const double th = 0.5 * (aqq - app) / apq;
            const double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
            s_c = 1.0 / sqrt(t * t + 1.0);
            s_s = t * s_c;
          }
        }
        __syncthreads();
        if (s_go) {
          const double c = s_c, sn = s_s;
          for (int k = threadIdx.x; k < b; k += blockDim.x) {     // columns p, q
            const double tkp = T[k + p * b], tkq = T[k + q * b];
            T[k + p * b] = c * tkp - sn * tkq;
            T[k + q * b] = sn * tkp + c * tkq;
            const double qkp = Q[k + p * b], qkq = Q[k + q * b];
            Q[k + p * b] = c * qkp - sn * qkq;
            Q[k + q * b] = sn * qkp + c * qkq;
          }
          __syncthreads();
          for (int k = threadIdx.x; k < b; k += blockDim.x) {     // rows p, q
            const double tpk = T[p + k * b], tqk = T[q + k * b];
            T[p + k * b] = c * tpk - sn * tqk;
            T[q + k * b] = sn * tpk + c * tqk;
          }
        }
        __syncthreads();
      }
    }
  }
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) Qout[e] = Q[e];
  for (int i = threadIdx.x; i < b; i += blockDim.x) ev[i] = T[i + i * b];
  if (threadIdx.x == 0) {
    int im = 0;
    for (int i = 1; i < b; ++i)
      if (T[i + i * b] > T[im + im * b]) im = i;
    *top = im;
  }
}

// The top Ritz pair's vector x = V q and residual r = W q - lam x (q = column
// *top of Q, lam = ev[*top]); per block the partial sums of |x|^2 and |r|^2.
__global__ void k_writz(const double* __restrict__ V, const double* __restrict__ W, int m, int b,
                        const double* __restrict__ Q, const double* __restrict__ ev, const int* __restrict__ top,
                        double* __restrict__ x, double* __restrict__ part) {
  __shared__ double sx[256], sr[256];
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  const int t = *top;
  const double lam = ev[t];
  double xv = 0.0, rv = 0.0;
  if (row < m) {
    double wq = 0.0;
    for (int i = 0; i < b; ++i) {
      const double qi = Q[i + (size_t)t * b];
      xv = fma(V[row + (size_t)i * m], qi, xv);
      wq = fma(W[row + (size_t)i * m], qi, wq);
    }
    x[row] = xv;
    rv = wq - lam * xv;
  }
  sx[threadIdx.x] = xv * xv;
  sr[threadIdx.x] = rv * rv;
  __syncthreads();
  for (int s2 = 128; s2 > 0; s2 >>= 1) {
    if (threadIdx.x < s2) {
      sx[threadIdx.x] += sx[threadIdx.x + s2];
      sr[threadIdx.x] += sr[threadIdx.x + s2];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = sx[0];
    part[2 * blockIdx.x + 1] = sr[0];
  }
}

// ---------------------------------------------------------------- host helpers
// Gauss-Legendre nodes and weights on [-1, 1] by Newton's method on P_n.
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = std::cos(pi * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      const double pn = n == 1 ? z : p1, pm = n == 1 ? 1.0 : p0;
      dp = n * (z * pn - pm) / (z * z - 1.0);
      const double dz = pn / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = -z;
    x[n - 1 - i] = z;
    w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// ---------------------------------------------------------------- driver
// Launch helpers of the dense kernels: C = op(A) B with the inner dimension
// split so that the GPU holds at least ~4 blocks per SM (partials in P, then
// summed in a fixed order), or straight into C.
static cudaError_t wgemm(bool ta, int m, int n, int kdim, const double* A, int lda, const double* B, int ldb,
                         double* C, int ldc, bool sym, double* P, size_t pcap, int sms, cudaStream_t st) {
  const int tm = (m + WG_T - 1) / WG_T, tn = (n + WG_T - 1) / WG_T;
  const long long tiles = sym ? (long long)tm * (tm + 1) / 2 : (long long)tm * tn;
  int ks = (int)std::max<long long>(1, (4LL * sms + tiles - 1) / tiles);
  ks = std::min(ks, std::max(1, kdim / WG_KC));
  const size_t cn = (size_t)ldc * n;
  if ((size_t)ks * cn > pcap) ks = (int)std::max<size_t>(1, pcap / cn);
  dim3 grid(tm, tn, ks);
  double* out = ks > 1 ? P : C;
  if (ta)
    k_wgemm<true><<<grid, 256, 0, st>>>(m, n, kdim, ks, A, lda, B, ldb, out, ldc, cn, sym ? 1 : 0);
  else
    k_wgemm<false><<<grid, 256, 0, st>>>(m, n, kdim, ks, A, lda, B, ldb, out, ldc, cn, sym ? 1 : 0);
  if (ks > 1) k_wsum<<<(unsigned)((cn + 255) / 256), 256, 0, st>>>(P, ks, cn, cn, C);
  return cudaGetLastError();
}

// Shifted CholeskyQR3: X (m x b) <- an orthonormal basis of its columns.
static cudaError_t wortho(double* X, int m, int b, double* G, double* P, size_t pcap, int* bad, int sms,
                          cudaStream_t st) {
  const size_t smem = sizeof(double) * (size_t)b * b;
  for (int pass = 0; pass < 3; ++pass) {
    cudaError_t e = wgemm(true, b, b, m, X, m, X, m, G, b, true, P, pcap, sms, st);
    if (e != cudaSuccess) return e;
    k_wchol<<<1, 256, smem, st>>>(G, b, m, pass == 0 ? 1 : 0, bad);
    k_wtrsm<<<(m + 127) / 128, 128, smem, st>>>(X, m, b, G);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Status codes follow slsht.h (0 ok, -1 argument, -3 memory, -5 no
// convergence, -6 CUDA); the caller supplies device scratch allocation.
int window_ellipse_run(int L, double theta_c, double a, int n_phi, int n_theta, void* (*alloc)(size_t, void*),
                       void (*release)(void*, size_t, void*), void* actx, cudaStream_t st, std::vector<double>& h,
                       double* lambda_out, char* errbuf, size_t errlen) {
  if (L < 1 || L > 256 || !(a > 0.0) || !(theta_c >= 0.0) || theta_c > a || a >= 3.14159265358979323846 / 2)
    return -1;
  if (n_phi <= 0) n_phi = 8 * L + 64;
  if (n_theta <= 0) n_theta = 2 * L + 24;
  const int M = L * (L + 1) / 2;
  const size_t npts = (size_t)n_phi * n_theta;
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  std::vector<double> glx, glw;
  gauss_legendre(n_theta, glx, glw);
  const int bmax = std::min(M, 96);
  const size_t bytes_nodes = sizeof(double) * (3 * npts + 2 * (size_t)n_theta);
  const size_t bytes_A = sizeof(double) * npts * M;
  const size_t bytes_K = sizeof(double) * (size_t)M * M;
  // V, W (M x bmax); G, Q (bmax^2); ev, x, partial norms; split-K partials
  const size_t pcap = std::max<size_t>((size_t)8 * M * bmax, (size_t)64 * bmax * bmax);
  const size_t n_small = 2 * (size_t)M * bmax + 2 * (size_t)bmax * bmax + bmax + M + 2 * 4096;
  const size_t bytes_V = sizeof(double) * (n_small + pcap) + 256;
  double* nodes = (double*)alloc(bytes_nodes, actx);
  double* A = (double*)alloc(bytes_A, actx);
  double* K = (double*)alloc(bytes_K, actx);
  double* Vd = (double*)alloc(bytes_V, actx);
  int status = 0;
  auto fail = [&](int code, const char* what) {
    if (errbuf && errlen) snprintf(errbuf, errlen, "%s", what);
    status = code;
  };
  do {
    if (!nodes || !A || !K || !Vd) { fail(-3, "window generator: device memory"); break; }
    double* ct = nodes;
    double* ph = ct + npts;
    double* sw = ph + npts;
    double* gt = sw + npts;
    double* gw = gt + n_theta;
    if (cudaMemcpyAsync(gt, glx.data(), sizeof(double) * n_theta, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(gw, glw.data(), sizeof(double) * n_theta, cudaMemcpyHostToDevice, st) != cudaSuccess) {
      fail(-6, "window generator: copy of the Gauss-Legendre rule");
      break;
    }
    k_region_nodes<<<(n_phi + 127) / 128, 128, 0, st>>>(theta_c, a, n_phi, n_theta, gt, gw, ct, ph, sw);
    dim3 grid((unsigned)((npts + 255) / 256), L);
    k_window_basis<<<grid, 256, 0, st>>>(ct, ph, sw, (int)npts, L, A);
    if (cudaGetLastError() != cudaSuccess) { fail(-6, "window generator: node / basis kernels"); break; }
    double* V = Vd;
    double* W = V + (size_t)M * bmax;
    double* G = W + (size_t)M * bmax;
    double* Q = G + (size_t)bmax * bmax;
    double* ev = Q + (size_t)bmax * bmax;
    double* x = ev + bmax;
    double* part = x + M;
    double* P = part + 2 * 4096;
    int* flags = (int*)(P + pcap);                 // [0] bad pivot, [1] top index
    // K = A^T A (A: npts x M, column-major)
    if (wgemm(true, M, M, (int)npts, A, (int)npts, A, (int)npts, K, M, true, P, pcap, sms, st) != cudaSuccess) {
      fail(-6, "window generator: Gram matrix");
      break;
    }
    // Shannon number trace(K): the count of eigenvalues near 1
    std::vector<double> Kdiag(M);
    if (cudaMemcpy2DAsync(Kdiag.data(), sizeof(double), K, sizeof(double) * (M + 1), sizeof(double), M,
                          cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      fail(-6, "window generator: trace");
      break;
    }
    double shannon = 0.0;
    for (double v : Kdiag) shannon += v;
    const int b = std::min(M, std::max(16, std::min(bmax, (int)std::ceil(2.0 * shannon) + 8)));
    // seeded start block (splitmix64 -> [-1, 1)), orthonormalised on the device
    std::vector<double> V0((size_t)M * b);
    uint64_t seed = 0x9E3779B97F4A7C15ull;
    for (auto& v : V0) {
      seed += 0x9E3779B97F4A7C15ull;
      uint64_t z = seed;
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      z ^= z >> 31;
      v = (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
    }
    const size_t smem2 = 2 * sizeof(double) * (size_t)b * b;
    if (cudaFuncSetAttribute(k_wjacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2) != cudaSuccess ||
        cudaFuncSetAttribute(k_wchol, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(smem2 / 2)) != cudaSuccess ||
        cudaFuncSetAttribute(k_wtrsm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(smem2 / 2)) != cudaSuccess ||
        cudaMemsetAsync(flags, 0, 2 * sizeof(int), st) != cudaSuccess ||
        cudaMemcpyAsync(V, V0.data(), sizeof(double) * V0.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        wortho(V, M, b, G, P, pcap, flags, sms, st) != cudaSuccess) {
      fail(-6, "window generator: start block");
      break;
    }
    const int nblk = (M + 255) / 256;
    double prev = -1.0, lam = 0.0, last_res = -1.0, last_change = -1.0;
    bool converged = false;
    std::vector<double> pn(2 * (size_t)nblk);
    if (b == M) {
      // the block spans the whole space: K's own eigenpairs (Jacobi on K)
      int top = 0;
      k_wjacobi<<<1, 128, smem2, st>>>(K, M, Q, ev, flags + 1);
      if (cudaGetLastError() != cudaSuccess ||
          cudaMemcpyAsync(&top, flags + 1, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess ||
          cudaMemcpyAsync(&lam, ev + top, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaMemcpyAsync(x, Q + (size_t)top * M, sizeof(double) * M, cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
        fail(-6, "window generator: eigenpairs of K");
        break;
      }
      converged = true;
    }
    for (int it = 0; it < 400 && !status && !converged; ++it) {
      // W = K V
      if (wgemm(false, M, b, M, K, M, V, M, W, M, false, P, pcap, sms, st) != cudaSuccess) {
        fail(-6, "window generator: block product");
        break;
      }
      if (it % 3 == 2) {
        // Rayleigh-Ritz: T = V^T W, its eigenpairs, the top Ritz pair's residual
        int top = 0;
        if (wgemm(true, b, b, M, V, M, W, M, G, b, false, P, pcap, sms, st) != cudaSuccess) {
          fail(-6, "window generator: Rayleigh quotient");
          break;
        }
        k_wjacobi<<<1, 128, smem2, st>>>(G, b, Q, ev, flags + 1);
        k_writz<<<nblk, 256, 0, st>>>(V, W, M, b, Q, ev, flags + 1, x, part);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(pn.data(), part, sizeof(double) * pn.size(), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(&top, flags + 1, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess ||
            cudaMemcpyAsync(&lam, ev + top, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
          fail(-6, "window generator: Rayleigh-Ritz");
          break;
        }
        double xn = 0.0, rn = 0.0;
        for (int i = 0; i < nblk; ++i) { xn += pn[2 * i]; rn += pn[2 * i + 1]; }
        last_res = std::sqrt(rn / xn);
        last_change = std::fabs(lam - prev);
        // the Ritz value settled to a few units in the last place of lambda <= 1
        if (last_res < 1e-13 && last_change < 4e-15) { converged = true; break; }
        prev = lam;
      }
      // the next block: an orthonormal basis of K V
      std::swap(V, W);
      if (wortho(V, M, b, G, P, pcap, flags, sms, st) != cudaSuccess) {
        fail(-6, "window generator: orthonormalisation");
        break;
      }
    }
    if (status) break;
    int bad = 0;
    std::vector<double> top(M);
    if (cudaMemcpyAsync(&bad, flags, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(top.data(), x, sizeof(double) * M, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      fail(-6, "window generator: result");
      break;
    }
    (void)bad;                       // pivots replaced along the way; the convergence test decides
    if (!converged) {
      if (errbuf && errlen)
        snprintf(errbuf, errlen, "window generator: subspace iteration did not converge (residual %.3g, change %.3g)",
                 last_res, last_change);
      status = -5;
      break;
    }
    // real even basis -> complex coefficients, unit energy, h_0^0 > 0
    double nrm = 0.0;
    for (double v : top) nrm += v * v;
    nrm = std::sqrt(nrm);
    const double sgn = top[0] < 0 ? -1.0 : 1.0;
    h.assign(2 * (size_t)L * L, 0.0);
    const double r2 = std::sqrt(0.5);
    for (int l = 0; l < L; ++l) {
      h[2 * ((size_t)l * l + l)] = sgn * top[(size_t)l * (l + 1) / 2] / nrm;
      for (int m = 1; m <= l; ++m) {
        const double c = sgn * top[(size_t)l * (l + 1) / 2 + m] / nrm * r2;
        h[2 * ((size_t)l * l + l + m)] = c;
        h[2 * ((size_t)l * l + l - m)] = (m & 1) ? -c : c;
      }
    }
    if (lambda_out) *lambda_out = lam;
  } while (0);
  cudaStreamSynchronize(st);
  if (nodes) release(nodes, bytes_nodes, actx);
  if (A) release(A, bytes_A, actx);
  if (K) release(K, bytes_K, actx);
  if (Vd) release(Vd, bytes_V, actx);
  return status;
}
