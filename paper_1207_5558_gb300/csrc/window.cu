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
// A[pt][a] = sqrt(w_pt) u_a(pt), K = A^T A (one symmetric rank-k update on
// the tensor-core-free FP64 path of cuBLAS: a plain library product).  The top
// eigenpair by block subspace iteration (block larger than the Shannon number
// trace(K), where the eigenvalues cluster near 1) with a Rayleigh-Ritz step
// on the host; the block products K V run on the device.
#include <cublas_v2.h>

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

// Modified Gram-Schmidt on the columns of V (m x b, column-major), twice.
static void orthonormalise(std::vector<double>& V, int m, int b) {
  for (int pass = 0; pass < 2; ++pass) {
    for (int j = 0; j < b; ++j) {
      double* vj = &V[(size_t)j * m];
      for (int k = 0; k < j; ++k) {
        const double* vk = &V[(size_t)k * m];
        double d = 0.0;
        for (int i = 0; i < m; ++i) d += vk[i] * vj[i];
        for (int i = 0; i < m; ++i) vj[i] -= d * vk[i];
      }
      double nrm = 0.0;
      for (int i = 0; i < m; ++i) nrm += vj[i] * vj[i];
      nrm = std::sqrt(nrm);
      if (nrm > 0.0)
        for (int i = 0; i < m; ++i) vj[i] /= nrm;
    }
  }
}

// Cyclic Jacobi eigen-decomposition of the symmetric b x b matrix T
// (column-major); eigenvalues to ev, eigenvectors (columns) to Q.
static void jacobi_eig(std::vector<double> T, int b, std::vector<double>& ev, std::vector<double>& Q) {
  Q.assign((size_t)b * b, 0.0);
  for (int i = 0; i < b; ++i) Q[(size_t)i * b + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < b; ++p)
      for (int q = p + 1; q < b; ++q) off += T[(size_t)q * b + p] * T[(size_t)q * b + p];
    if (off < 1e-30) break;
    for (int p = 0; p < b; ++p) {
      for (int q = p + 1; q < b; ++q) {
        const double apq = T[(size_t)q * b + p];
        if (std::fabs(apq) < 1e-300) continue;
        const double app = T[(size_t)p * b + p], aqq = T[(size_t)q * b + q];
        const double th = 0.5 * (aqq - app) / apq;
        const double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < b; ++k) {            // T <- J^T T J
          const double tkp = T[(size_t)p * b + k], tkq = T[(size_t)q * b + k];
          T[(size_t)p * b + k] = c * tkp - s * tkq;
          T[(size_t)q * b + k] = s * tkp + c * tkq;
        }
        for (int k = 0; k < b; ++k) {
          const double tpk = T[(size_t)k * b + p], tqk = T[(size_t)k * b + q];
          T[(size_t)k * b + p] = c * tpk - s * tqk;
          T[(size_t)k * b + q] = s * tpk + c * tqk;
        }
        for (int k = 0; k < b; ++k) {
          const double qkp = Q[(size_t)p * b + k], qkq = Q[(size_t)q * b + k];
          Q[(size_t)p * b + k] = c * qkp - s * qkq;
          Q[(size_t)q * b + k] = s * qkp + c * qkq;
        }
      }
    }
  }
  ev.resize(b);
  for (int i = 0; i < b; ++i) ev[i] = T[(size_t)i * b + i];
}

// ---------------------------------------------------------------- driver
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
  std::vector<double> glx, glw;
  gauss_legendre(n_theta, glx, glw);
  const size_t bytes_nodes = sizeof(double) * (3 * npts + 2 * (size_t)n_theta);
  const size_t bytes_A = sizeof(double) * npts * M;
  const size_t bytes_K = sizeof(double) * (size_t)M * M;
  int bmax = std::min(M, 96);
  const size_t bytes_V = sizeof(double) * (size_t)M * bmax * 2;
  double* nodes = (double*)alloc(bytes_nodes, actx);
  double* A = (double*)alloc(bytes_A, actx);
  double* K = (double*)alloc(bytes_K, actx);
  double* Vd = (double*)alloc(bytes_V, actx);
  int status = 0;
  cublasHandle_t hb = nullptr;
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
    if (cublasCreate(&hb) != CUBLAS_STATUS_SUCCESS || cublasSetStream(hb, st) != CUBLAS_STATUS_SUCCESS) {
      fail(-6, "window generator: cuBLAS handle");
      break;
    }
    const double one = 1.0, zero = 0.0;
    // K = A^T A (lower triangle), A: npts x M column-major
    if (cublasDsyrk(hb, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_T, M, (int)npts, &one, A, (int)npts, &zero, K, M) !=
        CUBLAS_STATUS_SUCCESS) {
      fail(-6, "window generator: cublasDsyrk");
      break;
    }
    // Shannon number trace(K): the count of eigenvalues near 1
    std::vector<double> Kdiag(M);
    if (cublasGetVector(M, sizeof(double), K, M + 1, Kdiag.data(), 1) != CUBLAS_STATUS_SUCCESS) {
      fail(-6, "window generator: trace");
      break;
    }
    double shannon = 0.0;
    for (double v : Kdiag) shannon += v;
    const int b = std::min(M, std::max(16, std::min(bmax, (int)std::ceil(2.0 * shannon) + 8)));
    // block subspace iteration with Rayleigh-Ritz
    std::vector<double> V((size_t)M * b), W((size_t)M * b), ev, Q, T((size_t)b * b);
    uint64_t seed = 0x9E3779B97F4A7C15ull;
    for (auto& v : V) {                        // splitmix64 -> [-1, 1)
      seed += 0x9E3779B97F4A7C15ull;
      uint64_t z = seed;
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      z ^= z >> 31;
      v = (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
    }
    orthonormalise(V, M, b);
    double* Vdev = Vd;
    double* Wdev = Vd + (size_t)M * bmax;
    double prev = -1.0, lam = 0.0;
    bool converged = false;
    std::vector<double> top(M);
    for (int it = 0; it < 400; ++it) {
      if (cudaMemcpyAsync(Vdev, V.data(), sizeof(double) * V.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
          cublasDsymm(hb, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_LOWER, M, b, &one, K, M, Vdev, M, &zero, Wdev, M) !=
              CUBLAS_STATUS_SUCCESS ||
          cudaMemcpyAsync(W.data(), Wdev, sizeof(double) * W.size(), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess) {
        fail(-6, "window generator: block product");
        break;
      }
      // Rayleigh-Ritz: T = V^T K V
      for (int j = 0; j < b; ++j)
        for (int i = 0; i < b; ++i) {
          double d = 0.0;
          const double* vi = &V[(size_t)i * M];
          const double* wj = &W[(size_t)j * M];
          for (int k = 0; k < M; ++k) d += vi[k] * wj[k];
          T[(size_t)j * b + i] = d;
        }
      for (int j = 0; j < b; ++j)              // symmetrise
        for (int i = j + 1; i < b; ++i) {
          const double s = 0.5 * (T[(size_t)j * b + i] + T[(size_t)i * b + j]);
          T[(size_t)j * b + i] = T[(size_t)i * b + j] = s;
        }
      jacobi_eig(T, b, ev, Q);
      int imax = 0;
      for (int i = 1; i < b; ++i)
        if (ev[i] > ev[imax]) imax = i;
      lam = ev[imax];
      // residual of the top Ritz pair: r = W q - lam V q
      double rn = 0.0, vn = 0.0;
      for (int k = 0; k < M; ++k) {
        double wv = 0.0, vv = 0.0;
        for (int i = 0; i < b; ++i) {
          wv += W[(size_t)i * M + k] * Q[(size_t)imax * b + i];
          vv += V[(size_t)i * M + k] * Q[(size_t)imax * b + i];
        }
        top[k] = vv;
        rn += (wv - lam * vv) * (wv - lam * vv);
        vn += vv * vv;
      }
      if (std::sqrt(rn / vn) < 1e-13 && std::fabs(lam - prev) < 1e-15) { converged = true; break; }
      prev = lam;
      V = W;                                   // next block: orth(K V)
      orthonormalise(V, M, b);
    }
    if (status) break;
    if (!converged) { fail(-5, "window generator: subspace iteration did not converge"); break; }
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
  if (hb) cublasDestroy(hb);
  cudaStreamSynchronize(st);
  if (nodes) release(nodes, bytes_nodes, actx);
  if (A) release(A, bytes_A, actx);
  if (K) release(K, bytes_K, actx);
  if (Vd) release(Vd, bytes_V, actx);
  return status;
}
