// g at arbitrary orientations gamma from the grid's gamma samples (the remark
// on steerable windows in Sec. IV-B: by linearity, the distribution at any
// gamma follows from a few basis orientations).
//
// g depends on gamma only through e^{-i q' gamma}, |q'| <= Q, where Q is the
// largest azimuthal order of the window (Eq. alternative_harmonic_formulation_wigner
// with D from Eq. Dlm): Q = L_h - 1 for a general window, N - 1 for a steerable
// window with h_p^q' = 0 for |q'| >= N.  With N_gamma >= 2Q + 1 samples
// gamma_c = 2 pi c / N_gamma the samples determine the Q-band trigonometric
// polynomial exactly, and
//   g(gamma) = sum_c w_c(gamma) g(gamma_c),
//   w_c(gamma) = (1 + 2 sum_{q'=1..Q} cos(q' (gamma - gamma_c))) / N_gamma,
// a real weight (the Dirichlet kernel of the band), so every output is a real
// combination of one row of N_gamma grid samples.
#include "common.cuh"

// W[k][c] = w_c(gamma_k), FP64
__global__ void k_steer_weights(const double* __restrict__ gam, int ng, int Ngam, int Q, double* __restrict__ W) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)ng * Ngam) return;
  const int k = (int)(t / Ngam), c = (int)(t % Ngam);
  const double pi = 3.14159265358979323846;
  const double d = gam[k] - 2.0 * pi * c / Ngam;
  double s = 1.0;
  for (int q = 1; q <= Q; ++q) s += 2.0 * cos(q * d);
  W[t] = s / Ngam;
}

// out[row][k] = sum_c W[k][c] g[row][c]; one thread per (row, k), the row's
// samples and the weights from L1/L2 (rows of N_gamma <= 255 values)
template <typename T2>
__global__ void k_steer(const T2* __restrict__ g, long long rows, int Ngam, const double* __restrict__ W, int ng,
                        T2* __restrict__ out) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows * ng) return;
  const long long row = t / ng;
  const int k = (int)(t % ng);
  const T2* src = g + row * Ngam;
  const double* w = W + (size_t)k * Ngam;
  double re = 0.0, im = 0.0;
  for (int c = 0; c < Ngam; ++c) {
    const T2 v = src[c];
    re = fma(w[c], (double)v.x, re);
    im = fma(w[c], (double)v.y, im);
  }
  typedef decltype(T2().x) T;
  out[t] = mk2((T)re, (T)im);
}

cudaError_t launch_steer_gamma(const void* g, int prec, long long rows, int Ngam, const double* gam, int ng, int Q,
                               double* W, void* out, cudaStream_t st) {
  if (rows <= 0 || ng <= 0) return cudaSuccess;
  const long long nw = (long long)ng * Ngam;
  k_steer_weights<<<(unsigned)((nw + 255) / 256), 256, 0, st>>>(gam, ng, Ngam, Q, W);
  const long long n = rows * ng;
  const unsigned blocks = (unsigned)((n + 255) / 256);
  if (prec == 0)
    k_steer<double2><<<blocks, 256, 0, st>>>((const double2*)g, rows, Ngam, W, ng, (double2*)out);
  else
    k_steer<float2><<<blocks, 256, 0, st>>>((const float2*)g, rows, Ngam, W, ng, (float2*)out);
  return cudaGetLastError();
}
