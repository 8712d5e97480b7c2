// Inverse directional SLSHT (Sec. III-C, Eq. inversion_1, inversion_2, and the
// exact SO(3) quadrature of Eq. sig_reconstruction_discrete):
//   f_lm = (2 pi/Na)(2 pi/Ng) sum_{a,b,c} q_b g[a][b][c] / (sqrt(16 pi^3) h_0^0).
// A bandwidth-bound reduction: each CTA sums a fixed slab of alpha rows of one
// pair in a fixed order (strided per-thread sums, then a fixed tree), and a
// second kernel adds the slab sums in order, so results are bitwise
// reproducible.  Accumulation is FP64 for both input precisions.
#include "common.cuh"

#define INV_THREADS 256

template <typename T2>
__global__ void __launch_bounds__(INV_THREADS)
k_inverse_partial(const T2* __restrict__ g, const double* __restrict__ wb, int Na, int Nb, int Ng,
                  int nslab, double2* __restrict__ partial) {
  __shared__ double sre[INV_THREADS], sim[INV_THREADS];
  const int slab = blockIdx.x, pair = blockIdx.y;
  const int rows_per = (Na + nslab - 1) / nslab;
  const int a0 = slab * rows_per, a1 = min(Na, a0 + rows_per);
  const size_t J = (size_t)Nb * Ng;
  const T2* base = g + (size_t)pair * Na * J;
  double re = 0.0, im = 0.0;
  // j advances by INV_THREADS: keep (b, c) = (j / Ng, j % Ng) by increments
  const int db = INV_THREADS / Ng, dc = INV_THREADS % Ng;
  for (int a = a0; a < a1; ++a) {
    const T2* row = base + (size_t)a * J;
    int b = threadIdx.x / Ng, c = threadIdx.x % Ng;
    for (size_t j = threadIdx.x; j < J; j += INV_THREADS) {
      const double w = wb[b];
      const T2 v = row[j];
      re = fma(w, (double)v.x, re);
      im = fma(w, (double)v.y, im);
      b += db;
      c += dc;
      if (c >= Ng) { c -= Ng; ++b; }
    }
  }
  sre[threadIdx.x] = re;
  sim[threadIdx.x] = im;
  __syncthreads();
  for (int s = INV_THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sre[threadIdx.x] += sre[threadIdx.x + s];
      sim[threadIdx.x] += sim[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[(size_t)pair * nslab + slab] = make_double2(sre[0], sim[0]);
}

__global__ void k_inverse_final(const double2* __restrict__ partial, int nslab, int npairs,
                                double sre, double sim, double2* __restrict__ fout) {
  const int pair = blockIdx.x * blockDim.x + threadIdx.x;
  if (pair >= npairs) return;
  double re = 0.0, im = 0.0;
  for (int s = 0; s < nslab; ++s) {
    const double2 v = partial[(size_t)pair * nslab + s];
    re += v.x;
    im += v.y;
  }
  fout[pair] = make_double2(re * sre - im * sim, re * sim + im * sre);
}

template <typename T2>
static cudaError_t launch_inverse_t(const T2* g, const double* wb, int Na, int Nb, int Ng,
                                    int npairs, double2* partial, int nslab, cudaStream_t st) {
  if (npairs <= 0) return cudaSuccess;
  dim3 grid(nslab, npairs);
  k_inverse_partial<T2><<<grid, INV_THREADS, 0, st>>>(g, wb, Na, Nb, Ng, nslab, partial);
  return cudaGetLastError();
}

cudaError_t launch_inverse_f64(const double2* g, const double* wb, int Na, int Nb, int Ng,
                               int npairs, double2* partial, int nslab, cudaStream_t st) {
  return launch_inverse_t<double2>(g, wb, Na, Nb, Ng, npairs, partial, nslab, st);
}
cudaError_t launch_inverse_f32(const float2* g, const double* wb, int Na, int Nb, int Ng,
                               int npairs, double2* partial, int nslab, cudaStream_t st) {
  return launch_inverse_t<float2>(g, wb, Na, Nb, Ng, npairs, partial, nslab, st);
}

cudaError_t launch_inverse_final(const double2* partial, int nslab, int npairs, double scale_re,
                                 double scale_im, double2* fout, cudaStream_t st) {
  if (npairs <= 0) return cudaSuccess;
  k_inverse_final<<<(npairs + 127) / 128, 128, 0, st>>>(partial, nslab, npairs, scale_re, scale_im,
                                                         fout);
  return cudaGetLastError();
}
