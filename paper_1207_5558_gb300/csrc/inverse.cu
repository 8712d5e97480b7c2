// Inverse directional SLSHT (Sec. III-C, Eq. inversion_1, inversion_2, and the
// exact SO(3) quadrature of Eq. sig_reconstruction_discrete):
//   f_lm = (2 pi/Na)(2 pi/Ng) sum_{a,b,c} q_b g[a][b][c] / (sqrt(16 pi^3) h_0^0).
// A bandwidth-bound reduction, reordered as
//   f_lm ~ sum_j q_{b(j)} S_j,     S_j = sum_a g[a][j]   (j = b*Ng + c),
// so the inner loop is a plain column sum: thread j of a CTA walks down the
// alpha rows of one slab of its pair (eight rows in flight, consecutive
// threads on consecutive columns), weights its column once, and the CTA adds
// its columns in a fixed tree; a second kernel adds the CTA sums of a pair in
// a fixed order, so results are bitwise reproducible.  FP64 accumulation for
// both precisions; for complex64 g the eight rows of a step are first added
// in FP32 (g itself carries ~1e-7 relative error), keeping the per-sample work
// off the FP64 pipe.
#include "common.cuh"

#define INV_THREADS 256

template <typename T2>
__global__ void __launch_bounds__(INV_THREADS)
k_inverse_cols(const T2* __restrict__ g, const double* __restrict__ wb, int Na, int Nb, int Ng, int nslab,
               double2* __restrict__ partial) {
  __shared__ double sre[INV_THREADS], sim[INV_THREADS];
  const int cb = blockIdx.x, pair = blockIdx.y, slab = blockIdx.z;
  const size_t J = (size_t)Nb * Ng;
  const size_t j = (size_t)cb * INV_THREADS + threadIdx.x;
  const int rows_per = (Na + nslab - 1) / nslab;
  const int a0 = slab * rows_per, a1 = min(Na, a0 + rows_per);
  double re = 0.0, im = 0.0;
  if (j < J) {
    const T2* col = g + (size_t)pair * Na * J + j;
    int a = a0;
    for (; a + 7 < a1; a += 8) {
      T2 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = __ldcs(col + (size_t)(a + u) * J);
      if constexpr (sizeof(T2) == sizeof(double2)) {     // pairwise: short FP64 add chains
        re += ((v[0].x + v[1].x) + (v[2].x + v[3].x)) + ((v[4].x + v[5].x) + (v[6].x + v[7].x));
        im += ((v[0].y + v[1].y) + (v[2].y + v[3].y)) + ((v[4].y + v[5].y) + (v[6].y + v[7].y));
      } else {
        const float sr = ((v[0].x + v[1].x) + (v[2].x + v[3].x)) + ((v[4].x + v[5].x) + (v[6].x + v[7].x));
        const float si = ((v[0].y + v[1].y) + (v[2].y + v[3].y)) + ((v[4].y + v[5].y) + (v[6].y + v[7].y));
        re += (double)sr;
        im += (double)si;
      }
    }
    for (; a < a1; ++a) {
      const T2 v = __ldcs(col + (size_t)a * J);
      re += (double)v.x;
      im += (double)v.y;
    }
    const double w = wb[j / Ng];
    re *= w;
    im *= w;
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
  if (threadIdx.x == 0)
    partial[((size_t)pair * nslab + slab) * gridDim.x + cb] = make_double2(sre[0], sim[0]);
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

int inverse_col_blocks(int Nb, int Ng) { return (int)(((size_t)Nb * Ng + INV_THREADS - 1) / INV_THREADS); }

template <typename T2>
static cudaError_t launch_inverse_t(const T2* g, const double* wb, int Na, int Nb, int Ng,
                                    int npairs, double2* partial, int nslab, cudaStream_t st) {
  if (npairs <= 0) return cudaSuccess;
  const int ncb = inverse_col_blocks(Nb, Ng);
  if (nslab > 65535) return cudaErrorInvalidValue;
  const size_t per_pair = (size_t)Na * Nb * Ng;
  for (int p0 = 0; p0 < npairs; p0 += 65535) {      // grid.y limit
    const int np = npairs - p0 < 65535 ? npairs - p0 : 65535;
    dim3 grid(ncb, np, nslab);
    k_inverse_cols<T2><<<grid, INV_THREADS, 0, st>>>(g + per_pair * p0, wb, Na, Nb, Ng, nslab,
                                                     partial + (size_t)p0 * nslab * ncb);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
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
