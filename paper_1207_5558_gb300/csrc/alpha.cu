// alpha stage on CUDA cores (FP64 path; also an FP32 variant):
//   g[a][j] = sum_q X_q[j] e^{-i q alpha_a}
//           = X_0[j] + sum_{r=1}^{Lh-1} ( P_r[j] cos(r alpha_a) - i M_r[j] sin(r alpha_a) ),
// with P_r = X_r + X_-r and M_r = X_r - X_-r from the gamma stage: pairing +q
// and -q halves the multiply-adds of the direct sum (4(Lh-1) + 2 per sample).
// One thread per column j = (beta, gamma) sample; its 2Lh-1 coefficients sit
// in shared memory; each thread produces ABLK consecutive alpha rows per pass
// so a coefficient load feeds 4*ABLK fused multiply-adds.  Stores are
// coalesced: for a fixed row a, a warp writes 32 consecutive columns.
#include "common.cuh"

#define ABLK 4

// NT columns per CTA: 128, or 64 when the 2Lh-1 staged coefficients of 128
// columns would not fit in shared memory (FP64 at Lh = 64).
template <typename T, int NT>
__global__ void __launch_bounds__(NT)
k_alpha_cc(const typename vec2<T>::t* __restrict__ Xs, const typename vec2<T>::t* __restrict__ csa,
           int Lh, int Na, int J, typename vec2<T>::t* __restrict__ g, const int2* __restrict__ slots) {
  typedef typename vec2<T>::t T2;
  extern __shared__ unsigned char smem_raw[];
  T2* sx = reinterpret_cast<T2*>(smem_raw);      // [2Lh-1][NT]
  const int K = 2 * Lh - 1;
  const int pair = blockIdx.y;
  const int j0 = blockIdx.x * NT;
  const int t = threadIdx.x;
  const int j = j0 + t;
  const T2* src = Xs + (size_t)pair * K * J;
  for (int c = 0; c < K; ++c)
    sx[c * NT + t] = (j < J) ? src[(size_t)c * J + j] : mk2((T)0, (T)0);
  __syncthreads();
  if (j >= J) return;
  // output slot and, for a mirrored pair, the slot of (l, -m) with (-1)^m
  const int2 sl = slots != nullptr ? slots[pair] : make_int2(pair, -1);
  T2* dst = g + (size_t)sl.x * Na * J + j;
  T2* mdst = sl.y >= 0 ? g + (size_t)(sl.y >> 1) * Na * J + j : nullptr;
  const T ms = (sl.y & 1) ? (T)-1 : (T)1;
  const T2 x0 = sx[t];
  for (int a0 = 0; a0 < Na; a0 += ABLK) {
    T re[ABLK], im[ABLK];
#pragma unroll
    for (int u = 0; u < ABLK; ++u) { re[u] = x0.x; im[u] = x0.y; }
    for (int r = 1; r < Lh; ++r) {
      const T2 P = sx[(2 * r - 1) * NT + t];
      const T2 M = sx[(2 * r) * NT + t];
#pragma unroll
      for (int u = 0; u < ABLK; ++u) {
        const int a = min(a0 + u, Na - 1);
        const T2 cs = csa[(size_t)a * Lh + r];
        re[u] = fma(P.x, cs.x, re[u]);
        re[u] = fma(M.y, cs.y, re[u]);
        im[u] = fma(P.y, cs.x, im[u]);
        im[u] = fma(-M.x, cs.y, im[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < ABLK; ++u)
      if (a0 + u < Na) dst[(size_t)(a0 + u) * J] = mk2(re[u], im[u]);
    if (mdst != nullptr) {
#pragma unroll
      for (int u = 0; u < ABLK; ++u)
        if (a0 + u < Na) mdst[(size_t)(a0 + u) * J] = mk2(ms * re[u], -ms * im[u]);
    }
  }
}

template <typename T>
static cudaError_t launch_alpha_t(const typename vec2<T>::t* Xs, const typename vec2<T>::t* csa,
                                  int Lh, int Na, int J, int npairs, typename vec2<T>::t* g,
                                  const int2* slots, cudaStream_t st) {
  if (npairs <= 0 || J <= 0) return cudaSuccess;
  typedef typename vec2<T>::t T2;
  const size_t smem128 = sizeof(T2) * (size_t)(2 * Lh - 1) * 128;
  if (smem128 <= 200 * 1024) {
    if (smem128 > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(k_alpha_cc<T, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem128);
      if (e != cudaSuccess) return e;
    }
    dim3 grid((J + 127) / 128, npairs);
    k_alpha_cc<T, 128><<<grid, 128, smem128, st>>>(Xs, csa, Lh, Na, J, g, slots);
    return cudaGetLastError();
  }
  const size_t smem64 = smem128 / 2;
  if (smem64 > 200 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_alpha_cc<T, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem64);
  if (e != cudaSuccess) return e;
  dim3 grid((J + 63) / 64, npairs);
  k_alpha_cc<T, 64><<<grid, 64, smem64, st>>>(Xs, csa, Lh, Na, J, g, slots);
  return cudaGetLastError();
}

cudaError_t launch_alpha_f64(const double2* Xs, const double2* csa, int Lh, int Na, int J,
                             int npairs, double2* g, const int2* slots, cudaStream_t st) {
  return launch_alpha_t<double>(Xs, csa, Lh, Na, J, npairs, g, slots, st);
}
cudaError_t launch_alpha_f32(const float2* Xs, const float2* csa, int Lh, int Na, int J,
                             int npairs, float2* g, const int2* slots, cudaStream_t st) {
  return launch_alpha_t<float>(Xs, csa, Lh, Na, J, npairs, g, slots, st);
}
