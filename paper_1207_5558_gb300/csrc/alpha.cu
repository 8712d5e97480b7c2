// alpha stage on CUDA cores (FP64 path; also an FP32 variant):
//   g[a][j] = sum_q X_q[j] e^{-i q alpha_a}
//           = X_0[j] + sum_{r=1}^{Lh-1} ( P_r[j] cos(r alpha_a) - i M_r[j] sin(r alpha_a) ),
// with P_r = X_r + X_-r and M_r = X_r - X_-r from the gamma stage: pairing +q
// and -q halves the multiply-adds of the direct sum (4(Lh-1) + 2 per sample).
// One thread per column j = (beta, gamma) sample; its 2Lh-1 coefficients sit
// in shared memory; each thread produces ALPHA_ABLK consecutive alpha rows per pass
// so a coefficient load feeds 4*ALPHA_ABLK fused multiply-adds.  Stores are
// coalesced: for a fixed row a, a warp writes 32 consecutive columns.
#include "alpha_dev.cuh"

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
  // paired layout of Xs: row 0 X_0, row 2r-1 P_r, row 2r M_r
  alpha_direct_column<T>(sx + t, NT, 0, -1, 2, 0, 2, Lh, Na, J, csa, dst, mdst, ms, 0, ALPHA_ABLK);
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

// ---------------------------------------------------------------- split DFT
// The alpha sum as the split DFT of alpha_split_column (alpha_dev.cuh); the
// paired input rows are unpaired into X_q, row q + Lh - 1, in shared memory.
template <typename T, int P, int NT>
__global__ void __launch_bounds__(NT)
k_alpha_split(const typename vec2<T>::t* __restrict__ Xs, const typename vec2<T>::t* __restrict__ tw, int Lh,
              int Na, int J, typename vec2<T>::t* __restrict__ g, const int2* __restrict__ slots) {
  typedef typename vec2<T>::t T2;
  constexpr int H = (P - 1) / 2;
  extern __shared__ unsigned char smem_raw[];
  T2* sx = reinterpret_cast<T2*>(smem_raw);      // [q + Lh - 1][NT]: X_q
  __shared__ T cpr[H + 1][H + 1], spr[H + 1][H + 1];   // cos / sin(2 pi r s / P), r, s >= 1
  const int K = 2 * Lh - 1;
  const int pair = blockIdx.y;
  const int t = threadIdx.x;
  const int j = blockIdx.x * NT + t;
  const T2* src = Xs + (size_t)pair * K * J;
  alpha_split_consts<T, P>(cpr, spr, t);
  if (j < J) {
    const T2 x0 = src[j];
    sx[(Lh - 1) * NT + t] = x0;
    for (int r = 1; r < Lh; ++r) {
      const T2 pr = src[(size_t)(2 * r - 1) * J + j], mr = src[(size_t)(2 * r) * J + j];
      sx[(Lh - 1 + r) * NT + t] = mk2((T)0.5 * (pr.x + mr.x), (T)0.5 * (pr.y + mr.y));
      sx[(Lh - 1 - r) * NT + t] = mk2((T)0.5 * (pr.x - mr.x), (T)0.5 * (pr.y - mr.y));
    }
  }
  __syncthreads();
  if (j >= J) return;
  const int2 sl = slots != nullptr ? slots[pair] : make_int2(pair, -1);
  T2* dst = g + (size_t)sl.x * Na * J + j;
  T2* mdst = sl.y >= 0 ? g + (size_t)(sl.y >> 1) * Na * J + j : nullptr;
  const T ms = (sl.y & 1) ? (T)-1 : (T)1;
  alpha_split_column<T, P>(sx + t, NT, Lh, Na, J, tw, cpr, spr, dst, mdst, ms, 0, 1);
}

// The split factor for Na: the odd P in {9, 7, 5, 3} dividing Na with the
// fewest multiply-adds per sample (about 4K/P + P + 3), or 0 (direct sum).
int alpha_split_factor(int Lh, int Na) {
  const int K = 2 * Lh - 1;
  const double direct = 4.0 * (Lh - 1) + 2.0;
  int best = 0;
  double cost = direct;
  const int cand[4] = {9, 7, 5, 3};
  for (int i = 0; i < 4; ++i) {
    const int P = cand[i];
    if (Na % P != 0 || Na / P < 1) continue;
    const double c = 4.0 * K / P + P + 3.0;
    if (c < cost) { cost = c; best = P; }
  }
  return best;
}

template <typename T, int P>
static cudaError_t launch_split_p(const typename vec2<T>::t* Xs, const typename vec2<T>::t* tw, int Lh, int Na,
                                  int J, int npairs, typename vec2<T>::t* g, const int2* slots, cudaStream_t st) {
  typedef typename vec2<T>::t T2;
  const size_t smem128 = sizeof(T2) * (size_t)(2 * Lh - 1) * 128;
  if (smem128 <= 200 * 1024) {
    if (smem128 > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(k_alpha_split<T, P, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem128);
      if (e != cudaSuccess) return e;
    }
    dim3 grid((J + 127) / 128, npairs);
    k_alpha_split<T, P, 128><<<grid, 128, smem128, st>>>(Xs, tw, Lh, Na, J, g, slots);
    return cudaGetLastError();
  }
  const size_t smem64 = smem128 / 2;
  if (smem64 > 200 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_alpha_split<T, P, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem64);
  if (e != cudaSuccess) return e;
  dim3 grid((J + 63) / 64, npairs);
  k_alpha_split<T, P, 64><<<grid, 64, smem64, st>>>(Xs, tw, Lh, Na, J, g, slots);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_split_t(const typename vec2<T>::t* Xs, const typename vec2<T>::t* tw, int Lh, int Na,
                                  int J, int npairs, typename vec2<T>::t* g, const int2* slots, cudaStream_t st) {
  if (npairs <= 0 || J <= 0) return cudaSuccess;
  switch (alpha_split_factor(Lh, Na)) {
    case 9: return launch_split_p<T, 9>(Xs, tw, Lh, Na, J, npairs, g, slots, st);
    case 7: return launch_split_p<T, 7>(Xs, tw, Lh, Na, J, npairs, g, slots, st);
    case 5: return launch_split_p<T, 5>(Xs, tw, Lh, Na, J, npairs, g, slots, st);
    case 3: return launch_split_p<T, 3>(Xs, tw, Lh, Na, J, npairs, g, slots, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_alpha_split_f64(const double2* Xs, const double2* tw, int Lh, int Na, int J, int npairs,
                                   double2* g, const int2* slots, cudaStream_t st) {
  return launch_split_t<double>(Xs, tw, Lh, Na, J, npairs, g, slots, st);
}
cudaError_t launch_alpha_split_f32(const float2* Xs, const float2* tw, int Lh, int Na, int J, int npairs,
                                   float2* g, const int2* slots, cudaStream_t st) {
  return launch_split_t<float>(Xs, tw, Lh, Na, J, npairs, g, slots, st);
}
