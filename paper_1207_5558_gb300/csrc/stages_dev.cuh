// Block bodies of the rotated-window stage, shared by the per-call kernel
// (k_rotwin_smem) and the batch kernel (k_batch_rotwin).
//
// H^p_q(j) = sum_{q'} h_p^{q'} d^p_{q,q'}(beta_b) e^{-i q' gamma_c}, j = b*Ng + c:
// the window's coefficients rotated by (0, beta_b, gamma_c) (Eq. rotation_non_symm
// with Eq. Dlm), stored at H[h_index(p*p + p + q, j, Lh*Lh)].
#pragma once

#include "common.cuh"

// Shared memory of rotwin_block_smem: the (2p+1)^2 products and the Ng x
// (2p+1) gamma phases of the largest degree p = Lh - 1.
__host__ __device__ __forceinline__ size_t rotwin_smem_bytes(int Lh, int Ng, size_t el2) {
  const size_t K = 2 * (size_t)Lh - 1;
  return el2 * (K * K + (size_t)Ng * K);
}

// One (beta row b, degree p) block: the (2p+1)^2 products h_p^{q'}
// d^p_{q,q'}(beta_b) and the gamma phases of the orders |q'| <= p are staged
// in shared memory once, then each output (q, c) is a (2p+1)-term dot product
// read from shared memory (a warp shares q: broadcast rows of the products,
// odd-stride phase rows without bank conflicts).  dblk = the degree-p block
// of d(beta_b); eg[c * (2Lh-1) + q' + Lh - 1] = (cos, sin)(q' gamma_c).  All
// threads of the block take part (one __syncthreads).
// store(index, re, im) receives each output with its h_index position.
template <typename T, typename Store>
__device__ __forceinline__ void rotwin_block_smem_to(const double2* __restrict__ h, const T* __restrict__ dblk,
                                                     const typename vec2<T>::t* __restrict__ eg, int Lh, int Ng,
                                                     int b, int p, Store store, unsigned char* smem) {
  typedef typename vec2<T>::t T2;
  const int K = 2 * Lh - 1, n2 = Lh * Lh, w = 2 * p + 1;
  T2* hd = reinterpret_cast<T2*>(smem);       // [q + p][q' + p]
  T2* ep = hd + w * w;                        // [c][q' + p]
  for (int t = threadIdx.x; t < w * w; t += blockDim.x) {
    const int qp = t % w;
    const double2 hv = __ldg(h + p * p + qp);
    const T d = __ldg(dblk + t);
    hd[t] = mk2(d * (T)hv.x, d * (T)hv.y);
  }
  for (int t = threadIdx.x; t < Ng * w; t += blockDim.x) {
    const int c = t / w, qp = t % w;
    ep[t] = eg[(size_t)c * K + (Lh - 1) - p + qp];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < w * Ng; t += blockDim.x) {
    const int qi = t / Ng, c = t % Ng;
    const T2* hr = hd + qi * w;
    const T2* er = ep + c * w;
    T re = 0, im = 0;
    for (int u = 0; u < w; ++u) {                // h d (cos - i sin)
      const T2 a = hr[u], E = er[u];
      re = fma(a.x, E.x, re); re = fma(a.y, E.y, re);
      im = fma(a.y, E.x, im); im = fma(-a.x, E.y, im);
    }
    store(h_index(p * p + qi, b * Ng + c, n2), re, im);
  }
}

template <typename T>
struct RotwinStore {
  typename vec2<T>::t* H;
  __device__ __forceinline__ void operator()(size_t i, T re, T im) const { H[i] = mk2(re, im); }
};

template <typename T>
__device__ __forceinline__ void rotwin_block_smem(const double2* __restrict__ h, const T* __restrict__ dblk,
                                                  const typename vec2<T>::t* __restrict__ eg, int Lh, int Ng, int b,
                                                  int p, typename vec2<T>::t* __restrict__ H, unsigned char* smem) {
  rotwin_block_smem_to<T>(h, dblk, eg, Lh, Ng, b, p, RotwinStore<T>{H}, smem);
}

// The same block without shared memory (windows whose staged products would
// not fit): each output reads h, d and the phases through the cache.
template <typename T, typename Store>
__device__ __forceinline__ void rotwin_block_direct_to(const double2* __restrict__ h, const T* __restrict__ dblk,
                                                       const typename vec2<T>::t* __restrict__ eg, int Lh, int Ng,
                                                       int b, int p, Store store) {
  typedef typename vec2<T>::t T2;
  const int K = 2 * Lh - 1, n2 = Lh * Lh, w = 2 * p + 1;
  for (int t = threadIdx.x; t < w * Ng; t += blockDim.x) {
    const int qi = t / Ng, c = t % Ng;
    const T* drow = dblk + qi * w;
    const T2* erow = eg + (size_t)c * K + (Lh - 1) - p;
    T re = 0, im = 0;
    for (int u = 0; u < w; ++u) {
      const double2 hv = __ldg(h + p * p + u);
      const T d = __ldg(drow + u);
      const T2 E = erow[u];
      const T ar = d * (T)hv.x, ai = d * (T)hv.y;
      re = fma(ar, E.x, re); re = fma(ai, E.y, re);
      im = fma(ai, E.x, im); im = fma(-ar, E.y, im);
    }
    store(h_index(p * p + qi, b * Ng + c, n2), re, im);
  }
}
