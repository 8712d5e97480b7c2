// Block bodies of the rotated-window stage, shared by the per-call kernel
// (k_rotwin_smem) and the batch kernel (k_batch_rotwin).
//
// H^p_q(j) = sum_{q'} h_p^{q'} d^p_{q,q'}(beta_b) e^{-i q' gamma_c}, j = b*Ng + c:
// the window's coefficients rotated by (0, beta_b, gamma_c) (Eq. rotation_non_symm
// with Eq. Dlm), stored at H[h_index(p*p + p + q, j, Lh*Lh)].
#pragma once

#include <type_traits>

#include "common.cuh"

// Shared-memory chunking of a rotated-window block.  With the window folded
// into the gamma phases,
//   H^p_q(b, c) = sum_{q'} d^p_{q,q'}(beta_b) B_p(q', c),
//   B_p(q', c)  = h_p^{q'} e^{-i q' gamma_c},
// each (degree p) slice is a real-by-complex matrix product whose rows are the
// (beta row, q) pairs.  A block (beta rows b .. b + ROTWIN_NB - 1, degree p,
// column chunk z) stages B_p for CC <= 32 gamma columns once, then passes over
// its ROTWIN_NB (2p+1) rows QC at a time, staging their d rows (transposed)
// for each pass.  nq = 1 (kept for the batch block lists).
#define ROTWIN_SMEM_LIMIT (200 * 1024)
#define ROTWIN_NB 4          // beta rows a block serves
#define ROTWIN_CC 32         // gamma columns of a chunk
#define ROTWIN_THREADS 128   // 16 row groups x 8 column groups
struct RotChunks {
  int QC, CC, nq, nc;
  // d rows of one pass ([2Lh-1][QC] reals) and B ([2Lh-1][CC] complex)
  __host__ __device__ size_t smem(int Lh, size_t el2) const {
    return (el2 / 2) * (size_t)QC * (2 * Lh - 1) + el2 * (size_t)CC * (2 * Lh - 1);
  }
};
// Rows a thread holds: four (float, one 16-byte load of d) or two (double).
__host__ __device__ inline int rot_tq(size_t el2) { return el2 == 8 ? 4 : 2; }
__host__ __device__ inline RotChunks rot_chunks(int Lh, int Ng, size_t el2) {
  (void)Lh;
  RotChunks r;
  r.QC = 16 * rot_tq(el2);
  r.CC = ROTWIN_CC;
  r.nq = 1;
  r.nc = (Ng + r.CC - 1) / r.CC;
  return r;
}

// Asynchronous 4- or 8-byte global -> shared copy (cp.async), and the wait
// for all of this thread's copies.
template <typename T>
__device__ __forceinline__ void cp_async_el(T* dst, const T* src) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8, "cp.async element");
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  if (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

__device__ __forceinline__ void rot_unpack(const float4 v, float* d) { d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w; }
__device__ __forceinline__ void rot_unpack(const double2 v, double* d) { d[0] = v.x; d[1] = v.y; }

// Orders q' of the window that take part in the sums: bit q' + 63 of the four
// words of qmask (null: every order).  A window whose coefficients vanish at
// some orders for every degree -- a steerable window, azimuthally band-limited
// (|q'| < N < L_h), or a window with only even orders -- then costs only its
// active orders: the sums over q' skip terms that are zero.
__device__ __forceinline__ bool rot_order_on(const uint32_t* qmask, int qp) {
  if (qmask == nullptr) return true;
  const int bit = qp + 63;
  return (__ldg(qmask + (bit >> 5)) >> (bit & 31)) & 1u;
}

// One (beta rows b0 .. b0 + nb - 1, degree p, column chunk z) block of the
// rotated window (see RotChunks).  dblk0 = the degree-p block of d(beta_b0),
// consecutive beta rows dstride apart, row-major [q + p][q' + p];
// eg[c * (2Lh-1) + q' + Lh - 1] = (cos, sin)(q' gamma_c).  The d rows are read
// through the symmetry d^p_{q,q'} = (-1)^{q-q'} d^p_{q',q}, so that the
// staging copies run along q (coalesced, cp.async: a pass's loads all in
// flight) and land in [q'][row] order; the sign (-1)^{q'+p} is folded into
// the staged B rows and (-1)^{q+p} into the outputs.  A thread holds TQ consecutive
// rows x 4 columns (c0 + cg + 8 k), 2 multiply-adds a term.  Only the orders
// that qmask marks active are staged and summed (in increasing q', so with
// every order active the sums are those of the full window).
// All threads of the block take part.  store(index, re, im) receives each
// output with its h_index position.
template <typename T, typename Store>
__device__ __forceinline__ void rotwin_block_smem_to(const double2* __restrict__ h, const T* __restrict__ dblk0,
                                                     size_t dstride, int nb, const typename vec2<T>::t* __restrict__ eg,
                                                     int Lh, int Ng, int b0, int p, const RotChunks& ch, int z,
                                                     Store store, unsigned char* smem,
                                                     const uint32_t* qmask = nullptr) {
  typedef typename vec2<T>::t T2;
  constexpr int TQ = sizeof(T) == 4 ? 4 : 2;
  typedef typename std::conditional<sizeof(T) == 4, float4, double2>::type TV;   // TQ values of T
  const int K = 2 * Lh - 1, n2 = Lh * Lh, w = 2 * p + 1;
  const int QC = ch.QC, CC = ch.CC;
  if (QC != 16 * TQ || CC != ROTWIN_CC) return;   // the tiling below assumes rot_chunks' shape
  const int c0 = z * CC, ncr = min(CC, Ng - c0);
  T* sd = reinterpret_cast<T*>(smem);                          // [active order][row of the pass]
  T2* sB = reinterpret_cast<T2*>(sd + (size_t)QC * K);         // [active order][c - c0]
  // the active orders of degree p as u = q' + p, increasing
  __shared__ int s_ul[2 * SLSHT_MAX_LH - 1];
  __shared__ int s_nu;
  __syncthreads();                            // s_ul of a previous block of this CTA is read
  if (threadIdx.x == 0) {
    int n = 0;
    for (int u = 0; u < w; ++u)
      if (rot_order_on(qmask, u - p)) s_ul[n++] = u;
    s_nu = n;
  }
  __syncthreads();
  const int nu = s_nu;
  // (-1)^{q'+p} B_p(q', c) = (-1)^{q'+p} h_p^{q'} (cos - i sin)(q' gamma_c); zero beyond the chunk
  for (int t = threadIdx.x; t < nu * CC; t += ROTWIN_THREADS) {
    const int i = t / CC, c = t - i * CC, u = s_ul[i];
    T2 v = mk2((T)0, (T)0);
    if (c < ncr) {
      const double2 hv = __ldg(h + p * p + u);
      const T2 e = eg[(size_t)(c0 + c) * K + (Lh - 1) - p + u];
      const T hx = (u & 1) ? -(T)hv.x : (T)hv.x, hy = (u & 1) ? -(T)hv.y : (T)hv.y;
      v = mk2(hx * e.x + hy * e.y, hy * e.x - hx * e.y);
    }
    sB[t] = v;
  }
  const int rows = nb * w;
  const int rg = threadIdx.x >> 3, cg = threadIdx.x & 7;
  // staging: a thread always fills row rr of the pass, every ustep-th u
  constexpr int QCc = 16 * TQ, ustep = ROTWIN_THREADS / QCc;
  const int rr = threadIdx.x % QCc, u0 = threadIdx.x / QCc;
  for (int r0 = 0; r0 < rows; r0 += QCc) {
    __syncthreads();                          // sB ready; the previous pass's d rows read
    // d rows of the pass, transposed: sd[i][rr] = d[u][q + p] = (-1)^{q+u}
    // d^p_{q,u-p}(beta_b), u = s_ul[i], for row r0 + rr = (b - b0) w + q + p (rows past the
    // end are left as they are: they feed only outputs that are not stored)
    {
      const int r = r0 + rr;
      if (r < rows) {
        const int bi = r / w, qi = r - bi * w;
        const T* src = dblk0 + (size_t)bi * dstride + qi;
        for (int i = u0; i < nu; i += ustep) cp_async_el(sd + (size_t)i * QCc + rr, src + (size_t)s_ul[i] * w);
      }
      cp_async_wait_all();
    }
    __syncthreads();
    T re[TQ][4], im[TQ][4];
#pragma unroll
    for (int a = 0; a < TQ; ++a)
#pragma unroll
      for (int k = 0; k < 4; ++k) re[a][k] = im[a][k] = (T)0;
    const T* dp = sd + rg * TQ;
    const T2* bp = sB + cg;
    for (int i = 0; i < nu; ++i) {
      T dq[TQ];
      rot_unpack(*reinterpret_cast<const TV*>(dp + (size_t)i * QCc), dq);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const T2 bv = bp[(size_t)i * CC + 8 * k];
#pragma unroll
        for (int a = 0; a < TQ; ++a) {
          re[a][k] = fma(dq[a], bv.x, re[a][k]);
          im[a][k] = fma(dq[a], bv.y, im[a][k]);
        }
      }
    }
#pragma unroll
    for (int a = 0; a < TQ; ++a) {
      const int r = r0 + rg * TQ + a;
      if (r >= rows) continue;
      const int bi = r / w, qi = r - bi * w;
      const int jb = (b0 + bi) * Ng + c0;
      const T sg = (qi & 1) ? (T)-1 : (T)1;             // (-1)^{q+p}
      const int hr = h_row(p, qi - p, Lh, sizeof(T) == 4 && h_order_major(Lh));
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int c = cg + 8 * k;
        if (c < ncr) store(h_index(hr, jb + c, n2), sg * re[a][k], sg * im[a][k]);
      }
    }
  }
}

template <typename T>
struct RotwinStore {
  typename vec2<T>::t* H;
  __device__ __forceinline__ void operator()(size_t i, T re, T im) const { H[i] = mk2(re, im); }
};
