// Block bodies of the rotated-window stage, shared by the per-call kernel
// (k_rotwin_smem) and the batch kernel (k_batch_rotwin).
//
// H^p_q(j) = sum_{q'} h_p^{q'} d^p_{q,q'}(beta_b) e^{-i q' gamma_c}, j = b*Ng + c:
// the window's coefficients rotated by (0, beta_b, gamma_c) (Eq. rotation_non_symm
// with Eq. Dlm), stored at H[h_index(p*p + p + q, j, Lh*Lh)].
#pragma once

#include "common.cuh"

// Shared-memory chunking of a rotated-window block: a block (beta row b,
// degree p, chunk z) forms the outputs (q, c) with q + p in [q0, q0 + QC) and
// c in [c0, c0 + CC), staging QC rows of the (2p+1)^2 products h d and CC
// rows of gamma phases.  Whole blocks (QC = 2Lh-1, CC = Ng, one chunk) when
// they fit ROTWIN_SMEM_TARGET (four blocks an SM); otherwise CC <= 32 gamma
// columns and as many q rows as fit beside them.  ROTWIN_SMEM_LIMIT bounds
// the launches' dynamic shared memory.
#define ROTWIN_SMEM_LIMIT (200 * 1024)
#define ROTWIN_SMEM_TARGET (48 * 1024)
struct RotChunks {
  int QC, CC, nq, nc;
  // QC product rows, CC phase rows and the window's degree-p row
  __host__ __device__ size_t smem(int Lh, size_t el2) const { return el2 * (size_t)(QC + CC + 1) * (2 * Lh - 1); }
};
__host__ __device__ inline RotChunks rot_chunks(int Lh, int Ng, size_t el2) {
  const int K = 2 * Lh - 1;
  RotChunks r;
  const long long rows = (long long)ROTWIN_SMEM_TARGET / ((long long)K * (long long)el2) - 1;   // QC + CC that fit
  if ((long long)K + Ng <= rows) {
    r.QC = K;
    r.CC = Ng;
  } else {
    r.CC = Ng < 32 ? Ng : 32;
    if (r.CC > rows - 1) r.CC = (int)(rows > 2 ? rows / 2 : 1);
    long long qc = rows - r.CC;
    r.QC = (int)(qc < 1 ? 1 : (qc > K ? K : qc));
  }
  r.nq = (K + r.QC - 1) / r.QC;
  r.nc = (Ng + r.CC - 1) / r.CC;
  return r;
}

// Beta rows a rotated-window block serves (the gamma phases and the
// window's degree-p row are staged once for all of them).
#define ROTWIN_NB 4

// One (beta rows b0 .. b0 + nb - 1, degree p, chunk z) block: the gamma
// phases of its columns and the window's degree-p row are staged in shared
// memory once; then for each beta row the products h_p^{q'} d^p_{q,q'}(beta_b)
// of its q rows are staged and each output (q, c) is a (2p+1)-term dot
// product read from shared memory (2 x 2 output blocks per thread: two
// product rows and two phase rows per step for four multiply-adds).  dblk0 =
// the degree-p block of d(beta_b0), consecutive rows dstride apart;
// eg[c * (2Lh-1) + q' + Lh - 1] = (cos, sin)(q' gamma_c).  All threads of the
// block take part; a chunk wholly beyond degree p returns at once (the same
// for the whole block).  store(index, re, im) receives each output with its
// h_index position.
template <typename T, typename Store>
__device__ __forceinline__ void rotwin_block_smem_to(const double2* __restrict__ h, const T* __restrict__ dblk0,
                                                     size_t dstride, int nb, const typename vec2<T>::t* __restrict__ eg,
                                                     int Lh, int Ng, int b0, int p, const RotChunks& ch, int z,
                                                     Store store, unsigned char* smem) {
  typedef typename vec2<T>::t T2;
  const int K = 2 * Lh - 1, n2 = Lh * Lh, w = 2 * p + 1;
  const int q0 = (z / ch.nc) * ch.QC, c0 = (z % ch.nc) * ch.CC;
  if (q0 >= w) return;
  const int nqr = min(ch.QC, w - q0), ncr = min(ch.CC, Ng - c0);
  T2* hd = reinterpret_cast<T2*>(smem);       // [q + p - q0][q' + p]
  T2* ep = hd + (size_t)nqr * w;              // [c - c0][q' + p]
  T2* hr = ep + (size_t)ncr * w;              // [q' + p]: h_p^{q'} in T
  // the window's degree-p row, converted once (a float/double conversion runs
  // on the FP64 pipe), and the gamma phases of the chunk's columns
  for (int t = threadIdx.x; t < w; t += blockDim.x) {
    const double2 hv = __ldg(h + p * p + t);
    hr[t] = mk2((T)hv.x, (T)hv.y);
  }
#pragma unroll 4
  for (int t = threadIdx.x; t < ncr * w; t += blockDim.x) {
    const int c = t / w, qp = t - c * w;
    ep[t] = eg[(size_t)(c0 + c) * K + (Lh - 1) - p + qp];
  }
  const int nqh = (nqr + 1) / 2, nch = (ncr + 1) / 2;
  for (int bi = 0; bi < nb; ++bi) {
    const int b = b0 + bi;
    const T* dblk = dblk0 + (size_t)bi * dstride;
    __syncthreads();                          // hr / ep ready; the previous row's products read
#pragma unroll 4
    for (int t = threadIdx.x; t < nqr * w; t += blockDim.x) {
      const int qp = t % w;
      const T2 hv = hr[qp];
      const T d = __ldg(dblk + (size_t)q0 * w + t);
      hd[t] = mk2(d * hv.x, d * hv.y);
    }
    __syncthreads();
    // each thread: rows qa, qa + nqh and columns ca, ca + nch of the chunk
    for (int t = threadIdx.x; t < nqh * nch; t += blockDim.x) {
      const int qa = t / nch, ca = t % nch, qb = qa + nqh, cb = ca + nch;
      const bool has_q = qb < nqr, has_c = cb < ncr;
      const T2* ha = hd + qa * w;
      const T2* hb = hd + (has_q ? qb : qa) * w;
      const T2* ea = ep + ca * w;
      const T2* eb = ep + (has_c ? cb : ca) * w;
      T r00 = 0, i00 = 0, r01 = 0, i01 = 0, r10 = 0, i10 = 0, r11 = 0, i11 = 0;
      for (int u = 0; u < w; ++u) {              // h d (cos - i sin)
        const T2 a = ha[u], b2 = hb[u], E = ea[u], F = eb[u];
        r00 = fma(a.x, E.x, r00); r00 = fma(a.y, E.y, r00); i00 = fma(a.y, E.x, i00); i00 = fma(-a.x, E.y, i00);
        r01 = fma(a.x, F.x, r01); r01 = fma(a.y, F.y, r01); i01 = fma(a.y, F.x, i01); i01 = fma(-a.x, F.y, i01);
        r10 = fma(b2.x, E.x, r10); r10 = fma(b2.y, E.y, r10); i10 = fma(b2.y, E.x, i10); i10 = fma(-b2.x, E.y, i10);
        r11 = fma(b2.x, F.x, r11); r11 = fma(b2.y, F.y, r11); i11 = fma(b2.y, F.x, i11); i11 = fma(-b2.x, F.y, i11);
      }
      const int ja = b * Ng + c0 + ca, jb = b * Ng + c0 + cb;
      store(h_index(p * p + q0 + qa, ja, n2), r00, i00);
      if (has_c) store(h_index(p * p + q0 + qa, jb, n2), r01, i01);
      if (has_q) store(h_index(p * p + q0 + qb, ja, n2), r10, i10);
      if (has_q && has_c) store(h_index(p * p + q0 + qb, jb, n2), r11, i11);
    }
  }
}

template <typename T>
struct RotwinStore {
  typename vec2<T>::t* H;
  __device__ __forceinline__ void operator()(size_t i, T re, T im) const { H[i] = mk2(re, im); }
};
