// FP32_BULK alpha stage on tcgen05 for wide windows, 16 < L_h <= 64: the
// contraction g[a][j] = sum_{|q| < L_h} X_q[j] e^{-i q alpha_a} with the
// orders +-q paired, as in the CUDA-core direct form:
//   g = X_0 + sum_{r >= 1} ( P_r cos(r alpha) - i M_r sin(r alpha) ),
//   P_r = X_r + X_-r, M_r = X_r - X_-r   (P_0 = X_0, M_0 = 0), so
//   Re g = sum_r ( Re P_r cos(r alpha) + Im M_r sin(r alpha) ),
//   Im g = sum_r ( Im P_r cos(r alpha) - Re M_r sin(r alpha) ).
// Both are real GEMMs against the SAME operand B[n][k] = (cos | sin)(r alpha_n):
//   D_re[j][n] = sum_k A_re[j][k] B[n][k],  D_im[j][n] = sum_k A_im[j][k] B[n][k],
// M = 128 columns j, N = 128 alpha rows, K = 64 NKF (NKF = 1 for L_h <= 32,
// 2 for L_h <= 64), with KP = K / 2 and the slot map
//   A_re[j][r] = Re P_r, A_re[j][KP + r] = Im M_r,
//   A_im[j][r] = Im P_r, A_im[j][KP + r] = -Re M_r,
//   B[n][r] = cos(r alpha_n), B[n][KP + r] = sin(r alpha_n)   (r < L_h; M slot 0 and all else zero).
// Per output sample that is 2K real products against 4 (2 L_h - 1) for the
// unpaired form, and the streamed operand B serves both GEMMs.  As in the
// narrow engine both operands are split into FP16 hi + lo (A after a
// per-column power-of-two scale that puts its largest entry in [2^14, 2^15))
// and D = A_hi B_hi + A_hi B_lo + A_lo B_hi accumulates in FP32.
//
// Two kernels: k_xaw_from_h (CUDA cores) forms X for one 128-column tile of
// a group of pairs from the rotated window H, folds it into P and M, scales,
// splits and writes the swizzled A operand (A_re and A_im, NKF K-chunks of
// 32 KB each) and the column scales to a blob in global memory; k_alpha_tcw
// (persistent, one CTA per SM, work item = (pair, tile)) keeps the item's
// whole A operand in shared memory, streams the E-table K-chunks (32 KB each)
// through a ring of 3 or 4 stages with cp.async.bulk, issues the MMAs from
// one thread into two TMEM accumulators (each 2 x 128 columns: D_re, D_im),
// and eight epilogue warps drain them and store g.  Every mbarrier wait is
// bounded; on expiry the CTA raises its abort flag, waits (bounded) for its
// copies and MMAs in flight, frees TMEM and exits, and the host reads the
// shared error word.
#include <cuda_fp16.h>

#include "common.cuh"
#include "tc.cuh"
#include "tc_ptx.cuh"

#define XW_COLS 16                      // columns per producer block
#define XW_PARTS (TC_M / XW_COLS)
#define XW_PP 4                         // pairs per producer block
#define XW_THREADS 256
#define TCW_NA 128                      // alpha rows per chunk (MMA N)

// A-operand K-chunks per tile: 2 NKF (A_re then A_im, NKF chunks of 64 each)
static inline int tcw_nk(int Lh) { return Lh <= 32 ? 2 : 4; }
static inline int tcw_tiles(int Nb, int Ng) { return (Nb * Ng + TC_M - 1) / TC_M; }
static inline int tcw_chunks(int Na) { return (Na + TCW_NA - 1) / TCW_NA; }

bool tcw_supported(int Lh, int Na) { return Lh > 16 && Lh <= 64 && Na >= 1; }

size_t tcw_etab_bytes(int Na, int Lh) { return (size_t)tcw_chunks(Na) * (tcw_nk(Lh) / 2) * TC_B_BYTES; }

// per pair: tiles x 2 NKF x 32 KB of A, one float scale per padded column,
// then room for the coupling rows of a producer group as floats, interleaved
// [pq][XW_PP] (the producer's operand; used in the group's first pair)
static inline size_t tcw_scales_bytes(size_t tiles) { return ((tiles * TC_M * sizeof(float)) + 1023) / 1024 * 1024; }
size_t tcw_xblob_bytes(int Nb, int Ng, int Lh) {
  const size_t t = (size_t)tcw_tiles(Nb, Ng);
  const size_t kf = ((size_t)Lh * Lh * XW_PP * sizeof(float2) + 1023) / 1024 * 1024;
  return t * (size_t)tcw_nk(Lh) * TC_A_BYTES + tcw_scales_bytes(t) + kf;
}

// The coupling rows of the launch's pairs as floats: one conversion per
// coefficient (float/double conversions share the slow FP64 pipe on this
// GPU; the producer then reads floats), pair i at [pq][i % XW_PP] of its
// group's first blob; the slots of a short last group are zero.
__global__ void k_kf_from_kc(const double2* __restrict__ kc, int n2, int npairs, unsigned char* __restrict__ xblob,
                             size_t blob_stride, size_t kf_off) {
  const int pair = blockIdx.y, g0 = pair - pair % XW_PP;
  float2* kf = reinterpret_cast<float2*>(xblob + (size_t)g0 * blob_stride + kf_off);
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n2; t += gridDim.x * blockDim.x) {
    float2 o = make_float2(0.f, 0.f);
    if (pair < npairs) {
      const double2 v = kc[(size_t)pair * n2 + t];
      o = make_float2((float)v.x, (float)v.y);
    }
    kf[(size_t)t * XW_PP + pair % XW_PP] = o;
  }
}

// ---------------------------------------------------------------- E tables
// chunk (c, kc) at (c NKF + kc) 32 KB: [hi: 128 rows x 64][lo]; row n ->
// alpha a = 128 c + n, slot k = 64 kc + kl -> cos(k alpha) for k < KP,
// sin((k - KP) alpha) above; zeros beyond Na, for r >= Lh and at M slot 0.
__global__ void k_tcw_etab(unsigned char* __restrict__ etab, int Na, int Lh, int nkf) {
  const int c = blockIdx.x / nkf, kc = blockIdx.x % nkf;
  const int KP = 32 * nkf;
  unsigned char* base = etab + (size_t)blockIdx.x * TC_B_BYTES;
  for (int t = threadIdx.x; t < TCW_NA * TC_KB; t += blockDim.x) {
    const int n = t / TC_KB, kl = t % TC_KB;
    const int slot = kc * TC_KB + kl;
    const bool sin_part = slot >= KP;
    const int r = sin_part ? slot - KP : slot;
    const int a = c * TCW_NA + n;
    double v = 0.0;
    if (a < Na && r < Lh && !(sin_part && r == 0)) {
      double sn, co;
      sincos_2pi_frac((long long)r * a, Na, &sn, &co);
      v = sin_part ? sn : co;
    }
    const __half hi = __double2half(v);
    const __half lo = __double2half(v - (double)__half2float(hi));
    *reinterpret_cast<__half*>(base + sw128_off(n, kl)) = hi;
    *reinterpret_cast<__half*>(base + TC_B_HALF + sw128_off(n, kl)) = lo;
  }
}

cudaError_t launch_tcw_etab(void* etab, int Na, int Lh, cudaStream_t st) {
  if (!tcw_supported(Lh, Na)) return cudaErrorInvalidValue;
  const int nkf = tcw_nk(Lh) / 2;
  k_tcw_etab<<<tcw_chunks(Na) * nkf, 256, 0, st>>>((unsigned char*)etab, Na, Lh, nkf);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- A operand from H
// X_q(j) = sum_{p>=|q|} k(p,q) H^p_q(j) for up to XW_PP pairs and one eighth
// of a 128-column tile: a block serves XW_COLS columns of XW_PP pairs, so every
// H value it loads feeds the multiply-adds of all its pairs (H is read from L2
// once per group of XW_PP pairs); the groups of one tile are adjacent blocks,
// so each H tile is read from HBM about once.
//   phase 1: one item per (q, two adjacent columns), its degrees p >= |q| (H
//            loads coalesced across columns, k broadcast through the cache)
//            into the shared tiles sX[pair][q + Lh - 1][column] (complex);
//   phase 2: per (pair, column), the largest |entry| of A_re and A_im (from
//            P_r and M_r) -> scale 2^e into [2^14, 2^15);
//   phase 3: per (pair, column, operand, 8 slots): P_r / M_r, scale, split
//            into FP16 hi/lo, store swizzled into its K-chunk.  Columns
//            beyond J are zero.

// H values of columns j, j + 1 (the second zero when two is false)
__device__ __forceinline__ float4 xw_ld2(const float2* p, bool two) {
  if (two) return __ldg(reinterpret_cast<const float4*>(p));
  const float2 a = __ldg(p);
  return make_float4(a.x, a.y, 0.f, 0.f);
}
// x_v += k_v h for the four pairs v of a group and two columns: acc[v] =
// (re, im) of both columns, h = (H of column 0, H of column 1)
__device__ __forceinline__ void xw_mac2(float4* acc, float4 k01, float4 k23, float4 h) {
  const float kr[XW_PP] = {k01.x, k01.z, k23.x, k23.z}, ki[XW_PP] = {k01.y, k01.w, k23.y, k23.w};
#pragma unroll
  for (int v = 0; v < XW_PP; ++v) {
    acc[v].x = fmaf(kr[v], h.x, acc[v].x); acc[v].x = fmaf(-ki[v], h.y, acc[v].x);
    acc[v].y = fmaf(kr[v], h.y, acc[v].y); acc[v].y = fmaf(ki[v], h.x, acc[v].y);
    acc[v].z = fmaf(kr[v], h.z, acc[v].z); acc[v].z = fmaf(-ki[v], h.w, acc[v].z);
    acc[v].w = fmaf(kr[v], h.w, acc[v].w); acc[v].w = fmaf(ki[v], h.z, acc[v].w);
  }
}

// slot k of operand m (0: A_re, 1: A_im) of one column from its X row xs
// (xs[(q + Lh - 1) * XW_COLS] = X_q)
__device__ __forceinline__ float xw_slot(const float2* xs, int Lh, int KP, int m, int k) {
  const int r = k < KP ? k : k - KP;
  if (r >= Lh) return 0.f;
  const float2 xp = xs[(size_t)(Lh - 1 + r) * XW_COLS];
  if (k < KP) {                                     // P_r
    if (r == 0) return m == 0 ? xp.x : xp.y;
    const float2 xm = xs[(size_t)(Lh - 1 - r) * XW_COLS];
    return m == 0 ? xp.x + xm.x : xp.y + xm.y;
  }
  if (r == 0) return 0.f;                           // M_0
  const float2 xm = xs[(size_t)(Lh - 1 - r) * XW_COLS];
  return m == 0 ? xp.y - xm.y : -(xp.x - xm.x);    // Im M_r | -Re M_r
}

__global__ void __launch_bounds__(XW_THREADS, 3)
k_xaw_from_h(const float2* __restrict__ H, int Lh, int J, int nkf, unsigned char* __restrict__ xblob,
             size_t blob_stride, int tiles, size_t kf_off, int npairs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int K = 2 * Lh - 1, KF = 64 * nkf, KP = KF / 2;
  float2* sX = reinterpret_cast<float2*>(smem_raw);                     // [XW_PP][K][XW_COLS]
  int* sEx = reinterpret_cast<int*>(sX + (size_t)XW_PP * K * XW_COLS);  // [XW_PP][XW_COLS]
  // pair groups vary fastest: the blocks of one H tile run together and share it in L2
  const int groups = (npairs + XW_PP - 1) / XW_PP;
  const int pb = (int)(blockIdx.x % groups) * XW_PP, part = (int)(blockIdx.x / groups);
  const int tile = part / XW_PARTS, r0 = (part % XW_PARTS) * XW_COLS;
  const int npp = min(XW_PP, npairs - pb);
  const int n2 = Lh * Lh;
  // k(p,q) of the group's pairs: two 16-byte loads per pq
  const float4* kp = reinterpret_cast<const float4*>(xblob + (size_t)pb * blob_stride + kf_off);
  const int jt = tile * TC_M + r0;
  // items (q, column pair): one 16-byte H load serves two adjacent columns
  for (int it = threadIdx.x; it < K * (XW_COLS / 2); it += XW_THREADS) {
    const int u = it / (XW_COLS / 2), r = 2 * (it % (XW_COLS / 2));
    const int q = u - (Lh - 1), aq = q < 0 ? -q : q;
    const int j = jt + r;
    float4 acc[XW_PP];                              // (re, im) of columns r and r + 1
#pragma unroll
    for (int v = 0; v < XW_PP; ++v) acc[v] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (j < J) {
      // j is even, so (j, j + 1) share a 128-column tile and a 16-byte H word
      const float2* hp = H + h_index(0, j, n2);      // row pq at hp + pq * 128
      const bool two = j + 1 < J;
      int p = aq;
      for (; p + 3 < Lh; p += 4) {                  // four degrees' loads in flight per step
        float4 hv[4];
#pragma unroll
        for (int w = 0; w < 4; ++w) hv[w] = xw_ld2(hp + (size_t)((p + w) * (p + w) + (p + w) + q) * 128, two);
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          const int pq = (p + w) * (p + w) + (p + w) + q;
          xw_mac2(acc, __ldg(kp + 2 * pq), __ldg(kp + 2 * pq + 1), hv[w]);
        }
      }
      for (; p < Lh; ++p) {
        const int pq = p * p + p + q;
        xw_mac2(acc, __ldg(kp + 2 * pq), __ldg(kp + 2 * pq + 1), xw_ld2(hp + (size_t)pq * 128, two));
      }
    }
#pragma unroll
    for (int v = 0; v < XW_PP; ++v) *reinterpret_cast<float4*>(sX + ((size_t)v * K + u) * XW_COLS + r) = acc[v];
  }
  __syncthreads();
  {   // four threads per (pair, column), then a shuffle across the four
    const int col = threadIdx.x / 4, sub = threadIdx.x % 4;      // col < XW_PP * XW_COLS = 64
    const float2* xs = sX + (size_t)(col / XW_COLS) * K * XW_COLS + (col % XW_COLS);
    float mx = 0.f;
    for (int k = sub; k < KF; k += 4)
      mx = fmaxf(mx, fmaxf(fabsf(xw_slot(xs, Lh, KP, 0, k)), fabsf(xw_slot(xs, Lh, KP, 1, k))));
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
    if (sub == 0) {
      int ex = 0;
      if (mx > 0.f) frexpf(mx, &ex);
      sEx[col] = mx > 0.f ? min(125, max(-125, 15 - ex)) : 0;
    }
  }
  __syncthreads();
  // items (pair v, operand m, 8-slot chunk k0, column r), column fastest
  for (int it = threadIdx.x; it < npp * 2 * (KF / 8) * XW_COLS; it += XW_THREADS) {
    const int r = it % XW_COLS, k0 = ((it / XW_COLS) % (KF / 8)) * 8;
    const int m = (it / (XW_COLS * (KF / 8))) % 2, v = it / (XW_COLS * (KF / 8) * 2);
    const int e = sEx[v * XW_COLS + r];
    const float sc = __int_as_float((127 + e) << 23);
    const float2* xs = sX + (size_t)v * K * XW_COLS + r;
    __align__(16) __half hi[8], lo[8];
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      const float x = xw_slot(xs, Lh, KP, m, k0 + w) * sc;
      hi[w] = __float2half_rn(x);
      lo[w] = __float2half_rn(x - __half2float(hi[w]));
    }
    unsigned char* blob = xblob + (size_t)(pb + v) * blob_stride;
    unsigned char* cb = blob + ((size_t)tile * 2 * nkf + m * nkf + k0 / TC_KB) * TC_A_BYTES;
    *reinterpret_cast<uint4*>(cb + sw128_off(r0 + r, k0 % TC_KB)) = *reinterpret_cast<uint4*>(hi);
    *reinterpret_cast<uint4*>(cb + TC_A_HALF + sw128_off(r0 + r, k0 % TC_KB)) = *reinterpret_cast<uint4*>(lo);
    if (k0 == 0 && m == 0) {
      float* scales = reinterpret_cast<float*>(blob + (size_t)tiles * 2 * nkf * TC_A_BYTES);
      scales[jt + r] = jt + r < J ? __int_as_float((127 - e) << 23) : 0.f;
    }
  }
}

static size_t xaw_smem(int Lh) {
  return sizeof(float2) * (size_t)XW_PP * (2 * Lh - 1) * XW_COLS + sizeof(int) * XW_PP * XW_COLS;
}

cudaError_t launch_xaw_from_h(const double2* kc, const float2* H, int Lh, int Nb, int Ng, int npairs, void* xblob,
                              cudaStream_t st) {
  if (npairs <= 0) return cudaSuccess;
  if (Lh <= 16 || Lh > 64) return cudaErrorInvalidValue;
  const int nkf = tcw_nk(Lh) / 2, tiles = tcw_tiles(Nb, Ng);
  const long long blocks = (long long)((npairs + XW_PP - 1) / XW_PP) * XW_PARTS * tiles;
  static_assert(XW_PP == 4, "xw_mac2 takes the coupling rows of four pairs");
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  // the ceiling of the largest case (L_h = 64), set once (never inside a stream capture)
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_xaw_from_h, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xaw_smem(64));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const size_t stride = tcw_xblob_bytes(Nb, Ng, Lh);
  const size_t kf_off = (size_t)tiles * 2 * nkf * TC_A_BYTES + tcw_scales_bytes(tiles);
  const int groups = (npairs + XW_PP - 1) / XW_PP;
  k_kf_from_kc<<<dim3((Lh * Lh + 255) / 256, groups * XW_PP), 256, 0, st>>>(kc, Lh * Lh, npairs,
                                                                           (unsigned char*)xblob, stride, kf_off);
  k_xaw_from_h<<<(unsigned)blocks, XW_THREADS, xaw_smem(Lh), st>>>(H, Lh, Nb * Ng, nkf, (unsigned char*)xblob,
                                                                   stride, tiles, kf_off, npairs);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- the kernel
#define TCW_MAX_BS 4
#define TCW_ACC 2                       // TMEM accumulators (2 x (D_re, D_im) x 128 columns: all 512)
struct TcwBars {
  uint64_t a_full, a_empty, b_full[TCW_MAX_BS], b_empty[TCW_MAX_BS], acc_full[TCW_ACC], acc_empty[TCW_ACC], drain;
  uint32_t tmem_base;
  int abort_flag;
};

// E-table ring depth: what fits beside the A operand (3 stages at NKF = 2, 4 at NKF = 1).
#define TCW_BS(NKF) ((NKF) == 2 ? 3 : 4)
#define TCW_SMEM(NKF) (2 * (NKF) * TC_A_BYTES + TCW_BS(NKF) * TC_B_BYTES + 1024 + 256)

template <int NKF>
__global__ void __launch_bounds__(TC_THREADS, 1)
k_alpha_tcw(const unsigned char* __restrict__ xblob, size_t blob_stride, int tiles,
            const unsigned char* __restrict__ etab, int Na, int J, int npairs, float2* __restrict__ g,
            int* __restrict__ err, const int2* __restrict__ slots, int wait_test) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  constexpr int BS = TCW_BS(NKF), NK = 2 * NKF;
  unsigned char* sA = sm;                               // NK x 32 KB: the item's A operand (A_re, A_im)
  unsigned char* sB = sm + NK * TC_A_BYTES;             // BS x 32 KB: ring of E-table K-chunks
  TcwBars* bars = reinterpret_cast<TcwBars*>(sB + BS * TC_B_BYTES);
  volatile int* abort_flag = &bars->abort_flag;
  const uint32_t wlim = wait_test ? (1u << 14) : TC_WAIT_LIMIT;   // short limit for the timeout test
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nch = (Na + TCW_NA - 1) / TCW_NA;
  const long long nitems = (long long)npairs * tiles;

  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bars->a_full), 1);
    mbar_init(smem_u32(&bars->a_empty), 1);
    for (int i = 0; i < BS; ++i) {
      mbar_init(smem_u32(&bars->b_full[i]), 1);
      mbar_init(smem_u32(&bars->b_empty[i]), 1);
    }
    for (int i = 0; i < TCW_ACC; ++i) {
      mbar_init(smem_u32(&bars->acc_full[i]), 1);
      mbar_init(smem_u32(&bars->acc_empty[i]), 32 * TC_EPI_WARPS);
    }
    mbar_init(smem_u32(&bars->drain), 1);
    bars->abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {   // TMEM: TCW_ACC accumulators of 128 x TC_N FP32
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                     smem_u32(&bars->tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = bars->tmem_base;

  if (warp == 0) {
    // ---------------- loader: the item's A operand, then its E K-chunks in order
    if (lane == 0) {
      int a_armed = -1, b_armed[BS];
#pragma unroll
      for (int i = 0; i < BS; ++i) b_armed[i] = -1;
      long long bc = 0;
      int li = 0;
      bool ok = true;
      for (long long it = blockIdx.x; it < nitems && ok; it += gridDim.x, ++li) {
        const int pair = (int)(it / tiles), tile = (int)(it % tiles);
        const uint32_t pa = (uint32_t)(li & 1);
        if (!(ok = mbar_wait_n(smem_u32(&bars->a_empty), pa ^ 1u, abort_flag, wlim))) break;
        if (!(wait_test && li == 0)) {   // wait_test: the first A operand is never fetched
          const uint32_t fa = smem_u32(&bars->a_full);
          mbar_expect_tx(fa, NK * TC_A_BYTES);
          const unsigned char* src = xblob + (size_t)pair * blob_stride + (size_t)tile * NK * TC_A_BYTES;
          for (int o = 0; o < NK * TC_A_BYTES; o += 16384) bulk_g2s(smem_u32(sA + o), src + o, 16384, fa);
          a_armed = (int)pa;
        }
        for (int c = 0; c < nch && ok; ++c) {
          for (int kc = 0; kc < NKF; ++kc, ++bc) {
            const int sb = (int)(bc % BS);
            const uint32_t pb = (uint32_t)((bc / BS) & 1);
            if (!(ok = mbar_wait_n(smem_u32(&bars->b_empty[sb]), pb ^ 1u, abort_flag, wlim))) break;
            const uint32_t fb = smem_u32(&bars->b_full[sb]);
            mbar_expect_tx(fb, TC_B_BYTES);
            const unsigned char* bsrc = etab + ((size_t)c * NKF + kc) * TC_B_BYTES;
            for (int o = 0; o < TC_B_BYTES; o += 16384)
              bulk_g2s(smem_u32(sB + sb * TC_B_BYTES + o), bsrc + o, 16384, fb);
#pragma unroll
            for (int i = 0; i < BS; ++i)
              if (i == sb) b_armed[i] = (int)pb;
          }
        }
      }
      if (!ok) *abort_flag = 1;
      // copies in flight must land before the CTA may exit
      if (a_armed >= 0) {
        uint32_t n = 0;
        while (!mbar_test(smem_u32(&bars->a_full), (uint32_t)a_armed) && ++n < TC_WAIT_LIMIT) {}
      }
#pragma unroll
      for (int i = 0; i < BS; ++i) {
        if (b_armed[i] >= 0) {
          uint32_t n = 0;
          while (!mbar_test(smem_u32(&bars->b_full[i]), (uint32_t)b_armed[i]) && ++n < TC_WAIT_LIMIT) {}
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer
    if (lane == 0) {
      const uint32_t idesc = umma_idesc_f16(TC_M, TC_N);
      long long bc = 0, ac = 0;
      int li = 0;
      bool ok = true;
      for (long long it = blockIdx.x; it < nitems && ok; it += gridDim.x, ++li) {
        if (!(ok = mbar_wait_n(smem_u32(&bars->a_full), (uint32_t)(li & 1), abort_flag, wlim))) break;
        for (int c = 0; c < nch && ok; ++c, ++ac) {
          const int acc = (int)(ac % TCW_ACC);
          if (!(ok = mbar_wait_n(smem_u32(&bars->acc_empty[acc]), (uint32_t)(((ac / TCW_ACC) & 1) ^ 1),
                                 abort_flag, wlim)))
            break;
          const uint32_t d = tmem + (uint32_t)(acc * 2 * TC_N);     // D_re, then D_im 128 columns on
          for (int kc = 0; kc < NKF; ++kc, ++bc) {
            const int sb = (int)(bc % BS);
            if (!(ok = mbar_wait_n(smem_u32(&bars->b_full[sb]), (uint32_t)((bc / BS) & 1), abort_flag, wlim))) break;
            tc_fence_after();
            const uint32_t b_hi = smem_u32(sB + sb * TC_B_BYTES), b_lo = b_hi + TC_B_HALF;
#pragma unroll
            for (int m = 0; m < 2; ++m) {                // the E chunk serves A_re and A_im
              const uint32_t a_hi = smem_u32(sA + (m * NKF + kc) * TC_A_BYTES), a_lo = a_hi + TC_A_HALF;
              const uint32_t as[3] = {a_hi, a_hi, a_lo};
              const uint32_t bs[3] = {b_hi, b_lo, b_hi};
#pragma unroll
              for (int pr = 0; pr < 3; ++pr) {
                const uint64_t ad = sw128_desc(as[pr]), bd = sw128_desc(bs[pr]);
#pragma unroll
                for (int s = 0; s < TC_KB / 16; ++s)     // K = 16 per MMA: +32 bytes
                  umma_f16(d + (uint32_t)(m * TC_N), ad + (uint64_t)(2 * s), bd + (uint64_t)(2 * s), idesc,
                           (kc | pr | s) != 0);
              }
            }
            umma_commit(smem_u32(&bars->b_empty[sb]));
          }
          if (!ok) break;
          umma_commit(smem_u32(&bars->acc_full[acc]));
        }
        if (!ok) break;
        umma_commit(smem_u32(&bars->a_empty));
      }
      if (!ok) *abort_flag = 1;
      // every MMA issued by this thread completes before TMEM is released
      umma_commit(smem_u32(&bars->drain));
      uint32_t n = 0;
      while (!mbar_test(smem_u32(&bars->drain), 0u) && ++n < TC_WAIT_LIMIT) {}
    }
  } else {
    // ---------------- epilogue: warps 2..9; TMEM lane quadrant = warp % 4,
    // half = which 64 of the chunk's 128 alpha rows (two passes of 32)
    const int quad = warp & 3;
    const int half = (warp - 2) >> 2;
    const int row = quad * 32 + lane;
    long long ac = 0;
    bool ok = true;
    for (long long it = blockIdx.x; it < nitems && ok; it += gridDim.x) {
      const int pair = (int)(it / tiles), tile = (int)(it % tiles);
      const int j = tile * TC_M + row;
      const bool jin = j < J;
      const float* scales = reinterpret_cast<const float*>(xblob + (size_t)pair * blob_stride +
                                                           (size_t)tiles * NK * TC_A_BYTES);
      const float sc = jin ? scales[j] : 0.f;
      const int2 sl = slots != nullptr ? slots[pair] : make_int2(pair, -1);
      float2* gp = g + (size_t)sl.x * Na * J + (jin ? j : 0);
      float2* gm = sl.y >= 0 ? g + (size_t)(sl.y >> 1) * Na * J + (jin ? j : 0) : nullptr;
      const float msc = (sl.y & 1) ? -sc : sc;
      for (int c = 0; c < nch; ++c, ++ac) {
        const int acc = (int)(ac % TCW_ACC);
        // one lane waits, the warp follows: tcgen05.ld needs a converged warp
        int got = 0;
        if (lane == 0)
          got = mbar_wait_n(smem_u32(&bars->acc_full[acc]), (uint32_t)((ac / TCW_ACC) & 1), abort_flag, wlim);
        got = __shfl_sync(0xffffffffu, got, 0);
        __syncwarp();
        if (!(ok = got != 0)) break;
        tc_fence_after();
        const uint32_t tbase = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(acc * 2 * TC_N);
#pragma unroll 1
        for (int ps = 0; ps < 2; ++ps) {
          const int cb = half * (TCW_NA / 2) + ps * 32;
          uint32_t vr[32], vi[32];
          TMEM_LD32(tbase + (uint32_t)cb, vr);
          TMEM_LD32(tbase + (uint32_t)(TC_N + cb), vi);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          const int a0 = c * TCW_NA + cb;
          if (jin) {
            float2* p = gp + (size_t)a0 * J;
            if (a0 + 32 <= Na) {
#pragma unroll
              for (int u = 0; u < 32; ++u) {
                __stcs(p, make_float2(__uint_as_float(vr[u]) * sc, __uint_as_float(vi[u]) * sc));
                p += J;
              }
            } else {
#pragma unroll
              for (int u = 0; u < 32; ++u) {
                if (a0 + u < Na) __stcs(p, make_float2(__uint_as_float(vr[u]) * sc, __uint_as_float(vi[u]) * sc));
                p += J;
              }
            }
          }
          if (jin && gm != nullptr) {     // (l, -m): (-1)^m conj g (real f and h)
            float2* p = gm + (size_t)a0 * J;
#pragma unroll
            for (int u = 0; u < 32; ++u) {
              if (a0 + u < Na)
                __stcs(p, make_float2(__uint_as_float(vr[u]) * msc, -__uint_as_float(vi[u]) * msc));
              p += J;
            }
          }
        }
        tc_fence_before();
        mbar_arrive(smem_u32(&bars->acc_empty[acc]));
      }
    }
    if (!ok) *abort_flag = 1;
  }
  __syncthreads();
  if (*abort_flag && threadIdx.x == 0) atomicExch(err, 1);
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
  }
}

template <int NKF>
static cudaError_t launch_tcw_t(const void* xblob, const void* etab, int Lh, int Na, int Nb, int Ng, int npairs,
                                float2* g, int num_sms, const int2* slots, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e =
        cudaFuncSetAttribute(k_alpha_tcw<NKF>, cudaFuncAttributeMaxDynamicSharedMemorySize, TCW_SMEM(NKF));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  int* err = tc_error_word();
  if (!err) return cudaErrorMemoryAllocation;
  const int tiles = tcw_tiles(Nb, Ng);
  const long long items = (long long)npairs * tiles;
  const int grid = (int)(items < num_sms ? items : num_sms);
  k_alpha_tcw<NKF><<<grid, TC_THREADS, TCW_SMEM(NKF), st>>>((const unsigned char*)xblob, tcw_xblob_bytes(Nb, Ng, Lh),
                                                          tiles, (const unsigned char*)etab, Na, Nb * Ng, npairs, g,
                                                          err, slots, tc_take_wait_test());
  return cudaGetLastError();
}

cudaError_t launch_alpha_tcw(const void* xblob, const void* etab, int Lh, int Na, int Nb, int Ng, int npairs,
                             float2* g, int num_sms, const int2* slots, cudaStream_t st) {
  if (npairs <= 0) return cudaSuccess;
  if (!tcw_supported(Lh, Na)) return cudaErrorInvalidValue;
  if (tcw_nk(Lh) == 2) return launch_tcw_t<1>(xblob, etab, Lh, Na, Nb, Ng, npairs, g, num_sms, slots, st);
  return launch_tcw_t<2>(xblob, etab, Lh, Na, Nb, Ng, npairs, g, num_sms, slots, st);
}
