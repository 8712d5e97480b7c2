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
// The producer (two passes: k_xw_tc on the tensor cores, or k_xw_x on the
// CUDA cores for small grids, forms X in FP32 for a group of up to 16 pairs
// from the rotated window H; k_xaw_split folds X into P and M, scales each
// column by its largest slot, splits and writes the swizzled A operand --
// A_re and A_im, NKF K-chunks of 32 KB each -- and the column scales to a
// blob in global memory); k_alpha_tcw
// (persistent, one CTA per SM, work item = (pair, tile)) keeps the item's
// whole A operand in shared memory, streams the E-table K-chunks (32 KB each)
// through a ring of 3 or 4 stages with cp.async.bulk, issues the MMAs from
// one thread into two TMEM accumulators (each 2 x 128 columns: D_re, D_im),
// and eight epilogue warps drain them and store g.  Every mbarrier wait is
// bounded; on expiry the CTA raises its abort flag, waits (bounded) for its
// copies and MMAs in flight, frees TMEM and exits, and the host reads the
// shared error word.
#include <cuda_fp16.h>

#include <algorithm>

#include "common.cuh"
#include "tc.cuh"
#include "tc_ptx.cuh"

#define TCW_NA 128                      // alpha rows per chunk (MMA N)

// A-operand K-chunks per tile: 2 NKF (A_re then A_im, NKF chunks of 64 each)
static inline int tcw_nk(int Lh) { return Lh <= 32 ? 2 : 4; }
static inline int tcw_tiles(int Nb, int Ng) { return (Nb * Ng + TC_M - 1) / TC_M; }
static inline int tcw_chunks(int Na) { return (Na + TCW_NA - 1) / TCW_NA; }

bool tcw_supported(int Lh, int Na) { return Lh > 16 && Lh <= 64 && Na >= 1; }

size_t tcw_etab_bytes(int Na, int Lh) { return (size_t)tcw_chunks(Na) * (tcw_nk(Lh) / 2) * TC_B_BYTES; }

// per pair: tiles x 2 NKF x 32 KB of A, one float scale per padded column,
// room for the coupling rows of a producer group of up to XA_MAXP pairs as
// floats, interleaved [pq][XA_MAXP] (used in the group's first pair), the
// group's coupling operand of the first pass (likewise), and the pair's
// X_q(j) in FP32, [tile][q + L_h - 1][128 columns] (the producer's first pass
// writes it, its second pass scales and splits it into A)
#define XA_MAXP 16
// The first pass's coupling operand (k_xwb, in the group's first blob): per
// order u = q + L_h - 1 and chunk c of XT_DEG degrees one XT_BIMG image, then
// one float per (u, c) undoing its scale.
#define XT_DEG 32                       // degrees per K chunk of the first pass
#define XT_MAXCH 2                      // chunks per order (L_h <= 64)
#define XT_BATOM (64 * 128)             // one 64-row K atom (64 FP16, 128-byte swizzle) of a coupling image
#define XT_BIMG (2 * XT_BATOM)          // coupling image of a chunk: 64 rows x K = 128 (16 KB)
static inline size_t tcw_scales_bytes(size_t tiles) { return ((tiles * TC_M * sizeof(float)) + 1023) / 1024 * 1024; }
static inline size_t tcw_kf_bytes(int Lh) { return ((size_t)Lh * Lh * XA_MAXP * sizeof(float2) + 1023) / 1024 * 1024; }
static inline size_t tcw_kb_bytes(int Lh) {
  const size_t n = (size_t)(2 * Lh - 1) * XT_MAXCH;
  return n * XT_BIMG + (n * sizeof(float) + 1023) / 1024 * 1024;
}
static inline size_t tcw_xf_bytes(size_t tiles, int Lh) { return tiles * (size_t)(2 * Lh - 1) * TC_M * sizeof(float2); }
// The first pass runs on the tensor cores (k_xw_tc, persistent) when the
// grid gives its CTAs at least 32 (tile, order) items each on 152 SMs;
// below that the pipeline's start-up outweighs its rate and the CUDA-core
// first pass (k_xw_x, one block per item) is faster.  Only then does a blob
// hold the coupling images.
#define XT_MIN_ITEMS (32 * 152)
static inline bool xt_use_tc(long long tiles, int Lh) { return tiles * (2 * Lh - 1) >= XT_MIN_ITEMS; }
size_t tcw_xblob_bytes(int Nb, int Ng, int Lh) {
  const size_t t = (size_t)tcw_tiles(Nb, Ng);
  return t * (size_t)tcw_nk(Lh) * TC_A_BYTES + tcw_scales_bytes(t) + tcw_kf_bytes(Lh) +
         (xt_use_tc((long long)t, Lh) ? tcw_kb_bytes(Lh) : 0) + tcw_xf_bytes(t, Lh);
}

// The coupling rows of a group of up to XA_MAXP pairs as floats: one
// conversion per coefficient (float/double conversions share the slow FP64
// pipe on this GPU; the producer then reads floats), pair v of the group at
// [pq][v]; the slots past the group's last pair are zero.
__global__ void k_kf_from_kc(const double2* __restrict__ kc, int n2, int npairs, unsigned char* __restrict__ xblob,
                             size_t blob_stride, size_t kf_off) {
  // group blockIdx.y: pairs g0 .. g0 + ng - 1, its table in the group's first blob
  const int g0 = blockIdx.y * XA_MAXP, ng = min(XA_MAXP, npairs - g0);
  kc += (size_t)g0 * n2;
  float2* kf = reinterpret_cast<float2*>(xblob + (size_t)g0 * blob_stride + kf_off);
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n2 * XA_MAXP; t += gridDim.x * blockDim.x) {
    const int pq = t / XA_MAXP, v = t % XA_MAXP;
    float2 o = make_float2(0.f, 0.f);
    if (v < ng) {
      const double2 x = kc[(size_t)v * n2 + pq];
      o = make_float2((float)x.x, (float)x.y);
    }
    kf[t] = o;
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
// Two passes.  The first: X_q(j) = sum_{p>=|q|} k(p,q) H^p_q(j) for a group
// of up to XA_MAXP pairs, per (128-column tile, order q), into the pair's
// FP32 region, by k_xw_tc (below) on large grids and by k_xw_x on small ones.  k_xaw_split: one thread per (pair, column, 8 orders
// r): P_r = X_r + X_-r, M_r = X_r - X_-r (P_0 = X_0, M_0 = 0), the column's
// largest slot (a shuffle over the lanes of the column) sets its scale 2^e
// into [2^14, 2^15), every slot scaled, split into FP16 hi/lo and stored
// swizzled into its K-chunk (A_re[r] = Re P_r, A_re[KP + r] = Im M_r,
// A_im[r] = Im P_r, A_im[KP + r] = -Re M_r; zero for r >= L_h), and 2^-e goes
// to the pair's scale array.  Columns beyond J are zero.

// k_xw_x: one block per (128-column tile, order q), one thread per column;
// the thread keeps its column's sums for every pair of the group in
// registers, so each H value (one coalesced row per degree; the order's rows
// are one run of the order-major tile) feeds 4 NP multiply-adds, with the
// group's k(., q) in shared memory (broadcast reads) and the next four
// degrees' H loads issued before the current four are used.
template <int NP>
__device__ __forceinline__ void xw_mac(const float2 (*sk)[NP], int i, float2 h, float* ar, float* ai) {
#pragma unroll
  for (int v = 0; v < NP; ++v) {
    const float2 kv = sk[i][v];
    ar[v] = fmaf(kv.x, h.x, ar[v]); ar[v] = fmaf(-kv.y, h.y, ar[v]);
    ai[v] = fmaf(kv.x, h.y, ai[v]); ai[v] = fmaf(kv.y, h.x, ai[v]);
  }
}

template <int NP>
__global__ void __launch_bounds__(TC_M) k_xw_x(const float2* __restrict__ H, int Lh, int J, int npairs,
                                               unsigned char* __restrict__ xblob, size_t blob_stride, size_t kf_off,
                                               size_t xf_off) {
  __shared__ float2 sk[64][NP];                     // k(p, q) of the group, p = |q| + row
  // group blockIdx.z: pairs g0 .. g0 + ng - 1 (blobs from g0), couplings in g0's blob
  const int g0 = blockIdx.z * XA_MAXP, ng = min(NP, npairs - g0);
  xblob += (size_t)g0 * blob_stride;
  const float2* kf = reinterpret_cast<const float2*>(xblob + kf_off);
  const int tile = blockIdx.x, u = blockIdx.y, q = u - (Lh - 1), aq = q < 0 ? -q : q;
  const int n2 = Lh * Lh, P = Lh - aq, K = 2 * Lh - 1;
  for (int t = threadIdx.x; t < P * NP; t += TC_M) {
    const int i = t / NP, v = t % NP, pd = aq + i;
    sk[i][v] = kf[(size_t)(pd * pd + pd + q) * XA_MAXP + v];
  }
  __syncthreads();
  const int col = threadIdx.x, j = tile * TC_M + col;
  float ar[NP], ai[NP];
#pragma unroll
  for (int v = 0; v < NP; ++v) ar[v] = ai[v] = 0.f;
  if (j < J) {                                       // H past column J is never written
    // degree aq + i of order q at hp + i * 128
    const float2* hp = H + ((size_t)tile * n2 + h_row(aq, q, Lh, true)) * TC_M + col;
    float2 cur[4], nxt[4];
#pragma unroll
    for (int w = 0; w < 4; ++w) cur[w] = w < P ? __ldg(hp + (size_t)w * TC_M) : make_float2(0.f, 0.f);
    for (int i = 0; i < P; i += 4) {
#pragma unroll
      for (int w = 0; w < 4; ++w)                    // the next four degrees, in flight meanwhile
        nxt[w] = i + 4 + w < P ? __ldg(hp + (size_t)(i + 4 + w) * TC_M) : make_float2(0.f, 0.f);
#pragma unroll
      for (int w = 0; w < 4; ++w)
        if (i + w < P) xw_mac<NP>(sk, i + w, cur[w], ar, ai);
#pragma unroll
      for (int w = 0; w < 4; ++w) cur[w] = nxt[w];
    }
  }
#pragma unroll
  for (int v = 0; v < NP; ++v)
    if (v < ng)
      reinterpret_cast<float2*>(xblob + (size_t)v * blob_stride + xf_off)[((size_t)tile * K + u) * TC_M + col] =
          make_float2(ar[v], ai[v]);
}

// FP16 hi and lo of 8 scaled values as two 16-byte units
__device__ __forceinline__ void xw_split8(const float* x, float sc, uint4* hi, uint4* lo) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int w = 0; w < 4; ++w) {
    const float x0 = x[2 * w] * sc, x1 = x[2 * w + 1] * sc;
    const __half2 a = __floats2half2_rn(x0, x1);
    const float2 af = __half22float2(a);
    const __half2 b = __floats2half2_rn(x0 - af.x, x1 - af.y);
    h[w] = *reinterpret_cast<const uint32_t*>(&a);
    l[w] = *reinterpret_cast<const uint32_t*>(&b);
  }
  *hi = make_uint4(h[0], h[1], h[2], h[3]);
  *lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// One thread per (pair, column, group of 8 orders r): the warp's lanes are 32
// / NRG columns x the NRG = KP / 8 groups, so each of its 16-byte stores
// (8 slots of one part) fills whole rows of the swizzled image (512 or 256
// contiguous bytes per instruction).
__global__ void __launch_bounds__(256) k_xaw_split(int Lh, int J, int nkf, unsigned char* __restrict__ xblob,
                                                   size_t blob_stride, int tiles, size_t xf_off) {
  const int KP = 32 * nkf, K = 2 * Lh - 1, nrg = KP / 8, cpw = 32 / nrg;
  const int pair = blockIdx.y, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int col = (blockIdx.x * 8 + warp) * cpw + lane / nrg;     // column of the pair's padded list
  const int rg = lane % nrg, tile = col / TC_M, row = col % TC_M, j = col;
  if (tile >= tiles) return;                         // whole warps: tiles x 128 is a multiple of cpw
  unsigned char* blob = xblob + (size_t)pair * blob_stride;
  // X_q of the column at x0[q * 128], q = -(Lh-1) .. Lh-1
  const float2* x0 = reinterpret_cast<const float2*>(blob + xf_off) + ((size_t)tile * K + (Lh - 1)) * TC_M + row;
  float* scales = reinterpret_cast<float*>(blob + (size_t)tiles * 2 * nkf * TC_A_BYTES);
  float a[4][8];                                     // Re P, Im P, Im M, -Re M of the group's 8 orders
#pragma unroll
  for (int w = 0; w < 8; ++w) {
    const int r = rg * 8 + w;
    float2 xp = make_float2(0.f, 0.f), xm = make_float2(0.f, 0.f);
    if (r < Lh) xp = __ldg(x0 + (ptrdiff_t)r * TC_M);
    if (r > 0 && r < Lh) xm = __ldg(x0 - (ptrdiff_t)r * TC_M);
    const bool z = r == 0;
    a[0][w] = z ? xp.x : xp.x + xm.x;
    a[1][w] = z ? xp.y : xp.y + xm.y;
    a[2][w] = z ? 0.f : xp.y - xm.y;
    a[3][w] = z ? 0.f : -(xp.x - xm.x);
  }
  float mx = 0.f;                                    // the column's largest slot: its nrg lanes together
#pragma unroll
  for (int g = 0; g < 4; ++g)
#pragma unroll
    for (int w = 0; w < 8; ++w) mx = fmaxf(mx, fabsf(a[g][w]));
  for (int o = nrg >> 1; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (j >= J) mx = 0.f;
  int ex = 0;
  if (mx > 0.f) frexpf(mx, &ex);
  const int e = mx > 0.f ? min(125, max(-125, 15 - ex)) : 0;
  const float sc = __int_as_float((127 + e) << 23);
  // A_re K-chunks, then A_im: (m * nkf + slot / 64) x 32 KB, hi then lo;
  // A_re P part (Re P), A_im P part (Im P), A_re M part (Im M), A_im M part (-Re M)
  unsigned char* ab = blob + (size_t)tile * 2 * nkf * TC_A_BYTES;
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    const int m = g & 1, k = (g < 2 ? 0 : KP) + rg * 8;
    unsigned char* cb = ab + (size_t)(m * nkf + (k >> 6)) * TC_A_BYTES + sw128_off(row, k & 63);
    uint4 hi, lo;
    xw_split8(a[g], sc, &hi, &lo);
    *reinterpret_cast<uint4*>(cb) = hi;
    *reinterpret_cast<uint4*>(cb + TC_A_HALF) = lo;
  }
  if (rg == 0) scales[j] = j < J ? __int_as_float((127 - e) << 23) : 0.f;
}

// ---------------------------------------------------------------- first pass on the tensor cores
// The first pass as one GEMM per (128-column tile, order q): M = the tile's
// columns j, K = the degrees p >= |q| in chunks of XT_DEG = 32.  H arrives
// in the order-major tile layout, so a chunk's rows are one contiguous run.
// Both operands are split into FP16 hi and lo after a power-of-two scale that
// puts the largest entry in [2^14, 2^15): H per (column, chunk) by the
// converter warps, which write each column's A row straight into a TMEM
// stage (thread = column = TMEM lane), the couplings per (order, chunk) once
// per group (k_xwb).  For each half h of the chunk's degrees the A row holds
// the K = 16 slices [Re H hi | Im H hi | Re H lo | Im H lo], and the coupling
// operand has N = 64 rows, so that one MMA per slice gives all three split
// products:
//   rows n < 32 (hi):  [Bre hi | Bim hi | Bre hi | Bim hi],
//   rows 32 + n (lo):  [Bre lo | Bim lo |   0    |   0   ],
// with, for pair v, Bre = Re k_v, Bim = -Im k_v in row v (Re X) and Bre =
// Im k_v, Bim = Re k_v in row 16 + v (Im X), so that
//   X[n] = D[n] + D[32 + n] = sum_p (A_hi B_hi + A_lo B_hi + A_hi B_lo)
//   (the lo x lo product dropped, about 22 significant bits as the rotated
//   window and the alpha stage).
// A chunk is 4 or 8 MMAs (8 with both degree halves live) from one issuing
// thread and one commit; each chunk accumulates in FP32 in a TMEM accumulator
// of its own (64 columns), and the epilogue undoes both scales while it sums
// the chunks.  One bulk copy brings a chunk's rows, one its coupling image.

// FP16 hi and lo of a pair of floats, packed
__device__ __forceinline__ uint32_t xt_split2(float a, float b, uint32_t* lo_word) {
  const __half2 h = __floats2half2_rn(a, b);
  const float2 hf = __half22float2(h);
  const __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
  *lo_word = *reinterpret_cast<const uint32_t*>(&l);
  return *reinterpret_cast<const uint32_t*>(&h);
}

// One block per (order u, chunk c, group), each thread four 16-byte units of
// the image: row n of the 64, unit k8 of the 16 (K slots 8 k8 .., slice
// st = k8 / 2: degree half st / 4, part st % 4 as in the A row).  The
// chunk's coefficients of every pair set the scale.
__global__ void __launch_bounds__(256) k_xwb(int Lh, int npairs, unsigned char* __restrict__ xblob,
                                             size_t blob_stride, size_t kf_off, size_t kb_off) {
  __shared__ float s_max[8];
  const int u = blockIdx.x, c = blockIdx.y, g0 = blockIdx.z * XA_MAXP, ng = min(XA_MAXP, npairs - g0);
  const int q = u - (Lh - 1), aq = q < 0 ? -q : q, P = Lh - aq, K = 2 * Lh - 1;
  if (c * XT_DEG >= P) return;                       // the order has no such chunk (block-uniform)
  unsigned char* blob = xblob + (size_t)g0 * blob_stride;
  const float2* kf = reinterpret_cast<const float2*>(blob + kf_off);
  unsigned char* img = blob + kb_off + ((size_t)u * XT_MAXCH + c) * XT_BIMG;
  float* bsc = reinterpret_cast<float*>(blob + kb_off + (size_t)K * XT_MAXCH * XT_BIMG);
  float x[4][8], mx = 0.f;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int t4 = threadIdx.x + 256 * r, n = t4 >> 4, k8 = t4 & 15;
    const int st = k8 >> 1, h = st >> 2, part = st & 3, lo_row = n >> 5, rv = n & 31;
    const int v = rv & 15, im_row = rv >> 4;
    const bool zero = lo_row && part >= 2;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int i = c * XT_DEG + 16 * h + 8 * (k8 & 1) + e, p = aq + i;
      float val = 0.f;
      if (!zero && v < ng && i < P) {
        const float2 kv = kf[(size_t)(p * p + p + q) * XA_MAXP + v];
        val = (part & 1) ? (im_row ? kv.x : -kv.y) : (im_row ? kv.y : kv.x);
      }
      x[r][e] = val;
      mx = fmaxf(mx, fabsf(val));
    }
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = mx;
  __syncthreads();
  mx = 0.f;
#pragma unroll
  for (int w = 0; w < 8; ++w) mx = fmaxf(mx, s_max[w]);
  int ex = 0;
  if (mx > 0.f) frexpf(mx, &ex);
  const int es = mx > 0.f ? min(125, max(-125, 15 - ex)) : 0;
  const float sc = __int_as_float((127 + es) << 23);
  if (threadIdx.x == 0) bsc[u * XT_MAXCH + c] = __int_as_float((127 - es) << 23);
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int t4 = threadIdx.x + 256 * r, n = t4 >> 4, k8 = t4 & 15;
    uint32_t hw[4], lw[4];
#pragma unroll
    for (int w = 0; w < 4; ++w) hw[w] = xt_split2(x[r][2 * w] * sc, x[r][2 * w + 1] * sc, &lw[w]);
    const uint4 o = (n >> 5) ? make_uint4(lw[0], lw[1], lw[2], lw[3]) : make_uint4(hw[0], hw[1], hw[2], hw[3]);
    *reinterpret_cast<uint4*>(img + (k8 >> 3) * XT_BATOM + sw128_off(n, (k8 & 7) * 8)) = o;
  }
}

#define XT_ROWB (TC_M * 8)              // one H row of a tile: 128 columns x float2
#define XT_HSTAGE (XT_DEG * XT_ROWB)    // ring stage: a chunk's H rows, 32 KB
#define XT_NS 4                         // H ring stages
#define XT_NACC 2                       // TMEM accumulators
#define XT_ACC (XT_MAXCH * 64)          // columns of one accumulator (64 a chunk)
#define XT_NA 4                         // TMEM A stages, and the coupling image ring (same index)
#define XT_ASTAGE 64                    // TMEM columns of one A stage
#define XT_ACOL (XT_NACC * XT_ACC)      // first TMEM column of the A stages
#ifndef XT_GROUPS
#define XT_GROUPS 2                     // converter groups of 4 warps, taking the chunks in turn
#endif
#define XT_CONV (4 * XT_GROUPS)         // converter warps
#define XT_META (XT_NA + XT_NACC + XT_GROUPS)   // per-item scale slots (reuse distance, see the converters)
#define XT_EPI0 (3 + XT_CONV)           // first epilogue warp
#define XT_THREADS (32 * (XT_EPI0 + 4)) // H loader, MMA issuer, image loader, converters, 4 epilogue warps
#define XT_META_BYTES (XT_META * XT_MAXCH * TC_M * 4)
#define XT_SMEM (XT_NA * XT_BIMG + XT_NS * XT_HSTAGE + XT_META_BYTES + 1024 + 512)

struct XtBars {
  uint64_t full[XT_NS], free[XT_NS], bfull[XT_NA], ready[XT_NA], afree[XT_NA], acc_full[XT_NACC],
      acc_empty[XT_NACC], meta_full[XT_META], drain;
  uint32_t tmem_base;
  int abort_flag;
};

// D += A B with A (128 x 16 FP16, row i in TMEM lane i, 8 columns) in tensor
// memory and B described in shared memory
__device__ __forceinline__ void umma_f16_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d_tmem),
      "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate));
}
// this thread's 32 consecutive 32-bit TMEM columns of its lane (warp-collective)
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
      "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]),
      "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]), "r"(v[17]),
      "r"(v[18]), "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]), "r"(v[25]),
      "r"(v[26]), "r"(v[27]), "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])
      : "memory");
}

// Contiguous item ranges (item t = tile * K + u) of equal traffic: an item
// reads its P = L_h - |q| H rows and writes ng X rows (KB).
__host__ __device__ inline long long xt_cost(int u, int Lh, int ng) {
  const int q = u - (Lh - 1);
  return (long long)(Lh - (q < 0 ? -q : q)) + ng;
}
// first item whose predecessors cost x or more (ctile: the cost of one tile)
__device__ inline int xt_first(long long x, int Lh, int ng, long long ctile) {
  const int K = 2 * Lh - 1;
  const long long tile = x / ctile, rem = x - tile * ctile;
  long long cb = 0;
  int u = 0;
  while (u < K && cb < rem) cb += xt_cost(u++, Lh, ng);
  return (int)(tile * K + u);
}

__global__ void __launch_bounds__(XT_THREADS, 1)
k_xw_tc(const float2* __restrict__ H, int Lh, int J, int tiles, int npairs, unsigned char* __restrict__ xblob,
        size_t blob_stride, size_t kb_off, size_t xf_off, int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* bring = sm;                                      // XT_NA x a chunk's coupling image
  unsigned char* ring = sm + XT_NA * XT_BIMG;                     // XT_NS x a chunk's H rows
  float* meta = reinterpret_cast<float*>(ring + XT_NS * XT_HSTAGE);   // [XT_META][XT_MAXCH][128]
  XtBars* bars = reinterpret_cast<XtBars*>(ring + XT_NS * XT_HSTAGE + XT_META_BYTES);
  volatile int* abort_flag = &bars->abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int K = 2 * Lh - 1, n2 = Lh * Lh;
  const int g0 = blockIdx.y * XA_MAXP, ng = min(XA_MAXP, npairs - g0);
  long long ctile = 0;
  for (int u = 0; u < K; ++u) ctile += xt_cost(u, Lh, ng);
  const long long C = ctile * tiles;
  const int i0 = xt_first(C * blockIdx.x / gridDim.x, Lh, ng, ctile);
  const int i1 = xt_first(C * (blockIdx.x + 1) / gridDim.x, Lh, ng, ctile);
  xblob += (size_t)g0 * blob_stride;
  const unsigned char* kb = xblob + kb_off;
  const float* bsc = reinterpret_cast<const float*>(kb + (size_t)K * XT_MAXCH * XT_BIMG);

  if (threadIdx.x == 0) {
    for (int i = 0; i < XT_NS; ++i) {
      mbar_init(smem_u32(&bars->full[i]), 1);
      mbar_init(smem_u32(&bars->free[i]), 4);      // the converter group's 4 warps: rows read
    }
    for (int i = 0; i < XT_NA; ++i) {
      mbar_init(smem_u32(&bars->bfull[i]), 1);
      mbar_init(smem_u32(&bars->ready[i]), 4);
      // MMA commit: the products of the A stage and of the image slot of this
      // index completed
      mbar_init(smem_u32(&bars->afree[i]), 1);
    }
    for (int i = 0; i < XT_NACC; ++i) {
      mbar_init(smem_u32(&bars->acc_full[i]), 1);
      mbar_init(smem_u32(&bars->acc_empty[i]), 4);
    }
    for (int i = 0; i < XT_META; ++i) mbar_init(smem_u32(&bars->meta_full[i]), XT_CONV);
    mbar_init(smem_u32(&bars->drain), 1);
    bars->abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                     smem_u32(&bars->tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = bars->tmem_base;

  if (warp == 0) {
    // ---------------- H loader: per chunk its H rows (one contiguous run of the
    // order-major tile, one bulk copy) into a ring stage the converters have read
    if (lane == 0) {
      int armed[XT_NS];
#pragma unroll
      for (int i = 0; i < XT_NS; ++i) armed[i] = -1;
      long long bc = 0;
      bool ok = true;
      for (int t = i0; t < i1 && ok; ++t) {
        const int tile = t / K, u = t - tile * K, q = u - (Lh - 1), aq = q < 0 ? -q : q, P = Lh - aq;
        const unsigned char* hb =
            reinterpret_cast<const unsigned char*>(H + (size_t)tile * n2 * TC_M) + (size_t)h_row(aq, q, Lh, true) * XT_ROWB;
        for (int c = 0; c * XT_DEG < P; ++c, ++bc) {
          const int s = (int)(bc % XT_NS);
          const uint32_t ph = (uint32_t)((bc / XT_NS) & 1);
          if (!(ok = mbar_wait_n(smem_u32(&bars->free[s]), ph ^ 1u, abort_flag, TC_WAIT_LIMIT))) break;
          const int rows = min(XT_DEG, P - c * XT_DEG);
          const uint32_t fb = smem_u32(&bars->full[s]);
          mbar_expect_tx(fb, (uint32_t)(rows * XT_ROWB));
          bulk_g2s(smem_u32(ring + (size_t)s * XT_HSTAGE), hb + (size_t)c * XT_DEG * XT_ROWB, (uint32_t)(rows * XT_ROWB), fb);
#pragma unroll
          for (int i = 0; i < XT_NS; ++i)
            if (i == s) armed[i] = (int)ph;
        }
      }
      if (!ok) *abort_flag = 1;
#pragma unroll
      for (int i = 0; i < XT_NS; ++i) {   // copies in flight land before the CTA may exit
        if (armed[i] >= 0) {
          uint32_t n = 0;
          while (!mbar_test(smem_u32(&bars->full[i]), (uint32_t)armed[i]) && ++n < TC_WAIT_LIMIT) {}
        }
      }
    }
  } else if (warp == 2) {
    // ---------------- image loader: per chunk its coupling image into the slot
    // of its A stage index, once that slot's previous products have completed
    if (lane == 0) {
      int armed[XT_NA];
#pragma unroll
      for (int i = 0; i < XT_NA; ++i) armed[i] = -1;
      long long bc = 0;
      bool ok = true;
      for (int t = i0; t < i1 && ok; ++t) {
        const int u = t % K, q = u - (Lh - 1), P = Lh - (q < 0 ? -q : q);
        for (int c = 0; c * XT_DEG < P; ++c, ++bc) {
          const int s = (int)(bc % XT_NA);
          const uint32_t ph = (uint32_t)((bc / XT_NA) & 1);
          if (!(ok = mbar_wait_n(smem_u32(&bars->afree[s]), ph ^ 1u, abort_flag, TC_WAIT_LIMIT))) break;
          const uint32_t fb = smem_u32(&bars->bfull[s]);
          mbar_expect_tx(fb, XT_BIMG);
          bulk_g2s(smem_u32(bring + (size_t)s * XT_BIMG), kb + ((size_t)u * XT_MAXCH + c) * XT_BIMG, XT_BIMG, fb);
#pragma unroll
          for (int i = 0; i < XT_NA; ++i)
            if (i == s) armed[i] = (int)ph;
        }
      }
      if (!ok) *abort_flag = 1;
#pragma unroll
      for (int i = 0; i < XT_NA; ++i) {
        if (armed[i] >= 0) {
          uint32_t n = 0;
          while (!mbar_test(smem_u32(&bars->bfull[i]), (uint32_t)armed[i]) && ++n < TC_WAIT_LIMIT) {}
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer: per chunk c of item i, one N = 64 product per
    // live K = 16 slice of the TMEM A stage and the chunk's coupling image,
    // into accumulator i % XT_NACC, columns 64 c ..; one commit a chunk frees
    // the A stage and the image slot
    if (lane == 0) {
      const uint32_t idesc = umma_idesc_f16(128, 64);
      long long bc = 0;
      int li = 0;
      bool ok = true;
      for (int t = i0; t < i1 && ok; ++t, ++li) {
        const int u = t % K, q = u - (Lh - 1), P = Lh - (q < 0 ? -q : q);
        const int a = li % XT_NACC;
        if (!(ok = mbar_wait_n(smem_u32(&bars->acc_empty[a]), (uint32_t)(((li / XT_NACC) & 1) ^ 1), abort_flag,
                               TC_WAIT_LIMIT)))
          break;
        tc_fence_after();
        for (int c = 0; c * XT_DEG < P; ++c, ++bc) {
          const int sa = (int)(bc % XT_NA);
          const uint32_t ph = (uint32_t)((bc / XT_NA) & 1);
          if (!(ok = mbar_wait_n(smem_u32(&bars->bfull[sa]), ph, abort_flag, TC_WAIT_LIMIT))) break;
          if (!(ok = mbar_wait_n(smem_u32(&bars->ready[sa]), ph, abort_flag, TC_WAIT_LIMIT))) break;
          tc_fence_after();
          const int nst = P - c * XT_DEG > 16 ? 8 : 4;   // slices of the live degree halves
          const uint32_t at = tmem + (uint32_t)(XT_ACOL + sa * XT_ASTAGE);
          const uint32_t bb = smem_u32(bring + (size_t)sa * XT_BIMG);
          const uint32_t d = tmem + (uint32_t)(a * XT_ACC + c * 64);
          for (int st = 0; st < nst; ++st)
            umma_f16_ta(d, at + (uint32_t)(8 * st), sw128_desc(bb + (uint32_t)((st >> 2) * XT_BATOM)) + (uint64_t)(2 * (st & 3)),
                        idesc, st > 0 ? 1u : 0u);
          umma_commit(smem_u32(&bars->afree[sa]));
        }
        if (!ok) break;
        umma_commit(smem_u32(&bars->acc_full[a]));
      }
      if (!ok) *abort_flag = 1;
      umma_commit(smem_u32(&bars->drain));   // every MMA completes before TMEM is released
      uint32_t n = 0;
      while (!mbar_test(smem_u32(&bars->drain), 0u) && ++n < TC_WAIT_LIMIT) {}
    }
  } else if (warp < XT_EPI0) {
    // ---------------- converters: XT_GROUPS groups of four warps taking the
    // chunks in turn, thread = column of the tile = TMEM lane (warp % 4
    // picks the lane quadrant).  Per chunk: the column's largest |value|
    // over the staged rows (zero past the order's degrees and past column
    // J) and its scale; once the A stage's previous products have completed,
    // per live half of the degrees the split A row into the stage's TMEM
    // columns; then the ring stage is released and the inverse scale goes to
    // the item's meta slot.  Slot li % XT_META is written after the A stage
    // wait, so the products of the chunk XT_NA earlier have completed; its
    // item is at most XT_NA items back and was issued only after the
    // epilogue had released item li - XT_NA - XT_NACC, so the epilogue has
    // read that slot's previous item.  Every converter warp arrives on the
    // item's meta barrier, also when its group had none of the item's chunks:
    // a warp arriving for item li has passed the A stage wait of one of its
    // chunks in the XT_GROUPS items before, so the epilogue has released item
    // li - XT_GROUPS - XT_NA - XT_NACC, and XT_GROUPS more slots of distance
    // keep the warp from completing a slot's next phase before the epilogue
    // has waited on the current one.
    const int grp = (warp - 3) >> 2, quad = warp & 3, col = quad * 32 + lane;
    const uint32_t tl = (uint32_t)(quad * 32) << 16;
    long long bc = 0;
    bool ok = true;
    int li = 0;
    for (int t = i0; t < i1 && ok; ++t, ++li) {
      const int tile = t / K, u = t - tile * K, q = u - (Lh - 1), P = Lh - (q < 0 ? -q : q);
      const bool live = tile * TC_M + col < J;
      const int ms = li % XT_META;
      for (int c = 0; c * XT_DEG < P; ++c, ++bc) {
        if ((int)(bc % XT_GROUPS) != grp) continue;
        const int s = (int)(bc % XT_NS), sa = (int)(bc % XT_NA);
        int got = 0;
        if (lane == 0) got = mbar_wait_n(smem_u32(&bars->full[s]), (uint32_t)((bc / XT_NS) & 1), abort_flag, TC_WAIT_LIMIT);
        got = __shfl_sync(0xffffffffu, got, 0);
        if (!(ok = got != 0)) break;
        const float2* hs = reinterpret_cast<const float2*>(ring + (size_t)s * XT_HSTAGE) + col;
        const int rows = live ? min(XT_DEG, P - c * XT_DEG) : 0;
        float mx = 0.f;
        for (int i = 0; i < rows; ++i) {
          const float2 h = hs[(size_t)i * TC_M];
          mx = fmaxf(mx, fmaxf(fabsf(h.x), fabsf(h.y)));
        }
        int ex = 0;
        if (mx > 0.f) frexpf(mx, &ex);
        const int es = mx > 0.f ? min(125, max(-125, 15 - ex)) : 0;
        const float sc = __int_as_float((127 + es) << 23);
        if (lane == 0)
          got = mbar_wait_n(smem_u32(&bars->afree[sa]), (uint32_t)(((bc / XT_NA) & 1) ^ 1), abort_flag, TC_WAIT_LIMIT);
        got = __shfl_sync(0xffffffffu, got, 0);
        if (!(ok = got != 0)) break;
        tc_fence_after();
        const int nh = P - c * XT_DEG > 16 ? 2 : 1;   // live degree halves (warp-uniform)
        for (int h = 0; h < nh; ++h) {
          uint32_t w[32];   // Re hi, Im hi, Re lo, Im lo: 8 columns each, two FP16 a column
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int i0 = 16 * h + 2 * e;
            float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f);
            if (i0 < rows) a = hs[(size_t)i0 * TC_M];
            if (i0 + 1 < rows) b = hs[(size_t)(i0 + 1) * TC_M];
            w[e] = xt_split2(a.x * sc, b.x * sc, &w[16 + e]);
            w[8 + e] = xt_split2(a.y * sc, b.y * sc, &w[24 + e]);
          }
          tmem_st32(tmem + tl + (uint32_t)(XT_ACOL + sa * XT_ASTAGE + 32 * h), w);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&bars->free[s]));   // the rows are read
        meta[(ms * XT_MAXCH + c) * TC_M + col] = __int_as_float((127 - es) << 23);
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&bars->ready[sa]));
      }
      if (!ok) break;
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bars->meta_full[ms]));
    }
    if (!ok) *abort_flag = 1;
  } else {
    // ---------------- epilogue: the last four warps, TMEM lane quadrant warp % 4 =
    // the tile's columns; X of the group's pairs: the sum of each chunk's hi
    // and lo column halves, both scales undone
    const int quad = warp & 3, row = quad * 32 + lane;
    bool ok = true;
    int li = 0;
    for (int t = i0; t < i1 && ok; ++t, ++li) {
      const int tile = t / K, u = t - tile * K, q = u - (Lh - 1), P = Lh - (q < 0 ? -q : q);
      const int a = li % XT_NACC, ms = li % XT_META;
      int got = 0;
      if (lane == 0)
        got = mbar_wait_n(smem_u32(&bars->acc_full[a]), (uint32_t)((li / XT_NACC) & 1), abort_flag, TC_WAIT_LIMIT) &&
              mbar_wait_n(smem_u32(&bars->meta_full[ms]), (uint32_t)((li / XT_META) & 1), abort_flag, TC_WAIT_LIMIT);
      got = __shfl_sync(0xffffffffu, got, 0);
      __syncwarp();
      if (!(ok = got != 0)) break;
      tc_fence_after();
      float x[32];
#pragma unroll
      for (int n = 0; n < 32; ++n) x[n] = 0.f;
      const uint32_t tb = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(a * XT_ACC);
#pragma unroll 1
      for (int c = 0; c * XT_DEG < P; ++c) {
        const float sf = meta[(ms * XT_MAXCH + c) * TC_M + row] * __ldg(bsc + u * XT_MAXCH + c);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          uint32_t dh[16], dl[16];
          TMEM_LD16(tb + (uint32_t)(c * 64 + 16 * h), dh);
          TMEM_LD16(tb + (uint32_t)(c * 64 + 32 + 16 * h), dl);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int n = 0; n < 16; ++n)
            x[16 * h + n] = fmaf(sf, __uint_as_float(dh[n]) + __uint_as_float(dl[n]), x[16 * h + n]);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bars->acc_empty[a]));
      const size_t xo = xf_off + (((size_t)tile * K + u) * TC_M + row) * sizeof(float2);
#pragma unroll
      for (int v = 0; v < XA_MAXP; ++v)
        if (v < ng) *reinterpret_cast<float2*>(xblob + (size_t)v * blob_stride + xo) = make_float2(x[v], x[16 + v]);
    }
    if (!ok) *abort_flag = 1;
  }
  __syncthreads();
  if (*abort_flag && threadIdx.x == 0) atomicExch(err, 1);
  tc_fence_after();
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
}

cudaError_t launch_xaw_from_h(const double2* kc, const float2* H, int Lh, int Nb, int Ng, int npairs, void* xblob,
                              cudaStream_t st) {
  if (npairs <= 0) return cudaSuccess;
  if (Lh <= 16 || Lh > 64) return cudaErrorInvalidValue;
  const int nkf = tcw_nk(Lh) / 2, tiles = tcw_tiles(Nb, Ng), n2 = Lh * Lh;
  if (npairs > 65535) return cudaErrorInvalidValue;
  const size_t stride = tcw_xblob_bytes(Nb, Ng, Lh);
  const size_t sc_off = (size_t)tiles * 2 * nkf * TC_A_BYTES;
  const size_t kf_off = sc_off + tcw_scales_bytes(tiles);
  const size_t kb_off = kf_off + tcw_kf_bytes(Lh);
  const size_t xf_off = kb_off + (xt_use_tc(tiles, Lh) ? tcw_kb_bytes(Lh) : 0);
  unsigned char* xb = (unsigned char*)xblob;
  // first pass, every group of up to XA_MAXP pairs in one launch: X in FP32
  const int groups = (npairs + XA_MAXP - 1) / XA_MAXP;
  if (groups > 65535) return cudaErrorInvalidValue;
  k_kf_from_kc<<<dim3((n2 * XA_MAXP + 255) / 256, groups), 256, 0, st>>>(kc, n2, npairs, xb, stride, kf_off);
  if (!xt_use_tc(tiles, Lh)) {
    const dim3 grid(tiles, 2 * Lh - 1, groups);
    if (npairs <= 4)
      k_xw_x<4><<<grid, TC_M, 0, st>>>(H, Lh, Nb * Ng, npairs, xb, stride, kf_off, xf_off);
    else if (npairs <= 8)
      k_xw_x<8><<<grid, TC_M, 0, st>>>(H, Lh, Nb * Ng, npairs, xb, stride, kf_off, xf_off);
    else
      k_xw_x<16><<<grid, TC_M, 0, st>>>(H, Lh, Nb * Ng, npairs, xb, stride, kf_off, xf_off);
  } else {
    static bool attr = false;
    static int nsm = 0;
    if (!attr) {
      cudaError_t e = cudaFuncSetAttribute(k_xw_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, XT_SMEM);
      if (e != cudaSuccess) return e;
      int dev = 0;
      if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
      if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
      attr = true;
    }
    int* err = tc_error_word();
    if (!err) return cudaErrorMemoryAllocation;
    k_xwb<<<dim3(2 * Lh - 1, XT_MAXCH, groups), 256, 0, st>>>(Lh, npairs, xb, stride, kf_off, kb_off);
    // persistent: one CTA per SM per group, each over a contiguous item range
    const long long items = (long long)tiles * (2 * Lh - 1);
    const int gx = (int)std::min<long long>(items, nsm);
    k_xw_tc<<<dim3(gx, groups), XT_THREADS, XT_SMEM, st>>>(H, Lh, Nb * Ng, tiles, npairs, xb, stride, kb_off, xf_off,
                                                           err);
  }
  // second pass: scales and the split A operands
  const int cols_per_block = 8 * (32 / (4 * nkf));   // 8 warps of 32 / (KP / 8) columns
  k_xaw_split<<<dim3((tiles * TC_M + cols_per_block - 1) / cols_per_block, npairs), 256, 0, st>>>(
      Lh, Nb * Ng, nkf, xb, stride, tiles, xf_off);
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

static_assert(sizeof(XtBars) <= 512, "the first pass's bookkeeping fits the space XT_SMEM keeps for it");
static_assert(XT_ACOL + XT_NA * XT_ASTAGE <= 512, "the first pass's accumulators and A stages fit TMEM");
static_assert(XT_SMEM <= 232448, "one CTA's shared memory");
