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
// The producer (CUDA cores, two passes: k_xw_x forms X in FP32 for a group
// of up to 16 pairs from the rotated window H, with each column's slot bound;
// k_xaw_split folds X into P and M, scales, splits and writes the swizzled A
// operand -- A_re and A_im, NKF K-chunks of 32 KB each -- and the column
// scales to a blob in global memory); k_alpha_tcw
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

#define TCW_NA 128                      // alpha rows per chunk (MMA N)

// A-operand K-chunks per tile: 2 NKF (A_re then A_im, NKF chunks of 64 each)
static inline int tcw_nk(int Lh) { return Lh <= 32 ? 2 : 4; }
static inline int tcw_tiles(int Nb, int Ng) { return (Nb * Ng + TC_M - 1) / TC_M; }
static inline int tcw_chunks(int Na) { return (Na + TCW_NA - 1) / TCW_NA; }

bool tcw_supported(int Lh, int Na) { return Lh > 16 && Lh <= 64 && Na >= 1; }

size_t tcw_etab_bytes(int Na, int Lh) { return (size_t)tcw_chunks(Na) * (tcw_nk(Lh) / 2) * TC_B_BYTES; }

// per pair: tiles x 2 NKF x 32 KB of A, one float scale per padded column,
// room for the coupling rows of a producer group of up to XA_MAXP pairs as
// floats, interleaved [pq][XA_MAXP] (used in the group's first pair), and the
// pair's X_q(j) in FP32, [tile][q + L_h - 1][128 columns] (the producer's
// first pass writes it, its second pass scales and splits it into A)
#define XA_MAXP 16
static inline size_t tcw_scales_bytes(size_t tiles) { return ((tiles * TC_M * sizeof(float)) + 1023) / 1024 * 1024; }
static inline size_t tcw_kf_bytes(int Lh) { return ((size_t)Lh * Lh * XA_MAXP * sizeof(float2) + 1023) / 1024 * 1024; }
static inline size_t tcw_xf_bytes(size_t tiles, int Lh) { return tiles * (size_t)(2 * Lh - 1) * TC_M * sizeof(float2); }
size_t tcw_xblob_bytes(int Nb, int Ng, int Lh) {
  const size_t t = (size_t)tcw_tiles(Nb, Ng);
  return t * (size_t)tcw_nk(Lh) * TC_A_BYTES + tcw_scales_bytes(t) + tcw_kf_bytes(Lh) + tcw_xf_bytes(t, Lh);
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
// Two passes.  k_xw_x: X_q(j) = sum_{p>=|q|} k(p,q) H^p_q(j) for a group of
// up to XA_MAXP pairs, one block per (128-column tile, order q), one thread
// per column: the thread keeps its column's sums for every pair of the group
// in registers, so each H value (one coalesced row of the tiled layout per
// degree, read from HBM once per group) feeds 4 NP multiply-adds, with the
// group's k(., q) in shared memory (broadcast reads) and the next four
// degrees' H loads issued before the current four are used.  X goes to the
// pair's FP32 region, and 2 max(|Re X|, |Im X|), a bound of every slot built
// from the column's X (|Re P_r| <= |Re X_r| + |Re X_-r|, ...) and at most
// twice the largest one (X_r = (P_r + M_r) / 2), raises the column's entry in
// the pair's scale array (atomicMax on the float bits, entries >= 0).
// k_xaw_split: one thread per (pair, column, 8 orders r): scale 2^e from
// that bound into [2^13, 2^15), P_r = X_r + X_-r, M_r = X_r - X_-r (P_0 = X_0,
// M_0 = 0), every slot scaled, split into FP16 hi/lo and stored swizzled into
// its K-chunk (A_re[r] = Re P_r, A_re[KP + r] = Im M_r, A_im[r] = Im P_r,
// A_im[KP + r] = -Re M_r; zero for r >= L_h).  Columns beyond J are zero.

// Complex multiply-adds of the group's pairs for one column: sk[i][v] =
// k(p, q) of pair v, h = H^p_q of the column.
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
                                               size_t xf_off, size_t sc_off) {
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
    const float2* hp = H + (size_t)tile * n2 * TC_M + col;   // row pq at hp + pq * 128
    float2 cur[4], nxt[4];
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const int pd = aq + w;
      cur[w] = w < P ? __ldg(hp + (size_t)(pd * pd + pd + q) * TC_M) : make_float2(0.f, 0.f);
    }
    for (int i = 0; i < P; i += 4) {
#pragma unroll
      for (int w = 0; w < 4; ++w) {                  // the next four degrees, in flight meanwhile
        const int pd = aq + i + 4 + w;
        nxt[w] = i + 4 + w < P ? __ldg(hp + (size_t)(pd * pd + pd + q) * TC_M) : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int w = 0; w < 4; ++w)
        if (i + w < P) xw_mac<NP>(sk, i + w, cur[w], ar, ai);
#pragma unroll
      for (int w = 0; w < 4; ++w) cur[w] = nxt[w];
    }
  }
#pragma unroll
  for (int v = 0; v < NP; ++v)
    if (v < ng) {
      unsigned char* blob = xblob + (size_t)v * blob_stride;
      reinterpret_cast<float2*>(blob + xf_off)[((size_t)tile * K + u) * TC_M + col] = make_float2(ar[v], ai[v]);
      if (j < J) atomicMax(reinterpret_cast<int*>(blob + sc_off) + j, __float_as_int(2.f * fmaxf(fabsf(ar[v]), fabsf(ai[v]))));
    }
}

// The column maxima of every pair cleared (before k_xw_x raises them).
__global__ void k_xw_clear(int n, int ng, unsigned char* __restrict__ xblob, size_t blob_stride, size_t sc_off) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < (long long)n * ng;
       t += (long long)gridDim.x * blockDim.x)
    reinterpret_cast<int*>(xblob + (size_t)(t / n) * blob_stride + sc_off)[t % n] = 0;
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
  const float mx = j < J ? scales[j] : 0.f;          // the column's slot bound (k_xw_x)
  int ex = 0;
  if (mx > 0.f) frexpf(mx, &ex);
  const int e = mx > 0.f ? min(125, max(-125, 15 - ex)) : 0;
  const float sc = __int_as_float((127 + e) << 23);
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
  __syncwarp();                                      // every lane has read the column's bound
  if (rg == 0) scales[j] = j < J ? __int_as_float((127 - e) << 23) : 0.f;
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
  const size_t xf_off = kf_off + tcw_kf_bytes(Lh);
  unsigned char* xb = (unsigned char*)xblob;
  // first pass, every group of up to XA_MAXP pairs in one launch: X in FP32
  // and the columns' slot bounds
  const int groups = (npairs + XA_MAXP - 1) / XA_MAXP;
  if (groups > 65535) return cudaErrorInvalidValue;
  k_kf_from_kc<<<dim3((n2 * XA_MAXP + 255) / 256, groups), 256, 0, st>>>(kc, n2, npairs, xb, stride, kf_off);
  const int n = tiles * TC_M;
  k_xw_clear<<<(unsigned)std::min<long long>(((long long)n * npairs + 255) / 256, 8192), 256, 0, st>>>(n, npairs, xb,
                                                                                                     stride, sc_off);
  const dim3 grid(tiles, 2 * Lh - 1, groups);
  if (npairs <= 4)
    k_xw_x<4><<<grid, TC_M, 0, st>>>(H, Lh, Nb * Ng, npairs, xb, stride, kf_off, xf_off, sc_off);
  else if (npairs <= 8)
    k_xw_x<8><<<grid, TC_M, 0, st>>>(H, Lh, Nb * Ng, npairs, xb, stride, kf_off, xf_off, sc_off);
  else
    k_xw_x<16><<<grid, TC_M, 0, st>>>(H, Lh, Nb * Ng, npairs, xb, stride, kf_off, xf_off, sc_off);
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
