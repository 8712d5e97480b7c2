// The rotated window on the tensor cores (FP32_BULK outputs).  For each
// degree p the window rotated to (0, beta_b, gamma_c) (Eq. rotation_non_symm
// with Eq. Dlm) is a real-by-complex matrix product,
//   H^p_q(b, c) = sum_{q'} B_p(q', c) d^p_{q,q'}(beta_b),   B_p(q', c) = h_p^{q'} e^{-i q' gamma_c},
// with depth the 2p + 1 orders q'.  One tcgen05 MMA tile puts the gamma
// samples c on M (128 TMEM lanes) and 128 consecutive (beta, q) rows of the
// degree on N, so the accumulator holds H transposed: a warp's lanes are 32
// consecutive gamma samples of one output row, which are 32 consecutive
// elements of H's tiled layout (h_index), and the stores coalesce.
//
// Both operands are split into FP16 hi and lo parts, scaled by powers of two
// so that their largest entries lie below 2^15, and the three products hi hi,
// hi lo, lo hi accumulate in FP32 in TMEM (about 22 significant bits, as the
// alpha stage of this path).  The d operand depends only on (L_h, N_beta): its
// split parts, already in the 128-byte swizzled K-major image the MMAs read,
// are built once per context from the FP32 d(beta) table (launch_rotwin_tc_table,
// one 32 KB image of hi and lo parts per (degree, 128-row tile, 64-wide K
// chunk), and one scale per row).  The window operand B_p changes with h: a
// small kernel per call (launch_rotwin_tc_window) writes it per degree in the
// same image form, with the window's inactive orders (qmask) as zero columns.
//
// The kernel is persistent (one CTA per SM over a contiguous range of the
// (degree, row tile) list, the ranges of equal traffic) and warp-specialised:
// warp 0 streams the d chunks through a ring of three stages with
// cp.async.bulk and, when the degree changes and the previous degree's
// products have completed, the new degree's window operand; warp 1 issues the
// MMAs into two TMEM accumulators (2 x (Re, Im) x 128 columns: all 512) and
// commits them to mbarriers; warps 2..9 drain the accumulators (two warps per
// TMEM lane quadrant, each half of the 128 rows) while the next tile's
// products run.  Every wait is bounded: on expiry the CTA raises its abort
// flag, every role leaves its loop, copies and products in flight complete,
// and the error word is set.
#include <cuda_fp16.h>

#include "common.cuh"
#include "stages_dev.cuh"
#include "tc.cuh"
#include "tc_ptx.cuh"

#define RT_ROWS 128                     // (beta, q) rows per tile (MMA N)
#define RT_PART (128 * 64 * 2)          // one 64-wide K chunk of 128 rows, FP16: 16 KB
#define RT_STAGE (2 * RT_PART)          // hi and lo parts of one d chunk: 32 KB
#define RT_RING 3
#define RT_EPI_WARPS 8
#define RT_THREADS (64 + 32 * RT_EPI_WARPS)
#define RT_WA_BYTES (8 * RT_PART)       // window operand: {Re, Im} x {hi, lo} x 2 K chunks
#define RT_SMEM (RT_WA_BYTES + RT_RING * RT_STAGE + 1024 + 1024)   // + alignment + RtBars

struct RtBars {
  uint64_t full[RT_RING], empty[RT_RING], acc_full[2], acc_empty[2], wfull, wempty, drain;
  uint32_t tmem_base;
  int abort_flag;
};

bool rotwin_tc_supported(int Lh, int Ng) { return Lh >= 2 && Lh <= SLSHT_MAX_LH && Ng >= 1 && Ng <= 128; }

// Tiles of degree p: ceil(Nb (2p+1) / 128); K chunks of 64 orders per tile.
__host__ __device__ inline int rt_tiles_of(int p, int Nb) { return (Nb * (2 * p + 1) + RT_ROWS - 1) / RT_ROWS; }
__host__ __device__ inline int rt_nch(int p) { return (2 * p + 1 + 63) >> 6; }

// Position in the (degree, tile) list: degree p, index of its first tile,
// index of its first 32 KB chunk image.
struct RtPos {
  int p, tb, cb;
};
__host__ __device__ inline void rt_seek(RtPos& s, int t, int Nb, int Lh) {
  while (s.p < Lh - 1 && t >= s.tb + rt_tiles_of(s.p, Nb)) {
    const int n = rt_tiles_of(s.p, Nb);
    s.tb += n;
    s.cb += n * rt_nch(s.p);
    ++s.p;
  }
}

// Splitting the tile list into contiguous ranges of equal traffic: a tile
// writes 128 rows of N_gamma complex64 outputs and reads rt_nch 32 KB chunks
// (cost in KB).  rt_first(x) is the first tile whose preceding tiles cost x
// or more, so the ranges [rt_first(k C / G), rt_first((k+1) C / G)) of
// G CTAs tile the list.
__host__ __device__ inline long long rt_cost(int p, int Ng) { return Ng + 32LL * rt_nch(p); }
__host__ __device__ inline int rt_first(long long x, int Lh, int Nb, int Ng) {
  long long cb = 0;
  int tb = 0;
  for (int p = 0; p < Lh; ++p) {
    const int n = rt_tiles_of(p, Nb);
    const long long c = rt_cost(p, Ng);
    if (cb + n * c >= x) {
      const long long r = x > cb ? (x - cb + c - 1) / c : 0;
      return tb + (int)r;
    }
    cb += n * c;
    tb += n;
  }
  return tb;
}

static void rt_counts(int Lh, int Nb, int* tiles, long long* chunks) {
  int t = 0;
  long long c = 0;
  for (int p = 0; p < Lh; ++p) {
    t += rt_tiles_of(p, Nb);
    c += (long long)rt_tiles_of(p, Nb) * rt_nch(p);
  }
  *tiles = t;
  *chunks = c;
}

size_t rotwin_tc_table_bytes(int Lh, int Nb) {
  int t;
  long long c;
  rt_counts(Lh, Nb, &t, &c);
  return (size_t)c * RT_STAGE + (size_t)t * RT_ROWS * sizeof(float);
}

// ---------------------------------------------------------------- the d image
// Eight threads per row (b, q) of a tile, each owning 8 consecutive orders of
// every K chunk: the row's largest |d| sets its scale 2^(15 - e) (e its binary
// exponent), the scaled values split into FP16 hi and lo, each group of 8
// stored as one 16-byte unit at its swizzled place.  Rows past the degree's
// last (b, q) and orders past 2p + 1 are zeros.
__global__ void k_rt_table(const float* __restrict__ dt, int Lh, int Nb, long long nthreads,
                           unsigned char* __restrict__ img, float* __restrict__ rs) {
  const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gt >= nthreads) return;   // nthreads = 1024 x tiles: whole warps, a row's eight threads together
  const int row = (int)(gt >> 3), sub = (int)(gt & 7);
  const int tile = row >> 7, r = row & 127;
  RtPos s{0, 0, 0};
  rt_seek(s, tile, Nb, Lh);
  const int p = s.p, w = 2 * p + 1, rt = tile - s.tb, nc = rt_nch(p);
  const int R = rt * RT_ROWS + r, b = R / w, qi = R - b * w;
  const bool live = b < Nb;
  const float* drow = dt + (size_t)(live ? b : 0) * blk_off(Lh) + blk_off(p) + (size_t)qi * w;
  float v[2][8];
  float mx = 0.f;
#pragma unroll
  for (int kc = 0; kc < 2; ++kc)
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int u = kc * 64 + sub * 8 + e;
      v[kc][e] = (live && kc < nc && u < w) ? drow[u] : 0.f;
      mx = fmaxf(mx, fabsf(v[kc][e]));
    }
  mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
  mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
  mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 4));
  int ex = 0;
  if (mx > 0.f) frexpf(mx, &ex);
  const float sc = ldexpf(1.f, 15 - ex);
  if (sub == 0) rs[row] = ldexpf(1.f, ex - 15);
#pragma unroll
  for (int kc = 0; kc < 2; ++kc) {
    if (kc >= nc) break;
    uint32_t hi[4], lo[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float x0 = v[kc][2 * e] * sc, x1 = v[kc][2 * e + 1] * sc;
      const __half2 h2 = __floats2half2_rn(x0, x1);
      const float2 hf = __half22float2(h2);
      const __half2 l2 = __floats2half2_rn(x0 - hf.x, x1 - hf.y);
      hi[e] = *reinterpret_cast<const uint32_t*>(&h2);
      lo[e] = *reinterpret_cast<const uint32_t*>(&l2);
    }
    unsigned char* base = img + (size_t)(s.cb + (long long)rt * nc + kc) * RT_STAGE + sw128_off(r, sub * 8);
    *reinterpret_cast<uint4*>(base) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
    *reinterpret_cast<uint4*>(base + RT_PART) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
  }
}

cudaError_t launch_rotwin_tc_table(const float* dt, int Lh, int Nb, void* tab, cudaStream_t st) {
  if (Lh < 1 || Lh > SLSHT_MAX_LH || Nb < 1) return cudaErrorInvalidValue;
  int tiles;
  long long chunks;
  rt_counts(Lh, Nb, &tiles, &chunks);
  const long long n = (long long)tiles * RT_ROWS * 8;
  unsigned char* img = (unsigned char*)tab;
  float* rs = (float*)(img + (size_t)chunks * RT_STAGE);
  k_rt_table<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(dt, Lh, Nb, n, img, rs);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- the window operand
// Window operand part (0 Re hi, 1 Re lo, 2 Im hi, 3 Im lo) of K chunk kc, in
// shared memory and in the per-degree images (RT_WA_BYTES each).
__host__ __device__ __forceinline__ size_t rt_wa_off(int part, int kc) { return (size_t)(part * 2 + kc) * RT_PART; }

size_t rotwin_tc_window_bytes(int Lh) { return (size_t)Lh * RT_WA_BYTES + 256 * sizeof(float); }

// Four blocks per degree p (blockIdx.y: which quarter of the (row, group)
// units): B_p(q', c) = h_p^{q'} e^{-i q' gamma_c} over the
// active orders (zero elsewhere and for c >= N_gamma), scaled by 2^(15 - e)
// with e the binary exponent of the largest |h_p^{q'}| (a bound of every
// entry), split into FP16 hi and lo, 16-byte units at their swizzled places;
// dsc[p] = 2^(e - 15) undoes the scale.
__global__ void __launch_bounds__(256) k_rt_window(const double2* __restrict__ h, const float2* __restrict__ eg,
                                                   const uint32_t* __restrict__ qmask, int Lh, int Ng,
                                                   unsigned char* __restrict__ wimg, float* __restrict__ dsc) {
  __shared__ float s_max[8];
  const int p = blockIdx.x, w = 2 * p + 1, nc = rt_nch(p), K = 2 * Lh - 1;
  float hm = 0.f;
  for (int u = threadIdx.x; u < w; u += blockDim.x)
    if (rot_order_on(qmask, u - p)) {
      const double2 hv = h[p * p + u];
      hm = fmaxf(hm, sqrtf((float)(hv.x * hv.x + hv.y * hv.y)));
    }
  for (int o = 16; o > 0; o >>= 1) hm = fmaxf(hm, __shfl_xor_sync(0xffffffffu, hm, o));
  if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = hm;
  __syncthreads();
  hm = 0.f;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) hm = fmaxf(hm, s_max[i]);
  int eb = 0;
  if (hm > 0.f) frexpf(hm, &eb);
  const float bsc = ldexpf(1.f, 15 - eb);
  if (threadIdx.x == 0 && blockIdx.y == 0) dsc[p] = ldexpf(1.f, eb - 15);
  unsigned char* dst = wimg + (size_t)p * RT_WA_BYTES;
  for (int it = blockIdx.y * blockDim.x + threadIdx.x; it < 128 * 8 * nc; it += gridDim.y * blockDim.x) {
    const int row = it & 127, gk = it >> 7, kc = gk >> 3, g = gk & 7;
    uint32_t v[4][4];
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      float re[2], im[2];
#pragma unroll
      for (int y = 0; y < 2; ++y) {
        const int u = kc * 64 + g * 8 + 2 * x + y;
        re[y] = 0.f;
        im[y] = 0.f;
        if (row < Ng && u < w && rot_order_on(qmask, u - p)) {
          const double2 hv = h[p * p + u];
          const float2 ph = eg[(size_t)row * K + (Lh - 1) - p + u];   // (cos, sin)(q' gamma_c)
          const float hx = (float)hv.x, hy = (float)hv.y;
          re[y] = (hx * ph.x + hy * ph.y) * bsc;
          im[y] = (hy * ph.x - hx * ph.y) * bsc;
        }
      }
      const __half2 a2 = __floats2half2_rn(re[0], re[1]);
      const float2 af = __half22float2(a2);
      const __half2 b2 = __floats2half2_rn(re[0] - af.x, re[1] - af.y);
      const __half2 c2 = __floats2half2_rn(im[0], im[1]);
      const float2 cf = __half22float2(c2);
      const __half2 d2 = __floats2half2_rn(im[0] - cf.x, im[1] - cf.y);
      v[0][x] = *reinterpret_cast<const uint32_t*>(&a2);
      v[1][x] = *reinterpret_cast<const uint32_t*>(&b2);
      v[2][x] = *reinterpret_cast<const uint32_t*>(&c2);
      v[3][x] = *reinterpret_cast<const uint32_t*>(&d2);
    }
    const uint32_t off = sw128_off(row, g * 8);
#pragma unroll
    for (int part = 0; part < 4; ++part)
      *reinterpret_cast<uint4*>(dst + rt_wa_off(part, kc) + off) = make_uint4(v[part][0], v[part][1], v[part][2], v[part][3]);
  }
}

cudaError_t launch_rotwin_tc_window(const double2* h, const float2* eg, const uint32_t* qmask, int Lh, int Ng,
                                   void* wbuf, cudaStream_t st) {
  if (!rotwin_tc_supported(Lh, Ng)) return cudaErrorInvalidValue;
  unsigned char* wimg = (unsigned char*)wbuf;
  float* dsc = (float*)(wimg + (size_t)Lh * RT_WA_BYTES);
  k_rt_window<<<dim3(Lh, 4), 256, 0, st>>>(h, eg, qmask, Lh, Ng, wimg, dsc);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- the kernel
__global__ void __launch_bounds__(RT_THREADS, 1)
k_rotwin_tc(const unsigned char* __restrict__ img, const float* __restrict__ rs, const unsigned char* __restrict__ wimg,
            const float* __restrict__ dsc, int Lh, int Nb, int Ng, long long total_cost, float2* __restrict__ H,
            int* __restrict__ err, int wait_test) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* ring = sm + RT_WA_BYTES;
  RtBars* bars = reinterpret_cast<RtBars*>(ring + RT_RING * RT_STAGE);
  volatile int* abort_flag = &bars->abort_flag;
  const uint32_t wlim = wait_test ? (1u << 14) : TC_WAIT_LIMIT;   // short limit for the timeout test
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t0 = rt_first(total_cost * blockIdx.x / gridDim.x, Lh, Nb, Ng);
  const int t1 = rt_first(total_cost * (blockIdx.x + 1) / gridDim.x, Lh, Nb, Ng);

  if (threadIdx.x == 0) {
    for (int i = 0; i < RT_RING; ++i) {
      mbar_init(smem_u32(&bars->full[i]), 1);
      mbar_init(smem_u32(&bars->empty[i]), 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(smem_u32(&bars->acc_full[i]), 1);
      mbar_init(smem_u32(&bars->acc_empty[i]), RT_EPI_WARPS);
    }
    mbar_init(smem_u32(&bars->wfull), 1);
    mbar_init(smem_u32(&bars->wempty), 1);
    mbar_init(smem_u32(&bars->drain), 1);
    bars->abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {   // TMEM: two accumulators of 128 lanes x (Re, Im) x 128 FP32 columns
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                     smem_u32(&bars->tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = bars->tmem_base;

  if (warp == 0) {
    // ---------------- loader: the window operand of each degree (once its
    // previous one is no longer read) and the d chunk images, in tile order
    if (lane == 0) {
      int armed[RT_RING];
#pragma unroll
      for (int i = 0; i < RT_RING; ++i) armed[i] = -1;
      int w_armed = -1;
      RtPos s{0, 0, 0};
      int cur_p = -1;
      uint32_t wph = 0;
      long long bc = 0;
      bool ok = true;
      for (int t = t0; t < t1 && ok; ++t) {
        rt_seek(s, t, Nb, Lh);
        const int nc = rt_nch(s.p);
        if (s.p != cur_p) {
          if (cur_p >= 0 && !(ok = mbar_wait_n(smem_u32(&bars->wempty), wph ^ 1u, abort_flag, wlim))) break;
          const uint32_t fw = smem_u32(&bars->wfull);
          mbar_expect_tx(fw, 4 * nc * RT_PART);
          const unsigned char* src = wimg + (size_t)s.p * RT_WA_BYTES;
          for (int part = 0; part < 4; ++part)
            for (int kc = 0; kc < nc; ++kc)
              bulk_g2s(smem_u32(sm + rt_wa_off(part, kc)), src + rt_wa_off(part, kc), RT_PART, fw);
          w_armed = (int)wph;
          wph ^= 1u;
          cur_p = s.p;
        }
        const unsigned char* src = img + ((size_t)s.cb + (size_t)(t - s.tb) * nc) * RT_STAGE;
        for (int kc = 0; kc < nc; ++kc, ++bc) {
          const int sb = (int)(bc % RT_RING);
          const uint32_t pb = (uint32_t)((bc / RT_RING) & 1);
          if (!(ok = mbar_wait_n(smem_u32(&bars->empty[sb]), pb ^ 1u, abort_flag, wlim))) break;
          if (wait_test && bc == 0) continue;   // wait_test: the first d chunk is never fetched
          const uint32_t fb = smem_u32(&bars->full[sb]);
          mbar_expect_tx(fb, RT_STAGE);
          bulk_g2s(smem_u32(ring + sb * RT_STAGE), src + (size_t)kc * RT_STAGE, RT_PART, fb);
          bulk_g2s(smem_u32(ring + sb * RT_STAGE + RT_PART), src + (size_t)kc * RT_STAGE + RT_PART, RT_PART, fb);
#pragma unroll
          for (int i = 0; i < RT_RING; ++i)
            if (i == sb) armed[i] = (int)pb;
        }
      }
      if (!ok) *abort_flag = 1;
      // copies in flight land before the CTA may exit
      if (w_armed >= 0) {
        uint32_t n = 0;
        while (!mbar_test(smem_u32(&bars->wfull), (uint32_t)w_armed) && ++n < TC_WAIT_LIMIT) {}
      }
#pragma unroll
      for (int i = 0; i < RT_RING; ++i) {
        if (armed[i] >= 0) {
          uint32_t n = 0;
          while (!mbar_test(smem_u32(&bars->full[i]), (uint32_t)armed[i]) && ++n < TC_WAIT_LIMIT) {}
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer: D(c, n) = sum_k B_p(k, c) d(n, k), Re and Im
    if (lane == 0) {
      const uint32_t idesc = umma_idesc_f16(128, RT_ROWS);
      RtPos s{0, 0, 0};
      int cur_p = -1;
      uint32_t wph = 0;
      long long bc = 0;
      bool ok = true;
      int i = 0;
      for (int t = t0; t < t1 && ok; ++t, ++i) {
        rt_seek(s, t, Nb, Lh);
        if (s.p != cur_p) {
          // the previous degree's products release its window operand, then
          // the new degree's operand lands
          if (cur_p >= 0) umma_commit(smem_u32(&bars->wempty));
          if (!(ok = mbar_wait_n(smem_u32(&bars->wfull), wph, abort_flag, wlim))) break;
          wph ^= 1u;
          cur_p = s.p;
        }
        const int acc = i & 1;
        if (!(ok = mbar_wait_n(smem_u32(&bars->acc_empty[acc]), (uint32_t)(((i >> 1) & 1) ^ 1), abort_flag, wlim)))
          break;
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(acc * 256);   // Re columns 0..127, Im 128..255
        const int nc = rt_nch(s.p), ks_all = (2 * s.p + 1 + 15) >> 4;
        for (int kc = 0; kc < nc; ++kc, ++bc) {
          const int sb = (int)(bc % RT_RING);
          if (!(ok = mbar_wait_n(smem_u32(&bars->full[sb]), (uint32_t)((bc / RT_RING) & 1), abort_flag, wlim)))
            break;
          tc_fence_after();
          const uint64_t bh = sw128_desc(smem_u32(ring + sb * RT_STAGE));
          const uint64_t bl = sw128_desc(smem_u32(ring + sb * RT_STAGE + RT_PART));
          const int ks_n = min(4, ks_all - 4 * kc);
#pragma unroll
          for (int m = 0; m < 2; ++m) {    // Re, Im
            const uint64_t ah = sw128_desc(smem_u32(sm + rt_wa_off(2 * m, kc)));
            const uint64_t al = sw128_desc(smem_u32(sm + rt_wa_off(2 * m + 1, kc)));
            for (int ks = 0; ks < ks_n; ++ks) {   // K = 16 per MMA: +32 bytes
              const uint64_t o = (uint64_t)(2 * ks);
              umma_f16(d + (uint32_t)(m * 128), ah + o, bh + o, idesc, (kc | ks) != 0);
              umma_f16(d + (uint32_t)(m * 128), ah + o, bl + o, idesc, 1u);
              umma_f16(d + (uint32_t)(m * 128), al + o, bh + o, idesc, 1u);
            }
          }
          umma_commit(smem_u32(&bars->empty[sb]));
        }
        if (!ok) break;
        umma_commit(smem_u32(&bars->acc_full[acc]));
      }
      if (!ok) *abort_flag = 1;
      // every MMA issued by this thread completes before TMEM is released
      umma_commit(smem_u32(&bars->drain));
      uint32_t n = 0;
      while (!mbar_test(smem_u32(&bars->drain), 0u) && ++n < TC_WAIT_LIMIT) {}
    }
  } else {
    // ---------------- epilogue: warps 2..9, TMEM lane quadrant warp % 4 (the
    // gamma samples), half = which 64 of the tile's 128 rows
    const int quad = warp & 3, half = (warp - 2) >> 2;
    const int c = quad * 32 + lane;
    const int n2 = Lh * Lh;
    const size_t jstride = (size_t)n2 * 128;          // elements between 128-column tiles of H
    RtPos s{0, 0, 0};
    bool ok = true;
    int i = 0;
    for (int t = t0; t < t1 && ok; ++t, ++i) {
      rt_seek(s, t, Nb, Lh);
      const int p = s.p, w = 2 * p + 1, rt = t - s.tb;
      // this lane's row of each pass, ahead of the wait: its scale, beta row
      // (Nb or more: a padding row) and H row offset, broadcast per row below
      const float dinv = __ldg(dsc + p);
      float rsc[2];
      int rb[2], roff[2];
#pragma unroll
      for (int ps = 0; ps < 2; ++ps) {
        const int n = half * 64 + ps * 32 + lane;
        const int R = rt * RT_ROWS + n;
        const int bb = R / w;
        rsc[ps] = __ldg(rs + (size_t)t * RT_ROWS + n);
        rb[ps] = bb;
        roff[ps] = h_row(p, R - bb * w - p, Lh, h_order_major(Lh)) * 128;
      }
      const int acc = i & 1;
      // one lane waits, the warp follows: tcgen05.ld needs a converged warp
      int got = 0;
      if (lane == 0) got = mbar_wait_n(smem_u32(&bars->acc_full[acc]), (uint32_t)((i >> 1) & 1), abort_flag, wlim);
      got = __shfl_sync(0xffffffffu, got, 0);
      __syncwarp();
      if (!(ok = got != 0)) break;
      tc_fence_after();
      const uint32_t tb = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(acc * 256);
#pragma unroll 1
      for (int ps = 0; ps < 2; ++ps) {
        const int n0 = half * 64 + ps * 32;
        uint32_t vr[32], vi[32];
        TMEM_LD32(tb + (uint32_t)n0, vr);
        TMEM_LD32(tb + (uint32_t)(128 + n0), vi);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const float my_sc = (ps ? rsc[1] : rsc[0]) * dinv;
        const int my_b = ps ? rb[1] : rb[0], my_off = ps ? roff[1] : roff[0];
#pragma unroll
        for (int u = 0; u < 32; ++u) {
          const float sc = __shfl_sync(0xffffffffu, my_sc, u);
          const int bb = __shfl_sync(0xffffffffu, my_b, u);
          const int ro = __shfl_sync(0xffffffffu, my_off, u);
          const int j = bb * Ng + c;
          if (bb < Nb && c < Ng)
            __stcs(H + (size_t)(j >> 7) * jstride + ro + (j & 127),
                   make_float2(__uint_as_float(vr[u]) * sc, __uint_as_float(vi[u]) * sc));
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bars->acc_empty[acc]));
    }
    if (!ok) *abort_flag = 1;
  }
  __syncthreads();
  if (*abort_flag && threadIdx.x == 0) atomicExch(err, 1);
  tc_fence_after();
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
}

cudaError_t launch_rotwin_tc(const void* tab, const void* wbuf, int Lh, int Nb, int Ng, float2* H, int num_sms,
                             cudaStream_t st) {
  if (!rotwin_tc_supported(Lh, Ng) || Nb < 1) return cudaErrorInvalidValue;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_rotwin_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, RT_SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  int* err = tc_error_word();
  if (!err) return cudaErrorMemoryAllocation;
  int tiles;
  long long chunks;
  rt_counts(Lh, Nb, &tiles, &chunks);
  const unsigned char* img = (const unsigned char*)tab;
  const float* rs = (const float*)(img + (size_t)chunks * RT_STAGE);
  const unsigned char* wimg = (const unsigned char*)wbuf;
  const float* dsc = (const float*)(wimg + (size_t)Lh * RT_WA_BYTES);
  long long cost = 0;
  for (int p = 0; p < Lh; ++p) cost += rt_tiles_of(p, Nb) * rt_cost(p, Ng);
  const int grid = tiles < num_sms ? tiles : num_sms;
  k_rotwin_tc<<<grid, RT_THREADS, RT_SMEM, st>>>(img, rs, wimg, dsc, Lh, Nb, Ng, cost, H, err, tc_take_wait_test());
  return cudaGetLastError();
}

static_assert(sizeof(RtBars) <= 1024, "the CTA's bookkeeping fits the space RT_SMEM keeps for it");
static_assert(RT_SMEM <= 232448, "one CTA's shared memory");
