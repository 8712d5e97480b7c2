// FP32_BULK forward transform, rotated-window route, as ONE persistent
// tcgen05 kernel: the beta/gamma producer and the alpha stage fused.
//
// For one pair (l, m) and columns j = (beta_b, gamma_c) (Sec. IV-B,
// Eq. alternative_harmonic_formulation_wigner with the sums over q' and p
// regrouped):
//   X_q(j)   = sum_{p >= |q|} k_lm(p, q) H^p_q(j),
//   g[a][j]  = sum_q X_q(j) e^{-i q alpha_a},
// where H^p_q(j) = sum_q' h_p^q' d^p_{q,q'}(beta_b) e^{-i q' gamma_c} is the
// rotated window (pair independent, computed once per call).  The alpha sum
// is the real GEMM of the tensor-core alpha stage (same split-FP16 operands,
// same 128-byte swizzled K-major layout, same E tables); what changes is where
// A comes from: producer warps build the A tile of the next (pair, 128-column
// tile) item directly in shared memory while the tensor cores and the
// epilogue work on the current one, so the A operand never travels through
// HBM and no second kernel competes for the SMs.
//
// Warp roles (608 threads, one CTA per SM):
//   warp 0      streams E-table chunks (TC_NC = 64 alpha rows, 32 KB) into a
//               double-buffered B stage with cp.async.bulk;
//   warp 1      allocates TMEM, issues tcgen05.mma from one thread into four
//               128 x TC_N FP32 accumulators;
//   warps 2-9   X producers: thread t owns column j = tile*128 + (t & 127)
//               and the sign half t >> 7 of q; it sums k(p,q) H^p_q(j) for
//               its orders (H rows from a shared-memory ring, k broadcast
//               from shared memory), the two halves exchange the column
//               maximum, scale the column by 2^e (largest entry into
//               [2^14, 2^15)), split into FP16 hi/lo and write their halves
//               of the 128-byte swizzled A row; the per-column 2^-e goes to
//               shared memory beside the A stage;
//   warps 10-17 epilogue: TMEM -> registers, rescale, streaming stores of g;
//   warp 18     streams the item's H tile (H resident in L2, tiled so that
//               a tile's rows are contiguous) into a 5-stage ring of 16 rows
//               (16 KB a stage, one cp.async.bulk each).
// Hand-offs (mbarriers; every wait is bounded):
//   a_full[s]   X producers -> MMA and epilogue (256 arrivals, after a
//               proxy fence so the tensor core sees the generic stores);
//   a_empty[s]  MMA commit + every epilogue thread once it has read the
//               stage's scales -> X producers (257 arrivals);
//   h_full[s] / h_empty[s]  H ring: loader (+ bytes) -> producers (256
//               arrivals when a stage's rows are consumed) -> loader;
//   b_full[s] / b_empty[s]  E loader (+ bytes) -> MMA (commit) -> E loader;
//   acc_full[i] / acc_empty[i]  MMA (commit) -> epilogue (256 arrivals) -> MMA.
// On a bounded wait's expiry the CTA raises its abort flag, every role leaves
// its loop (the producer warps decide together through one named barrier so
// they cannot split), waits (bounded) for its copies and MMAs in flight,
// frees TMEM and exits; the host reads the error word.
#include <cuda_fp16.h>

#include "common.cuh"
#include "tc.cuh"
#include "tc_ptx.cuh"

#define FU_XWARPS 8
#define FU_X0 2                                  // first producer warp
#define FU_E0 (FU_X0 + FU_XWARPS)                // first epilogue warp
#define FU_HL (FU_E0 + TC_EPI_WARPS)             // H-ring loader warp
#define FU_THREADS (32 * (FU_HL + 1))            // 608
#define FU_XBAR 1                                // named barrier of the producer warps
#define FU_HR 16                                 // H rows per ring stage
#define FU_HS 5                                  // ring stages
#define FU_H_BYTES (FU_HS * FU_HR * TC_M * 8)    // 80 KB

#define FU_ACC 4                                 // TMEM accumulators (TC_N columns each)

struct FuShared {
  uint64_t a_full[2], a_empty[2], b_full[2], b_empty[2], acc_full[FU_ACC], acc_empty[FU_ACC], drain;
  uint64_t h_full[FU_HS], h_empty[FU_HS];
  uint32_t tmem_base;
  int abort_flag;
  int x_ok[2];
  float scale[2][TC_M];         // 2^-e per column of each A stage (0 beyond J)
  float xmax[2][TC_M];          // per-column partial maxima of the two q halves
  float2 k[2][16 * 16];         // coupling row of the item's pair, FP32
};

#define FU_SMEM (2 * TC_A_BYTES + 2 * TC_B_BYTES + FU_H_BYTES + 1024 + (int)sizeof(FuShared))

__device__ __forceinline__ uint32_t pack_h2(float a, float b, uint32_t* lo_word) {
  const __half ha = __float2half_rn(a), hb = __float2half_rn(b);
  const __half la = __float2half_rn(a - __half2float(ha)), lb = __float2half_rn(b - __half2float(hb));
  __half2 h = __halves2half2(ha, hb), l = __halves2half2(la, lb);
  *lo_word = *reinterpret_cast<uint32_t*>(&l);
  return *reinterpret_cast<uint32_t*>(&h);
}

__device__ __forceinline__ void named_bar_sync(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// LHB: compile-time bound on the window band limit (Lh <= LHB); rows of
// degree p >= Lh are read clamped to a valid row and weighted by k = 0.
__host__ __device__ constexpr int isqrt_c(int n) {
  int r = 0;
  while ((r + 1) * (r + 1) <= n) ++r;
  return r;
}

// One column's sums X_q = sum_p k(p,q) H^p_q over the item's H tile for one
// sign half of q (NEG: q in [-(LHB-1), 0] into accumulator q + LHB - 1;
// else q in [1, LHB-1] into accumulator q - 1), reading the ring stage by
// stage.  Every producer thread waits for and releases every stage.
template <int LHB, bool NEG>
__device__ __forceinline__ void accumulate_half(float* ar, float* ai, const float2* sH, const float2* sk, int col,
                                                FuShared* S, int& h_slot, uint32_t& h_phase,
                                                volatile int* abort_flag, uint32_t wlim) {
  constexpr int NST = LHB * LHB / FU_HR;
#pragma unroll
  for (int st = 0; st < NST; ++st) {
    const int slot = h_slot;
    // on expiry: raise the abort flag and go on with stale rows (in bounds);
    // the item is dropped at the next hand-off
    if (!mbar_wait_n(smem_u32(&S->h_full[slot]), h_phase, abort_flag, wlim)) *abort_flag = 1;
    if (++h_slot == FU_HS) { h_slot = 0; h_phase ^= 1u; }
    const float2* hst = sH + (size_t)slot * FU_HR * TC_M + col;
#pragma unroll
    for (int r = 0; r < FU_HR; ++r) {
      const int pq = st * FU_HR + r;
      const int p = isqrt_c(pq), q = pq - p * p - p;
      if (NEG ? (q > 0) : (q <= 0)) continue;
      const int a = NEG ? q + LHB - 1 : q - 1;
      const float2 hv = hst[r * TC_M];
      const float2 kv = sk[pq];
      ar[a] = fmaf(kv.x, hv.x, ar[a]);
      ar[a] = fmaf(-kv.y, hv.y, ar[a]);
      ai[a] = fmaf(kv.x, hv.y, ai[a]);
      ai[a] = fmaf(kv.y, hv.x, ai[a]);
    }
    mbar_arrive(smem_u32(&S->h_empty[slot]));
  }
}

template <int LHB>
__global__ void __launch_bounds__(FU_THREADS, 1)
k_alpha_fused(const double2* __restrict__ kc, const float2* __restrict__ H, int Lh, int J, int tiles,
              const unsigned char* __restrict__ etab, int Na, int npairs, float2* __restrict__ g,
              int* __restrict__ err, uint32_t wlim, int wait_test, const int2* __restrict__ slots) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sA = sm;                               // 2 x 32 KB
  unsigned char* sB = sm + 2 * TC_A_BYTES;              // 2 x 32 KB (double-buffered E chunk)
  float2* sH = reinterpret_cast<float2*>(sB + 2 * TC_B_BYTES);   // [stage][row][128 columns]
  FuShared* S = reinterpret_cast<FuShared*>(sB + 2 * TC_B_BYTES + FU_H_BYTES);
  volatile int* abort_flag = &S->abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nch = (Na + TC_NC - 1) / TC_NC;
  const long long nitems = (long long)npairs * tiles;
  const int n2 = Lh * Lh;
  constexpr int NST = LHB * LHB / FU_HR;         // ring stages per item
  static_assert(LHB * LHB % FU_HR == 0, "whole ring stages per item");

  if (threadIdx.x == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(smem_u32(&S->a_full[i]), 32 * FU_XWARPS);
      mbar_init(smem_u32(&S->a_empty[i]), 1 + 32 * TC_EPI_WARPS);
      mbar_init(smem_u32(&S->b_full[i]), 1);
      mbar_init(smem_u32(&S->b_empty[i]), 1);
    }
    for (int i = 0; i < FU_ACC; ++i) {
      mbar_init(smem_u32(&S->acc_full[i]), 1);
      mbar_init(smem_u32(&S->acc_empty[i]), 32 * TC_EPI_WARPS);
    }
    mbar_init(smem_u32(&S->drain), 1);
    for (int i = 0; i < FU_HS; ++i) {
      mbar_init(smem_u32(&S->h_full[i]), 1);
      mbar_init(smem_u32(&S->h_empty[i]), 32 * FU_XWARPS);
    }
    S->abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {   // TMEM: 512 columns = FU_ACC accumulators of 128 x TC_N FP32
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                     smem_u32(&S->tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S->tmem_base;

  if (warp == 0) {
    // ---------------- E-table loader
    if (lane == 0) {
      int b_armed[2] = {-1, -1};
      long long bc = 0;
      bool ok = true;
      for (long long it = blockIdx.x; it < nitems && ok; it += gridDim.x) {
        for (int c = 0; c < nch; ++c, ++bc) {
          const int sb = (int)(bc & 1);                    // E stage of this chunk
          const uint32_t pb = (uint32_t)((bc >> 1) & 1);   // its use parity
          if (!(ok = mbar_wait_n(smem_u32(&S->b_empty[sb]), pb ^ 1u, abort_flag, wlim))) break;
          const uint32_t fb = smem_u32(&S->b_full[sb]);
          mbar_expect_tx(fb, TC_B_BYTES);
          const unsigned char* bsrc = etab + (size_t)c * TC_B_BYTES;
          for (int o = 0; o < TC_B_BYTES; o += 16384)
            bulk_g2s(smem_u32(sB + sb * TC_B_BYTES + o), bsrc + o, 16384, fb);
          if (sb == 0) b_armed[0] = (int)pb; else b_armed[1] = (int)pb;
        }
      }
      if (!ok) *abort_flag = 1;
      for (int i = 0; i < 2; ++i) {   // copies in flight must land before the CTA may exit
        if (b_armed[i] >= 0) {
          uint32_t n = 0;
          while (!mbar_test(smem_u32(&S->b_full[i]), (uint32_t)b_armed[i]) && ++n < TC_WAIT_LIMIT) {}
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
        const int sa = li & 1;
        if (!(ok = mbar_wait_n(smem_u32(&S->a_full[sa]), (uint32_t)((li >> 1) & 1), abort_flag, wlim))) break;
        tc_fence_after();
        const uint32_t a_hi = smem_u32(sA + sa * TC_A_BYTES), a_lo = a_hi + TC_A_HALF;
        for (int c = 0; c < nch; ++c, ++bc, ++ac) {
          const int acc = (int)(ac % FU_ACC);
          const int sb = (int)(bc & 1);
          if (!(ok = mbar_wait_n(smem_u32(&S->b_full[sb]), (uint32_t)((bc >> 1) & 1), abort_flag, wlim))) break;
          if (!(ok = mbar_wait_n(smem_u32(&S->acc_empty[acc]), (uint32_t)(((ac / FU_ACC) & 1) ^ 1), abort_flag,
                                 wlim)))
            break;
          tc_fence_after();
          const uint32_t b_hi = smem_u32(sB + sb * TC_B_BYTES), b_lo = b_hi + TC_B_HALF;
          const uint32_t d = tmem + (uint32_t)(acc * TC_N);
          const uint32_t as[3] = {a_hi, a_hi, a_lo};
          const uint32_t bs[3] = {b_hi, b_lo, b_hi};
#pragma unroll
          for (int pr = 0; pr < 3; ++pr) {
            const uint64_t ad = sw128_desc(as[pr]), bd = sw128_desc(bs[pr]);
#pragma unroll
            for (int s = 0; s < TC_KB / 16; ++s)       // K = 16 per MMA: +32 bytes
              umma_f16(d, ad + (uint64_t)(2 * s), bd + (uint64_t)(2 * s), idesc, (pr | s) != 0);
          }
          umma_commit(smem_u32(&S->b_empty[sb]));
          umma_commit(smem_u32(&S->acc_full[acc]));
        }
        if (!ok) break;
        umma_commit(smem_u32(&S->a_empty[sa]));
      }
      if (!ok) *abort_flag = 1;
      // every MMA issued by this thread completes before TMEM is released
      umma_commit(smem_u32(&S->drain));
      uint32_t n = 0;
      while (!mbar_test(smem_u32(&S->drain), 0u) && ++n < TC_WAIT_LIMIT) {}
    }
  } else if (warp < FU_E0) {
    // ---------------- X producers: thread x owns column x & 127 and the
    // half x >> 7 of the orders q (0: q <= 0, 1: q > 0)
    const int x = threadIdx.x - 32 * FU_X0;
    const int col = x & (TC_M - 1);
    const int neg = x < TC_M;                     // warp-uniform
    int li = 0;
    int h_slot = 0;              // ring position of the next stage and its phase parity
    uint32_t h_phase = 0;
    for (long long it = blockIdx.x; it < nitems; it += gridDim.x, ++li) {
      const int pair = (int)(it / tiles), tile = (int)(it % tiles);
      const int sa = li & 1;
      // the pair's coupling row, FP32, zero beyond the band (double-buffered
      // by item parity: the named barrier of the previous item separates
      // these writes from the last reads of the same buffer)
      float2* sk = S->k[sa];
      for (int t = x; t < LHB * LHB; t += 32 * FU_XWARPS) {
        float2 v = make_float2(0.f, 0.f);
        if (t < n2) {
          const double2 dv = kc[(size_t)pair * n2 + t];
          v = make_float2((float)dv.x, (float)dv.y);
        }
        sk[t] = v;
      }
      if (x == 0)
        S->x_ok[sa] = mbar_wait_n(smem_u32(&S->a_empty[sa]), (uint32_t)(((li >> 1) & 1) ^ 1), abort_flag, wlim) ? 1 : 0;
      named_bar_sync(FU_XBAR, 32 * FU_XWARPS);
      if (!S->x_ok[sa]) break;          // uniform across the producer warps

      const int j = tile * TC_M + col;
      const bool jin = j < J;
      // accumulator i: q = i - (LHB - 1) (neg half) or q = i + 1 (other half)
      float ar[LHB], ai[LHB];
#pragma unroll
      for (int i = 0; i < LHB; ++i) ar[i] = ai[i] = 0.f;
      if (neg)
        accumulate_half<LHB, true>(ar, ai, sH, sk, col, S, h_slot, h_phase, abort_flag, wlim);
      else
        accumulate_half<LHB, false>(ar, ai, sH, sk, col, S, h_slot, h_phase, abort_flag, wlim);
      if (!jin) {            // padding columns of the last tile: exact zeros
#pragma unroll
        for (int i = 0; i < LHB; ++i) ar[i] = ai[i] = 0.f;
      }
      // the column's largest entry over both halves
      float mx = 0.f;
#pragma unroll
      for (int i = 0; i < LHB; ++i) mx = fmaxf(mx, fmaxf(fabsf(ar[i]), fabsf(ai[i])));
      S->xmax[neg][col] = mx;
      named_bar_sync(FU_XBAR, 32 * FU_XWARPS);
      mx = fmaxf(mx, S->xmax[!neg][col]);
      int ex = 0;
      if (mx > 0.f) frexpf(mx, &ex);
      const int e = mx > 0.f ? min(125, max(-125, 15 - ex)) : 0;
      const float sc = jin ? __int_as_float((127 + e) << 23) : 0.f;
      if (neg) S->scale[sa][col] = jin ? __int_as_float((127 - e) << 23) : 0.f;
      // A row of the column: slot k = 15 + q holds Re X_q, 47 + q holds Im X_q.
      // The neg half writes the 16-byte chunks 0, 1, 4, 5 (q in [-15, 0]),
      // the other half 2, 3, 6, 7 (q in [1, 15] and the two zero slots).
      unsigned char* ahi = sA + sa * TC_A_BYTES;
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        const int c = (cc & 1) + 4 * (cc >> 1) + (neg ? 0 : 2);
        uint32_t wh[4], wl[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          float val[2];
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int k = 8 * ((cc & 1) + 4 * (cc >> 1)) + 2 * v + u;   // slot in the neg half's chunks
            // the neg half's slot k maps to q = (k & 31) - 15 <= 0; the other
            // half's slot k + 16 maps to q = (k & 31) + 1
            float y;
            if (neg) {
              const int q = (k & 31) - 15;
              y = (q > -LHB) ? ((k < 32) ? ar[q + LHB - 1] : ai[q + LHB - 1]) : 0.f;
            } else {
              const int q = (k & 31) + 1;
              y = (q < LHB && (k & 31) < 15) ? ((k < 32) ? ar[q - 1] : ai[q - 1]) : 0.f;
            }
            val[u] = y * sc;
          }
          wh[v] = pack_h2(val[0], val[1], &wl[v]);
        }
        *reinterpret_cast<uint4*>(ahi + sw128_off(col, 8 * c)) = make_uint4(wh[0], wh[1], wh[2], wh[3]);
        *reinterpret_cast<uint4*>(ahi + TC_A_HALF + sw128_off(col, 8 * c)) = make_uint4(wl[0], wl[1], wl[2], wl[3]);
      }
      // generic-proxy stores -> visible to the tensor core's async proxy
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      // wait_test: the first item's A tile is never handed over, so the
      // issuer's and the epilogue's bounded waits run out (timeout path test)
      if (!(wait_test && li == 0)) mbar_arrive(smem_u32(&S->a_full[sa]));
    }
  } else if (warp == FU_HL) {
    // ---------------- H-ring loader: the item's n2 rows, FU_HR rows a stage
    if (lane == 0) {
      int armed[FU_HS];
#pragma unroll
      for (int i = 0; i < FU_HS; ++i) armed[i] = -1;
      int slot = 0;
      uint32_t use = 0;
      bool ok = true;
      for (long long it = blockIdx.x; it < nitems && ok; it += gridDim.x) {
        const int tile = (int)(it % tiles);
        for (int s = 0; s < NST; ++s) {
          if (!(ok = mbar_wait_n(smem_u32(&S->h_empty[slot]), use ^ 1u, abort_flag, wlim))) break;
          const uint32_t fb = smem_u32(&S->h_full[slot]);
          mbar_expect_tx(fb, (uint32_t)(FU_HR * TC_M * 8));
          const float2* tsrc = H + (size_t)tile * n2 * TC_M;        // the tile's rows, contiguous
          float2* dst = sH + (size_t)slot * FU_HR * TC_M;
          if ((s + 1) * FU_HR <= n2) {
            bulk_g2s(smem_u32(dst), tsrc + (size_t)s * FU_HR * TC_M, FU_HR * TC_M * 8, fb);
          } else {
            for (int r = 0; r < FU_HR; ++r) {               // rows beyond the band: any valid row
              const int row = min(s * FU_HR + r, n2 - 1);
              bulk_g2s(smem_u32(dst + (size_t)r * TC_M), tsrc + (size_t)row * TC_M, TC_M * 8, fb);
            }
          }
#pragma unroll
          for (int i = 0; i < FU_HS; ++i)
            if (i == slot) armed[i] = (int)use;
          if (++slot == FU_HS) { slot = 0; use ^= 1u; }
        }
      }
      if (!ok) *abort_flag = 1;
      // copies in flight must land before the CTA may exit
#pragma unroll
      for (int i = 0; i < FU_HS; ++i) {
        if (armed[i] >= 0) {
          uint32_t n = 0;
          while (!mbar_test(smem_u32(&S->h_full[i]), (uint32_t)armed[i]) && ++n < TC_WAIT_LIMIT) {}
        }
      }
    }
  } else {
    // ---------------- epilogue: TMEM lane quadrant = warp % 4, half = which
    // TC_NC / 2 of the chunk's TC_NC alpha rows
    const int quad = warp & 3;
    const int half = (warp - FU_E0) >> 2;
    const int row = quad * 32 + lane;
    long long ac = 0;
    int li = 0;
    bool ok = true;
    for (long long it = blockIdx.x; it < nitems && ok; it += gridDim.x, ++li) {
      const int pair = (int)(it / tiles), tile = (int)(it % tiles);
      const int sa = li & 1;
      const int j = tile * TC_M + row;
      const bool jin = j < J;
      // the item's scales: every lane waits for the A stage itself, then
      // releases it (its MMAs release it too)
      const int w_ok = mbar_wait_n(smem_u32(&S->a_full[sa]), (uint32_t)((li >> 1) & 1), abort_flag, wlim) ? 1 : 0;
      if (!(ok = __all_sync(0xffffffffu, w_ok) != 0)) break;
      const float sc = S->scale[sa][row];
      mbar_arrive(smem_u32(&S->a_empty[sa]));
      // output slot of the pair and, for a mirrored pair, of (l, -m) with its sign
      const int2 sl = slots != nullptr ? slots[pair] : make_int2(pair, -1);
      float2* gp = g + (size_t)sl.x * Na * J + (jin ? j : 0);
      float2* gm = sl.y >= 0 ? g + (size_t)(sl.y >> 1) * Na * J + (jin ? j : 0) : nullptr;
      const float msc = (sl.y & 1) ? -sc : sc;
      for (int c = 0; c < nch; ++c, ++ac) {
        const int acc = (int)(ac % FU_ACC);
        // one lane waits, the warp follows: tcgen05.ld needs a converged warp
        int got = 0;
        if (lane == 0) got = mbar_wait_n(smem_u32(&S->acc_full[acc]), (uint32_t)((ac / FU_ACC) & 1), abort_flag, wlim);
        got = __shfl_sync(0xffffffffu, got, 0);
        __syncwarp();
        if (!(ok = got != 0)) break;
        tc_fence_after();
        const uint32_t tbase = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(acc * TC_N);
#pragma unroll 1
        for (int cb = half * (TC_NC / 2); cb < half * (TC_NC / 2) + TC_NC / 2; cb += 16) {
          uint32_t vr[16], vi[16];
          TMEM_LD16(tbase + (uint32_t)cb, vr);
          TMEM_LD16(tbase + (uint32_t)(TC_NC + cb), vi);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          const int a0 = c * TC_NC + cb;
          if (jin) {
            float2* p = gp + (size_t)a0 * J;
            if (a0 + 16 <= Na) {
#pragma unroll
              for (int u = 0; u < 16; ++u) {
                __stcs(p, make_float2(__uint_as_float(vr[u]) * sc, __uint_as_float(vi[u]) * sc));
                p += J;
              }
            } else {
#pragma unroll
              for (int u = 0; u < 16; ++u) {
                if (a0 + u < Na) __stcs(p, make_float2(__uint_as_float(vr[u]) * sc, __uint_as_float(vi[u]) * sc));
                p += J;
              }
            }
          }
          if (jin && gm != nullptr) {     // (l, -m): (-1)^m conj g (real f and h)
            float2* p = gm + (size_t)a0 * J;
#pragma unroll
            for (int u = 0; u < 16; ++u) {
              if (a0 + u < Na)
                __stcs(p, make_float2(__uint_as_float(vr[u]) * msc, -__uint_as_float(vi[u]) * msc));
              p += J;
            }
          }
        }
        tc_fence_before();
        mbar_arrive(smem_u32(&S->acc_empty[acc]));
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

template <int LHB>
static cudaError_t launch_fused_t(const double2* kc, const float2* H, const void* etab, int Lh, int Na, int J,
                                  int tiles, int npairs, float2* g, int* err, int grid, int wait_test,
                                  const int2* slots, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_alpha_fused<LHB>, cudaFuncAttributeMaxDynamicSharedMemorySize, FU_SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  // the wait test uses a short limit so the expiry comes quickly
  const uint32_t wlim = wait_test ? (1u << 14) : TC_WAIT_LIMIT;
  k_alpha_fused<LHB><<<grid, FU_THREADS, FU_SMEM, st>>>(kc, H, Lh, J, tiles, (const unsigned char*)etab, Na,
                                                        npairs, g, err, wlim, wait_test, slots);
  return cudaGetLastError();
}

cudaError_t launch_alpha_fused(const double2* kc, const float2* H, const void* etab, int Lh, int Na, int Nb,
                               int Ng, int npairs, float2* g, int num_sms, int wait_test, const int2* slots,
                               cudaStream_t st) {
  if (npairs <= 0) return cudaSuccess;
  if (!tc_supported(Lh, Na) || Lh > 16) return cudaErrorInvalidValue;
  // bulk copies of whole 1 KB rows of the tiled H need a 16-byte aligned base
  if (((uintptr_t)H & 15) != 0) return cudaErrorInvalidValue;
  int* err = tc_error_word();
  if (!err) return cudaErrorMemoryAllocation;
  const int J = Nb * Ng;
  const int tiles = (J + TC_M - 1) / TC_M;
  const long long items = (long long)npairs * tiles;
  const int grid = (int)(items < num_sms ? items : num_sms);
  if (Lh <= 4) return launch_fused_t<4>(kc, H, etab, Lh, Na, J, tiles, npairs, g, err, grid, wait_test, slots, st);
  if (Lh <= 8) return launch_fused_t<8>(kc, H, etab, Lh, Na, J, tiles, npairs, g, err, grid, wait_test, slots, st);
  return launch_fused_t<16>(kc, H, etab, Lh, Na, J, tiles, npairs, g, err, grid, wait_test, slots, st);
}
