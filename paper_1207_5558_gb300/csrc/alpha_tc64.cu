// FP64 alpha stage on the tensor cores for L_h <= 16: the contraction
//   g[a][j] = sum_{|q| < L_h} X_q[j] e^{-i q alpha_a}
// evaluated to double precision from exact integer products.
//
// Operands.  Per column j, X (formed in double-float arithmetic from the
// double-float window H and couplings k) is scaled by 2^-e_j so that its
// largest component lies in [0.5, 1) and cut into S = 7 signed base-256
// digits, x = sum_{i=1..7} d_i 256^-i + r (|d_1| <= 256, |d_i| <= 129, |r| <
// 256^-7); the table entries cos and sin (q alpha_a) are cut the same way,
// e = sum_{j=1..7} c_j 256^-j.  Every digit is an integer that FP16 holds
// exactly.  The real GEMM layout is the narrow engine's (K = 64 slots: Re X_q
// at 15 + q, Im X_q at 47 + q; B rows n < 16: (cos | sin), rows 16 + n:
// (-sin | cos) of alpha row 16 c + n), one GEMM per digit pair (i, j).
//
// Exactness.  A digit product is at most 2^16 and K has at most 62 non-zero
// terms, so the sum over the products of one weight w = i + j (at most w - 1
// of them) stays below 2^24 in magnitude: every partial sum is an integer
// that FP32 represents exactly, whatever the order of accumulation.  The
// 28 products with w <= 8 go to seven TMEM accumulators A_w (w = 2..8), each
// exact; the dropped products (w >= 9) are below 2^-50 of the column's scale.
//   x e = 2^-16 sum_{w=2..8} A_w 256^-(w-2),
// combined in the epilogue with error-free transformations (TwoSum, dd.cuh)
// for the three leading weights and FP32 sums for the tail (below 2^-48
// relative), then assembled as a double with integer operations
// (dd_to_double).  No FP64 instruction runs per sample.
//
// Kernels: k_tc64_etab (the digit tables, once per N_alpha), k_xa64 (per
// (pair, 128-column tile): X in double-float, the column scale and the seven
// digit operands, swizzled), k_alpha_tc64 (persistent, one CTA per SM, item =
// (pair, tile)): a loader warp (the item's 7 x 16 KB of A resident; the
// 7 x 4 KB B digits of each 16-row alpha chunk through a 3-stage ring), an
// MMA warp (per chunk 7 x 4 MMAs of 128 x 32(7 - i) x 16, one per A digit
// i and K step, into one of two accumulator sets of 7 x 32 TMEM columns), sixteen epilogue warps (combine, store
// complex128 g: the epilogue's integer and FP32 work per sample is the
// kernel's bound, so it gets the warps).  Every mbarrier wait is bounded; on expiry the CTA raises its
// abort flag, waits (bounded) for its copies and MMAs in flight, frees TMEM and
// exits, and the host reads the shared error word.
#include <cuda_fp16.h>

#include "common.cuh"
#include "dd.cuh"
#include "tc.cuh"
#include "tc_ptx.cuh"

#define T64_S 7                         // base-256 digits per operand
#define T64_NW 7                        // accumulators: weights 2..8
#define T64_NA 16                       // alpha rows per chunk
#define T64_N (2 * T64_NA)              // MMA N (Re and Im rows)
#define T64_A_SLICE (TC_M * TC_KB * 2)  // 16 KB: one digit of a 128-column tile
#define T64_B_SLICE (T64_N * TC_KB * 2) // 4 KB: one digit of an alpha chunk
#define T64_A_BYTES (T64_S * T64_A_SLICE)
#define T64_B_BYTES (T64_S * T64_B_SLICE)
#define T64_BS 3                        // B ring stages
#define T64_SET (T64_NW * T64_N)        // TMEM columns of one accumulator set (224)
#define T64_SMEM (T64_A_BYTES + T64_BS * T64_B_BYTES + 1024 + 256)
#ifndef T64_EPI_WARPS
#define T64_EPI_WARPS 16                // four per TMEM lane quadrant, 4 alpha rows each (8: two, 8 rows)
#endif
#define T64_RPW (4 * T64_NA / T64_EPI_WARPS)   // alpha rows per epilogue warp and chunk
#define T64_THREADS (64 + 32 * T64_EPI_WARPS)

static inline int t64_tiles(int Nb, int Ng) { return (Nb * Ng + TC_M - 1) / TC_M; }
static inline int t64_chunks(int Na) { return (Na + T64_NA - 1) / T64_NA; }

bool tc64_supported(int Lh, int Na) { return Lh >= 1 && Lh <= 16 && Na >= 1; }

size_t tc64_etab_bytes(int Na) { return (size_t)t64_chunks(Na) * T64_B_BYTES; }

// per pair: tiles x 7 x 16 KB of A digits, then one int exponent per padded column
static inline size_t t64_scales_bytes(size_t tiles) { return ((tiles * TC_M * sizeof(int)) + 1023) / 1024 * 1024; }
size_t tc64_xblob_bytes(int Nb, int Ng) {
  const size_t t = (size_t)t64_tiles(Nb, Ng);
  return t * T64_A_BYTES + t64_scales_bytes(t);
}

// ---------------------------------------------------------------- digit tables
// chunk c at c * T64_B_BYTES: digit j (0..6) at + j * 4 KB, 32 rows x 64 slots
// swizzled; row n < 16 -> alpha a = 16 c + n: cos(q alpha) at slot 15 + q,
// sin at 47 + q; row 16 + n: -sin | cos.  All |q| <= 15 (the A operand is
// zero beyond the window); zeros beyond Na.
__global__ void k_tc64_etab(unsigned char* __restrict__ etab, int Na) {
  const int c = blockIdx.x;
  unsigned char* base = etab + (size_t)c * T64_B_BYTES;
  for (int t = threadIdx.x; t < T64_N * TC_KB; t += blockDim.x) {
    const int r = t / TC_KB, k = t % TC_KB;
    const int n = r % T64_NA, a = c * T64_NA + n;
    double v = 0.0;
    if (a < Na && (k & 31) < 31) {
      const int q = (k & 31) - 15;
      double s, co;
      sincos_2pi_frac((long long)q * a, Na, &s, &co);
      const bool is_sin = k >= 32;
      v = r < T64_NA ? (is_sin ? s : co) : (is_sin ? co : -s);
    }
    // base-256 digits with round to nearest: each step exact in FP64
    for (int j = 0; j < T64_S; ++j) {
      v *= 256.0;
      const double d = rint(v);
      v -= d;
      *reinterpret_cast<__half*>(base + j * T64_B_SLICE + sw128_off(r, k)) = __double2half((double)d);
    }
  }
}

cudaError_t launch_tc64_etab(void* etab, int Na, cudaStream_t st) {
  if (Na < 1) return cudaErrorInvalidValue;
  k_tc64_etab<<<t64_chunks(Na), 256, 0, st>>>((unsigned char*)etab, Na);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- A digits from H
// One CTA per (128-column tile, pair):
//   phase 1: one item per (q, column): X_q = sum_{p>=|q|} k(p,q) H^p_q in
//            double-float (inputs scaled by 2^-kexp and 2^-hexp) into the
//            shared tile sX[slot][column] (Re at 15 + q, Im at 47 + q, as
//            (hi, lo) float pairs; unused slots zero);
//   phase 2: per column, the exponent e_j of its largest |hi|;
//   phase 3: per (column, 8 slots): x 2^-e_j cut into 7 digits (each step
//            exact: a power-of-two scaling, a rounding to an integer, an exact
//            subtraction, TwoSum renormalisation), stored swizzled, one
//            16-byte row segment per digit.  The column's output exponent
//            e_j + kexp + hexp - 16 goes to the scales.  Columns beyond J: zeros.
__global__ void __launch_bounds__(256)
k_xa64(const float4* __restrict__ kdd, const int* __restrict__ kexp, const float4* __restrict__ Hdd,
       const int* __restrict__ hexp, int Lh, int J, unsigned char* __restrict__ xblob, size_t blob_stride,
       int tiles) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* sX = reinterpret_cast<float2*>(smem_raw);                // [TC_KB][TC_M]
  int* sEx = reinterpret_cast<int*>(sX + (size_t)TC_KB * TC_M);     // [TC_M]
  const int tile = blockIdx.x, pair = blockIdx.y;
  const int n2 = Lh * Lh;
  const float4* kp = kdd + (size_t)pair * n2;
  const int jt = tile * TC_M;
  for (int it = threadIdx.x; it < 32 * TC_M; it += blockDim.x) {
    const int u = it / TC_M, r = it % TC_M;
    const int q = u - 15, aq = q < 0 ? -q : q;
    const int j = jt + r;
    dd_acc xr = dd_acc_zero(), xi = dd_acc_zero();
    if (u < 31 && aq < Lh && j < J) {
      for (int p0 = aq; p0 < Lh; p0 += 4) {
        float4 hv[4], kv[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int p = p0 + v;
          if (p < Lh) {
            const int pq = p * p + p + q;
            hv[v] = __ldg(Hdd + h_index(pq, j, n2));
            kv[v] = __ldg(kp + pq);
          } else {
            hv[v] = make_float4(0.f, 0.f, 0.f, 0.f);
            kv[v] = make_float4(0.f, 0.f, 0.f, 0.f);
          }
        }
#pragma unroll
        for (int v = 0; v < 4; ++v) {      // k H: (kr hr - ki hi) + i (kr hi + ki hr)
          dd_mac(xr, kv[v].x, kv[v].z, hv[v].x, hv[v].z);
          dd_mac(xr, -kv[v].y, -kv[v].w, hv[v].y, hv[v].w);
          dd_mac(xi, kv[v].x, kv[v].z, hv[v].y, hv[v].w);
          dd_mac(xi, kv[v].y, kv[v].w, hv[v].x, hv[v].z);
        }
      }
    }
    float rh, rl, ih, il;
    dd_acc_get(xr, &rh, &rl);
    dd_acc_get(xi, &ih, &il);
    sX[u * TC_M + r] = make_float2(rh, rl);
    sX[(32 + u) * TC_M + r] = make_float2(ih, il);
  }
  __syncthreads();
  const int sc0 = kexp[pair] + *hexp - 16;
  for (int r = threadIdx.x; r < TC_M; r += blockDim.x) {
    float mx = 0.f;
#pragma unroll 8
    for (int k = 0; k < TC_KB; ++k) mx = fmaxf(mx, fabsf(sX[k * TC_M + r].x));
    int ex = 0;
    if (mx > 0.f) frexpf(mx, &ex);   // mx 2^-ex in [0.5, 1)
    sEx[r] = mx > 0.f ? max(-126, min(126, ex)) : 0;
  }
  __syncthreads();
  unsigned char* blob = xblob + (size_t)pair * blob_stride;
  unsigned char* tb = blob + (size_t)tile * T64_A_BYTES;
  int* scales = reinterpret_cast<int*>(blob + (size_t)tiles * T64_A_BYTES);
  for (int it = threadIdx.x; it < TC_M * (TC_KB / 8); it += blockDim.x) {
    const int r = it % TC_M, k0 = (it / TC_M) * 8;
    const int ex = sEx[r];
    const float down = __int_as_float((127 - ex) << 23);          // 2^-ex, |ex| <= 126
    __align__(16) __half dg[T64_S][8];
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      const float2 x = sX[(k0 + v) * TC_M + r];
      float h = x.x * down, l = x.y * down;                        // exact: powers of two
#pragma unroll
      for (int i = 0; i < T64_S; ++i) {
        h *= 256.f;
        l *= 256.f;
        const float d = rintf(h);
        h -= d;                                                    // exact (|h - d| <= 1/2)
        float e;
        h = two_sum(h, l, &e);                                     // renormalise the remainder
        l = e;
        dg[i][v] = __float2half_rn(d);                             // an integer, |d| <= 256
      }
    }
#pragma unroll
    for (int i = 0; i < T64_S; ++i)
      *reinterpret_cast<uint4*>(tb + i * T64_A_SLICE + sw128_off(r, k0)) = *reinterpret_cast<uint4*>(dg[i]);
    if (k0 == 0) scales[jt + r] = sc0 + ex;
  }
}

static size_t xa64_smem() { return sizeof(float2) * (size_t)TC_KB * TC_M + sizeof(int) * TC_M; }

cudaError_t launch_xa64(const float4* kdd, const int* kexp, const float4* Hdd, const int* hexp, int Lh, int Nb,
                        int Ng, int npairs, void* xblob, cudaStream_t st) {
  if (npairs <= 0) return cudaSuccess;
  if (Lh < 1 || Lh > 16 || npairs > 65535) return cudaErrorInvalidValue;
  if (!kdd || !kexp || !Hdd || !hexp || !xblob) return cudaErrorInvalidValue;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_xa64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xa64_smem());
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int tiles = t64_tiles(Nb, Ng);
  dim3 grid(tiles, npairs);
  k_xa64<<<grid, 256, xa64_smem(), st>>>(kdd, kexp, Hdd, hexp, Lh, Nb * Ng, (unsigned char*)xblob,
                                         tc64_xblob_bytes(Nb, Ng), tiles);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- the kernel
#define TMEM_LD4(taddr, v)                                                                          \
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"                         \
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])                                     \
               : "r"(taddr))
#define TMEM_LD8(taddr, v)                                                                          \
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"             \
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), \
                 "=r"(v[7])                                                                         \
               : "r"(taddr))

struct T64Bars {
  uint64_t a_full, a_empty, b_full[T64_BS], b_empty[T64_BS], acc_full[2], acc_empty[2], drain;
  uint32_t tmem_base;
  int abort_flag;
};

// sum_{w=2..8} A_w 256^-(w-2) (a[w-2], integers below 2^24) as a double-float.
// The three leading weights by TwoSum: s2 + e1 + e2 is their exact sum (and
// e1 = 0 or e2 = 0 wherever s or s2 cancels, the partial sums then being
// exact multiples of 2^-8 or 2^-16 below 2^16 or 2^8); the tail (weights 5..8,
// about 2^-24 of the lead) and the two error terms in FP32, so the only
// roundings fall on terms of order 2^-24 of the result.
__device__ __forceinline__ void t64_combine(const float* a, float* h, float* l) {
  const float tail = fmaf(a[3], 0x1p-24f, fmaf(a[4], 0x1p-32f, fmaf(a[5], 0x1p-40f, a[6] * 0x1p-48f)));
  float e1, e2;
  const float s = two_sum(a[0], a[1] * 0x1p-8f, &e1);
  const float s2 = two_sum(s, a[2] * 0x1p-16f, &e2);
  const float err = (e1 + e2) + tail;
  *h = two_sum(s2, err, l);
}

// The same for the real and imaginary parts at once on packed FP32 pairs
// (bit for bit the scalar combination of each, half the instructions).
__device__ __forceinline__ void t64_combine2(const float* ar, const float* ai, float* rh, float* rl, float* ih,
                                             float* il) {
  f2p A[T64_NW];
#pragma unroll
  for (int w = 0; w < T64_NW; ++w) A[w] = pk2(ar[w], ai[w]);
  const f2p c8 = pk2(0x1p-8f, 0x1p-8f), c16 = pk2(0x1p-16f, 0x1p-16f), c24 = pk2(0x1p-24f, 0x1p-24f);
  const f2p c32 = pk2(0x1p-32f, 0x1p-32f), c40 = pk2(0x1p-40f, 0x1p-40f), c48 = pk2(0x1p-48f, 0x1p-48f);
  const f2p tail = fma2(A[3], c24, fma2(A[4], c32, fma2(A[5], c40, mul2(A[6], c48))));
  f2p e1, e2, l;
  const f2p s = two_sum2(A[0], mul2(A[1], c8), &e1);
  const f2p s2 = two_sum2(s, mul2(A[2], c16), &e2);
  const f2p err = add2(add2(e1, e2), tail);
  const f2p h = two_sum2(s2, err, &l);
  up2(h, rh, ih);
  up2(l, rl, il);
}

__global__ void __launch_bounds__(T64_THREADS, 1)
k_alpha_tc64(const unsigned char* __restrict__ xblob, size_t blob_stride, int tiles,
             const unsigned char* __restrict__ etab, int Na, int J, int npairs, double2* __restrict__ g,
             int* __restrict__ err, const int2* __restrict__ slots, int wait_test) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sA = sm;                               // 7 x 16 KB: the item's A digits
  unsigned char* sB = sm + T64_A_BYTES;                 // T64_BS x 28 KB: ring of B digit chunks
  T64Bars* bars = reinterpret_cast<T64Bars*>(sB + T64_BS * T64_B_BYTES);
  volatile int* abort_flag = &bars->abort_flag;
  const uint32_t wlim = wait_test ? (1u << 14) : TC_WAIT_LIMIT;   // short limit for the timeout test
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nch = (Na + T64_NA - 1) / T64_NA;
  const long long nitems = (long long)npairs * tiles;

  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bars->a_full), 1);
    mbar_init(smem_u32(&bars->a_empty), 1);
    for (int i = 0; i < T64_BS; ++i) {
      mbar_init(smem_u32(&bars->b_full[i]), 1);
      mbar_init(smem_u32(&bars->b_empty[i]), 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(smem_u32(&bars->acc_full[i]), 1);
      mbar_init(smem_u32(&bars->acc_empty[i]), 32 * T64_EPI_WARPS);
    }
    mbar_init(smem_u32(&bars->drain), 1);
    bars->abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {   // TMEM: two sets of 7 accumulators of 128 x 32 FP32 (448 of 512 columns)
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                     smem_u32(&bars->tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = bars->tmem_base;

  if (warp == 0) {
    // ---------------- loader: the item's A digits, then its B digit chunks in order
    if (lane == 0) {
      int a_armed = -1, b_armed[T64_BS];
#pragma unroll
      for (int i = 0; i < T64_BS; ++i) b_armed[i] = -1;
      long long bc = 0;
      int li = 0;
      bool ok = true;
      for (long long it = blockIdx.x; it < nitems && ok; it += gridDim.x, ++li) {
        const int pair = (int)(it / tiles), tile = (int)(it % tiles);
        const uint32_t pa = (uint32_t)(li & 1);
        if (!(ok = mbar_wait_n(smem_u32(&bars->a_empty), pa ^ 1u, abort_flag, wlim))) break;
        if (!(wait_test && li == 0)) {   // wait_test: the first A digits are never fetched
          const uint32_t fa = smem_u32(&bars->a_full);
          mbar_expect_tx(fa, T64_A_BYTES);
          const unsigned char* src = xblob + (size_t)pair * blob_stride + (size_t)tile * T64_A_BYTES;
          for (int o = 0; o < T64_A_BYTES; o += 16384) bulk_g2s(smem_u32(sA + o), src + o, 16384, fa);
          a_armed = (int)pa;
        }
        for (int c = 0; c < nch && ok; ++c, ++bc) {
          const int sb = (int)(bc % T64_BS);
          const uint32_t pb = (uint32_t)((bc / T64_BS) & 1);
          if (!(ok = mbar_wait_n(smem_u32(&bars->b_empty[sb]), pb ^ 1u, abort_flag, wlim))) break;
          const uint32_t fb = smem_u32(&bars->b_full[sb]);
          mbar_expect_tx(fb, T64_B_BYTES);
          const unsigned char* bsrc = etab + (size_t)c * T64_B_BYTES;
          // 28 KB in one 16 KB and one 12 KB copy
          bulk_g2s(smem_u32(sB + sb * T64_B_BYTES), bsrc, 16384, fb);
          bulk_g2s(smem_u32(sB + sb * T64_B_BYTES + 16384), bsrc + 16384, T64_B_BYTES - 16384, fb);
#pragma unroll
          for (int i = 0; i < T64_BS; ++i)
            if (i == sb) b_armed[i] = (int)pb;
        }
      }
      if (!ok) *abort_flag = 1;
      // copies in flight must land before the CTA may exit
      if (a_armed >= 0) {
        uint32_t n = 0;
        while (!mbar_test(smem_u32(&bars->a_full), (uint32_t)a_armed) && ++n < TC_WAIT_LIMIT) {}
      }
#pragma unroll
      for (int i = 0; i < T64_BS; ++i) {
        if (b_armed[i] >= 0) {
          uint32_t n = 0;
          while (!mbar_test(smem_u32(&bars->b_full[i]), (uint32_t)b_armed[i]) && ++n < TC_WAIT_LIMIT) {}
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer
    if (lane == 0) {
      long long bc = 0, ac = 0;
      int li = 0;
      bool ok = true;
      for (long long it = blockIdx.x; it < nitems && ok; it += gridDim.x, ++li) {
        if (!(ok = mbar_wait_n(smem_u32(&bars->a_full), (uint32_t)(li & 1), abort_flag, wlim))) break;
        for (int c = 0; c < nch && ok; ++c, ++bc, ++ac) {
          const int set = (int)(ac & 1), sb = (int)(bc % T64_BS);
          if (!(ok = mbar_wait_n(smem_u32(&bars->b_full[sb]), (uint32_t)((bc / T64_BS) & 1), abort_flag, wlim))) break;
          if (!(ok = mbar_wait_n(smem_u32(&bars->acc_empty[set]), (uint32_t)(((ac >> 1) & 1) ^ 1), abort_flag, wlim)))
            break;
          tc_fence_after();
          const uint32_t d0 = tmem + (uint32_t)(set * T64_SET);
          const uint64_t bd = sw128_desc(smem_u32(sB + sb * T64_B_BYTES));
          const uint32_t a0 = smem_u32(sA);
          // A digit i against B digits j = 0 .. 6 - i in ONE MMA: the B digits
          // are consecutive 32-row blocks of the chunk and the accumulators
          // consecutive 32-column blocks of the set, so N = 32 (7 - i) columns
          // from d0 + 32 i put A_i c_j into accumulator i + j.  i = 0 covers
          // every accumulator first and overwrites it.
#pragma unroll
          for (int i = 0; i < T64_S; ++i) {
            const uint64_t ad = sw128_desc(a0 + (uint32_t)(i * T64_A_SLICE));
            const uint32_t idesc = umma_idesc_f16(TC_M, T64_N * (T64_NW - i));
            const uint32_t d = d0 + (uint32_t)(i * T64_N);
#pragma unroll
            for (int s = 0; s < TC_KB / 16; ++s)         // K = 16 per MMA: +32 bytes
              umma_f16(d, ad + (uint64_t)(2 * s), bd + (uint64_t)(2 * s), idesc, (i | s) != 0);
          }
          umma_commit(smem_u32(&bars->b_empty[sb]));
          umma_commit(smem_u32(&bars->acc_full[set]));
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
    // ---------------- epilogue: warps 2 .. 1 + T64_EPI_WARPS; TMEM lane
    // quadrant = warp % 4, part = which T64_RPW of the chunk's 16 alpha rows
    const int quad = warp & 3;
    const int part = (warp - 2) >> 2;
    const int row = quad * 32 + lane;
    long long ac = 0;
    bool ok = true;
    for (long long it = blockIdx.x; it < nitems && ok; it += gridDim.x) {
      const int pair = (int)(it / tiles), tile = (int)(it % tiles);
      const int j = tile * TC_M + row;
      const bool jin = j < J;
      const int* scales = reinterpret_cast<const int*>(xblob + (size_t)pair * blob_stride +
                                                       (size_t)tiles * T64_A_BYTES);
      const int sc = jin ? scales[j] : 0;
      const int2 sl = slots != nullptr ? slots[pair] : make_int2(pair, -1);
      double2* gp = g + (size_t)sl.x * Na * J + (jin ? j : 0);
      double2* gm = sl.y >= 0 ? g + (size_t)(sl.y >> 1) * Na * J + (jin ? j : 0) : nullptr;
      const unsigned long long msgn = (sl.y & 1) ? (1ull << 63) : 0ull;
      for (int c = 0; c < nch; ++c, ++ac) {
        const int set = (int)(ac & 1);
        // one lane waits, the warp follows: tcgen05.ld needs a converged warp
        int got = 0;
        if (lane == 0) got = mbar_wait_n(smem_u32(&bars->acc_full[set]), (uint32_t)((ac >> 1) & 1), abort_flag, wlim);
        got = __shfl_sync(0xffffffffu, got, 0);
        __syncwarp();
        if (!(ok = got != 0)) break;
        tc_fence_after();
        const uint32_t tbase = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(set * T64_SET + part * T64_RPW);
        uint32_t vr[T64_NW][T64_RPW], vi[T64_NW][T64_RPW];
#pragma unroll
        for (int w = 0; w < T64_NW; ++w) {
#if T64_RPW == 4
          TMEM_LD4(tbase + (uint32_t)(w * T64_N), vr[w]);
          TMEM_LD4(tbase + (uint32_t)(w * T64_N + T64_NA), vi[w]);
#else
          TMEM_LD8(tbase + (uint32_t)(w * T64_N), vr[w]);
          TMEM_LD8(tbase + (uint32_t)(w * T64_N + T64_NA), vi[w]);
#endif
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        tc_fence_before();
        mbar_arrive(smem_u32(&bars->acc_empty[set]));   // the registers hold the chunk
        const int a0 = c * T64_NA + part * T64_RPW;
#pragma unroll
        for (int u = 0; u < T64_RPW; ++u) {
          float ar[T64_NW], ai[T64_NW];
#pragma unroll
          for (int w = 0; w < T64_NW; ++w) {
            ar[w] = __uint_as_float(vr[w][u]);
            ai[w] = __uint_as_float(vi[w][u]);
          }
          // padding columns past J and rows past N_alpha are exact zeros that
          // would take the assembly's FP64 branch: only live samples are formed
          const bool live = jin && a0 + u < Na;
          if (!live) continue;
          float rh, rl, ih, il;
          t64_combine2(ar, ai, &rh, &rl, &ih, &il);
          const double re = dd_to_double(rh, rl, sc), im = dd_to_double(ih, il, sc);
          __stcs(gp + (size_t)(a0 + u) * J, make_double2(re, im));
          if (gm != nullptr) {           // (l, -m): (-1)^m conj g, signs on the bit patterns
            const unsigned long long br = (unsigned long long)__double_as_longlong(re) ^ msgn;
            const unsigned long long bi = (unsigned long long)__double_as_longlong(im) ^ msgn ^ (1ull << 63);
            __stcs(gm + (size_t)(a0 + u) * J,
                   make_double2(__longlong_as_double((long long)br), __longlong_as_double((long long)bi)));
          }
        }
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

cudaError_t launch_alpha_tc64(const void* xblob, const void* etab, int Lh, int Na, int Nb, int Ng, int npairs,
                              double2* g, int num_sms, const int2* slots, cudaStream_t st) {
  if (npairs <= 0) return cudaSuccess;
  if (!tc64_supported(Lh, Na)) return cudaErrorInvalidValue;
  if (!xblob || !etab || !g) return cudaErrorInvalidValue;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_alpha_tc64, cudaFuncAttributeMaxDynamicSharedMemorySize, T64_SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  int* err = tc_error_word();
  if (!err) return cudaErrorMemoryAllocation;
  const int tiles = t64_tiles(Nb, Ng);
  const long long items = (long long)npairs * tiles;
  const int grid = (int)(items < num_sms ? items : num_sms);
  k_alpha_tc64<<<grid, T64_THREADS, T64_SMEM, st>>>((const unsigned char*)xblob, tc64_xblob_bytes(Nb, Ng), tiles,
                                                   (const unsigned char*)etab, Na, Nb * Ng, npairs, g, err, slots,
                                                   tc_take_wait_test());
  return cudaGetLastError();
}
