// FP32_BULK alpha stage on the 5th-generation tensor cores (tcgen05).
//
// For one pair, with complex columns j = (beta, gamma) sample and alpha rows a,
//   g[a][j] = sum_q X_q[j] e^{-i q alpha_a}
// is a real GEMM D[j][n] = sum_k A[j][k] B[n][k] with
//   A[j][k]      = Re X_q[j] at k = 15 + q,  Im X_q[j] at k = 47 + q   (|q| <= 15, zeros elsewhere)
//   B[n][k]      = cos(q alpha_a) at k = 15 + q,  sin(q alpha_a) at k = 47 + q   n = a - a0   (Re g)
//   B[128+n][k]  = -sin(q alpha_a) at k = 15 + q, cos(q alpha_a) at k = 47 + q               (Im g)
// so one M=128 x N=256 accumulator holds Re and Im of 128 columns x 128 alpha
// rows.  Precision: each operand is split into FP16 hi + lo (A after a
// per-row power-of-two scale so its largest entry is in [2^14, 2^15)), and
// D = A_hi B_hi + A_hi B_lo + A_lo B_hi is accumulated in FP32 (about 22
// significant bits per product), which keeps the relative L2 error of g near
// 1e-6.
//
// Kernel structure: persistent, one CTA per SM, work item = (pair, tile of
// 128 columns).  Warp 0 streams operands with cp.async.bulk into shared
// memory (A tile double-buffered, one B chunk stage: a chunk loads from L2 in
// well under the time the epilogue spends on the previous one), warp 1 issues
// tcgen05.mma from one thread into a double-buffered TMEM accumulator
// (2 x 256 columns), warps 2-9 drain the accumulator (tcgen05.ld; two warps
// per TMEM lane quadrant, each half of the 128 alpha rows), rescale and store
// g with coalesced 8-byte streaming stores (for a fixed alpha row a warp
// writes 32 consecutive columns).  The 129 KB of shared memory leave room on
// each SM for the producer kernels of the next chunk.  Every mbarrier wait is bounded: on expiry the
// CTA records an error word, stops, waits (bounded) for its own copies and
// MMAs in flight, frees TMEM and exits.
#include <cuda_fp16.h>

#include "common.cuh"
#include "tc.cuh"
#include "tc_ptx.cuh"

bool tc_supported(int Lh, int Na) { return Lh >= 1 && 2 * (2 * Lh - 1) <= TC_KB && Na >= 1; }

static inline int tc_tiles(int Nb, int Ng) { return (Nb * Ng + TC_M - 1) / TC_M; }
static inline int tc_chunks(int Na) { return (Na + TC_NC - 1) / TC_NC; }

size_t tc_etab_bytes(int Na, int Lh) { (void)Lh; return (size_t)tc_chunks(Na) * TC_B_BYTES; }

// per pair: tiles x 32 KB of A, then one float scale per padded column
size_t tc_xblob_bytes(int Nb, int Ng, int Lh) {
  (void)Lh;
  const size_t t = (size_t)tc_tiles(Nb, Ng);
  const size_t sc = ((t * TC_M * sizeof(float)) + 1023) / 1024 * 1024;
  return t * TC_A_BYTES + sc;
}

// ---------------------------------------------------------------- E tables
// chunk c: [hi part: TC_N = 128 rows x 64][lo part], rows n < TC_NC = 64 -> alpha
// a = c*64+n (cos at k = 15+q | sin at k = 47+q), rows 64+n -> (-sin | cos); zeros
// beyond Na and for |q| >= Lh.
__global__ void k_tc_etab(unsigned char* __restrict__ etab, int Na, int Lh) {
  const int c = blockIdx.x;
  unsigned char* base = etab + (size_t)c * TC_B_BYTES;
  for (int t = threadIdx.x; t < TC_N * TC_KB; t += blockDim.x) {
    const int r = t / TC_KB, k = t % TC_KB;
    const int n = r % TC_NC;
    const int a = c * TC_NC + n;
    double v = 0.0;
    const int q = (k & 31) - 15;
    if (a < Na && (k & 31) < 31 && abs(q) < Lh) {
      double s, co;
      sincos_2pi_frac((long long)q * a, Na, &s, &co);
      const bool is_sin = k >= 32;
      if (r < TC_NC) v = is_sin ? s : co;
      else v = is_sin ? co : -s;
    }
    const __half hi = __double2half(v);
    const __half lo = __double2half(v - (double)__half2float(hi));
    *reinterpret_cast<__half*>(base + sw128_off(r, k)) = hi;
    *reinterpret_cast<__half*>(base + TC_B_HALF + sw128_off(r, k)) = lo;
  }
}

cudaError_t launch_tc_etab(void* etab, int Na, int Lh, cudaStream_t st) {
  k_tc_etab<<<tc_chunks(Na), 256, 0, st>>>((unsigned char*)etab, Na, Lh);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- beta/gamma -> A
// Factoring-of-rotations route: G[q][q'](b) = Y[pair][b][q][q'] (the q''-DFT of
// the C tensor), for TC_NBB beta rows per CTA, then
//   X_q[c](b)   = G[q][0] + sum_{s>=1} (G[q][s] + G[q][-s]) cos(s gamma_c)
//                          - i (G[q][s] - G[q][-s]) sin(s gamma_c)
// and every row j = b*Ng + c is written as the A operand: scaled by 2^e (its
// largest entry into [2^14, 2^15)), split into FP16 hi/lo, swizzled.
#define TC_NBB 4

struct BgLayout {          // shared-memory carve-up of k_betagamma_tc
  int LhP, NgP;            // padded strides: Gp/Gm rows, phase and X rows (multiple of 4)
  size_t off_k, off_h, off_e, off_gp, off_gm, off_x, off_ex, total;
  __host__ __device__ BgLayout(int Lh, int Ng) {
    const int K = 2 * Lh - 1;
    LhP = Lh + 1;
    NgP = (Ng + 3) & ~3;
    // every region starts on a 16-byte boundary (float4 accesses)
    off_k = 0;
    off_h = a16(off_k + sizeof(float2) * Lh * Lh);
    off_e = a16(off_h + sizeof(float2) * Lh * Lh);
    off_gp = a16(off_e + sizeof(float2) * (size_t)Lh * NgP);
    off_gm = a16(off_gp + sizeof(float2) * (size_t)TC_NBB * K * LhP);
    off_x = a16(off_gm + sizeof(float2) * (size_t)TC_NBB * K * LhP);
    off_ex = a16(off_x + sizeof(float) * (size_t)TC_NBB * 2 * K * NgP);
    total = a16(off_ex + sizeof(int) * (size_t)TC_NBB * NgP);
  }
  __host__ __device__ static size_t a16(size_t n) { return (n + 15) & ~(size_t)15;
  }
};

__global__ void __launch_bounds__(256)
k_betagamma_tc(const double2* __restrict__ kc, const double2* __restrict__ h, const float* __restrict__ dT,
               const double2* __restrict__ Y, const float2* __restrict__ eg, int Lh, int Nb, int Ng,
               unsigned char* __restrict__ xblob, size_t blob_stride, int tiles) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int K = 2 * Lh - 1;
  const int b0 = blockIdx.x * TC_NBB, pair = blockIdx.y;
  const int nbb = min(TC_NBB, Nb - b0);
  const BgLayout L(Lh, Ng);
  float2* sk = reinterpret_cast<float2*>(smem_raw + L.off_k);
  float2* sh = reinterpret_cast<float2*>(smem_raw + L.off_h);
  float2* sE = reinterpret_cast<float2*>(smem_raw + L.off_e);     // [s][NgP]
  float2* sGp = reinterpret_cast<float2*>(smem_raw + L.off_gp);   // [bb][q][LhP]
  float2* sGm = reinterpret_cast<float2*>(smem_raw + L.off_gm);
  float* sX = reinterpret_cast<float*>(smem_raw + L.off_x);       // [bb][k][NgP], k < 2K: Re | Im
  int* sEx = reinterpret_cast<int*>(smem_raw + L.off_ex);         // [bb][c] row scale exponent
  const int n2 = Lh * Lh;
  for (int t = threadIdx.x; t < n2; t += blockDim.x) {
    const double2 kv = kc[(size_t)pair * n2 + t], hv = h[t];
    sk[t] = make_float2((float)kv.x, (float)kv.y);
    sh[t] = make_float2((float)hv.x, (float)hv.y);
  }
  for (int t = threadIdx.x; t < Lh * L.NgP; t += blockDim.x) {
    const int s = t / L.NgP, c = t % L.NgP;
    sE[t] = c < Ng ? eg[c * K + s + (Lh - 1)] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  // ---- G for the CTA's beta rows, folded into Gp / Gm
  for (int t = threadIdx.x; t < K * Lh; t += blockDim.x) {
    const int qi = t / Lh, s = t % Lh;
    float pr[TC_NBB], pi[TC_NBB], mr[TC_NBB], mi[TC_NBB];
#pragma unroll
    for (int u = 0; u < TC_NBB; ++u) pr[u] = pi[u] = mr[u] = mi[u] = 0.f;
    {
#pragma unroll
      for (int u = 0; u < TC_NBB; ++u) {
        if (u >= nbb) break;
        const double2* src = Y + (((size_t)pair * Nb + b0 + u) * K + qi) * K;
        const double2 vp = src[s + Lh - 1];
        pr[u] = (float)vp.x; pi[u] = (float)vp.y;
        if (s > 0) { const double2 vm = src[-s + Lh - 1]; mr[u] = (float)vm.x; mi[u] = (float)vm.y; }
      }
    }
#pragma unroll
    for (int u = 0; u < TC_NBB; ++u) {
      const int o = (u * K + qi) * L.LhP + s;
      if (s == 0) { sGp[o] = make_float2(pr[u], pi[u]); sGm[o] = sGp[o]; }
      else { sGp[o] = make_float2(pr[u] + mr[u], pi[u] + mi[u]); sGm[o] = make_float2(pr[u] - mr[u], pi[u] - mi[u]); }
    }
  }
  __syncthreads();
  // ---- gamma sum, four gamma columns per thread
  const int ncq = L.NgP / 4;
  for (int t = threadIdx.x; t < nbb * K * ncq; t += blockDim.x) {
    const int cq = t % ncq, qi = (t / ncq) % K, u = t / (ncq * K);
    const int c0 = 4 * cq;
    const float2* gp = sGp + (u * K + qi) * L.LhP;
    const float2* gm = sGm + (u * K + qi) * L.LhP;
    float re[4], im[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) { re[v] = gp[0].x; im[v] = gp[0].y; }
    for (int s = 1; s < Lh; ++s) {
      const float2 P = gp[s], M = gm[s];
      const float4 Ea = *reinterpret_cast<const float4*>(sE + s * L.NgP + c0);       // c0, c0+1
      const float4 Eb = *reinterpret_cast<const float4*>(sE + s * L.NgP + c0 + 2);   // c0+2, c0+3
      const float cs[4] = {Ea.x, Ea.z, Eb.x, Eb.z}, sn[4] = {Ea.y, Ea.w, Eb.y, Eb.w};
#pragma unroll
      for (int v = 0; v < 4; ++v) {            // (Gp cos - i Gm sin)
        re[v] = fmaf(P.x, cs[v], re[v]); re[v] = fmaf(M.y, sn[v], re[v]);
        im[v] = fmaf(P.y, cs[v], im[v]); im[v] = fmaf(-M.x, sn[v], im[v]);
      }
    }
    float* xr = sX + ((size_t)u * 2 * K + qi) * L.NgP + c0;
    float* xi = sX + ((size_t)u * 2 * K + K + qi) * L.NgP + c0;
    *reinterpret_cast<float4*>(xr) = make_float4(re[0], re[1], re[2], re[3]);
    *reinterpret_cast<float4*>(xi) = make_float4(im[0], im[1], im[2], im[3]);
  }
  __syncthreads();
  // ---- per row (u, c): e such that max |X| * 2^e lies in [2^14, 2^15), clamped
  // so that 2^e and 2^-e are normal floats
  unsigned char* blob = xblob + (size_t)pair * blob_stride;
  float* scales = reinterpret_cast<float*>(blob + (size_t)tiles * TC_A_BYTES);
  const int J = Nb * Ng;
  for (int t = threadIdx.x; t < nbb * L.NgP; t += blockDim.x) {
    const int u = t / L.NgP, c = t % L.NgP;
    if (c >= Ng) continue;
    const float* col = sX + (size_t)u * 2 * K * L.NgP + c;
    float mx = 0.f;
    for (int k = 0; k < 2 * K; ++k) mx = fmaxf(mx, fabsf(col[(size_t)k * L.NgP]));
    int ex = 0;
    if (mx > 0.f) frexpf(mx, &ex);
    const int e = mx > 0.f ? min(125, max(-125, 15 - ex)) : 0;
    sEx[t] = e;
    scales[(b0 + u) * Ng + c] = __int_as_float((127 - e) << 23);
  }
  __syncthreads();
  // ---- scale, split, store: one thread per (row, 16-byte chunk of 8 FP16 values),
  // rows fastest so a warp's shared-memory reads are consecutive columns
  for (int t = threadIdx.x; t < nbb * L.NgP * (TC_KB / 8); t += blockDim.x) {
    const int c = t % L.NgP, k0 = ((t / L.NgP) % (TC_KB / 8)) * 8, u = t / (L.NgP * (TC_KB / 8));
    if (c >= Ng) continue;
    const float sc = __int_as_float((127 + sEx[u * L.NgP + c]) << 23);
    const float* col = sX + (size_t)u * 2 * K * L.NgP + c;
    const int j = (b0 + u) * Ng + c;
    unsigned char* tb = blob + (size_t)(j / TC_M) * TC_A_BYTES;
    const int r = j % TC_M;
    __align__(16) __half hi[8], lo[8];
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      const int k = k0 + v;
      const int q = (k & 31) - 15;                 // Re X_q at 15 + q, Im X_q at 47 + q
      const int src = (k < 32 ? 0 : K) + q + (Lh - 1);
      const float x = ((k & 31) < 31 && abs(q) < Lh) ? col[(size_t)src * L.NgP] * sc : 0.f;
      hi[v] = __float2half_rn(x);
      lo[v] = __float2half_rn(x - __half2float(hi[v]));
    }
    *reinterpret_cast<uint4*>(tb + sw128_off(r, k0)) = *reinterpret_cast<uint4*>(hi);
    *reinterpret_cast<uint4*>(tb + TC_A_HALF + sw128_off(r, k0)) = *reinterpret_cast<uint4*>(lo);
  }
  // the CTA holding the last beta row also clears the padding rows of the last tile
  if (b0 + nbb == Nb) {
    for (int t = threadIdx.x; t < (tiles * TC_M - J) * (TC_KB / 8); t += blockDim.x) {
      const int j = J + t / (TC_KB / 8), k0 = (t % (TC_KB / 8)) * 8;
      unsigned char* tb = blob + (size_t)(j / TC_M) * TC_A_BYTES;
      const int r = j % TC_M;
      *reinterpret_cast<uint4*>(tb + sw128_off(r, k0)) = make_uint4(0, 0, 0, 0);
      *reinterpret_cast<uint4*>(tb + TC_A_HALF + sw128_off(r, k0)) = make_uint4(0, 0, 0, 0);
      if (k0 == 0) scales[j] = 0.f;
    }
  }
}

cudaError_t launch_betagamma_tc(const double2* kc, const double2* h, const float* dT, const double2* Y,
                                const float2* eg, int Lh, int Nb, int Ng, int npairs, void* xblob,
                                cudaStream_t st) {
  if (npairs <= 0) return cudaSuccess;
  const size_t smem = BgLayout(Lh, Ng).total;
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_betagamma_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  {
    cudaError_t e = cudaFuncSetAttribute(k_betagamma_tc, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
  }
  dim3 grid((Nb + TC_NBB - 1) / TC_NBB, npairs);
  if (Y == nullptr) return cudaErrorInvalidValue;       // the factoring route only
  k_betagamma_tc<<<grid, 256, smem, st>>>(kc, h, dT, Y, eg, Lh, Nb, Ng, (unsigned char*)xblob,
                                          tc_xblob_bytes(Nb, Ng, Lh), tc_tiles(Nb, Ng));
  return cudaGetLastError();
}

// ---------------------------------------------------------------- A operand from H
// Rotated-window route: X_q(j) = sum_{p>=|q|} k(p,q) H^p_q(j) (H from launch_rotwin_f32),
// for one pair and one 128-column tile per CTA.
//   phase 1: one item per (q, column): a loop over exactly its degrees p >= |q|,
//            H loads coalesced across columns, k(p,q) broadcast; X goes to a shared
//            tile [64 slots][128 columns] (Re X_q at slot 15+q, Im at 47+q);
//   phase 2: per column, the largest |entry| -> scale 2^e into [2^14, 2^15);
//   phase 3: per (column, 16-byte chunk): scale, split into FP16 hi/lo, store
//            swizzled.  Columns beyond J (padding of the last tile) are zero.
__global__ void __launch_bounds__(256)
k_xa_from_h(const double2* __restrict__ kc, const float2* __restrict__ H, int Lh, int J,
            unsigned char* __restrict__ xblob, size_t blob_stride, int tiles) {
  __shared__ float sX[TC_KB][TC_M];
  __shared__ float2 sk[16 * 16];
  __shared__ int sEx[TC_M];
  const int tile = blockIdx.x, pair = blockIdx.y;
  const int n2 = Lh * Lh;
  for (int t = threadIdx.x; t < n2; t += blockDim.x) {
    const double2 v = kc[(size_t)pair * n2 + t];
    sk[t] = make_float2((float)v.x, (float)v.y);
  }
  __syncthreads();
  const int jt = tile * TC_M;
  for (int it = threadIdx.x; it < 32 * TC_M; it += blockDim.x) {
    const int u = it / TC_M, r = it % TC_M;
    const int q = u - 15, aq = q < 0 ? -q : q;
    const int j = jt + r;
    float ar = 0.f, ai = 0.f;
    if (u < 31 && aq < Lh && j < J) {
      const float2* hp = H + h_index(0, j, n2);      // row pq at hp + pq * 128
      int p = aq;
      for (; p + 3 < Lh; p += 4) {                  // four loads in flight per step
        float2 hv[4], kv[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int pq = (p + v) * (p + v) + (p + v) + q;
          hv[v] = __ldg(hp + (size_t)pq * 128);
          kv[v] = sk[pq];
        }
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          ar = fmaf(kv[v].x, hv[v].x, ar); ar = fmaf(-kv[v].y, hv[v].y, ar);
          ai = fmaf(kv[v].x, hv[v].y, ai); ai = fmaf(kv[v].y, hv[v].x, ai);
        }
      }
      for (; p < Lh; ++p) {
        const int pq = p * p + p + q;
        const float2 hv = __ldg(hp + (size_t)pq * 128), kv = sk[pq];
        ar = fmaf(kv.x, hv.x, ar); ar = fmaf(-kv.y, hv.y, ar);
        ai = fmaf(kv.x, hv.y, ai); ai = fmaf(kv.y, hv.x, ai);
      }
    }
    sX[u][r] = ar;
    sX[32 + u][r] = ai;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < TC_M; r += blockDim.x) {
    float mx = 0.f;
#pragma unroll 8
    for (int k = 0; k < TC_KB; ++k) mx = fmaxf(mx, fabsf(sX[k][r]));
    int ex = 0;
    if (mx > 0.f) frexpf(mx, &ex);
    sEx[r] = mx > 0.f ? min(125, max(-125, 15 - ex)) : 0;
  }
  __syncthreads();
  unsigned char* blob = xblob + (size_t)pair * blob_stride;
  unsigned char* tb = blob + (size_t)tile * TC_A_BYTES;
  float* scales = reinterpret_cast<float*>(blob + (size_t)tiles * TC_A_BYTES);
  for (int it = threadIdx.x; it < TC_M * (TC_KB / 8); it += blockDim.x) {
    const int r = it % TC_M, k0 = (it / TC_M) * 8;
    const int e = sEx[r];
    const float sc = __int_as_float((127 + e) << 23);
    __align__(16) __half hi[8], lo[8];
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      const float x = sX[k0 + v][r] * sc;
      hi[v] = __float2half_rn(x);
      lo[v] = __float2half_rn(x - __half2float(hi[v]));
    }
    *reinterpret_cast<uint4*>(tb + sw128_off(r, k0)) = *reinterpret_cast<uint4*>(hi);
    *reinterpret_cast<uint4*>(tb + TC_A_HALF + sw128_off(r, k0)) = *reinterpret_cast<uint4*>(lo);
    if (k0 == 0) scales[jt + r] = jt + r < J ? __int_as_float((127 - e) << 23) : 0.f;
  }
}

cudaError_t launch_xa_from_h(const double2* kc, const float2* H, int Lh, int Nb, int Ng, int npairs, void* xblob,
                             cudaStream_t st) {
  if (npairs <= 0) return cudaSuccess;
  if (Lh > 16) return cudaErrorInvalidValue;
  const int tiles = tc_tiles(Nb, Ng);
  dim3 grid(tiles, npairs);
  k_xa_from_h<<<grid, 256, 0, st>>>(kc, H, Lh, Nb * Ng, (unsigned char*)xblob, tc_xblob_bytes(Nb, Ng, Lh), tiles);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- the kernel
struct TcBars {
  uint64_t a_full[2], a_empty[2], b_full, b_empty, acc_full[2], acc_empty[2], drain;
  uint32_t tmem_base;
  int abort_flag;
};

__global__ void __launch_bounds__(TC_THREADS, 1)
k_alpha_tc(const unsigned char* __restrict__ xblob, size_t blob_stride, int tiles,
           const unsigned char* __restrict__ etab, int Na, int J, int npairs, float2* __restrict__ g,
           int* __restrict__ err, const int2* __restrict__ slots, int wait_test) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sA = sm;                               // 2 x 32 KB
  unsigned char* sB = sm + 2 * TC_A_BYTES;              // 64 KB
  TcBars* bars = reinterpret_cast<TcBars*>(sB + TC_B_BYTES);
  volatile int* abort_flag = &bars->abort_flag;
  const uint32_t wlim = wait_test ? (1u << 14) : TC_WAIT_LIMIT;   // short limit for the timeout test
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nch = (Na + TC_NC - 1) / TC_NC;
  const long long nitems = (long long)npairs * tiles;

  if (threadIdx.x == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(smem_u32(&bars->a_full[i]), 1);
      mbar_init(smem_u32(&bars->a_empty[i]), 1);
      mbar_init(smem_u32(&bars->acc_full[i]), 1);
      mbar_init(smem_u32(&bars->acc_empty[i]), 32 * TC_EPI_WARPS);
    }
    mbar_init(smem_u32(&bars->b_full), 1);
    mbar_init(smem_u32(&bars->b_empty), 1);
    mbar_init(smem_u32(&bars->drain), 1);
    bars->abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {   // TMEM: 512 columns (two 128 x TC_N FP32 accumulators in use)
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                     smem_u32(&bars->tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = bars->tmem_base;

  if (warp == 0) {
    // ---------------- producer
    if (lane == 0) {
      int a_armed[2] = {-1, -1}, b_armed = -1;
      long long bc = 0;
      int li = 0;
      for (long long it = blockIdx.x; it < nitems && !*abort_flag; it += gridDim.x, ++li) {
        const int pair = (int)(it / tiles), tile = (int)(it % tiles);
        const int sa = li & 1;
        const uint32_t pa = (uint32_t)((li >> 1) & 1);
        if (!mbar_wait_n(smem_u32(&bars->a_empty[sa]), pa ^ 1u, abort_flag, wlim)) { *abort_flag = 1; break; }
        if (!(wait_test && li == 0)) {   // wait_test: the first A operand is never fetched
          const uint32_t fa = smem_u32(&bars->a_full[sa]);
          mbar_expect_tx(fa, TC_A_BYTES);
          const unsigned char* src = xblob + (size_t)pair * blob_stride + (size_t)tile * TC_A_BYTES;
          for (int o = 0; o < TC_A_BYTES; o += 16384)
            bulk_g2s(smem_u32(sA + sa * TC_A_BYTES + o), src + o, 16384, fa);
          a_armed[sa] = (int)pa;
        }
        for (int c = 0; c < nch; ++c, ++bc) {
          const uint32_t pb = (uint32_t)(bc & 1);
          if (!mbar_wait_n(smem_u32(&bars->b_empty), pb ^ 1u, abort_flag, wlim)) { *abort_flag = 1; break; }
          const uint32_t fb = smem_u32(&bars->b_full);
          mbar_expect_tx(fb, TC_B_BYTES);
          const unsigned char* bsrc = etab + (size_t)c * TC_B_BYTES;
          for (int o = 0; o < TC_B_BYTES; o += 16384)
            bulk_g2s(smem_u32(sB + o), bsrc + o, 16384, fb);
          b_armed = (int)pb;
        }
      }
      // copies in flight must land before the CTA may exit
      for (int i = 0; i < 2; ++i) {
        if (a_armed[i] >= 0) {
          uint32_t n = 0;
          while (!mbar_test(smem_u32(&bars->a_full[i]), (uint32_t)a_armed[i]) && ++n < TC_WAIT_LIMIT) {}
        }
      }
      if (b_armed >= 0) {
        uint32_t n = 0;
        while (!mbar_test(smem_u32(&bars->b_full), (uint32_t)b_armed) && ++n < TC_WAIT_LIMIT) {}
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
        if (!(ok = mbar_wait_n(smem_u32(&bars->a_full[sa]), (uint32_t)((li >> 1) & 1), abort_flag, wlim))) break;
        const uint32_t a_hi = smem_u32(sA + sa * TC_A_BYTES), a_lo = a_hi + TC_A_HALF;
        for (int c = 0; c < nch; ++c, ++bc, ++ac) {
          const int acc = (int)(ac & 1);
          if (!(ok = mbar_wait_n(smem_u32(&bars->b_full), (uint32_t)(bc & 1), abort_flag, wlim))) break;
          if (!(ok = mbar_wait_n(smem_u32(&bars->acc_empty[acc]), (uint32_t)(((ac >> 1) & 1) ^ 1), abort_flag, wlim))) break;
          tc_fence_after();
          const uint32_t b_hi = smem_u32(sB), b_lo = b_hi + TC_B_HALF;
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
          umma_commit(smem_u32(&bars->b_empty));
          umma_commit(smem_u32(&bars->acc_full[acc]));
        }
        if (!ok) break;
        umma_commit(smem_u32(&bars->a_empty[sa]));
      }
      if (!ok) *abort_flag = 1;
      // every MMA issued by this thread completes before TMEM is released
      umma_commit(smem_u32(&bars->drain));
      uint32_t n = 0;
      while (!mbar_test(smem_u32(&bars->drain), 0u) && ++n < TC_WAIT_LIMIT) {}
    }
  } else {
    // ---------------- epilogue: warps 2..9; TMEM lane quadrant = warp % 4,
    // half = which 64 of the chunk's 128 alpha rows
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
                                                           (size_t)tiles * TC_A_BYTES);
      const float sc = jin ? scales[j] : 0.f;
      const int2 sl = slots != nullptr ? slots[pair] : make_int2(pair, -1);
      float2* gp = g + (size_t)sl.x * Na * J + (jin ? j : 0);
      float2* gm = sl.y >= 0 ? g + (size_t)(sl.y >> 1) * Na * J + (jin ? j : 0) : nullptr;
      const float msc = (sl.y & 1) ? -sc : sc;
      for (int c = 0; c < nch; ++c, ++ac) {
        const int acc = (int)(ac & 1);
        // one lane waits, the warp follows: tcgen05.ld needs a converged warp
        int got = 0;
        if (lane == 0) got = mbar_wait_n(smem_u32(&bars->acc_full[acc]), (uint32_t)((ac >> 1) & 1), abort_flag, wlim);
        got = __shfl_sync(0xffffffffu, got, 0);
        __syncwarp();
        if (!(ok = got != 0)) break;
        tc_fence_after();
        const uint32_t tbase = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(acc * TC_N);
#pragma unroll 1
        for (int cb = half * (TC_NC / 2); cb < half * (TC_NC / 2) + TC_NC / 2; cb += 32) {
          uint32_t vr[32], vi[32];
          TMEM_LD32(tbase + (uint32_t)cb, vr);
          TMEM_LD32(tbase + (uint32_t)(TC_NC + cb), vi);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          const int a0 = c * TC_NC + cb;
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

static thread_local int t_wait_test = 0;
void tc_arm_wait_test() { t_wait_test = 1; }
int tc_take_wait_test() {
  const int v = t_wait_test;
  t_wait_test = 0;
  return v;
}

// Device word a tensor-core kernel sets when it gives up on a bounded wait.
int* tc_error_word() {
  static int* p = nullptr;
  if (!p) {
    if (cudaMalloc(&p, sizeof(int)) != cudaSuccess) { cudaGetLastError(); p = nullptr; return nullptr; }
    cudaMemset(p, 0, sizeof(int));
  }
  return p;
}

int tc_read_error(void) {
  int* p = tc_error_word();
  if (!p) return 0;
  int v = 0;
  if (cudaMemcpy(&v, p, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) { cudaGetLastError(); return 0; }
  if (v) cudaMemset(p, 0, sizeof(int));
  return v;
}

cudaError_t launch_alpha_tc(const void* xblob, const void* etab, int Lh, int Na, int Nb, int Ng, int npairs,
                            float2* g, int num_sms, const int2* slots, cudaStream_t st) {
  if (npairs <= 0) return cudaSuccess;
  if (!tc_supported(Lh, Na)) return cudaErrorInvalidValue;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_alpha_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    if (e != cudaSuccess) return e;
    // the whole unified L1/shared array as shared memory, so the producer
    // kernels of the next chunk fit beside this kernel's CTA on every SM
    e = cudaFuncSetAttribute(k_alpha_tc, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  int* err = tc_error_word();
  if (!err) return cudaErrorMemoryAllocation;
  const int tiles = tc_tiles(Nb, Ng);
  const long long items = (long long)npairs * tiles;
  const int grid = (int)(items < num_sms ? items : num_sms);
  k_alpha_tc<<<grid, TC_THREADS, TC_SMEM, st>>>((const unsigned char*)xblob, tc_xblob_bytes(Nb, Ng, Lh), tiles,
                                               (const unsigned char*)etab, Na, Nb * Ng, npairs, g, err, slots,
                                               tc_take_wait_test());
  return cudaGetLastError();
}
