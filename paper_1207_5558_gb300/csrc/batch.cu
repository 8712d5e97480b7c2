// Kernels of batch plans (see batch.cuh): the coupling gather, the rotated
// windows and the alpha stage of many analyses with different band limits,
// grids and precisions, one launch each.
//
// k_batch_alpha is persistent: each CTA takes the next tile from a counter in
// device memory.  A tile is (item, pair, block of nt columns j = (beta, gamma)
// samples); the CTA forms
//   X_q(j) = sum_{p >= |q|} k(p, q) H^p_q(j)        (|q| < Lh, the rotated-window
// regrouping of Eq. alternative_harmonic_formulation_wigner) in shared memory
// and then g(alpha_a, j) = sum_q X_q(j) e^{-i q alpha_a} for every alpha row,
// either directly (+-q paired) or as the split DFT of alpha_dev.cuh, with
// BA_THREADS / nt row groups per column.  Host code orders the tiles by
// decreasing cost, so large tiles start first and small ones fill the tail.
#include <algorithm>
#include <mutex>

#include "alpha_dd.cuh"
#include "alpha_dev.cuh"
#include "batch.cuh"
#include "couple_dev.cuh"
#include "stages_dev.cuh"

// ---------------------------------------------------------------- coupling
__global__ void __launch_bounds__(256) k_batch_couple(const BCouple* __restrict__ cpl,
                                                      const BCplBlk* __restrict__ blk) {
  const BCplBlk b = blk[blockIdx.x];
  const BCouple c = cpl[b.cpl];
  const int n2 = c.Lh * c.Lh;
  const long long idx = (long long)b.first + threadIdx.x;
  if (idx >= (long long)c.npairs * n2) return;
  const int pair = (int)(idx / n2), t = (int)(idx % n2);
  c.kc[idx] = couple_apply_one(c.f, c.Lh, c.lm[pair].y, c.coef + (size_t)pair * c.Lh * n2, c.meta[idx], t);
}

cudaError_t launch_batch_couple(const BCouple* cpl, const BCplBlk* blk, int nblk, cudaStream_t st) {
  if (nblk <= 0) return cudaSuccess;
  k_batch_couple<<<nblk, 256, 0, st>>>(cpl, blk);
  return cudaGetLastError();
}

// Largest |value| over a block (every thread gets it).
__device__ __forceinline__ double block_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double m = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
  __syncthreads();
  return m;
}

// Exponent e with |x| * 2^-e in [0.5, 1) for the largest |x| (0 for x = 0).
__device__ __forceinline__ int scale_exp(double mx) {
  int e = 0;
  if (mx > 0.0) frexp(mx, &e);
  return e;
}

// k of one pair (n2 entries at kp) as double-floats at kd, scaled by a power
// of two so its largest component lies in [0.5, 1); the exponent to *kexp.
// Every thread of the block takes part.
__device__ __forceinline__ void kdd_pair(const double2* __restrict__ kp, int n2, float4* __restrict__ kd,
                                         int* __restrict__ kexp, double* red) {
  double mx = 0.0;
  for (int t = threadIdx.x; t < n2; t += blockDim.x) {
    const double2 v = kp[t];
    mx = fmax(mx, fmax(fabs(v.x), fabs(v.y)));
  }
  const int e = scale_exp(block_max(mx, red));
  for (int t = threadIdx.x; t < n2; t += blockDim.x) {
    const double2 v = kp[t];
    float rh, rl, ih, il;
    dd_split(ldexp(v.x, -e), &rh, &rl);
    dd_split(ldexp(v.y, -e), &ih, &il);
    kd[t] = make_float4(rh, ih, rl, il);
  }
  if (threadIdx.x == 0) *kexp = e;
}

// block {cpl, pair}; blocks stride over the list (count nblk, or *n_dev)
__global__ void __launch_bounds__(256) k_batch_kdd(const BCouple* __restrict__ cpl, const BCplBlk* __restrict__ blk,
                                                   int nblk, const int* __restrict__ n_dev) {
  __shared__ double red[8];
  const int cnt = n_dev != nullptr ? *n_dev : nblk;
  for (int i = blockIdx.x; i < cnt; i += gridDim.x) {
    const BCplBlk b = blk[i];
    const BCouple c = cpl[b.cpl];
    const int n2 = c.Lh * c.Lh, pair = b.first;
    kdd_pair(c.kc + (size_t)pair * n2, n2, c.kdd + (size_t)pair * n2, c.kexp + pair, red);
  }
}

// one block per pair
__global__ void __launch_bounds__(256) k_kdd_pairs(const double2* __restrict__ kc, int n2, float4* __restrict__ kdd,
                                                   int* __restrict__ kexp) {
  __shared__ double red[8];
  const int pair = blockIdx.x;
  kdd_pair(kc + (size_t)pair * n2, n2, kdd + (size_t)pair * n2, kexp + pair, red);
}

cudaError_t launch_kdd_pairs(const double2* kc, int Lh, int npairs, float4* kdd, int* kexp, cudaStream_t st) {
  if (npairs <= 0) return cudaSuccess;
  k_kdd_pairs<<<npairs, 256, 0, st>>>(kc, Lh * Lh, kdd, kexp);
  return cudaGetLastError();
}

cudaError_t launch_batch_kdd(const BCouple* cpl, const BCplBlk* blk, int nblk, cudaStream_t st) {
  if (nblk <= 0) return cudaSuccess;
  k_batch_kdd<<<nblk, 256, 0, st>>>(cpl, blk, nblk, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_batch_kdd_n(const BCouple* cpl, const BCplBlk* blk, const int* n, int grid, cudaStream_t st) {
  k_batch_kdd<<<grid, 256, 0, st>>>(cpl, blk, 0, n);
  return cudaGetLastError();
}

static cudaError_t batch_attrs();

// ---------------------------------------------------------------- rotated windows
// FP64 outputs of a rotated window: the double H and/or its double-float copy
// scaled by 2^-e (each pointer may be null).
struct RotwinBoth {
  double2* H;
  float4* Hdd;
  int e;
  __device__ __forceinline__ void operator()(size_t i, double re, double im) const {
    if (H != nullptr) H[i] = make_double2(re, im);
    if (Hdd != nullptr) {
      float rh, rl, ih, il;
      dd_split(ldexp(re, -e), &rh, &rl);
      dd_split(ldexp(im, -e), &ih, &il);
      Hdd[i] = make_float4(rh, ih, rl, il);
    }
  }
};
// One (beta row, degree) block of an FP64 window: the double H and/or the
// double-float copy scaled by 2^-e, e from the window's largest coefficient
// (every block finds the same e; block (0, 0) records it in *hexp).
__device__ __forceinline__ void rotwin_block_fp64(const double2* __restrict__ h, const double* __restrict__ dblk,
                                                  size_t dstride, int nb, const double2* __restrict__ eg, int Lh,
                                                  int Ng, int b, int p, const RotChunks& ch, int z, double2* H,
                                                  float4* Hdd, int* hexp, unsigned char* smem,
                                                  const uint32_t* qmask) {
  __shared__ double red[4];
  int e = 0;
  if (Hdd != nullptr) {
    double mx = 0.0;
    for (int t = threadIdx.x; t < Lh * Lh; t += blockDim.x) {
      const double2 v = h[t];
      mx = fmax(mx, fmax(fabs(v.x), fabs(v.y)));
    }
    e = scale_exp(block_max(mx, red));
    if (b == 0 && p == 0 && z == 0 && threadIdx.x == 0) *hexp = e;
  }
  rotwin_block_smem_to<double>(h, dblk, dstride, nb, eg, Lh, Ng, b, p, ch, z, RotwinBoth{H, Hdd, e}, smem, qmask);
}

__global__ void __launch_bounds__(128) k_batch_rotwin(const BRot* __restrict__ rot, const BRotBlk* __restrict__ blk,
                                                      int nblk, const int* __restrict__ n_dev) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int cnt = n_dev != nullptr ? *n_dev : nblk;
  for (int i = blockIdx.x; i < cnt; i += gridDim.x) {
    const BRotBlk bb = blk[i];
    const BRot r = rot[bb.rot];
    const size_t S = blk_off(r.Lh);
    const size_t off = (size_t)bb.b * S + blk_off(bb.p);
    const int nb = min(ROTWIN_NB, r.Nb - bb.b);
    RotChunks ch;
    ch.QC = r.QC; ch.CC = r.CC; ch.nq = r.nq; ch.nc = r.nc;
    if (r.prec == 0) {
      rotwin_block_fp64(r.h, (const double*)r.dt + off, S, nb, (const double2*)r.eg, r.Lh, r.Ng, bb.b, bb.p, ch,
                        bb.z, (double2*)r.H, r.Hdd, r.hexp, smem_raw, r.qmask);
    } else {
      rotwin_block_smem_to<float>(r.h, (const float*)r.dt + off, S, nb, (const float2*)r.eg, r.Lh, r.Ng, bb.b, bb.p,
                                  ch, bb.z, RotwinStore<float>{(float2*)r.H}, smem_raw, r.qmask);
    }
    __syncthreads();               // the block's shared memory is reused by its next entry
  }
}

cudaError_t launch_batch_rotwin(const BRot* rot, const BRotBlk* blk, int nblk, size_t smem, cudaStream_t st) {
  if (nblk <= 0) return cudaSuccess;
  if (smem > ROTWIN_SMEM_LIMIT) return cudaErrorInvalidValue;
  cudaError_t e = batch_attrs();
  if (e != cudaSuccess) return e;
  k_batch_rotwin<<<nblk, 128, smem, st>>>(rot, blk, nblk, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_batch_rotwin_n(const BRot* rot, const BRotBlk* blk, const int* n, int grid, size_t smem,
                                  cudaStream_t st) {
  if (smem > ROTWIN_SMEM_LIMIT) return cudaErrorInvalidValue;
  cudaError_t e = batch_attrs();
  if (e != cudaSuccess) return e;
  k_batch_rotwin<<<grid, 128, smem, st>>>(rot, blk, 0, n);
  return cudaGetLastError();
}

// grid (Nb, Lh, chunks): the scaled double-float window of one call
__global__ void __launch_bounds__(128) k_rotwin_dd(const double2* __restrict__ h, const double* __restrict__ dt,
                                                   const double2* __restrict__ eg, int Lh, int Nb, int Ng,
                                                   RotChunks ch, float4* Hdd, int* hexp,
                                                   const uint32_t* __restrict__ qmask) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int b0 = blockIdx.x * ROTWIN_NB, p = blockIdx.y;
  const size_t S = blk_off(Lh);
  rotwin_block_fp64(h, dt + (size_t)b0 * S + blk_off(p), S, min(ROTWIN_NB, Nb - b0), eg, Lh, Ng, b0, p, ch,
                    blockIdx.z, nullptr, Hdd, hexp, smem_raw, qmask);
}

cudaError_t launch_rotwin_dd(const double2* h, const double* dt, const double2* eg, int Lh, int Nb, int Ng,
                             float4* Hdd, int* hexp, cudaStream_t st, const uint32_t* qmask) {
  const RotChunks ch = rot_chunks(Lh, Ng, sizeof(double2));
  cudaError_t e = batch_attrs();
  if (e != cudaSuccess) return e;
  dim3 grid((Nb + ROTWIN_NB - 1) / ROTWIN_NB, Lh, ch.nq * ch.nc);
  k_rotwin_dd<<<grid, 128, ch.smem(Lh, sizeof(double2)), st>>>(h, dt, eg, Lh, Nb, Ng, ch, Hdd, hexp, qmask);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- alpha stage
// Split-DFT constants sit after the X tile: cos and sin tables of
// ((P+1)/2)^2 entries each (P <= 9).
#define BA_CONST_ENTRIES 25

template <typename T, int P>
__device__ __forceinline__ void ba_split(const BItem& it, const BTile& tl, const typename vec2<T>::t* sx, const T* cst,
                                         typename vec2<T>::t* dst, typename vec2<T>::t* mdst, T sgn, int c, int s) {
  constexpr int H = (P - 1) / 2;
  const int S = BA_THREADS / it.nt;
  const T(*cpr)[H + 1] = reinterpret_cast<const T(*)[H + 1]>(cst);
  const T(*spr)[H + 1] = reinterpret_cast<const T(*)[H + 1]>(cst + BA_CONST_ENTRIES);
  alpha_split_column<T, P>(sx + c, it.nt, it.Lh, it.Na, it.J, reinterpret_cast<const typename vec2<T>::t*>(it.csa),
                           cpr, spr, dst, mdst, sgn, s, S);
}

template <typename T, int P>
__device__ __forceinline__ void ba_consts(T* cst) {
  constexpr int H = (P - 1) / 2;
  alpha_split_consts<T, P>(reinterpret_cast<T(*)[H + 1]>(cst), reinterpret_cast<T(*)[H + 1]>(cst + BA_CONST_ENTRIES),
                           threadIdx.x);
}

template <typename T>
__device__ __forceinline__ void ba_tile(const BItem& it, const BTile& tl, unsigned char* smem) {
  typedef typename vec2<T>::t T2;
  const int Lh = it.Lh, K = 2 * Lh - 1, n2 = Lh * Lh, NT = it.nt, S = BA_THREADS / NT;
  const int J = it.J, Na = it.Na, tid = threadIdx.x;
  T2* sx = reinterpret_cast<T2*>(smem);                      // [q + Lh - 1][NT]
  T* cst = reinterpret_cast<T*>(sx + (size_t)K * NT);       // split-DFT constants
  // the pair's k in T: FP32 tiles with L_h <= 32 convert it once into shared
  // memory (a float/double conversion runs on the slow FP64 pipe); wider
  // windows (the row would cost occupancy) and FP64 tiles read it as stored
  const double2* kd = it.kc + (size_t)tl.pair * n2;
  const bool staged = sizeof(T) == sizeof(float) && Lh <= 32;
  const T2* kp;
  if (staged) {
    T2* sk = reinterpret_cast<T2*>(cst + 2 * BA_CONST_ENTRIES);
    for (int t = tid; t < n2; t += BA_THREADS) {
      const double2 v = kd[t];
      sk[t] = mk2((T)v.x, (T)v.y);
    }
    __syncthreads();
    kp = sk;
  } else {
    kp = nullptr;
  }
  const T2* H = reinterpret_cast<const T2*>(it.H);
  const bool om = sizeof(T) == sizeof(float) && h_order_major(Lh);   // the FP32 wide window's row order
  // X_q for the tile's columns: four degrees' loads in flight per step
  for (int e = tid; e < K * NT; e += BA_THREADS) {
    const int qi = e / NT, c = e - qi * NT;
    const int q = qi - (Lh - 1), aq = q < 0 ? -q : q;
    const int j = tl.j0 + c;
    T xr = 0, xi = 0;
    if (j < J) {
      for (int p0 = aq; p0 < Lh; p0 += 4) {
        T2 hv[4], kv[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int p = p0 + v;
          if (p < Lh) {
            const int pq = p * p + p + q;
            hv[v] = H[h_index(om ? h_row(p, q, Lh, true) : pq, j, n2)];
            if (staged) {
              kv[v] = kp[pq];
            } else {
              const double2 k2 = __ldg(kd + pq);
              kv[v] = mk2((T)k2.x, (T)k2.y);
            }
          } else {
            hv[v] = mk2((T)0, (T)0);
            kv[v] = mk2((T)0, (T)0);
          }
        }
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const T kr = kv[v].x, ki = kv[v].y;
          xr = fma(kr, hv[v].x, xr); xr = fma(-ki, hv[v].y, xr);
          xi = fma(kr, hv[v].y, xi); xi = fma(ki, hv[v].x, xi);
        }
      }
    }
    sx[e] = mk2(xr, xi);
  }
  switch (it.form) {
    case 3: ba_consts<T, 3>(cst); break;
    case 5: ba_consts<T, 5>(cst); break;
    case 7: ba_consts<T, 7>(cst); break;
    case 9: ba_consts<T, 9>(cst); break;
    default: break;
  }
  __syncthreads();
  if (it.form == 0) {
    // +-q pairs in place: row Lh-1+r <- P_r = X_r + X_-r, row Lh-1-r <- M_r = X_r - X_-r
    for (int e = tid; e < (Lh - 1) * NT; e += BA_THREADS) {
      const int r = e / NT + 1, c = e - (r - 1) * NT;
      const T2 a = sx[(Lh - 1 + r) * NT + c], b = sx[(Lh - 1 - r) * NT + c];
      sx[(Lh - 1 + r) * NT + c] = mk2(a.x + b.x, a.y + b.y);
      sx[(Lh - 1 - r) * NT + c] = mk2(a.x - b.x, a.y - b.y);
    }
    __syncthreads();
  }
  const int c = tid % NT, s = tid / NT, j = tl.j0 + c;
  if (j >= J) return;
  // output slot and, for a mirrored pair, the slot of (l, -m) with (-1)^m
  const int2 sl = it.slots != nullptr ? it.slots[tl.pair] : make_int2(tl.out, -1);
  T2* g = reinterpret_cast<T2*>(it.g);
  T2* dst = g + (size_t)sl.x * Na * J + j;
  T2* mdst = sl.y >= 0 ? g + (size_t)(sl.y >> 1) * Na * J + j : nullptr;
  const T sgn = (sl.y & 1) ? (T)-1 : (T)1;
  switch (it.form) {
    case 0:
      alpha_direct_column<T>(sx + c, NT, Lh - 1, Lh - 1, 1, Lh - 1, -1, Lh, Na, J,
                             reinterpret_cast<const T2*>(it.csa), dst, mdst, sgn, s * ALPHA_ABLK, S * ALPHA_ABLK);
      break;
    case 3: ba_split<T, 3>(it, tl, sx, cst, dst, mdst, sgn, c, s); break;
    case 5: ba_split<T, 5>(it, tl, sx, cst, dst, mdst, sgn, c, s); break;
    case 7: ba_split<T, 7>(it, tl, sx, cst, dst, mdst, sgn, c, s); break;
    case 9: ba_split<T, 9>(it, tl, sx, cst, dst, mdst, sgn, c, s); break;
    default: break;
  }
}

// The tile of an FP64 item in double-float arithmetic: X_q from the scaled
// double-float k and H, the alpha sum (direct or split) from double-float
// tables, each output assembled as a double with the scale 2^(kexp + hexp).
template <int P>
__device__ __forceinline__ void ba_split_dd(const BItem& it, const float4* sx, const ddv* cst, const DdOut& out, int c,
                                            int s) {
  constexpr int H = (P - 1) / 2;
  alpha_split_column_dd<P>(sx + c, it.nt, it.Lh, it.Na, it.J, reinterpret_cast<const float4*>(it.csa), cst,
                           cst + (H + 1) * (H + 1), out, s, BA_THREADS / it.nt);
}

template <int P>
__device__ __forceinline__ void ba_consts_dd(ddv* cst) {
  constexpr int H = (P - 1) / 2;
  const int t = threadIdx.x;
  if (t < (H + 1) * (H + 1)) {
    const int r = t / (H + 1), s = t % (H + 1);
    double sv, cv;
    sincospi(2.0 * r * s / P, &sv, &cv);
    dd_split(cv, &cst[t].h, &cst[t].l);
    dd_split(sv, &cst[(H + 1) * (H + 1) + t].h, &cst[(H + 1) * (H + 1) + t].l);
  }
}

__device__ __forceinline__ void ba_tile_dd(const BItem& it, const BTile& tl, unsigned char* smem) {
  const int Lh = it.Lh, K = 2 * Lh - 1, n2 = Lh * Lh, NT = it.nt, S = BA_THREADS / NT;
  const int J = it.J, Na = it.Na, tid = threadIdx.x;
  float4* sx = reinterpret_cast<float4*>(smem);                    // [q + Lh - 1][NT]
  ddv* cst = reinterpret_cast<ddv*>(sx + (size_t)K * NT);          // split-DFT constants
  const float4* kp = it.kdd + (size_t)tl.pair * n2;
  const float4* H = reinterpret_cast<const float4*>(it.H);
  for (int e = tid; e < K * NT; e += BA_THREADS) {
    const int qi = e / NT, c = e - qi * NT;
    const int q = qi - (Lh - 1), aq = q < 0 ? -q : q;
    const int j = tl.j0 + c;
    dd_acc xr = dd_acc_zero(), xi = dd_acc_zero();
    if (j < J) {
      for (int p0 = aq; p0 < Lh; p0 += 4) {
        float4 hv[4], kv[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int p = p0 + v;
          if (p < Lh) {
            const int pq = p * p + p + q;
            hv[v] = __ldg(H + h_index(pq, j, n2));
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
    const ddv vr = ddv_of(xr), vi = ddv_of(xi);
    sx[e] = make_float4(vr.h, vi.h, vr.l, vi.l);
  }
  switch (it.form) {
    case 3: ba_consts_dd<3>(cst); break;
    case 5: ba_consts_dd<5>(cst); break;
    case 7: ba_consts_dd<7>(cst); break;
    case 9: ba_consts_dd<9>(cst); break;
    default: break;
  }
  __syncthreads();
  if (it.form == 0) {
    for (int e = tid; e < (Lh - 1) * NT; e += BA_THREADS) {
      const int r = e / NT + 1, c = e - (r - 1) * NT;
      const ddc a = ddc_load_smem(sx + (Lh - 1 + r) * NT + c), b = ddc_load_smem(sx + (Lh - 1 - r) * NT + c);
      sx[(Lh - 1 + r) * NT + c] = ddc_pack({ddv_add(a.re, b.re), ddv_add(a.im, b.im)});
      sx[(Lh - 1 - r) * NT + c] = ddc_pack({ddv_sub(a.re, b.re), ddv_sub(a.im, b.im)});
    }
    __syncthreads();
  }
  const int c = tid % NT, s = tid / NT, j = tl.j0 + c;
  if (j >= J) return;
  // output slot and, for a mirrored pair, the slot of (l, -m) with (-1)^m
  const int2 sl = it.slots != nullptr ? it.slots[tl.pair] : make_int2(tl.out, -1);
  double2* g = reinterpret_cast<double2*>(it.g);
  DdOut out;
  out.dst = g + (size_t)sl.x * Na * J + j;
  out.mdst = sl.y >= 0 ? g + (size_t)(sl.y >> 1) * Na * J + j : nullptr;
  out.sgn = (sl.y & 1) ? (1ull << 63) : 0ull;
  out.sc = it.kexp[tl.pair] + *it.hexp;
  switch (it.form) {
    case 0:
      alpha_direct_column_dd(sx + c, NT, Lh - 1, Lh - 1, 1, Lh - 1, -1, Lh, Na, J,
                             reinterpret_cast<const float4*>(it.csa), out, s * ALPHA_ABLK, S * ALPHA_ABLK);
      break;
    case 3: ba_split_dd<3>(it, sx, cst, out, c, s); break;
    case 5: ba_split_dd<5>(it, sx, cst, out, c, s); break;
    case 7: ba_split_dd<7>(it, sx, cst, out, c, s); break;
    case 9: ba_split_dd<9>(it, sx, cst, out, c, s); break;
    default: break;
  }
}

__global__ void __launch_bounds__(BA_THREADS) k_batch_alpha_dd(const BItem* __restrict__ items,
                                                               const BTile* __restrict__ tiles, int ntiles,
                                                               int* __restrict__ counter,
                                                               const int* __restrict__ n_dev) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_tile;
  if (n_dev != nullptr) ntiles = *n_dev;
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(counter, 1);
    __syncthreads();
    const int ti = s_tile;
    if (ti >= ntiles) return;
    const BTile tl = tiles[ti];
    const BItem it = items[tl.item];
    ba_tile_dd(it, tl, smem_raw);
    __syncthreads();
  }
}

// One item in FP64 or FP32 arithmetic, every (pair, column block) tile in
// index order, CTAs striding (equal tiles: no counter needed).
template <typename T>
__global__ void __launch_bounds__(BA_THREADS) k_alpha_single(const BItem it, int ntiles) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ntj = (it.J + it.nt - 1) / it.nt;
  for (int ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
    const BTile tl{0, ti / ntj, ti / ntj, (ti % ntj) * it.nt};
    ba_tile<T>(it, tl, smem_raw);
    __syncthreads();
  }
}

// The same for the double-float engine.
__global__ void __launch_bounds__(BA_THREADS) k_alpha_dd_single(const BItem it, int ntiles) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ntj = (it.J + it.nt - 1) / it.nt;
  for (int ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
    const BTile tl{0, ti / ntj, ti / ntj, (ti % ntj) * it.nt};
    ba_tile_dd(it, tl, smem_raw);
    __syncthreads();
  }
}

// One instantiation per precision: items of the other precision are never
// in its tile list.
template <typename T>
__global__ void __launch_bounds__(BA_THREADS) k_batch_alpha(const BItem* __restrict__ items,
                                                            const BTile* __restrict__ tiles, int ntiles,
                                                            int* __restrict__ counter, const int* __restrict__ n_dev) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_tile;
  if (n_dev != nullptr) ntiles = *n_dev;
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(counter, 1);
    __syncthreads();
    const int ti = s_tile;
    if (ti >= ntiles) return;
    const BTile tl = tiles[ti];
    const BItem it = items[tl.item];
    ba_tile<T>(it, tl, smem_raw);
    __syncthreads();   // the tile's shared memory and s_tile are reused
  }
}

size_t batch_alpha_smem(int prec, int Lh, int nt) {
  const size_t el2 = prec == 1 ? sizeof(float2) : 16;     // double2, or float4 double-float pairs
  const size_t cst = prec == 1 ? sizeof(float) : (prec == 0 ? sizeof(double) : sizeof(ddv));
  // X tile, split-DFT constants, and (FP32 kernel, L_h <= 32) the pair's k row as floats
  const size_t krow = (prec == 1 && Lh <= 32) ? sizeof(float2) * (size_t)Lh * Lh : 0;
  const size_t b = el2 * (size_t)(2 * Lh - 1) * nt + 2 * cst * BA_CONST_ENTRIES + krow;
  return (b + 15) / 16 * 16;
}

static const void* batch_alpha_fn(int prec) {
  return prec == 0 ? (const void*)k_batch_alpha<double>
                   : (prec == 1 ? (const void*)k_batch_alpha<float> : (const void*)k_batch_alpha_dd);
}

// The batch kernels' dynamic shared-memory ceiling is set once, to
// BA_SMEM_LIMIT, before any launch: a per-plan value could be lowered by a
// later plan under the graph nodes of an earlier one, and the attribute call
// is kept out of stream captures.
static cudaError_t g_attr_status = cudaErrorNotReady;
static std::once_flag g_attr_once;

static cudaError_t batch_attrs() {
  std::call_once(g_attr_once, [] {
    cudaError_t e = cudaFuncSetAttribute(k_batch_alpha<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         BA_SMEM_LIMIT);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_batch_alpha<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, BA_SMEM_LIMIT);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_batch_alpha_dd, cudaFuncAttributeMaxDynamicSharedMemorySize, BA_SMEM_LIMIT);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_alpha_dd_single, cudaFuncAttributeMaxDynamicSharedMemorySize, BA_SMEM_LIMIT);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_alpha_single<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, BA_SMEM_LIMIT);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_alpha_single<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, BA_SMEM_LIMIT);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_rotwin_dd, cudaFuncAttributeMaxDynamicSharedMemorySize, BA_SMEM_LIMIT);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_batch_rotwin, cudaFuncAttributeMaxDynamicSharedMemorySize, BA_SMEM_LIMIT);
    g_attr_status = e;
  });
  return g_attr_status;
}

int batch_alpha_occupancy(int prec, size_t smem) {
  if (batch_attrs() != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_alpha_fn(prec), BA_THREADS, smem) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return n > 0 ? n : 1;
}

cudaError_t launch_batch_alpha(int prec, const BItem* items, const BTile* tiles, int ntiles, int* counter, int grid,
                               size_t smem, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  if (smem > BA_SMEM_LIMIT) return cudaErrorInvalidValue;
  cudaError_t e = batch_attrs();
  if (e != cudaSuccess) return e;
  if (prec == 0) k_batch_alpha<double><<<grid, BA_THREADS, smem, st>>>(items, tiles, ntiles, counter, nullptr);
  else if (prec == 1) k_batch_alpha<float><<<grid, BA_THREADS, smem, st>>>(items, tiles, ntiles, counter, nullptr);
  else k_batch_alpha_dd<<<grid, BA_THREADS, smem, st>>>(items, tiles, ntiles, counter, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_batch_alpha_n(int prec, const BItem* items, const BTile* tiles, const int* n, int* counter,
                                 int grid, size_t smem, cudaStream_t st) {
  if (smem > BA_SMEM_LIMIT) return cudaErrorInvalidValue;
  cudaError_t e = batch_attrs();
  if (e != cudaSuccess) return e;
  if (prec == 0) k_batch_alpha<double><<<grid, BA_THREADS, smem, st>>>(items, tiles, 0, counter, n);
  else if (prec == 1) k_batch_alpha<float><<<grid, BA_THREADS, smem, st>>>(items, tiles, 0, counter, n);
  else k_batch_alpha_dd<<<grid, BA_THREADS, smem, st>>>(items, tiles, 0, counter, n);
  return cudaGetLastError();
}

int batch_rotwin_occupancy(size_t smem) {
  if (batch_attrs() != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_rotwin, 128, smem) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return n > 0 ? n : 1;
}

cudaError_t launch_alpha_dd_call(const BItem& item, int npairs, int num_sms, cudaStream_t st) {
  return launch_alpha_call(item, npairs, num_sms, st);
}

cudaError_t launch_alpha_call(const BItem& item, int npairs, int num_sms, cudaStream_t st) {
  if (npairs <= 0 || item.J <= 0) return cudaSuccess;
  const size_t smem = batch_alpha_smem(item.prec, item.Lh, item.nt);
  if (smem > BA_SMEM_LIMIT) return cudaErrorInvalidValue;
  cudaError_t e = batch_attrs();
  if (e != cudaSuccess) return e;
  const void* fn = item.prec == 2 ? (const void*)k_alpha_dd_single
                   : (item.prec == 0 ? (const void*)k_alpha_single<double> : (const void*)k_alpha_single<float>);
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, BA_THREADS, smem) != cudaSuccess) {
    cudaGetLastError();
    occ = 1;
  }
  const long long ntiles = (long long)npairs * ((item.J + item.nt - 1) / item.nt);
  if (ntiles > 0x7fffffffLL) return cudaErrorInvalidValue;
  const int grid = (int)std::min<long long>((long long)num_sms * std::max(occ, 1), ntiles);
  if (item.prec == 2) k_alpha_dd_single<<<grid, BA_THREADS, smem, st>>>(item, (int)ntiles);
  else if (item.prec == 0) k_alpha_single<double><<<grid, BA_THREADS, smem, st>>>(item, (int)ntiles);
  else k_alpha_single<float><<<grid, BA_THREADS, smem, st>>>(item, (int)ntiles);
  return cudaGetLastError();
}
