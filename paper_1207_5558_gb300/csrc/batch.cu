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
#include <mutex>

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

static cudaError_t batch_attrs();

// ---------------------------------------------------------------- rotated windows
__global__ void __launch_bounds__(128) k_batch_rotwin(const BRot* __restrict__ rot, const BRotBlk* __restrict__ blk) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const BRotBlk bb = blk[blockIdx.x];
  const BRot r = rot[bb.rot];
  const size_t off = (size_t)bb.b * blk_off(r.Lh) + blk_off(bb.p);
  if (r.prec == 0) {
    const double* d = (const double*)r.dt + off;
    if (r.smem_ok)
      rotwin_block_smem<double>(r.h, d, (const double2*)r.eg, r.Lh, r.Ng, bb.b, bb.p, (double2*)r.H, smem_raw);
    else
      rotwin_block_direct<double>(r.h, d, (const double2*)r.eg, r.Lh, r.Ng, bb.b, bb.p, (double2*)r.H);
  } else {
    const float* d = (const float*)r.dt + off;
    if (r.smem_ok)
      rotwin_block_smem<float>(r.h, d, (const float2*)r.eg, r.Lh, r.Ng, bb.b, bb.p, (float2*)r.H, smem_raw);
    else
      rotwin_block_direct<float>(r.h, d, (const float2*)r.eg, r.Lh, r.Ng, bb.b, bb.p, (float2*)r.H);
  }
}

cudaError_t launch_batch_rotwin(const BRot* rot, const BRotBlk* blk, int nblk, size_t smem, cudaStream_t st) {
  if (nblk <= 0) return cudaSuccess;
  if (smem > BA_SMEM_LIMIT) return cudaErrorInvalidValue;
  cudaError_t e = batch_attrs();
  if (e != cudaSuccess) return e;
  k_batch_rotwin<<<nblk, 128, smem, st>>>(rot, blk);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- alpha stage
// Split-DFT constants sit after the X tile: cos and sin tables of
// ((P+1)/2)^2 entries each (P <= 9).
#define BA_CONST_ENTRIES 25

template <typename T, int P>
__device__ __forceinline__ void ba_split(const BItem& it, const BTile& tl, const typename vec2<T>::t* sx, const T* cst,
                                         typename vec2<T>::t* dst, int c, int s) {
  constexpr int H = (P - 1) / 2;
  const int S = BA_THREADS / it.nt;
  const T(*cpr)[H + 1] = reinterpret_cast<const T(*)[H + 1]>(cst);
  const T(*spr)[H + 1] = reinterpret_cast<const T(*)[H + 1]>(cst + BA_CONST_ENTRIES);
  alpha_split_column<T, P>(sx + c, it.nt, it.Lh, it.Na, it.J, reinterpret_cast<const typename vec2<T>::t*>(it.csa),
                           cpr, spr, dst, nullptr, (T)1, s, S);
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
  const double2* kp = it.kc + (size_t)tl.pair * n2;
  const T2* H = reinterpret_cast<const T2*>(it.H);
  // X_q for the tile's columns: four degrees' loads in flight per step
  for (int e = tid; e < K * NT; e += BA_THREADS) {
    const int qi = e / NT, c = e - qi * NT;
    const int q = qi - (Lh - 1), aq = q < 0 ? -q : q;
    const int j = tl.j0 + c;
    T xr = 0, xi = 0;
    if (j < J) {
      for (int p0 = aq; p0 < Lh; p0 += 4) {
        T2 hv[4];
        double2 kv[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int p = p0 + v;
          if (p < Lh) {
            const int pq = p * p + p + q;
            hv[v] = H[h_index(pq, j, n2)];
            kv[v] = __ldg(kp + pq);
          } else {
            hv[v] = mk2((T)0, (T)0);
            kv[v] = make_double2(0.0, 0.0);
          }
        }
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const T kr = (T)kv[v].x, ki = (T)kv[v].y;
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
  T2* dst = reinterpret_cast<T2*>(it.g) + (size_t)tl.out * Na * J + j;
  switch (it.form) {
    case 0:
      alpha_direct_column<T>(sx + c, NT, Lh - 1, Lh - 1, 1, Lh - 1, -1, Lh, Na, J,
                             reinterpret_cast<const T2*>(it.csa), dst, nullptr, (T)1, s * ALPHA_ABLK,
                             S * ALPHA_ABLK);
      break;
    case 3: ba_split<T, 3>(it, tl, sx, cst, dst, c, s); break;
    case 5: ba_split<T, 5>(it, tl, sx, cst, dst, c, s); break;
    case 7: ba_split<T, 7>(it, tl, sx, cst, dst, c, s); break;
    case 9: ba_split<T, 9>(it, tl, sx, cst, dst, c, s); break;
    default: break;
  }
}

// One instantiation per precision: items of the other precision are never
// in its tile list.
template <typename T>
__global__ void __launch_bounds__(BA_THREADS) k_batch_alpha(const BItem* __restrict__ items,
                                                            const BTile* __restrict__ tiles, int ntiles,
                                                            int* __restrict__ counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_tile;
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
  const size_t el = prec == 0 ? sizeof(double) : sizeof(float);
  const size_t b = 2 * el * (size_t)(2 * Lh - 1) * nt + 2 * el * BA_CONST_ENTRIES;
  return (b + 15) / 16 * 16;
}

static const void* batch_alpha_fn(int prec) {
  return prec == 0 ? (const void*)k_batch_alpha<double> : (const void*)k_batch_alpha<float>;
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
  if (prec == 0) k_batch_alpha<double><<<grid, BA_THREADS, smem, st>>>(items, tiles, ntiles, counter);
  else k_batch_alpha<float><<<grid, BA_THREADS, smem, st>>>(items, tiles, ntiles, counter);
  return cudaGetLastError();
}
