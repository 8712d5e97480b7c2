// Device tables: Delta = d(pi/2) by the Trapani-Navaza recursion, Wigner-d at
// the beta samples through the factorisation of rotations, phase tables and
// beta quadrature weights.  All generated in FP64 (cast on store where the
// FP32 path wants float).
#include "common.cuh"

// Writes the eight symmetric images of Delta^p_{m,m'} (0 <= m' <= m <= p).
// At beta = pi/2:  Delta_{-m,m'} = (-1)^{p+m'} Delta_{m,m'},
//                  Delta_{m,-m'} = (-1)^{p+m} Delta_{m,m'},
//                  Delta_{m',m}  = (-1)^{m-m'} Delta_{m,m'}   (Sec. IV-B symmetries).
__device__ __forceinline__ void delta_store8(double* blk, int p, int m, int mp, double v) {
  const int W = 2 * p + 1;
  const double s_pm = ((p + m) & 1) ? -1.0 : 1.0;
  const double s_pmp = ((p + mp) & 1) ? -1.0 : 1.0;
  const double s_t = ((m - mp) & 1) ? -1.0 : 1.0;
#define AT(a, b) blk[((a) + p) * W + ((b) + p)]
  AT(m, mp) = v;
  AT(-m, mp) = s_pmp * v;
  AT(m, -mp) = s_pm * v;
  AT(-m, -mp) = s_t * v;
  AT(mp, m) = s_t * v;
  AT(-mp, m) = s_pm * s_t * v;
  AT(mp, -m) = s_pmp * s_t * v;
  AT(-mp, -m) = v;
#undef AT
}

// One CTA, degrees in sequence.  For degree p the edge row Delta^p_{p,m'} is
// obtained from the previous edge,
//   Delta^p_{p,0}  = -sqrt((2p-1)/(2p)) Delta^{p-1}_{p-1,0},
//   Delta^p_{p,m'} =  sqrt(p(2p-1)/(2(p+m')(p+m'-1))) Delta^{p-1}_{p-1,m'-1},
// and thread m' then runs the three-term recurrence downward in m,
//   Delta_{m,m'} = [2m' Delta_{m+1,m'} - sqrt((p-m-1)(p+m+2)) Delta_{m+2,m'}]
//                  / sqrt((p-m)(p+m+1)),
// which follows from the J_z relation d(b) J_z = (J_z cos b + J_x sin b) d(b)
// at b = pi/2, down to m = m' (the eighth 0 <= m' <= m <= p).
__global__ void k_delta(double* __restrict__ D, int Lh) {
  __shared__ double edge_prev[SLSHT_MAX_LH];
  __shared__ double edge_cur[SLSHT_MAX_LH];
  const int t = threadIdx.x;
  for (int p = 0; p < Lh; ++p) {
    if (t <= p) {
      double e;
      if (p == 0) e = 1.0;
      else if (t == 0) e = -sqrt((2.0 * p - 1.0) / (2.0 * p)) * edge_prev[0];
      else e = sqrt(p * (2.0 * p - 1.0) / (2.0 * (p + t) * (p + t - 1.0))) * edge_prev[t - 1];
      edge_cur[t] = e;
    }
    __syncthreads();
    if (t <= p) {
      double* blk = D + blk_off(p);
      double a1 = edge_cur[t], a2 = 0.0;
      delta_store8(blk, p, p, t, a1);
      for (int m = p - 1; m >= t; --m) {
        const double v = (2.0 * t * a1 - sqrt((double)(p - m - 1) * (double)(p + m + 2)) * a2) /
                         sqrt((double)(p - m) * (double)(p + m + 1));
        delta_store8(blk, p, m, t, v);
        a2 = a1;
        a1 = v;
      }
    }
    __syncthreads();
    if (t <= p) edge_prev[t] = edge_cur[t];
    __syncthreads();
  }
}

cudaError_t launch_delta(double* D, int Lh, cudaStream_t st) {
  k_delta<<<1, SLSHT_MAX_LH, 0, st>>>(D, Lh);
  return cudaGetLastError();
}

__device__ __forceinline__ int degree_of(int idx, int Lh) {
  int p = 0;
  while (p + 1 < Lh && blk_off(p + 1) <= idx) ++p;
  return p;
}

// d^p_{q,q'}(beta_b) = Re[ i^{q-q'} sum_{q''} Delta^p_{q''q} Delta^p_{q''q'} e^{-i q'' beta_b} ]
// (Eq. WignerD_expansion_new at alpha = gamma = 0), beta_b = 2 pi b / (2 Nb - 1).
// Layout [b][S].  A block serves one beta row: the 2Lh-1 phases e^{-i q'' beta_b}
// are computed once into shared memory, so an entry costs 2(2p+1) FP64
// multiply-adds.
template <typename T>
__global__ void k_dtable(const double* __restrict__ D, T* __restrict__ dt, int Lh, int Nb) {
  extern __shared__ double2 ph[];                 // [q'' + Lh - 1] = (cos, sin)(q'' beta_b)
  const int S = blk_off(Lh);
  const int b = blockIdx.y;
  const long long M = 2LL * Nb - 1;
  for (int t = threadIdx.x; t < 2 * Lh - 1; t += blockDim.x) {
    double s, c;
    sincos_2pi_frac((long long)(t - (Lh - 1)) * b, M, &s, &c);
    ph[t] = make_double2(c, s);
  }
  __syncthreads();
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < S; idx += gridDim.x * blockDim.x) {
    const int p = degree_of(idx, Lh);
    const int W = 2 * p + 1;
    const int r = idx - blk_off(p);
    const int q = r / W - p, qp = r % W - p;
    const double* blk = D + blk_off(p);
    double sr = 0.0, si = 0.0;
    for (int qpp = -p; qpp <= p; ++qpp) {
      const double w = blk[(qpp + p) * W + (q + p)] * blk[(qpp + p) * W + (qp + p)];
      const double2 e = ph[qpp + Lh - 1];
      sr = fma(w, e.x, sr);
      si = fma(-w, e.y, si);
    }
    double v;
    switch ((((q - qp) % 4) + 4) % 4) {
      case 0: v = sr; break;
      case 1: v = -si; break;
      case 2: v = -sr; break;
      default: v = si; break;
    }
    dt[(size_t)b * S + idx] = (T)v;
  }
}

cudaError_t launch_dtable_f64(const double* D, double* dt, int Lh, int Nb, cudaStream_t st) {
  const int S = blk_off(Lh);
  dim3 grid((S + 255) / 256, Nb);
  k_dtable<double><<<grid, 256, sizeof(double2) * (2 * Lh - 1), st>>>(D, dt, Lh, Nb);
  return cudaGetLastError();
}
cudaError_t launch_dtable_f32(const double* D, float* dt, int Lh, int Nb, cudaStream_t st) {
  const int S = blk_off(Lh);
  dim3 grid((S + 255) / 256, Nb);
  k_dtable<float><<<grid, 256, sizeof(double2) * (2 * Lh - 1), st>>>(D, dt, Lh, Nb);
  return cudaGetLastError();
}
template <typename T2>
__global__ void k_phase(T2* __restrict__ tab, int N, int R, int r0) {
  const long long n = (long long)N * R;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t / R), r = (int)(t % R);
    double s, c;
    sincos_2pi_frac((long long)(r0 + r) * i, N, &s, &c);
    tab[t] = mk2((decltype(tab[0].x))c, (decltype(tab[0].x))s);
  }
}

cudaError_t launch_phase_f64(double2* tab, int N, int R, int r0, cudaStream_t st) {
  const long long n = (long long)N * R;
  const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  k_phase<double2><<<blocks, 256, 0, st>>>(tab, N, R, r0);
  return cudaGetLastError();
}
cudaError_t launch_phase_f32(float2* tab, int N, int R, int r0, cudaStream_t st) {
  const long long n = (long long)N * R;
  const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  k_phase<float2><<<blocks, 256, 0, st>>>(tab, N, R, r0);
  return cudaGetLastError();
}

// The same table as double-float pairs: tab[i * R + r] = {cos.h, sin.h,
// cos.l, sin.l} with cos = cos.h + cos.l to about 2^-48.
__global__ void k_phase_dd(float4* __restrict__ tab, int N, int R, int r0) {
  const long long n = (long long)N * R;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t / R), r = (int)(t % R);
    double s, c;
    sincos_2pi_frac((long long)(r0 + r) * i, N, &s, &c);
    const float ch = __double2float_rn(c), sh = __double2float_rn(s);
    tab[t] = make_float4(ch, sh, __double2float_rn(c - (double)ch), __double2float_rn(s - (double)sh));
  }
}

cudaError_t launch_phase_dd(float4* tab, int N, int R, int r0, cudaStream_t st) {
  const long long n = (long long)N * R;
  const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  k_phase_dd<<<blocks, 256, 0, st>>>(tab, N, R, r0);
  return cudaGetLastError();
}

// q_b = (2/M) sum_{|k|<Nb} W(k) cos(k beta_b) (b >= 1), q_0 = (1/M) sum W(k),
// M = 2Nb - 1, W(k) = 2/(1-k^2) for even k and 0 for odd k: the printed w(m)
// of Sec. IV-A with the imaginary k = +-1 terms cancelling in the folded sum.
__global__ void k_beta_weights(double* __restrict__ w, int Nb) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= Nb) return;
  const long long M = 2LL * Nb - 1;
  double acc = 0.0;
  for (int k = -(Nb - 1); k <= Nb - 1; ++k) {
    if (k & 1) continue;
    double s, c;
    sincos_2pi_frac((long long)k * b, M, &s, &c);
    acc += 2.0 / (1.0 - (double)k * (double)k) * c;
  }
  w[b] = (b == 0 ? 1.0 : 2.0) * acc / (double)M;
}

cudaError_t launch_beta_weights(double* w, int Nb, cudaStream_t st) {
  k_beta_weights<<<(Nb + 127) / 128, 128, 0, st>>>(w, Nb);
  return cudaGetLastError();
}
