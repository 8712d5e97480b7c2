// Inverse directional SLSHT without the condition h_0^0 != 0: the
// reconstruction of the remark after Eq. inversion_2 (Sec. III-C).
//
// By the orthogonality of the Wigner D functions (Eq. WignerD_ortho), the
// projection of g(.; l, m) on conj(D^p_{q,q'}) is 8 pi^2/(2p+1) k_lm(p,q) h_p^q'.
// Summed against conj(h_p^q') over q' it leaves the window's energy at degree p,
// E_p = sum_q' |h_p^q'|^2, times k_lm(p, q):
//   khat_lm(q) = (2p+1)/(8 pi^2 E_p) int g(rho; l, m) conj(W^p_q(rho)) d rho,
//   W^p_q = sum_q' h_p^q' D^p_{q,q'} = e^{-i q alpha} H^p_q(beta, gamma),
// H^p_q the window's degree-p coefficients rotated to (0, beta, gamma), the
// quantity the forward transform builds once per call.  On the grid the
// integral is the SO(3) quadrature of the standard inverse, exact when every
// grid size is at least L_h + p.  Then the Wigner-3j orthogonality over q
// (sum_q (L p l; M q -m)(L' p l; M q -m) = delta_{LL'}/(2L+1), m = M + q)
// decouples the signal from k = sum_l' f_{l', m-q} T(l', m-q; p, q; l, m):
//   f_LM = (2L+1)/c^2 sum_q T(L, M; p, q; l, M+q) khat_{l, M+q}(q),
// c^2 = (2L+1)(2p+1)(2l+1)/(4 pi) (L p l; 0 0 0)^2.  With l = L + p the 3j
// symbols are "stretched" (closed form), and the ratio
//   rho(M, q) = (L p l; M q -m) (-1)^m / (L p l; 0 0 0)
// is positive with rho^2 = A(L, M) A(p, q) / A(L + p, m),
//   A(n, k) = C(2n, n+k) / C(2n, n) = prod_{i=1..|k|} (n - i + 1)/(n + i),
// so that f_LM = sqrt(4 pi (2L+1) / ((2p+1)(2l+1))) sum_q rho(M, q) khat_{l, M+q}(q).
//
// Kernels: k_ialt_cols reads g once (thread = column j = (beta_b, gamma_c),
// alpha rows walked down the column), forms G_q(j) = sum_a g[a][j] e^{i q alpha_a}
// for a block of IA_QB orders at a time, multiplies by q_b conj(H^p_q(j)) and
// reduces the CTA's columns in a fixed tree; k_ialt_khat adds the CTAs of a
// pair in a fixed order and scales; k_ialt_combine forms every f_LM.  Every
// reduction has a fixed order: results are bitwise reproducible.
#include "common.cuh"

#define IA_THREADS 128
#define IA_QB 8

template <typename T2>
struct ia_acc;                       // accumulation type of the alpha sum
template <>
struct ia_acc<double2> { typedef double t; typedef double2 t2; };
template <>
struct ia_acc<float2> { typedef float t; typedef float2 t2; };

// partial[((pair * ncb + cb) * K + q + p] over the CTA's columns
template <typename T2>
__global__ void __launch_bounds__(IA_THREADS)
k_ialt_cols(const T2* __restrict__ g, const double* __restrict__ wb, const double* __restrict__ dt, int S,
            const double2* __restrict__ hp, const typename ia_acc<T2>::t2* __restrict__ ea,
            const double2* __restrict__ eg, int Na, int Nb, int Ng, int p, double2* __restrict__ partial) {
  typedef typename ia_acc<T2>::t A;
  __shared__ double sre[IA_THREADS], sim[IA_THREADS];
  const int cb = blockIdx.x, pair = blockIdx.y, ncb = gridDim.x;
  const int K = 2 * p + 1;
  const size_t J = (size_t)Nb * Ng;
  const size_t j = (size_t)cb * IA_THREADS + threadIdx.x;
  const bool live = j < J;
  const int b = live ? (int)(j / Ng) : 0, c = live ? (int)(j % Ng) : 0;
  const T2* col = g + (size_t)pair * Na * J + (live ? j : 0);
  const double* db = dt + (size_t)b * S + blk_off(p);     // d^p_{q,q'}(beta_b) at [(q+p) K + q'+p]
  const double w = live ? wb[b] : 0.0;
  for (int q0 = -p; q0 <= p; q0 += IA_QB) {
    const int nq = min(IA_QB, p - q0 + 1);
    A gr[IA_QB], gi[IA_QB];
#pragma unroll
    for (int u = 0; u < IA_QB; ++u) gr[u] = gi[u] = (A)0;
    if (live) {
      for (int a = 0; a < Na; ++a) {
        const T2 v = __ldcs(col + (size_t)a * J);
        const A vr = (A)v.x, vi = (A)v.y;
        const typename ia_acc<T2>::t2* e = ea + (size_t)a * K + (q0 + p);
#pragma unroll
        for (int u = 0; u < IA_QB; ++u) {
          if (u < nq) {                       // (vr + i vi)(cos + i sin)(q alpha_a)
            const typename ia_acc<T2>::t2 cs = e[u];
            gr[u] = fma(vr, cs.x, fma(-vi, cs.y, gr[u]));
            gi[u] = fma(vr, cs.y, fma(vi, cs.x, gi[u]));
          }
        }
      }
    }
#pragma unroll
    for (int u = 0; u < IA_QB; ++u) {
      if (u >= nq) break;
      const int q = q0 + u;
      double cr = 0.0, ci = 0.0;               // w_b conj(H^p_q(b, c)) G_q
      if (live) {
        double hr = 0.0, hi = 0.0;             // conj(H) = sum_q' conj(h_p^q') d e^{+i q' gamma_c}
        for (int qp = -p; qp <= p; ++qp) {
          const double d = db[(q + p) * K + qp + p];
          const double2 hv = hp[qp + p];                  // h_p^q'
          const double2 e = eg[(size_t)c * K + qp + p];   // (cos, sin)(q' gamma_c)
          const double ar = d * hv.x, ai = -d * hv.y;     // d conj(h)
          hr = fma(ar, e.x, fma(-ai, e.y, hr));
          hi = fma(ar, e.y, fma(ai, e.x, hi));
        }
        const double xr = (double)gr[u], xi = (double)gi[u];
        cr = w * (hr * xr - hi * xi);
        ci = w * (hr * xi + hi * xr);
      }
      sre[threadIdx.x] = cr;
      sim[threadIdx.x] = ci;
      __syncthreads();
      for (int s = IA_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
          sre[threadIdx.x] += sre[threadIdx.x + s];
          sim[threadIdx.x] += sim[threadIdx.x + s];
        }
        __syncthreads();
      }
      if (threadIdx.x == 0)
        partial[((size_t)pair * ncb + cb) * K + q + p] = make_double2(sre[0], sim[0]);
      __syncthreads();
    }
  }
}

// khat[pair][q + p] = scale * sum over the pair's CTAs (fixed order)
__global__ void k_ialt_khat(const double2* __restrict__ partial, int ncb, int K, int npairs, double scale,
                            double2* __restrict__ khat) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)npairs * K) return;
  const int pair = (int)(t / K), qi = (int)(t % K);
  double re = 0.0, im = 0.0;
  for (int cb = 0; cb < ncb; ++cb) {
    const double2 v = partial[((size_t)pair * ncb + cb) * K + qi];
    re += v.x;
    im += v.y;
  }
  khat[t] = make_double2(re * scale, im * scale);
}

// rho(M, q)^2 = A(L, M) A(p, q) / A(L + p, M + q): the factors of A(L, M)
// and 1/A(L + p, m) taken together step by step (each ratio below 1 and close
// to it, so no partial product leaves the double range), then the rest.
__device__ __forceinline__ double ialt_rho(int L, int M, int p, int q) {
  const int J = L + p, aM = abs(M), am = abs(M + q), aq = abs(q);
  double r = 1.0;
  const int n = min(aM, am);
  for (int i = 1; i <= n; ++i) r *= ((double)(L - i + 1) * (double)(J + i)) / ((double)(L + i) * (double)(J - i + 1));
  for (int i = n + 1; i <= aM; ++i) r *= (double)(L - i + 1) / (double)(L + i);
  for (int i = n + 1; i <= am; ++i) r *= (double)(J + i) / (double)(J - i + 1);
  for (int i = 1; i <= aq; ++i) r *= (double)(p - i + 1) / (double)(p + i);
  return sqrt(r);
}

// f[o] for output (L, M) = lm_out[o]; rows[o * K + q + p] = the khat row of (L + p, M + q)
__global__ void k_ialt_combine(const double2* __restrict__ khat, const int2* __restrict__ lm_out,
                               const int* __restrict__ rows, int n_out, int p, double2* __restrict__ f) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n_out) return;
  const int K = 2 * p + 1;
  const int L = lm_out[o].x, M = lm_out[o].y, l = L + p;
  double re = 0.0, im = 0.0;
  for (int q = -p; q <= p; ++q) {
    const double r = ialt_rho(L, M, p, q);
    const double2 k = khat[(size_t)rows[(size_t)o * K + q + p] * K + q + p];
    re = fma(r, k.x, re);
    im = fma(r, k.y, im);
  }
  const double pre = sqrt(4.0 * 3.14159265358979323846 * (2.0 * L + 1.0) / ((2.0 * p + 1.0) * (2.0 * l + 1.0)));
  f[o] = make_double2(pre * re, pre * im);
}

int ialt_col_blocks(int Nb, int Ng) { return (int)(((size_t)Nb * Ng + IA_THREADS - 1) / IA_THREADS); }

cudaError_t launch_inverse_alt(const void* g, int prec, const double* wb, const double* dt, int Lh,
                               const double2* hp, const void* ea, const double2* eg, int Na, int Nb, int Ng, int p,
                               int n_in, double2* partial, double scale, double2* khat, const int2* lm_out,
                               const int* rows, int n_out, double2* f, cudaStream_t st) {
  if (n_in <= 0 || n_out <= 0) return cudaSuccess;
  const int ncb = ialt_col_blocks(Nb, Ng), K = 2 * p + 1, S = blk_off(Lh);
  for (int p0 = 0; p0 < n_in; p0 += 65535) {       // grid.y limit
    const int np = n_in - p0 < 65535 ? n_in - p0 : 65535;
    dim3 grid(ncb, np);
    const size_t per_pair = (size_t)Na * Nb * Ng;
    double2* part = partial + (size_t)p0 * ncb * K;
    if (prec == 0)
      k_ialt_cols<double2><<<grid, IA_THREADS, 0, st>>>((const double2*)g + per_pair * p0, wb, dt, S, hp,
                                                        (const double2*)ea, eg, Na, Nb, Ng, p, part);
    else
      k_ialt_cols<float2><<<grid, IA_THREADS, 0, st>>>((const float2*)g + per_pair * p0, wb, dt, S, hp,
                                                       (const float2*)ea, eg, Na, Nb, Ng, p, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const long long nk = (long long)n_in * K;
  k_ialt_khat<<<(unsigned)((nk + 127) / 128), 128, 0, st>>>(partial, ncb, K, n_in, scale, khat);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_ialt_combine<<<(n_out + 127) / 128, 128, 0, st>>>(khat, lm_out, rows, n_out, p, f);
  return cudaGetLastError();
}
