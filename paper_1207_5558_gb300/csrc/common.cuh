// Shared device helpers and launcher declarations for libslsht.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define SLSHT_MAX_LH 64          // largest window band limit (exclusive)
#define SLSHT_CHAIN_MAX 128      // >= 2*SLSHT_MAX_LH - 1: longest 3j chain in j1

// Offset of the (2p+1)^2 block of degree p in tables that store every degree
// p < Lh back to back: sum_{p' < p} (2p'+1)^2 = p (4p^2 - 1) / 3.
__host__ __device__ __forceinline__ int blk_off(int p) { return p * (4 * p * p - 1) / 3; }

// cos and sin of 2 pi k / N, with the integer product reduced modulo N first
// so the argument passed to sincospi lies in [0, 2).
__device__ __forceinline__ void sincos_2pi_frac(long long k, long long N, double* s, double* c) {
  long long r = k % N;
  if (r < 0) r += N;
  sincospi(2.0 * (double)r / (double)N, s, c);
}

template <typename T> struct vec2;
template <> struct vec2<double> { typedef double2 t; };
template <> struct vec2<float> { typedef float2 t; };

__device__ __forceinline__ double2 mk2(double a, double b) { return make_double2(a, b); }
__device__ __forceinline__ float2 mk2(float a, float b) { return make_float2(a, b); }

// ----------------------------------------------------------------- launchers
// Every launcher enqueues on `st` and returns the launch status
// (cudaGetLastError after the launch).

// Delta^p = d^p(pi/2), p < Lh, full (2p+1)^2 blocks at blk_off(p).
cudaError_t launch_delta(double* D, int Lh, cudaStream_t st);
// d^p_{q,q'}(beta_b) for b < Nb from Delta (Eq. WignerD_expansion_new):
// dt[b * S + blk_off(p) + (q+p)(2p+1) + (q'+p)], S = blk_off(Lh).
cudaError_t launch_dtable_f64(const double* D, double* dt, int Lh, int Nb, cudaStream_t st);
cudaError_t launch_dtable_f32(const double* D, float* dt, int Lh, int Nb, cudaStream_t st);
// tab[i * R + r] = (cos, sin)(2 pi (r0 + r) i / N), i < N, r < R.
cudaError_t launch_phase_f64(double2* tab, int N, int R, int r0, cudaStream_t st);
cudaError_t launch_phase_f32(float2* tab, int N, int R, int r0, cudaStream_t st);
// The same as double-float pairs {cos.h, sin.h, cos.l, sin.l}.
cudaError_t launch_phase_dd(float4* tab, int N, int R, int r0, cudaStream_t st);
// beta quadrature weights q_b, b < Nb (see the inverse).
cudaError_t launch_beta_weights(double* w, int Nb, cudaStream_t st);

// k_lm(p, q) for each pair: kc[pair * Lh*Lh + p*p + p + q] (complex128), by
// 3j chains in FP64.  work (nullable, device): nwork items (pair, mirror index
// of (l, -m) or -1), every pair in exactly one item (mirror_work on the host):
// the mirror's k comes from the same chains.
cudaError_t launch_couple(const double2* f, int Lf, int Lh, const int2* lm, int npairs, double2* kc, cudaStream_t st,
                          const int2* work = nullptr, int nwork = 0);

// The same k through a signal-independent table of Gaunt coefficients:
// launch_gaunt_table fills `table` (gaunt_table_bytes) for a pair list from
// nwork work items (pair, mirror index of (l, -m) or -1; every pair appears in
// exactly one item, as pair or as mirror), launch_couple_apply then forms k
// for any signal f with that pair list.
size_t gaunt_table_bytes(int Lh, int npairs);
cudaError_t launch_gaunt_table(int Lf, int Lh, const int2* lm, int npairs, const int2* work, int nwork, void* table,
                               cudaStream_t st);
cudaError_t launch_couple_apply(const double2* f, int Lh, const int2* lm, int npairs, const void* table, double2* kc,
                                cudaStream_t st);

// k by the SHT of the modulated signal (Appendix A): Gauss-Legendre
// quadrature of the band-limited triple products on msht_nodes(L_f, L_h, lmax)
// nodes (lmax = the largest requested l); scratch of msht_scratch_bytes.
int msht_nodes(int Lf, int Lh, int lmax);
size_t msht_scratch_bytes(int Lf, int Lh, int lmax, int npairs);
cudaError_t launch_couple_msht(const double2* f, int Lf, int Lh, const int2* lm, int npairs, int lmax, void* scratch,
                               double2* kc, cudaStream_t st);

// C_{q,q',q''}(l, m) (Eq. constant_alternative_formulation), [pair][q][q'][q''].
cudaError_t launch_ctensor(const double2* kc, const double2* h, const double* D, int Lh,
                           int npairs, double2* C, cudaStream_t st);
// Y[pair][b][q][q'] = sum_q'' C[q][q'][q''] e^{-i q'' beta_b}.
cudaError_t launch_beta_dft(const double2* C, int Lh, int Nb, int npairs, double2* Y,
                            cudaStream_t st);

// Output of the beta/gamma stage for the CUDA-core alpha stage: paired sums
// Xs[pair][c][j], j = b*Ng + gamma index, c = 0: X_0, c = 2r-1: X_r + X_-r,
// c = 2r: X_r - X_-r (r = 1 .. Lh-1).
// src_y == nullptr: beta sum from the d table (separation of variables);
// otherwise from Y of launch_beta_dft (factoring of rotations).
cudaError_t launch_betagamma_f64(const double2* kc, const double2* h, const double* dt,
                                 const double2* Y, const double2* eg, int Lh, int Nb, int Ng,
                                 int npairs, double2* Xs, cudaStream_t st);
cudaError_t launch_betagamma_f32(const double2* kc, const double2* h, const float* dt,
                                 const double2* Y, const float2* eg, int Lh, int Nb, int Ng,
                                 int npairs, float2* Xs, cudaStream_t st);

// Tiled layout of the rotated window: columns j in tiles of 128, each tile
// holding all n2 = Lh^2 rows pq = p*p + p + q back to back, so one tile's rows
// are one contiguous block (128 x n2 elements; columns past J in the last
// tile are never written).
__host__ __device__ __forceinline__ size_t h_index(int pq, int j, int n2) {
  return ((size_t)(j >> 7) * (size_t)n2 + (size_t)pq) * 128 + (size_t)(j & 127);
}
// Row of (p, q) in a tile of H.  In pq order it is p*p + p + q.  The FP32
// window of a band limit L_h > 16 is stored order-major instead: the rows of
// order q (its degrees p = |q| .. L_h - 1) are one contiguous run, the runs in
// order q = -(L_h - 1) .. L_h - 1, so that the wide engine's per-order
// products read each (tile, order) as one block.  Both orders use the same
// n2 = L_h^2 rows.
__host__ __device__ __forceinline__ int h_row(int p, int q, int Lh, bool order_major) {
  if (!order_major) return p * p + p + q;
  const int a = q < 0 ? -q : q, m = Lh - 1;
  const int off = q <= 0 ? (m - a) * (m - a + 1) / 2 : m * (m + 1) / 2 + q * Lh - q * (q - 1) / 2;
  return off + p - a;
}
// Whether the FP32 window of band limit Lh is stored order-major.
__host__ __device__ __forceinline__ bool h_order_major(int Lh) { return Lh > 16; }
// Elements of the tiled H for J columns.
__host__ __device__ __forceinline__ size_t h_elems(size_t J, int n2) { return (J + 127) / 128 * 128 * (size_t)n2; }

// Rotated window H^p_q(j) = sum_q' h_p^q' d^p_{q,q'}(beta_b) e^{-i q' gamma_c},
// at H[h_index(p*p+p+q, j, Lh*Lh)], j = b*Ng + c; dt in the [b][S] layout.
cudaError_t launch_rotwin_f64(const double2* h, const double* dt, const double2* eg, int Lh, int Nb, int Ng,
                              double2* H, cudaStream_t st, const uint32_t* qmask = nullptr);
cudaError_t launch_rotwin_f32(const double2* h, const float* dt, const float2* eg, int Lh, int Nb, int Ng,
                              float2* H, cudaStream_t st, const uint32_t* qmask = nullptr);
// The window's active orders for the rotated-window sums (qmask of
// rotwin_block_smem_to): bit q' + 63 of mask[0..3] is set when some degree
// has |Re h_p^q'| or |Im h_p^q'| above 2^-rel_exp of the window's largest
// component (rel_exp = 0: above zero).  One block.
cudaError_t launch_order_mask(const double2* h, int Lh, int rel_exp, uint32_t* mask, cudaStream_t st);
// g[pair][a][j] = X_0 + sum_r (P_r cos(r alpha_a) - i M_r sin(r alpha_a)).
// slots (nullable): per pair {output slot, mirror} as for launch_alpha_tc.
cudaError_t launch_alpha_f64(const double2* Xs, const double2* csa, int Lh, int Na, int J,
                             int npairs, double2* g, const int2* slots, cudaStream_t st);
cudaError_t launch_alpha_f32(const float2* Xs, const float2* csa, int Lh, int Na, int J,
                             int npairs, float2* g, const int2* slots, cudaStream_t st);

// The alpha sum as a split DFT (Na = P Q, P in {3,5,7,9}); tw[t * (2Lh-1) +
// q + Lh - 1] = (cos, sin)(2 pi q t / Na).  alpha_split_factor returns the P
// used for (Lh, Na), 0 when the direct sum is cheaper or no factor divides Na.
int alpha_split_factor(int Lh, int Na);
cudaError_t launch_alpha_split_f64(const double2* Xs, const double2* tw, int Lh, int Na, int J, int npairs,
                                   double2* g, const int2* slots, cudaStream_t st);
cudaError_t launch_alpha_split_f32(const float2* Xs, const float2* tw, int Lh, int Na, int J, int npairs,
                                   float2* g, const int2* slots, cudaStream_t st);

// Inverse: partial sums then final scaling (deterministic order).  The
// partial sums of one pair are nslab * inverse_col_blocks(Nb, Ng) entries.
int inverse_col_blocks(int Nb, int Ng);
// Inverse without h_0^0 (inverse_alt.cu): column blocks of the projection
// kernel, and the whole launch sequence.  prec 0: g complex128 and ea the
// FP64 table (cos, sin)(q alpha_a), q = -p..p; 1: complex64 g, FP32 ea.
// eg: (cos, sin)(q' gamma_c), q' = -p..p, FP64.  hp: h_p^q', q' = -p..p.
// partial: n_in * ialt_col_blocks * (2p+1); khat: n_in * (2p+1);
// rows[o * (2p+1) + q + p]: the g row of (L + p, M + q) for output o.
// g at arbitrary gamma (steer.cu): out[row][k] = sum_c w_c(gam[k]) g[row][c]
// over rows = pairs * n_alpha * n_beta rows of Ngam samples, the Dirichlet
// weights of the band |q'| <= Q written to W (ng * Ngam doubles).
cudaError_t launch_steer_gamma(const void* g, int prec, long long rows, int Ngam, const double* gam, int ng, int Q,
                               double* W, void* out, cudaStream_t st);
int ialt_col_blocks(int Nb, int Ng);
cudaError_t launch_inverse_alt(const void* g, int prec, const double* wb, const double* dt, int Lh,
                               const double2* hp, const void* ea, const double2* eg, int Na, int Nb, int Ng, int p,
                               int n_in, double2* partial, double scale, double2* khat, const int2* lm_out,
                               const int* rows, int n_out, double2* f, cudaStream_t st);
cudaError_t launch_inverse_f64(const double2* g, const double* wb, int Na, int Nb, int Ng,
                               int npairs, double2* partial, int nslab, cudaStream_t st);
cudaError_t launch_inverse_f32(const float2* g, const double* wb, int Na, int Nb, int Ng,
                               int npairs, double2* partial, int nslab, cudaStream_t st);
cudaError_t launch_inverse_final(const double2* partial, int nslab, int npairs, double scale_re,
                                 double scale_im, double2* fout, cudaStream_t st);
