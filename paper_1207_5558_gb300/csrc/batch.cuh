// Device descriptors and launchers of batch plans: many analyses (signal,
// window, pair list, grid, precision) evaluated by three launches, each over
// a host-built work list:
//   k_batch_couple  the Gaunt gather-sum k_lm(p, q) of every pair of every item,
//   k_batch_rotwin  every distinct rotated window H (one block per (beta row, degree)),
//   k_batch_alpha   a persistent kernel (one per precision) whose CTAs take tiles (item, pair,
//                   column block) from a shared counter: X_q for the tile's
//                   columns from H and k, then the alpha sum, stored to g.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define BA_THREADS 128           // threads of a k_batch_alpha CTA (columns x row groups)
#define BA_SMEM_LIMIT (200 * 1024)

struct BCouple {                 // one coupling output (a signal with a pair list)
  const double2* f;              // signal coefficients
  const int2* lm;                // pair list (l, m)
  const double* coef;            // Gaunt table rows [pair][i][t]
  const int2* meta;              // (first l', count) per [pair][t]
  double2* kc;                   // k [pair][t]
  float4* kdd;                   // double-float k scaled by 2^-kexp[pair] (null: not needed)
  int* kexp;
  int Lh, npairs;
  int Lf;                        // signal band limit (the serving path's 3j chains)
};
struct BCplBlk { int cpl, first; };        // 256 consecutive (pair, t) items of one BCouple

struct BRot {                    // one rotated window H
  const double2* h;
  const void* dt;                // d^p(beta_b) table [b][blk_off(Lh)], T
  const void* eg;                // gamma phases [c][2Lh-1], T2
  void* H;                       // tiled H (h_index), T2 (null: not needed)
  float4* Hdd;                   // FP64 windows: double-float H scaled by 2^-hexp[0] (null: not needed)
  int* hexp;
  const uint32_t* qmask;         // active orders of the window (null: all; launch_order_mask)
  int prec, Lh, Nb, Ng;          // prec 0: FP64, 1: FP32
  int QC, CC, nq, nc;            // shared-memory chunking (rot_chunks)
};
struct BRotBlk { int rot, b, p, z; };      // beta rows b .. b + ROTWIN_NB - 1; z: chunk of (q rows, gamma columns)

struct BItem {                   // one analysis of the batch (alpha stage view)
  const double2* kc;             // k [pair][Lh^2]
  const void* H;                 // tiled H, T2 (double-float items: the scaled float4 H)
  const void* csa;               // form 0: (cos, sin)(2 pi r a / Na) [a][Lh]; P: split twiddles [t][2Lh-1]
                                 // (double-float items: float4 {cos.h, sin.h, cos.l, sin.l})
  void* g;                       // output [pair][a][j], T2
  const float4* kdd;             // double-float items: scaled k and its exponents
  const int* kexp;
  const int* hexp;
  const int2* slots;             // double-float items (nullable): per pair {output slot, mirror}
                                 // as for launch_alpha_tc; null: pair p -> tile's out slot
  int prec, Lh, Na, J;           // prec 0: FP64, 1: FP32, 2: FP64 output from double-float arithmetic
  int nt;                        // columns per tile: 32, 64 or 128 (BA_THREADS / nt row groups)
  int form;                      // 0: direct sum, 3/5/7/9: split DFT with that factor
};
struct BTile { int item, pair, out, j0; };  // k of `pair`, output slot `out`, columns j0 .. j0+nt-1

// Shared memory of a k_batch_alpha tile: X_q for nt columns (prec 0, 1 or 2).
size_t batch_alpha_smem(int prec, int Lh, int nt);
// Resident CTAs of k_batch_alpha (precision prec) per SM with `smem` bytes of
// dynamic shared memory.
int batch_alpha_occupancy(int prec, size_t smem);

cudaError_t launch_batch_couple(const BCouple* cpl, const BCplBlk* blk, int nblk, cudaStream_t st);
// Double-float k of the couplings that need it: block list {cpl, pair}.
cudaError_t launch_batch_kdd(const BCouple* cpl, const BCplBlk* blk, int nblk, cudaStream_t st);
cudaError_t launch_batch_rotwin(const BRot* rot, const BRotBlk* blk, int nblk, size_t smem, cudaStream_t st);
// One call's pieces (the per-call path): k of npairs pairs scaled into
// kdd/kexp; the rotated window's scaled double-float copy; the alpha stage
// of one item over all its (pair, column block) tiles, tiles derived from
// the index (no list), CTAs striding over them.
cudaError_t launch_kdd_pairs(const double2* kc, int Lh, int npairs, float4* kdd, int* kexp, cudaStream_t st);
cudaError_t launch_rotwin_dd(const double2* h, const double* dt, const double2* eg, int Lh, int Nb, int Ng,
                             float4* Hdd, int* hexp, cudaStream_t st, const uint32_t* qmask = nullptr);
cudaError_t launch_alpha_dd_call(const BItem& item, int npairs, int num_sms, cudaStream_t st);
// The same for an item of any precision (item.prec 0 FP64, 1 FP32, 2 double-float).
cudaError_t launch_alpha_call(const BItem& item, int npairs, int num_sms, cudaStream_t st);

// Persistent: `grid` CTAs take tiles from *counter (reset to 0 before each
// launch); every tile's item has precision prec (0 FP64, 1 FP32, 2 double-float).
cudaError_t launch_batch_alpha(int prec, const BItem* items, const BTile* tiles, int ntiles, int* counter, int grid,
                               size_t smem, cudaStream_t st);

// The serving path's launches (fixed grids, work counts read from device
// memory, so that one captured graph serves ticks of any composition):
//   launch_serve_couple  k of the list of work items by 3j chains in the call
//                        (cls 0: L_h <= 16, 1: <= 32, 2: <= 64); an item is
//                        serve_couple_entry(coupling, pair, mirror): the
//                        mirror pair (l, -m) of the same coupling (-1: none)
//                        gets its k from the same chains
//   launch_batch_kdd_n, launch_batch_rotwin_n, launch_batch_alpha_n
//                        as above with the block / tile count *n.
#define SERVE_CPL_MAX 1024               // couplings a serving tick may list (its chunks)
__host__ __device__ inline int2 serve_couple_entry(int cpl, int pair, int mirror) {
  return make_int2(cpl + SERVE_CPL_MAX * (mirror + 1), pair);
}
cudaError_t launch_serve_couple(int cls, const BCouple* cpl, const int2* list, const int* n, int grid,
                                cudaStream_t st);
cudaError_t launch_batch_kdd_n(const BCouple* cpl, const BCplBlk* blk, const int* n, int grid, cudaStream_t st);
cudaError_t launch_batch_rotwin_n(const BRot* rot, const BRotBlk* blk, const int* n, int grid, size_t smem,
                                  cudaStream_t st);
cudaError_t launch_batch_alpha_n(int prec, const BItem* items, const BTile* tiles, const int* n, int* counter,
                                 int grid, size_t smem, cudaStream_t st);
// Resident CTAs per SM of the rotated-window kernel with `smem` bytes.
int batch_rotwin_occupancy(size_t smem);
