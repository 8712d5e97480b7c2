// Tensor-core (tcgen05) alpha stage of the FP32_BULK path: interface.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

// Whether the tensor-core alpha stage handles this window band limit / grid.
bool tc_supported(int Lh, int Na);
// Bytes of the per-grid E operand tables (split-FP16 cos / sin of q alpha_a).
size_t tc_etab_bytes(int Na, int Lh);
cudaError_t launch_tc_etab(void* etab, int Na, int Lh, cudaStream_t st);
// Bytes of the A operand (split-FP16 X, per-row scales) of ONE pair.
size_t tc_xblob_bytes(int Nb, int Ng, int Lh);
// Factoring route: gamma sum of Y (launch_beta_dft) writing the A operand blobs
// (FP32 sums); dt is unused (pass nullptr), Y is required.
cudaError_t launch_betagamma_tc(const double2* kc, const double2* h, const float* dt,
                                const double2* Y, const float2* eg, int Lh, int Nb, int Ng,
                                int npairs, void* xblob, cudaStream_t st);
// Rotated-window route: the A operand blobs from H (launch_rotwin_f32).
cudaError_t launch_xa_from_h(const double2* kc, const float2* H, int Lh, int Nb, int Ng, int npairs, void* xblob,
                             cudaStream_t st);
// alpha stage on tcgen05: g[pair][a][j] complex64.
// slots (nullable, device): per pair {output slot, mirror}, mirror = -1 or
// 2 * slot of (l, -m) + (m & 1): that slot receives (-1)^m conj of the pair's
// g (valid when f and h are real fields); without slots pair i writes slot i.
cudaError_t launch_alpha_tc(const void* xblob, const void* etab, int Lh, int Na, int Nb, int Ng,
                            int npairs, float2* g, int num_sms, const int2* slots, cudaStream_t st);
// Fused rotated-window producer + alpha stage (one persistent kernel): the A
// operand of every (pair, 128-column tile) is built in shared memory from H
// (launch_rotwin_f32, tiled layout of h_index) and the pair's coupling row
// kc, then multiplied by the E tables on tcgen05; g[pair][a][j] complex64.
// Lh <= 16.
// wait_test != 0: the launch withholds the first A tile of every CTA so its
// bounded waits expire and it reports through the error word (tests the
// timeout path; the output is not computed).
cudaError_t launch_alpha_fused(const double2* kc, const float2* H, const void* etab, int Lh, int Na, int Nb,
                               int Ng, int npairs, float2* g, int num_sms, int wait_test, const int2* slots,
                               cudaStream_t st);
// Wide windows, 16 < Lh <= 64 (alpha_tcw.cu): K split into 2 or 4 chunks of
// 64; the same E-table / A-blob / alpha-stage roles as the narrow engine.
bool tcw_supported(int Lh, int Na);
size_t tcw_etab_bytes(int Na, int Lh);
cudaError_t launch_tcw_etab(void* etab, int Na, int Lh, cudaStream_t st);
size_t tcw_xblob_bytes(int Nb, int Ng, int Lh);
cudaError_t launch_xaw_from_h(const double2* kc, const float2* H, int Lh, int Nb, int Ng, int npairs, void* xblob,
                              cudaStream_t st);
cudaError_t launch_alpha_tcw(const void* xblob, const void* etab, int Lh, int Na, int Nb, int Ng, int npairs,
                             float2* g, int num_sms, const int2* slots, cudaStream_t st);
// FP64 alpha stage on the tensor cores, Lh <= 16 (alpha_tc64.cu): base-256
// digit products, exact in FP32, into seven accumulators per output.
bool tc64_supported(int Lh, int Na);
size_t tc64_etab_bytes(int Na);
cudaError_t launch_tc64_etab(void* etab, int Na, cudaStream_t st);
size_t tc64_xblob_bytes(int Nb, int Ng);
// A digits from the double-float window Hdd (tiled layout of h_index, scaled
// by 2^-*hexp) and couplings kdd (per pair, scaled by 2^-kexp[pair])
cudaError_t launch_xa64(const float4* kdd, const int* kexp, const float4* Hdd, const int* hexp, int Lh, int Nb,
                        int Ng, int npairs, void* xblob, cudaStream_t st);
// g[pair][a][j] complex128; slots as launch_alpha_tc
cudaError_t launch_alpha_tc64(const void* xblob, const void* etab, int Lh, int Na, int Nb, int Ng, int npairs,
                              double2* g, int num_sms, const int2* slots, cudaStream_t st);
// Timeout-path test of the separate-producer tensor-core kernels
// (launch_alpha_tc, launch_alpha_tcw, launch_alpha_tc64): after
// tc_arm_wait_test() the next such launch from the same host thread withholds
// the first A operand of every CTA (the copy is never issued), so the
// issuer's and the epilogue's bounded waits expire, the kernel leaves cleanly
// and reports through the error word; that launch's output is not computed.
void tc_arm_wait_test();
int tc_take_wait_test();
// The rotated window of an FP32_BULK call on the tensor cores (rotwin_tc.cu):
// H (the tiled layout of h_index) from the split-FP16 d(beta) image `tab`
// (launch_rotwin_tc_table, built once per (Lh, Nb) from the FP32 d(beta)
// table dt, rotwin_tc_table_bytes bytes) and the window operand images of the
// call `wbuf` (launch_rotwin_tc_window from h, the FP32 gamma phases eg and
// qmask as for launch_rotwin_f32, rotwin_tc_window_bytes bytes).
// N_gamma <= 128.  Like the alpha kernels it takes tc_arm_wait_test() (the
// first d chunk is then never fetched).
bool rotwin_tc_supported(int Lh, int Ng);
size_t rotwin_tc_table_bytes(int Lh, int Nb);
cudaError_t launch_rotwin_tc_table(const float* dt, int Lh, int Nb, void* tab, cudaStream_t st);
size_t rotwin_tc_window_bytes(int Lh);
cudaError_t launch_rotwin_tc_window(const double2* h, const float2* eg, const uint32_t* qmask, int Lh, int Ng,
                                   void* wbuf, cudaStream_t st);
cudaError_t launch_rotwin_tc(const void* tab, const void* wbuf, int Lh, int Nb, int Ng, float2* H, int num_sms,
                             cudaStream_t st);
// Device error word shared by the tensor-core kernels (allocated on first use).
int* tc_error_word();
// Non-zero (and cleared) if a tensor-core kernel gave up on a bounded wait
// since the last call.  Synchronous.
int tc_read_error(void);
