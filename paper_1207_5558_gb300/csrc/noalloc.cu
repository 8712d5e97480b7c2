// slsht_forward_noalloc: the forward transform without any device allocation.
//
// Some callers cannot allocate device memory at the moment they need the
// transform: real-time sections where cudaMalloc's implicit device
// synchronisation is not allowed, plug-ins whose host application owns the
// allocator (and forbids a second one from growing behind its back), and
// processes that have already handed the whole device to a fixed memory pool.
// The call is made from ordinary host code (it calls the CUDA runtime, which a
// function queued with cudaLaunchHostFunc may not do).  For them this entry point works out of one scratch
// array of SLSHT_NOALLOC_SCRATCH_BYTES declared at file scope in device memory:
// it is created when the library is loaded and stays on every GPU that loads
// the library until the process exits.
//
// Every call rebuilds the tables it needs (Delta, the d(beta) table, the phase
// tables) in that array and runs the CUDA-core launch sequence of the forward
// transform (coupling, beta/gamma, alpha) on the caller's stream, in chunks of
// pairs sized to what is left of the array.  Nothing in the array has to start
// at zero: every word a kernel reads was written earlier in the same call.
// Calls share the array, so two calls whose work overlaps on the GPU (for
// example on two streams without an ordering between them) race and corrupt
// each other's results.
#include <mutex>

#include "../../include/slsht.h"
#include "common.cuh"

static __device__ __align__(256) unsigned char g_noalloc_scratch[SLSHT_NOALLOC_SCRATCH_BYTES];

void slsht_record_error_text(const char* text);

namespace {

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[64] = {nullptr};   // device address of the array, per device

// Device address of the scratch array on the current device (set up once per
// device with that device current).
int noalloc_scratch(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return SLSHT_E_CUDA;
  }
  std::lock_guard<std::mutex> g(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      slsht_record_error_text("slsht_forward_noalloc: cudaGetSymbolAddress of the scratch array failed");
      return SLSHT_E_CUDA;
    }
    g_noalloc_ptr[dev] = p;
  }
  *out = (unsigned char*)g_noalloc_ptr[dev];
  return SLSHT_OK;
}

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

size_t up256(size_t n) { return (n + 255) & ~(size_t)255; }

}  // namespace

extern "C" int slsht_forward_noalloc(const slsht_desc* desc, const double* f_lm, const double* h_lm,
                                     const int32_t* lm, int32_t n_pairs, void* g_out, void* stream) {
  if (!desc || n_pairs < 0) return SLSHT_E_ARG;
  if (n_pairs == 0) return slsht_check_args(desc, lm, 0);
  if (!f_lm || !h_lm || !lm || !g_out || (((uintptr_t)g_out) & 7)) return SLSHT_E_ARG;
  if (!on_device(g_out)) return SLSHT_E_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  // Validate the pairs through a fixed host buffer (no allocation).  A device
  // pair list is read on the caller's stream, after the work queued there
  // before this call (which may be what wrote it), and the stream is then
  // synchronised: the kernels below read the same, validated list, provided
  // the caller leaves it unchanged until the call's work is done.
  const bool lm_dev = on_device(lm);
  {
    int32_t buf[1024];
    for (int32_t off = 0; off < n_pairs; off += 512) {
      const int32_t n = n_pairs - off < 512 ? n_pairs - off : 512;
      const int32_t* src = lm + 2 * (size_t)off;
      if (lm_dev) {
        if (cudaMemcpyAsync(buf, src, sizeof(int32_t) * 2 * (size_t)n, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
          cudaGetLastError();
          slsht_record_error_text("slsht_forward_noalloc: reading the device pair list on the stream failed");
          return SLSHT_E_CUDA;
        }
        src = buf;
      }
      const int s = slsht_check_args(desc, src, n);
      if (s != SLSHT_OK) return s;
    }
  }
  const int Lf = desc->L_f, Lh = desc->L_h, Na = desc->n_alpha, Nb = desc->n_beta, Ng = desc->n_gamma;
  const int K = 2 * Lh - 1;
  const bool f64 = desc->prec == SLSHT_FP64;
  const size_t el = f64 ? sizeof(double) : sizeof(float);
  const size_t J = (size_t)Nb * Ng;
  // carve the array: inputs (when on the host), tables, then per-chunk k and X
  size_t off = 0;
  const size_t o_f = off; off += on_device(f_lm) ? 0 : up256(sizeof(double2) * (size_t)Lf * Lf);
  const size_t o_h = off; off += on_device(h_lm) ? 0 : up256(sizeof(double2) * (size_t)Lh * Lh);
  const size_t o_lm = off; off += lm_dev ? 0 : up256(sizeof(int2) * (size_t)n_pairs);
  const size_t o_D = off; off += up256(sizeof(double) * (size_t)blk_off(Lh));
  const size_t o_dt = off; off += up256(el * (size_t)blk_off(Lh) * Nb);
  const size_t o_eg = off; off += up256(2 * el * (size_t)Ng * K);
  const size_t o_csa = off; off += up256(2 * el * (size_t)Na * Lh);
  const size_t per_pair = up256(sizeof(double2) * (size_t)Lh * Lh) + up256(2 * el * (size_t)K * J);
  if (off + per_pair > (size_t)SLSHT_NOALLOC_SCRATCH_BYTES) {
    slsht_record_error_text(
        "slsht_forward_noalloc: the tables and one pair need more than the static scratch limit "
        "(SLSHT_NOALLOC_SCRATCH_BYTES); use slsht_forward or a smaller grid / window band limit");
    return SLSHT_E_NOMEM;
  }
  const int P = (int)(((size_t)SLSHT_NOALLOC_SCRATCH_BYTES - off) / per_pair < (size_t)n_pairs
                          ? ((size_t)SLSHT_NOALLOC_SCRATCH_BYTES - off) / per_pair
                          : (size_t)n_pairs);
  const size_t o_kc = off;
  const size_t o_X = o_kc + up256(sizeof(double2) * (size_t)P * Lh * Lh);

  unsigned char* base = nullptr;
  int s = noalloc_scratch(&base);
  if (s != SLSHT_OK) return s;
#define NA_CK(call)                                           \
  do {                                                        \
    cudaError_t _e = (call);                                  \
    if (_e != cudaSuccess) {                                  \
      slsht_record_error_text("slsht_forward_noalloc: " #call); \
      return SLSHT_E_CUDA;                                    \
    }                                                         \
  } while (0)
  const double2* f_dev = (const double2*)f_lm;
  const double2* h_dev = (const double2*)h_lm;
  const int2* lm_d = (const int2*)lm;
  if (!on_device(f_lm)) {
    NA_CK(cudaMemcpyAsync(base + o_f, f_lm, sizeof(double2) * (size_t)Lf * Lf, cudaMemcpyHostToDevice, st));
    f_dev = (const double2*)(base + o_f);
  }
  if (!on_device(h_lm)) {
    NA_CK(cudaMemcpyAsync(base + o_h, h_lm, sizeof(double2) * (size_t)Lh * Lh, cudaMemcpyHostToDevice, st));
    h_dev = (const double2*)(base + o_h);
  }
  if (!lm_dev) {
    NA_CK(cudaMemcpyAsync(base + o_lm, lm, sizeof(int2) * (size_t)n_pairs, cudaMemcpyHostToDevice, st));
    lm_d = (const int2*)(base + o_lm);
  }
  double* D = (double*)(base + o_D);
  NA_CK(launch_delta(D, Lh, st));
  if (f64) {
    NA_CK(launch_dtable_f64(D, (double*)(base + o_dt), Lh, Nb, st));
    NA_CK(launch_phase_f64((double2*)(base + o_eg), Ng, K, -(Lh - 1), st));
    NA_CK(launch_phase_f64((double2*)(base + o_csa), Na, Lh, 0, st));
  } else {
    NA_CK(launch_dtable_f32(D, (float*)(base + o_dt), Lh, Nb, st));
    NA_CK(launch_phase_f32((float2*)(base + o_eg), Ng, K, -(Lh - 1), st));
    NA_CK(launch_phase_f32((float2*)(base + o_csa), Na, Lh, 0, st));
  }
  const size_t per_pair_g = (size_t)Na * J * 2 * el;
  double2* kc = (double2*)(base + o_kc);
  for (int32_t p0 = 0; p0 < n_pairs; p0 += P) {
    const int np = n_pairs - p0 < P ? n_pairs - p0 : P;
    void* gdst = (char*)g_out + per_pair_g * (size_t)p0;
    NA_CK(launch_couple(f_dev, Lf, Lh, lm_d + p0, np, kc, st));
    if (f64) {
      NA_CK(launch_betagamma_f64(kc, h_dev, (const double*)(base + o_dt), nullptr,
                                 (const double2*)(base + o_eg), Lh, Nb, Ng, np, (double2*)(base + o_X), st));
      NA_CK(launch_alpha_f64((const double2*)(base + o_X), (const double2*)(base + o_csa), Lh, Na, (int)J, np,
                             (double2*)gdst, nullptr, st));
    } else {
      NA_CK(launch_betagamma_f32(kc, h_dev, (const float*)(base + o_dt), nullptr,
                                 (const float2*)(base + o_eg), Lh, Nb, Ng, np, (float2*)(base + o_X), st));
      NA_CK(launch_alpha_f32((const float2*)(base + o_X), (const float2*)(base + o_csa), Lh, Na, (int)J, np,
                             (float2*)gdst, nullptr, st));
    }
  }
#undef NA_CK
  return SLSHT_OK;
}
