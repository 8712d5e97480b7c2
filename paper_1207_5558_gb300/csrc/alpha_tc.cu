// Tensor-core alpha stage (placeholder until the tcgen05 kernel lands).
#include "tc.cuh"

bool tc_supported(int, int) { return false; }
size_t tc_etab_bytes(int, int) { return 0; }
cudaError_t launch_tc_etab(void*, int, int, cudaStream_t) { return cudaErrorNotSupported; }
size_t tc_xblob_bytes(int, int, int) { return 0; }
cudaError_t launch_betagamma_tc(const double2*, const double2*, const float*, const double2*,
                                const float2*, int, int, int, int, void*, cudaStream_t) {
  return cudaErrorNotSupported;
}
cudaError_t launch_alpha_tc(const void*, const void*, int, int, int, int, int, float2*, int,
                            cudaStream_t) {
  return cudaErrorNotSupported;
}
