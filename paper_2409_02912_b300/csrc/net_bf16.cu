// BF16 tensor-core path (placeholder until the tcgen05 kernels land).
#include "net_bf16.h"

nrx_status upload_bf16_weights(int, int, int, int, const std::vector<const float*>&, const float*, const float*,
                               const float*, const float*, const std::vector<IterWeightsF32>&,
                               std::vector<IterWeightsBF16>*, void**, ReadoutWeightsBF16*) {
  return NRX_EUNSUPPORTED;
}
cudaError_t launch_mp_bf16(const Geometry&, const IterWeightsBF16&, const __nv_bfloat16*, __nv_bfloat16*,
                           cudaStream_t) {
  return cudaErrorNotSupported;
}
cudaError_t launch_block_bf16(const Geometry&, const IterWeightsBF16&, int, const __nv_bfloat16*, __nv_bfloat16*,
                              __nv_bfloat16*, bool, cudaStream_t) {
  return cudaErrorNotSupported;
}
cudaError_t launch_readout_bf16(const Geometry&, const SlotTable&, const ReadoutWeightsBF16&, const __nv_bfloat16*,
                                float*, cudaStream_t) {
  return cudaErrorNotSupported;
}
cudaError_t launch_bf16_to_f32(const __nv_bfloat16*, float*, size_t, cudaStream_t) { return cudaErrorNotSupported; }
