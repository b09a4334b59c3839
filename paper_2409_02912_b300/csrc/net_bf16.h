// BF16 tensor-core (tcgen05) network kernels: weights and launchers.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <vector>

#include "../../include/nrx.h"
#include "common.cuh"
#include "kernels.h"

// Weights of one CGNN iteration for the BF16 path.
struct IterWeightsBF16 {
  const void* mp1;  // packed BF16 operand tiles (see net_bf16.cu)
  const void* mp2;
  const void* in;
  const float* mp1_b;
  const float* mp2_b;
  const float* in_b;
  const float* in_pe;  // [2][C] FP32 columns of the input layer for the PE features
  const void* pw1[4];
  const void* pw2[4];
  const float* pw1_b[4];
  const float* pw2_b[4];
  const float* dw1[4];
  const float* dw2[4];
};

struct ReadoutWeightsBF16 {
  const void* ro1;
  const float* ro1_b;
  const float* ro2;  // [m_max][C] FP32
  const float* ro2_b;
};

// blob_it: per iteration {mp1w, mp1b, mp2w, mp2b, inw, inb} then per block
// {dw1, pw1w, pw1b, dw2, pw2w, pw2b} (host pointers into the blob).
nrx_status upload_bf16_weights(int C, int R, int N_it, int m_max, const std::vector<const float*>& blob_it,
                               const float* ro1w, const float* ro1b, const float* ro2w, const float* ro2b,
                               const std::vector<IterWeightsF32>& it32, std::vector<IterWeightsBF16>* it16,
                               void** dev_alloc, ReadoutWeightsBF16* ro);

cudaError_t launch_mp_bf16(const Geometry& g, const IterWeightsBF16& w, const __nv_bfloat16* state,
                           __nv_bfloat16* z, cudaStream_t st);
cudaError_t launch_block_bf16(const Geometry& g, const IterWeightsBF16& w, int r, const __nv_bfloat16* z_in,
                              __nv_bfloat16* z_out, __nv_bfloat16* state, bool last, cudaStream_t st);
cudaError_t launch_readout_bf16(const Geometry& g, const SlotTable& tab, const ReadoutWeightsBF16& w,
                                const __nv_bfloat16* state, float* llr, cudaStream_t st);
cudaError_t launch_bf16_to_f32(const __nv_bfloat16* in, float* out, size_t n, cudaStream_t st);
