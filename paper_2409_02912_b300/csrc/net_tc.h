// Tensor-core (tcgen05) network kernels, FP16 or BF16 operands: weights and launchers.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <vector>

#include "../../include/nrx.h"
#include "common.cuh"
#include "kernels.h"

// Weights of one CGNN iteration for the tensor-core path.  Dense 64x64
// matrices are pre-packed on the host into the 8 KB K-major 128-byte-swizzle
// shared-memory image the MMA reads ([out][in] = N x K).  With BF16 operands
// each matrix is stored as two such images, W_hi = bf16(W) followed by
// W_lo = bf16(W - W_hi), and multiplied as A W_hi^T + A W_lo^T (the weight
// rounding error drops to that of a 16-bit mantissa).  Biases, depthwise taps
// and the PE columns of the input layer stay FP32.
//
// The message MLP's output layer is folded into the CNN-update input layer:
// with h_v = ReLU(W1 S_v + b1) and g_u = sum_{v != u} h_v, the aggregate is
// a_u = W2 g_u + (U-1) b2, so Win_a a_u = (Win_a W2) g_u + (U-1) Win_a b2.
// in_c holds Win_a W2 (formed in FP64 on the host) and cb2 = Win_a b2.
// Precision policies: T = activation storage / depthwise type; split = BF16
// weights as hi + lo images; fp8 = E4M3 MMA operands (per-row activation
// scales, per-output-channel weight scales) over FP16 storage.
struct PolBF16 {
  using T = __nv_bfloat16;
  static constexpr bool split = true, fp8 = false;
};
struct PolFP16 {
  using T = __half;
  static constexpr bool split = false, fp8 = false;
};
struct PolFP8 {
  using T = __half;
  static constexpr bool split = false, fp8 = true;
};

struct IterWeightsTC {
  const uint4* mp1;
  const uint4* in_s;   // input layer, columns acting on S
  const uint4* in_c;   // Win_a W2, acting on g
  const float* mp1_sc;   // E4M3 per-output-channel scales (FP8 policy only)
  const float* in_s_sc;
  const float* in_c_sc;
  const float* pw1_sc[4];
  const float* pw2_sc[4];
  const float* mp1_b;
  const float* in_b;
  const float* cb2;    // [C] Win_a b2
  const float* in_pe;  // [2][C]: columns acting on (dt, df)
  const uint4* pw1[4];
  const uint4* pw2[4];
  const float* pw1_b[4];
  const float* pw2_b[4];
  const float* dw1[4];
  const float* dw2[4];
  int* err;            // device word set when a bounded wait gives up
};

struct ReadoutWeightsTC {  // per Var-IO head (entry 0 only for a single-head network)
  const uint4* ro1[kMaxHeads];
  const float* ro1_sc[kMaxHeads];  // E4M3 scales (FP8 policy only)
  const float* ro1_b[kMaxHeads];
  const float* ro2[kMaxHeads];     // [m_max][C] FP32
  const float* ro2_b[kMaxHeads];
  int* err;
};

// blob_it: per iteration {mp1w, mp1b, mp2w, mp2b, inw, inb} then per block
// {dw1, pw1w, pw1b, dw2, pw2w, pw2b} (host pointers into the blob).  FP32
// device tensors (biases, taps, PE columns, readout head) are taken from the
// FP32 upload.  Only C = 64 is supported.  mode: 0 FP16, 1 BF16 (split
// weights), 2 FP8 (E4M3 with per-output-channel scales).
nrx_status upload_tc_weights(int mode, int C, int R, int N_it, const std::vector<const float*>& blob_it,
                             const std::vector<const float*>& ro1w_heads, const std::vector<IterWeightsF32>& it32,
                             const ReadoutWeightsF32& ro32, std::vector<IterWeightsTC>* out, void** dev_alloc,
                             ReadoutWeightsTC* ro, int** err_word);

template <typename P>
cudaError_t launch_mp_tc(const Geometry& g, const IterWeightsTC& w, const typename P::T* state, typename P::T* z,
                         cudaStream_t st);
template <typename P>
cudaError_t launch_block_tc(const Geometry& g, const IterWeightsTC& w, int r, const typename P::T* z_in,
                            typename P::T* z_out, typename P::T* state, bool last, cudaStream_t st);
template <typename P>
cudaError_t launch_readout_tc(const Geometry& g, const SlotTable& tab, const ReadoutWeightsTC& w,
                              const typename P::T* state, float* llr, cudaStream_t st);
template <typename T>
cudaError_t launch_to_f32(const T* in, float* out, size_t n, cudaStream_t st);

// Residual block for 16-bit operands (block_tc.cu): two tile pipelines per
// SM whose depthwise phases take turns, 12-subcarrier tiles, the residual and
// state added by identity-weight MMAs, input / state / output tiles moved by
// bulk tensor copies; requires S % 12 == 0 (always true: S = 12 N_PRB) and
// 16-byte aligned activations.
template <typename T>
cudaError_t launch_block16_tc(const Geometry& g, const IterWeightsTC& w, int r, const T* z_in, T* z_out, T* state,
                             bool last, cudaStream_t st);

// Message passing + CNN-update input layer for 16-bit operands (mp_tc.cu):
// eight worker warps and one issuer warp that runs the bulk tensor copies and
// the MMAs a tile ahead; requires 16-byte aligned activations.
template <typename T>
cudaError_t launch_mp16_tc(const Geometry& g, const IterWeightsTC& w, const T* state, T* z, cudaStream_t st);

// Number of SMs of the current device (cached).
int block_sms();

// cuTensorMapEncodeTiled through the runtime's driver entry point (null if
// the driver does not provide it).
#include <cudaTypedefs.h>
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();
