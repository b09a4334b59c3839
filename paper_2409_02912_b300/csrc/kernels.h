// Host-side launchers of the NRX / LMMSE kernels (CUDA path only).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <atomic>
#include <utility>

#include "common.cuh"

// Raise `Kernel`'s dynamic shared-memory limit to `bytes` once per device (the
// attribute is per device; later launches skip the driver call, which also
// keeps the launch sequence free of non-stream calls during graph capture).
template <auto Kernel>
inline cudaError_t ensure_smem(int bytes) {
  static std::atomic<unsigned long long> done{0};
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned long long bit = 1ull << (dev & 63);
  if (done.load(std::memory_order_acquire) & bit) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

// Launch with programmatic stream serialisation: the kernel may start while
// the previous kernel on the stream finishes (it calls griddepcontrol.wait
// before touching that kernel's outputs).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

constexpr int kStateInitTile = 16;  // subcarriers per StateInit CTA

// Bounds-checked build records, one per instrumented source file (debug.cuh):
// [0] violations, [1] site, [2] index and [3] extent of the first.  Without
// NRX_DEBUG they read as zero.
cudaError_t debug_read_frontend(unsigned long long* out, bool reset);
cudaError_t debug_read_net_f32(unsigned long long* out, bool reset);
cudaError_t debug_read_net_tc(unsigned long long* out, bool reset);
cudaError_t debug_read_block_tc(unsigned long long* out, bool reset);
cudaError_t debug_read_mp_tc(unsigned long long* out, bool reset);
cudaError_t debug_read_ldpc(unsigned long long* out, bool reset);
cudaError_t debug_read_train(unsigned long long* out, bool reset);

template <typename T>
__device__ __forceinline__ T store_cast(float v);
template <>
__device__ __forceinline__ float store_cast<float>(float v) {
  return v;
}
template <>
__device__ __forceinline__ __nv_bfloat16 store_cast<__nv_bfloat16>(float v) {
  return __float2bfloat16_rn(v);
}
template <>
__device__ __forceinline__ __half store_cast<__half>(float v) {
  return __float2half_rn(v);
}

// Weights of one CGNN iteration on the device (FP32 path: dense layers stored
// transposed, [in][out]; depthwise taps [C][9]).
struct IterWeightsF32 {
  const float* mp1_t;  // [C][C]
  const float* mp1_b;
  const float* mp2_t;  // [C][C]
  const float* mp2_b;
  const float* in_t;   // [2C+2][C]
  const float* in_b;
  const float* dw1[4];
  const float* pw1_t[4];
  const float* pw1_b[4];
  const float* dw2[4];
  const float* pw2_t[4];
  const float* pw2_b[4];
};

// Modulation-specific input / output layers (Var-IO, Sec. III): up to three
// heads (QPSK, 16-QAM, 64-QAM), selected per user by SlotTable::head.  A
// single-head network fills entry 0 only.
constexpr int kMaxHeads = 3;

// Entry h of a per-head parameter array without dynamic indexing (which
// would copy the kernel parameter struct to local memory).
template <typename T>
__device__ __forceinline__ T pick_head(const T (&a)[kMaxHeads], int h) {
  return h == 0 ? a[0] : (h == 1 ? a[1] : a[2]);
}

struct InitWeights {
  const float* w_pw[kMaxHeads];  // [C][F]
  const float* b_pw[kMaxHeads];  // [C]
  const float* k_dw[kMaxHeads];  // [C][9]
};

struct ReadoutWeightsF32 {
  const float* ro1_t[kMaxHeads];  // [C][C] transposed
  const float* ro1_b[kMaxHeads];
  const float* ro2[kMaxHeads];    // [m_max][C] (rows beyond the head's order are zero)
  const float* ro2_b[kMaxHeads];
};

size_t state_init_smem_bytes(int C, int B);

template <typename OutT>
cudaError_t launch_state_init(const Geometry& g, const SlotTable& tab, const float2* y, const InitWeights& w,
                              OutT* s_out, cudaStream_t st);

// f64_count (nullable): incremented by the number of REs solved in FP64.
cudaError_t launch_lmmse(const Geometry& g, const SlotTable& tab, const float2* y, float* llr,
                         unsigned long long* f64_count, cudaStream_t st);

// FP32 CUDA-core network kernels.
cudaError_t launch_mp_f32(const Geometry& g, const IterWeightsF32& w, const float* state, float* z,
                          cudaStream_t st);
cudaError_t launch_block_f32(const Geometry& g, const IterWeightsF32& w, int r, const float* z_in, float* z_out,
                             float* state, bool last, cudaStream_t st);
cudaError_t launch_readout_f32(const Geometry& g, const SlotTable& tab, const ReadoutWeightsF32& w,
                               const float* state, float* llr, cudaStream_t st);
