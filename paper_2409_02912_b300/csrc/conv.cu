// Soft-input Viterbi decoding of the rate-1/2, K=7 (133, 171) convolutional
// code, used to measure block error rates of the receivers' LLRs.  One warp
// decodes one block: lane l owns trellis states l and l + 32; predecessor
// metrics are exchanged with warp shuffles, the 64 decisions of a step are two
// ballots stored in shared memory, and lane 0 traces back.
#include <cuda_runtime.h>

#include <cmath>

#include "../../include/nrx_eval.h"

namespace {

constexpr int kMaxInfo = 4096;
constexpr int kTail = 6;
constexpr unsigned kG0 = 0133, kG1 = 0171;

__device__ __forceinline__ unsigned parity7(unsigned x) { return __popc(x & 0x7fu) & 1u; }

// Outputs (c0 | c1 << 1) of the transition into new state sp from predecessor
// ((sp << 1) & 63) | b.
__device__ __forceinline__ unsigned trans_out(unsigned sp, unsigned b) {
  const unsigned s = ((sp << 1) & 63u) | b;
  const unsigned reg = ((sp >> 5) << 6) | s;
  return parity7(reg & kG0) | (parity7(reg & kG1) << 1);
}

__device__ __forceinline__ float branch(float pm, unsigned o, float l0, float l1) {
  // Same addition order as the definition: (PM + m0) + m1.
  const float a = pm + ((o & 1u) ? l0 : 0.0f);
  return a + ((o & 2u) ? l1 : 0.0f);
}

__global__ void k_viterbi(int n_blocks, int n_info, const float* __restrict__ llr,
                          const int64_t* __restrict__ block_offset, const int32_t* __restrict__ perm,
                          uint8_t* __restrict__ out) {
  extern __shared__ uint2 s_dec[];
  const int T = n_info + kTail;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int blk = blockIdx.x * (blockDim.x >> 5) + warp;
  if (blk >= n_blocks) return;
  uint2* dec = s_dec + (size_t)warp * T;
  const float* l = llr + block_offset[blk];

  const unsigned sA = lane, sB = lane + 32;
  const unsigned p0 = (sA << 1) & 63u, p1 = p0 | 1u;  // shared by sA and sB
  const unsigned oA0 = trans_out(sA, 0), oA1 = trans_out(sA, 1);
  const unsigned oB0 = trans_out(sB, 0), oB1 = trans_out(sB, 1);
  const int src0 = p0 & 31, src1 = p1 & 31;
  const bool hi0 = p0 >= 32, hi1 = p1 >= 32;

  float pmA = lane == 0 ? 0.0f : -INFINITY;
  float pmB = -INFINITY;
  for (int t = 0; t < T; ++t) {
    const int i0 = 2 * t, i1 = 2 * t + 1;
    const float l0 = __ldg(l + (perm ? __ldg(perm + i0) : i0));
    const float l1 = __ldg(l + (perm ? __ldg(perm + i1) : i1));
    const float a0 = __shfl_sync(0xffffffffu, pmA, src0), b0 = __shfl_sync(0xffffffffu, pmB, src0);
    const float a1 = __shfl_sync(0xffffffffu, pmA, src1), b1 = __shfl_sync(0xffffffffu, pmB, src1);
    const float pm0 = hi0 ? b0 : a0, pm1 = hi1 ? b1 : a1;
    const float cA0 = branch(pm0, oA0, l0, l1), cA1 = branch(pm1, oA1, l0, l1);
    const float cB0 = branch(pm0, oB0, l0, l1), cB1 = branch(pm1, oB1, l0, l1);
    const bool tA = cA1 > cA0, tB = cB1 > cB0;
    const float nA = tA ? cA1 : cA0, nB = tB ? cB1 : cB0;
    const unsigned wA = __ballot_sync(0xffffffffu, tA), wB = __ballot_sync(0xffffffffu, tB);
    if (lane == 0) dec[t] = make_uint2(wA, wB);
    const float norm = __shfl_sync(0xffffffffu, nA, 0);
    pmA = nA - norm;
    pmB = nB - norm;
  }
  __syncwarp();
  if (lane == 0) {
    unsigned s = 0;
    uint8_t* o = out + (size_t)blk * n_info;
    for (int t = T - 1; t >= 0; --t) {
      if (t < n_info) o[t] = (uint8_t)(s >> 5);
      const uint2 w = dec[t];
      const unsigned word = (s >> 5) ? w.y : w.x;
      s = ((s << 1) & 63u) | ((word >> (s & 31u)) & 1u);
    }
  }
}

}  // namespace

extern "C" nrx_status nrx_conv_decode(int32_t n_blocks, int32_t n_info, const float* llr,
                                      const int64_t* block_offset, const int32_t* perm, uint8_t* info_bits,
                                      void* stream) {
  if (n_blocks < 0 || n_info < 1 || n_info > kMaxInfo || (n_blocks > 0 && (!llr || !block_offset || !info_bits)))
    return NRX_EINVAL;
  if (n_blocks == 0) return NRX_OK;
  const int T = n_info + kTail;
  int warps = (48 * 1024) / (T * (int)sizeof(uint2));
  warps = warps < 1 ? 1 : (warps > 8 ? 8 : warps);
  const int grid = (n_blocks + warps - 1) / warps;
  const size_t smem = (size_t)warps * T * sizeof(uint2);
  k_viterbi<<<grid, warps * 32, smem, static_cast<cudaStream_t>(stream)>>>(n_blocks, n_info, llr, block_offset,
                                                                         perm, info_bits);
  return cudaGetLastError() == cudaSuccess ? NRX_OK : NRX_ECUDA;
}
