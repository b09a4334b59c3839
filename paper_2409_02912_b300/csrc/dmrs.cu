// PUSCH DMRS base sequences from the TS 38.211 Sec. 5.2.1 pseudo-random
// sequence (Sec. 6.4.1.1.1.1 c_init), generated on the device so that callers
// can pass pilots produced next to the received grids.  One thread per
// (slot, DMRS symbol) steps both 31-bit LFSRs as machine words.
#include <cuda_runtime.h>

#include "../../include/nrx.h"

namespace {

constexpr int kMaxSlots = 64;
constexpr int kNc = 1600;

struct DmrsJobs {
  uint32_t c_init[kMaxSlots][2];
};

__device__ __forceinline__ void lfsr_step(uint32_t& x1, uint32_t& x2) {
  const uint32_t n1 = ((x1 >> 3) ^ x1) & 1u;
  const uint32_t n2 = ((x2 >> 3) ^ (x2 >> 2) ^ (x2 >> 1) ^ x2) & 1u;
  x1 = (x1 >> 1) | (n1 << 30);
  x2 = (x2 >> 1) | (n2 << 30);
}

__global__ void k_dmrs_gold(int n_slots, int n_dmrs, int M, DmrsJobs jobs, float2* __restrict__ out) {
  const int job = blockIdx.x * blockDim.x + threadIdx.x;
  if (job >= n_slots * n_dmrs) return;
  const int sl = job / n_dmrs, d = job % n_dmrs;
  uint32_t x1 = 1u, x2 = jobs.c_init[sl][d] & 0x7fffffffu;  // bit i = x(i), i < 31
  for (int i = 0; i < kNc; ++i) lfsr_step(x1, x2);
  const float a = 0.70710678118654752f;
  float2* o = out + (size_t)job * M;
  for (int m = 0; m < M; ++m) {
    const uint32_t c0 = (x1 ^ x2) & 1u;
    lfsr_step(x1, x2);
    const uint32_t c1 = (x1 ^ x2) & 1u;
    lfsr_step(x1, x2);
    o[m] = make_float2((1.0f - 2.0f * (float)c0) * a, (1.0f - 2.0f * (float)c1) * a);
  }
}

}  // namespace

extern "C" nrx_status nrx_dmrs_gold(int32_t n_slots, const int32_t* slot_numbers, int32_t n_id, int32_t n_scid,
                                    int32_t num_prb, int32_t num_dmrs_symbols, const int32_t* dmrs_symbols,
                                    void* out, void* stream) {
  if (n_slots < 1 || n_slots > kMaxSlots || !slot_numbers || n_id < 0 || n_id > 65535 || (n_scid != 0 && n_scid != 1) ||
      num_prb < 1 || num_prb > 275 || (num_dmrs_symbols != 1 && num_dmrs_symbols != 2) || !dmrs_symbols || !out)
    return NRX_EINVAL;
  DmrsJobs jobs;
  for (int s = 0; s < n_slots; ++s) {
    if (slot_numbers[s] < 0 || slot_numbers[s] > 159) return NRX_EINVAL;
    for (int d = 0; d < num_dmrs_symbols; ++d) {
      const int l = dmrs_symbols[d];
      if (l < 0 || l > 13) return NRX_EINVAL;
      const unsigned long long v = (1ull << 17) * (unsigned long long)(14 * slot_numbers[s] + l + 1) *
                                       (unsigned long long)(2 * n_id + 1) +
                                   2ull * (unsigned long long)n_id + (unsigned long long)n_scid;
      jobs.c_init[s][d] = (uint32_t)(v % (1ull << 31));
    }
  }
  const int n = n_slots * num_dmrs_symbols;
  k_dmrs_gold<<<(n + 63) / 64, 64, 0, static_cast<cudaStream_t>(stream)>>>(n_slots, num_dmrs_symbols, 6 * num_prb,
                                                                         jobs, static_cast<float2*>(out));
  return cudaGetLastError() == cudaSuccess ? NRX_OK : NRX_ECUDA;
}
