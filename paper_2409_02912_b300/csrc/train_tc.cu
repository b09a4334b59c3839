// BF16 tensor-core variant of the training GEMM (nrx_train_gemm_bf16): the
// same strided product and epilogues as the FP32 kernel, with both operands
// rounded to BF16 while they are staged in shared memory and FP32
// accumulation in tensor memory (BF16 compute, FP32 master weights and
// activations).  One CTA computes a 128 x 64 output tile over its K range in
// chunks of 64: all threads stage A (128 x 64) and B (64 x 64) in the 128-byte
// swizzled K-major layout, one thread issues four tcgen05.mma (K = 16) and
// commits to an mbarrier, every thread reads its accumulator row back.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "../../include/nrx_train.h"
#include "kernels.h"
#include "tc.cuh"

namespace {

constexpr int kThreads = 128;
constexpr int kTileM = 128, kTileN = 64, kChunkK = 64;
constexpr int kSmemA = 0, kSmemB = 16384;  // operand tiles; after the last MMA the
constexpr int kSmemOut = 0;                 // FP32 output tile [128][64] (32 KB) reuses them
constexpr int kSmemBar = 32768;
constexpr int kSmemBytes = kSmemBar + 16 + 1024;  // + alignment slack for the 1024-byte swizzle atoms

__device__ int g_train_tc_error;  // set when a bounded wait for the tensor cores gave up

struct GemmArgs {
  int M, N, K, k_per_cta;
  const float* A;
  long long sam, sak;
  const float* B;
  long long sbk, sbn;
  const float* bias;
  const float* R;
  long long ldr;
  float* C;
  long long ldc;
  int relu, atomic;
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

__global__ void __launch_bounds__(kThreads) k_gemm_bf16(GemmArgs a) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + kSmemBar);
  uint32_t* slot = reinterpret_cast<uint32_t*>(sm + kSmemBar + 8);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * kTileM, n0 = blockIdx.y * kTileN;
  const int kb = blockIdx.z * a.k_per_cta;
  const int ke = min(a.K, kb + a.k_per_cta);
  if (warp == 0) tc::tmem_alloc(slot, 64);
  if (tid == 0) {
    tc::mbar_init(bar, 1);
    tc::fence_mbar_init();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *slot;
  const uint32_t sa = tc::smem_u32(sm + kSmemA), sb = tc::smem_u32(sm + kSmemB);
  bool ok = true;
  uint32_t phase = 0;
  for (int k0 = kb; k0 < ke && ok; k0 += kChunkK) {
    // A(m, k) for m in [m0, m0 + 128), k in [k0, k0 + 64): element pairs along k.
    // Consecutive threads walk the operand's unit-stride index (coalesced).
    for (int i = tid; i < kTileM * (kChunkK / 2); i += kThreads) {
      int r, kp;
      if (a.sak == 1) {
        r = i / (kChunkK / 2);
        kp = i % (kChunkK / 2);
      } else {
        r = i % kTileM;
        kp = i / kTileM;
      }
      const int m = m0 + r, k = k0 + 2 * kp;
      float v0 = 0.f, v1 = 0.f;
      if (m < a.M) {
        if (k < ke) v0 = a.A[(long long)m * a.sam + (long long)k * a.sak];
        if (k + 1 < ke) v1 = a.A[(long long)m * a.sam + (long long)(k + 1) * a.sak];
      }
      *reinterpret_cast<uint32_t*>(sm + kSmemA + tc::sw128_offset(r, 2 * kp)) = pack_bf16(v0, v1);
    }
    // B(k, n) as the N x K (K-major) operand: row n, columns k.
    for (int i = tid; i < kTileN * (kChunkK / 2); i += kThreads) {
      int nn, kp;
      if (a.sbk == 1) {
        nn = i / (kChunkK / 2);
        kp = i % (kChunkK / 2);
      } else {
        nn = i % kTileN;
        kp = i / kTileN;
      }
      const int n = n0 + nn, k = k0 + 2 * kp;
      float v0 = 0.f, v1 = 0.f;
      if (n < a.N) {
        if (k < ke) v0 = a.B[(long long)k * a.sbk + (long long)n * a.sbn];
        if (k + 1 < ke) v1 = a.B[(long long)(k + 1) * a.sbk + (long long)n * a.sbn];
      }
      *reinterpret_cast<uint32_t*>(sm + kSmemB + tc::sw128_offset(nn, 2 * kp)) = pack_bf16(v0, v1);
    }
    tc::fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc::tc_fence_after();
      tc::mma_k64(tmem, sa, sb, tc::idesc_bf16_f32(kTileM, kTileN), k0 > kb);
      tc::mma_commit(bar);
    }
    // every thread waits for the chunk's MMAs (the next chunk overwrites the operands)
    int done = 1;
    if (tid == 0) done = tc::mbar_wait(bar, phase) ? 1 : 0;
    ok = __syncthreads_or(done == 0) == 0;
    phase ^= 1u;
    tc::tc_fence_after();
  }
  if (!ok) {
    if (tid == 0) atomicExch(&g_train_tc_error, 1);
  } else {
    // accumulator rows -> FP32 tile in shared memory (float4 chunk j of row r
    // at j ^ (r & 15)), then a coalesced write-out: 16 threads per output row
    float v[64];
    tc::tmem_row64(tmem + ((uint32_t)(warp * 32) << 16), v);
    const int r = warp * 32 + lane;
    float4* out = reinterpret_cast<float4*>(sm + kSmemOut);
#pragma unroll
    for (int j = 0; j < 16; ++j)
      out[r * 16 + (j ^ (r & 15))] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
    __syncthreads();
    const bool vec = !a.atomic && (a.ldc % 4 == 0) && ((reinterpret_cast<uintptr_t>(a.C) & 15) == 0);
    for (int idx = tid; idx < kTileM * 16; idx += kThreads) {
      const int rr = idx >> 4, j = idx & 15;
      const int m = m0 + rr, n = n0 + 4 * j;
      if (m >= a.M || n >= a.N) continue;
      const float4 q = out[rr * 16 + (j ^ (rr & 15))];
      float x[4] = {q.x, q.y, q.z, q.w};
      float* crow = a.C + (long long)m * a.ldc;
      if (a.atomic) {
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (n + e < a.N) atomicAdd(crow + n + e, x[e]);
        continue;
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        if (n + e >= a.N) break;
        if (a.bias) x[e] += a.bias[n + e];
        if (a.R) x[e] += a.R[(long long)m * a.ldr + n + e];
        if (a.relu) x[e] = fmaxf(x[e], 0.f);
      }
      if (vec && n + 4 <= a.N) {
        *reinterpret_cast<float4*>(crow + n) = make_float4(x[0], x[1], x[2], x[3]);
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (n + e < a.N) crow[n + e] = x[e];
      }
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 64);
}

nrx_status to_status(cudaError_t e) { return e == cudaSuccess ? NRX_OK : NRX_ECUDA; }

}  // namespace

extern "C" {

nrx_status nrx_train_gemm_bf16(int32_t M, int32_t N, int32_t K, const float* A, int64_t sam, int64_t sak,
                               const float* B, int64_t sbk, int64_t sbn, const float* bias, const float* R,
                               int64_t ldr, float* C, int64_t ldc, int32_t relu, int32_t accumulate, int32_t split_k,
                               void* stream) {
  if (M < 1 || N < 1 || K < 1 || !A || !B || !C || split_k < 1 || split_k > 65535) return NRX_EINVAL;
  if ((split_k > 1 && !accumulate) || (accumulate && (bias || R || relu))) return NRX_EINVAL;
  if (ensure_smem<k_gemm_bf16>(kSmemBytes) != cudaSuccess) return NRX_ECUDA;
  GemmArgs g;
  g.M = M;
  g.N = N;
  g.K = K;
  // K range per CTA: a whole number of 64-wide chunks
  const int per = (K + split_k - 1) / split_k;
  g.k_per_cta = (per + kChunkK - 1) / kChunkK * kChunkK;
  const int splits = (K + g.k_per_cta - 1) / g.k_per_cta;
  g.A = A;
  g.sam = sam;
  g.sak = sak;
  g.B = B;
  g.sbk = sbk;
  g.sbn = sbn;
  g.bias = bias;
  g.R = R;
  g.ldr = ldr;
  g.C = C;
  g.ldc = ldc;
  g.relu = relu;
  g.atomic = accumulate ? 1 : 0;
  dim3 grid((M + kTileM - 1) / kTileM, (N + kTileN - 1) / kTileN, splits);
  k_gemm_bf16<<<grid, kThreads, kSmemBytes, static_cast<cudaStream_t>(stream)>>>(g);
  return to_status(cudaGetLastError());
}

nrx_status nrx_train_check(void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaStreamSynchronize(s) != cudaSuccess) return NRX_ECUDA;
  int flag = 0;
  if (cudaMemcpyFromSymbol(&flag, g_train_tc_error, sizeof(int)) != cudaSuccess) return NRX_ECUDA;
  if (flag) {
    const int zero = 0;
    cudaMemcpyToSymbol(g_train_tc_error, &zero, sizeof(int));
    return NRX_ETIMEDOUT;
  }
  return NRX_OK;
}

}  // extern "C"
