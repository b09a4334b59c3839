// Layered normalised min-sum decoding of a quasi-cyclic LDPC code (the
// transport-block code behind the receivers' LLRs, Sec. II), declared in
// include/nrx_eval.h.
//
// One CTA per code block, one thread per check of the current layer (Z
// threads; a layer is one base-graph row).  The block's posteriors (nb Z
// FP32 values, L = ln P(0)/P(1)) live in shared memory; the check-to-variable
// messages of every edge in a caller-provided global scratch.  Rate recovery
// (TS 38.212 Sec. 5.4.2: undo the qm-row bit interleaver, fold the circular
// buffer back onto codeword positions 2 Z ..) runs in the same kernel.
// Within a layer the Z checks touch distinct variables (each nonzero block is
// a permutation), so the layer is race-free; layers are ordered by
// __syncthreads.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "../../include/nrx_eval.h"
#include "debug.cuh"
#include "kernels.h"

namespace {

constexpr int kMaxRows = 64;
constexpr int kMaxEdges = 320;
constexpr int kMaxDeg = 16;
constexpr int kMaxZ = 384;

// Base graph by value (kernel parameter space): edges in row-major order,
// shifts already reduced mod Z.
struct LdpcGraph {
  int mb, nb, nnz;
  int16_t row_ptr[kMaxRows + 1];
  int16_t col[kMaxEdges];
  int16_t shift[kMaxEdges];
};

__global__ void __launch_bounds__(kMaxZ) k_ldpc(LdpcGraph G, int Z, int kb, int E, int qm,
                                                const float* __restrict__ llr, const int64_t* __restrict__ offset,
                                                int iterations, float alpha, int stop_early, float* __restrict__ c2v,
                                                uint8_t* __restrict__ info) {
  extern __shared__ float post[];  // [nb Z]
  const int tid = threadIdx.x, nthr = blockDim.x, cb = blockIdx.x;
  const float* l = llr + offset[cb];
  float* msg = c2v + (size_t)cb * G.nnz * Z;
  const int N = G.nb * Z, ncb = (G.nb - 2) * Z, ecols = E / qm;
  for (int x = tid; x < N; x += nthr) post[x] = 0.f;
  for (int x = tid; x < G.nnz * Z; x += nthr) msg[x] = 0.f;
  __syncthreads();
  // rate recovery: received bit p is bit b = p % qm of symbol j = p / qm, i.e.
  // circular-buffer bit k = b (E / qm) + j, codeword bit 2 Z + k mod ncb
  for (int p = tid; p < E; p += nthr) {
    const int k = (p % qm) * ecols + p / qm;
    if (NRX_IN(2 * Z + k % ncb, N, 601)) atomicAdd(&post[2 * Z + k % ncb], -__ldg(l + p));
  }
  __syncthreads();
  const int i = tid;
  for (int it = 0; it < iterations; ++it) {
    for (int r = 0; r < G.mb; ++r) {
      if (i < Z) {
        const int e0 = G.row_ptr[r], d = G.row_ptr[r + 1] - e0;
        float t[kMaxDeg];
        int v[kMaxDeg];
        float m1 = INFINITY, m2 = INFINITY;
        int amin = 0;
        unsigned neg = 0, skip = 0;  // skip: edges whose indices fail the bounds check (debug build)
#pragma unroll
        for (int q = 0; q < kMaxDeg; ++q) {
          if (q < d) {
            const int e = e0 + q;
            int c = i + G.shift[e];
            c = c >= Z ? c - Z : c;
            v[q] = G.col[e] * Z + c;
            if (!NRX_IN(v[q], N, 602) || !NRX_IN((long long)e * Z + i, (long long)G.nnz * Z, 603)) {
              skip |= 1u << q;
              t[q] = 0.f;
              continue;
            }
            t[q] = post[v[q]] - msg[(size_t)e * Z + i];
            const float a = fabsf(t[q]);
            if (a < m1) {
              m2 = m1;
              m1 = a;
              amin = q;
            } else if (a < m2) {
              m2 = a;
            }
            neg ^= (t[q] < 0.f ? 1u : 0u) << q;
          }
        }
        const float total = (__popc(neg) & 1) ? -1.f : 1.f;
#pragma unroll
        for (int q = 0; q < kMaxDeg; ++q) {
          if (q < d && !((skip >> q) & 1u)) {
            const float s = ((neg >> q) & 1u) ? -total : total;  // product of the other signs
            // one rounding for the message and one for the posterior (never a fused multiply-add)
            const float nw = __fmul_rn(alpha * s, q == amin ? m2 : m1);
            msg[(size_t)(e0 + q) * Z + i] = nw;
            post[v[q]] = __fadd_rn(t[q], nw);
          }
        }
      }
      __syncthreads();
    }
    if (stop_early) {  // every check satisfied by the hard decisions?
      int bad = 0;
      if (i < Z) {
        for (int r = 0; r < G.mb && !bad; ++r) {
          unsigned par = 0;
          for (int e = G.row_ptr[r]; e < G.row_ptr[r + 1]; ++e) {
            int c = i + G.shift[e];
            c = c >= Z ? c - Z : c;
            par ^= post[G.col[e] * Z + c] < 0.f ? 1u : 0u;
          }
          bad = (int)par;
        }
      }
      if (!__syncthreads_or(bad)) break;
    }
  }
  uint8_t* out = info + (size_t)cb * kb * Z;
  for (int x = tid; x < kb * Z; x += nthr) out[x] = post[x] < 0.f ? 1 : 0;
}

}  // namespace

extern "C" nrx_status nrx_ldpc_decode(int32_t n_blocks, const float* llr, const int64_t* block_offset, int32_t E,
                                      int32_t qm, int32_t Z, int32_t kb, int32_t mb, const int32_t* row_ptr,
                                      const int32_t* col, const int32_t* shift, int32_t iterations, float alpha,
                                      int32_t stop_early, float* c2v, uint8_t* info_bits, void* stream) {
  if (n_blocks < 0 || Z < 1 || Z > kMaxZ || kb < 1 || mb < 1 || mb > kMaxRows || qm < 1 || qm > 8 || E < 1 ||
      E % qm || iterations < 1 || iterations > 100 || !(alpha > 0.f) || !row_ptr || !col || !shift)
    return NRX_EINVAL;
  const int nb = kb + mb;
  if (nb < 3 || (size_t)nb * Z * sizeof(float) > 227 * 1024) return NRX_EINVAL;
  LdpcGraph G;
  G.mb = mb;
  G.nb = nb;
  if (row_ptr[0] != 0) return NRX_EINVAL;
  for (int r = 0; r < mb; ++r) {
    const int d = row_ptr[r + 1] - row_ptr[r];
    if (d < 1 || d > kMaxDeg) return NRX_EINVAL;
  }
  G.nnz = row_ptr[mb];
  if (G.nnz > kMaxEdges) return NRX_EINVAL;
  for (int r = 0; r <= mb; ++r) G.row_ptr[r] = (int16_t)row_ptr[r];
  for (int e = 0; e < G.nnz; ++e) {
    if (col[e] < 0 || col[e] >= nb || shift[e] < 0) return NRX_EINVAL;
    G.col[e] = (int16_t)col[e];
    G.shift[e] = (int16_t)(shift[e] % Z);
  }
  if (n_blocks == 0) return NRX_OK;
  if (!llr || !block_offset || !c2v || !info_bits) return NRX_EINVAL;
  const size_t smem = (size_t)nb * Z * sizeof(float);
  if (ensure_smem<k_ldpc>(227 * 1024) != cudaSuccess) return NRX_ECUDA;
  const int threads = ((Z + 31) / 32) * 32;
  k_ldpc<<<n_blocks, threads, smem, static_cast<cudaStream_t>(stream)>>>(
      G, Z, kb, E, qm, llr, block_offset, iterations, alpha, stop_early ? 1 : 0, c2v, info_bits);
  return cudaGetLastError() == cudaSuccess ? NRX_OK : NRX_ECUDA;
}

NRX_DEBUG_READER(debug_read_ldpc)
