// Bounds-checked build.  Compiled with -DNRX_DEBUG, every instrumented
// shared-memory and global index is checked against the extent of the array
// it addresses; an index outside it is recorded (how many, and the site,
// index and extent of the first) and the access is skipped, so a fault in
// the index arithmetic shows up as a count rather than as a memory fault.
// Without NRX_DEBUG the checks compile to nothing.
//
// Each translation unit has its own record (a file-scope device array); its
// host reader is defined with NRX_DEBUG_READER(name) and collected by
// nrx_debug_counters() in nrx_api.cu.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#ifdef NRX_DEBUG
// [0] violations, [1] site of the first, [2] its index, [3] the extent it exceeded
static __device__ unsigned long long g_nrx_dbg[4];

__device__ __forceinline__ bool nrx_dbg_ok(long long i, long long n, int site) {
  if (i >= 0 && i < n) return true;
  if (atomicAdd(&g_nrx_dbg[0], 1ull) == 0ull) {
    g_nrx_dbg[1] = (unsigned long long)site;
    g_nrx_dbg[2] = (unsigned long long)i;
    g_nrx_dbg[3] = (unsigned long long)n;
  }
  return false;
}
#define NRX_IN(i, n, site) nrx_dbg_ok((long long)(i), (long long)(n), (site))
#define NRX_DEBUG_READER(name)                                                                   \
  cudaError_t name(unsigned long long* out, bool reset) {                                          \
    cudaError_t e = cudaMemcpyFromSymbol(out, g_nrx_dbg, sizeof(g_nrx_dbg));                       \
    if (e == cudaSuccess && reset) {                                                               \
      const unsigned long long z[4] = {0, 0, 0, 0};                                                \
      e = cudaMemcpyToSymbol(g_nrx_dbg, z, sizeof(z));                                             \
    }                                                                                              \
    return e;                                                                                      \
  }
#else
#define NRX_IN(i, n, site) true
#define NRX_DEBUG_READER(name)                                   \
  cudaError_t name(unsigned long long* out, bool) {                \
    for (int k = 0; k < 4; ++k) out[k] = 0;                        \
    return cudaSuccess;                                            \
  }
#endif
