// NRX forward pass that allocates no device memory.
//
// Some callers cannot call cudaMalloc: code that runs while a CUDA stream is
// being captured into a graph (allocation calls are not capturable), real-time
// baseband pipelines whose memory budget is fixed at start-up and that forbid
// allocation on the data path, and plug-ins hosted by a framework that owns
// every allocation on the GPU.  nrx_detect_noalloc serves them: the caller
// passes the weights, the received grid and the LLR buffer in device memory it
// already owns, and the network's activation scratch lives in the static
// device array below instead of context workspaces.
//
// The array costs kScratchBytes on every GPU that loads this library, for the
// life of the process.  Every call first copies the weights from the caller's
// blob into the array's weight region in kernel layout (one extra launch, up
// to 1 MiB of traffic), since the array may hold another net.  All calls
// share it and it keeps the last call's contents; every kernel of the forward
// pass writes each scratch element before reading it, so nothing needs
// clearing between calls.  Calls whose executions overlap on the GPU
// (different streams, or different host threads without ordering) race on
// the array: order them.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "../../include/nrx.h"
#include "common.cuh"
#include "kernels.h"

namespace {

constexpr size_t kScratchBytes = size_t(16) << 20;  // 16 MiB in total
constexpr size_t kWeightBytes = size_t(1) << 20;    // first MiB: weights in kernel layout
constexpr int kMaxDevices = 64;
constexpr int kMaxOps = 128;

static __device__ __align__(256) unsigned char g_nrx_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  The first call
// on each device looks it up with cudaGetSymbolAddress (host code cannot use
// the array's name as a device pointer) and keeps it for the life of the
// process: after a cudaDeviceReset the module is loaded again and the kept
// address is stale, so this entry point must not be used across a device
// reset.
nrx_status scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return NRX_ECUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_nrx_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return NRX_ECUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return NRX_OK;
}

// One copy of a blob tensor into the kernel layout, optionally transposed
// from [n_out][n_in] to [n_in][n_out].
struct CopyOp {
  int src, dst, n_out, n_in, transpose;
};
struct CopyPlan {
  int n_ops;
  CopyOp op[kMaxOps];
};

__global__ void k_layout_weights(CopyPlan plan, const float* __restrict__ blob, float* __restrict__ dst) {
  const CopyOp op = plan.op[blockIdx.y];
  const int n = op.n_out * op.n_in;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int o = i / op.n_in, k = i % op.n_in;
    const int d = op.transpose ? k * op.n_out + o : i;
    dst[op.dst + d] = __ldg(blob + op.src + i);
  }
}

size_t align4(size_t n) { return (n + 3) & ~size_t(3); }

}  // namespace

extern "C" nrx_status nrx_detect_noalloc(const void* weights_header, const float* weights_dev, const void* y,
                                         const nrx_slot_cfg* cfg, const int32_t* bits, float* llr,
                                         void* stream) {
  if (!weights_header || !weights_dev || !y || !cfg || !bits || !llr) return NRX_EINVAL;
  if ((reinterpret_cast<uintptr_t>(y) & 15) || (reinterpret_cast<uintptr_t>(llr) & 3) ||
      (reinterpret_cast<uintptr_t>(weights_dev) & 15))
    return NRX_EINVAL;
  int32_t h[8];
  memcpy(h, weights_header, sizeof(h));
  const int B = h[2], C = h[3], R = h[4], N_it = h[5], m_max = h[6];
  if (h[0] != 0x5758524E || h[1] != 1 || (B != 1 && B != 2 && B != 4 && B != 8) || (C != 32 && C != 64) || R < 1 ||
      R > 4 || N_it < 1 || N_it > 16 || m_max < 2 || m_max > 8)
    return NRX_EINVAL;
  const int F = 4 * B + 2;
  const long long expect = (long long)C * F + C + 9 * C +
                           (long long)N_it * (2 * ((long long)C * C + C) + (long long)C * (2 * C + 2) + C +
                                              (long long)R * (2 * (9 * C + (long long)C * C + C))) +
                           (long long)C * C + C + (long long)m_max * C + m_max;
  if (h[7] != expect) return NRX_EINVAL;
  // The copy plan and the weight region are fixed-size: reject nets that do
  // not fit from the header alone, before anything is built.  Ops: StateInit
  // (3), per iteration 6 + 6 R, read-out (4).  Floats: each tensor rounded up
  // to a multiple of 4.
  if (7 + N_it * (6 + 6 * R) > kMaxOps) return NRX_EINVAL;
  {
    const size_t cc = align4((size_t)C * C), c1 = align4(C), c9 = align4(9 * (size_t)C);
    const size_t floats = align4((size_t)C * F) + c1 + c9 +
                          (size_t)N_it * (2 * cc + 2 * c1 + align4((size_t)C * (2 * C + 2)) + c1 +
                                          (size_t)R * (2 * c9 + 2 * cc + 2 * c1)) +
                          cc + c1 + align4((size_t)m_max * C) + align4(m_max);
    if (floats * sizeof(float) > kWeightBytes) return NRX_EINVAL;
  }

  // Slot geometry and per-slot table (one slot).
  const nrx_slot_cfg& c = *cfg;
  if (c.num_prb < 1 || c.num_prb > 275 || c.num_users < 1 || c.num_users > NRX_MAX_USERS) return NRX_EINVAL;
  if (c.num_dmrs_symbols != 1 && c.num_dmrs_symbols != 2) return NRX_EINVAL;
  for (int d = 0; d < c.num_dmrs_symbols; ++d)
    if (c.dmrs_symbols[d] < 0 || c.dmrs_symbols[d] >= NRX_SYMBOLS) return NRX_EINVAL;
  if (c.num_dmrs_symbols == 2 && c.dmrs_symbols[1] <= c.dmrs_symbols[0]) return NRX_EINVAL;
  if (!c.dmrs_seq || (reinterpret_cast<uintptr_t>(c.dmrs_seq) & 7)) return NRX_EINVAL;
  const int its = c.iterations == 0 ? N_it : c.iterations;
  if (its < 1 || its > N_it) return NRX_EINVAL;
  Geometry g;
  SlotTable tab;
  memset(&g, 0, sizeof(g));
  memset(&tab, 0, sizeof(tab));
  g.n_slots = 1;
  g.S = 12 * c.num_prb;
  g.U = c.num_users;
  g.B = B;
  g.C = C;
  g.F = F;
  g.m_max = m_max;
  g.n_dmrs = c.num_dmrs_symbols;
  g.td0 = c.dmrs_symbols[0];
  g.td1 = c.num_dmrs_symbols == 2 ? c.dmrs_symbols[1] : c.dmrs_symbols[0];
  g.n_data = (NRX_SYMBOLS - g.n_dmrs) * g.S;
  for (int t = 0, di = 0; t < NRX_SYMBOLS; ++t)
    if (t != g.td0 && t != g.td1) g.data_t[di++] = (int8_t)t;
  tab.dmrs[0] = static_cast<const float2*>(c.dmrs_seq);
  tab.noise_var[0] = c.noise_var;
  size_t off = 0;
  for (int u = 0; u < g.U; ++u) {
    const int m = bits[u];
    if ((m != 2 && m != 4 && m != 6) || m > m_max) return NRX_EINVAL;
    tab.bits[0][u] = (int8_t)m;
    tab.llr_off[0][u] = (int32_t)off;
    off += (size_t)g.n_data * m;
  }
  tab.llr_total = (long long)off;

  // Weight layout plan (same layout the context path builds on the host).
  CopyPlan plan;
  memset(&plan, 0, sizeof(plan));
  size_t src = 0, dst = 0;
  bool plan_full = false;
  auto add = [&](int n_out, int n_in, bool tr) {
    const size_t at = dst;
    if (plan.n_ops == kMaxOps) {  // unreachable after the header checks; never write past the table
      plan_full = true;
      return at;
    }
    plan.op[plan.n_ops++] = {(int)src, (int)dst, n_out, n_in, tr ? 1 : 0};
    src += (size_t)n_out * n_in;
    dst = align4(dst + (size_t)n_out * n_in);
    return at;
  };
  const size_t o_init_w = add(C, F, false), o_init_b = add(1, C, false), o_init_dw = add(1, 9 * C, false);
  size_t o_it[16][6], o_blk[16][4][6];
  for (int k = 0; k < N_it; ++k) {
    o_it[k][0] = add(C, C, true);
    o_it[k][1] = add(1, C, false);
    o_it[k][2] = add(C, C, true);
    o_it[k][3] = add(1, C, false);
    o_it[k][4] = add(C, 2 * C + 2, true);
    o_it[k][5] = add(1, C, false);
    for (int r = 0; r < R; ++r) {
      o_blk[k][r][0] = add(1, 9 * C, false);
      o_blk[k][r][1] = add(C, C, true);
      o_blk[k][r][2] = add(1, C, false);
      o_blk[k][r][3] = add(1, 9 * C, false);
      o_blk[k][r][4] = add(C, C, true);
      o_blk[k][r][5] = add(1, C, false);
    }
  }
  const size_t o_ro1 = add(C, C, true), o_ro1b = add(1, C, false), o_ro2 = add(m_max, C, false),
               o_ro2b = add(1, m_max, false);
  if (plan_full) return NRX_EINVAL;

  // Scratch budget: weights in the first MiB, then S, z_a, z_b.
  const size_t act = (size_t)g.U * NRX_SYMBOLS * g.S * C;
  if (dst * sizeof(float) > kWeightBytes || 3 * act * sizeof(float) > kScratchBytes - kWeightBytes)
    return NRX_EINVAL;

  void* base = nullptr;
  nrx_status st = scratch_address(&base);
  if (st != NRX_OK) return st;
  float* W = static_cast<float*>(base);
  float* S = reinterpret_cast<float*>(static_cast<unsigned char*>(base) + kWeightBytes);
  float* za = S + act;
  float* zb = za + act;
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  k_layout_weights<<<dim3(16, plan.n_ops), 256, 0, s>>>(plan, weights_dev, W);
  if (cudaGetLastError() != cudaSuccess) return NRX_ECUDA;
  const float2* yy = static_cast<const float2*>(y);
  InitWeights iw{};
  iw.w_pw[0] = W + o_init_w;
  iw.b_pw[0] = W + o_init_b;
  iw.k_dw[0] = W + o_init_dw;
  if (launch_state_init<float>(g, tab, yy, iw, S, s) != cudaSuccess)
    return NRX_ECUDA;
  for (int k = 0; k < its; ++k) {
    IterWeightsF32 w;
    memset(&w, 0, sizeof(w));
    w.mp1_t = W + o_it[k][0];
    w.mp1_b = W + o_it[k][1];
    w.mp2_t = W + o_it[k][2];
    w.mp2_b = W + o_it[k][3];
    w.in_t = W + o_it[k][4];
    w.in_b = W + o_it[k][5];
    for (int r = 0; r < R; ++r) {
      w.dw1[r] = W + o_blk[k][r][0];
      w.pw1_t[r] = W + o_blk[k][r][1];
      w.pw1_b[r] = W + o_blk[k][r][2];
      w.dw2[r] = W + o_blk[k][r][3];
      w.pw2_t[r] = W + o_blk[k][r][4];
      w.pw2_b[r] = W + o_blk[k][r][5];
    }
    if (launch_mp_f32(g, w, S, za, s) != cudaSuccess) return NRX_ECUDA;
    float* zin = za;
    float* zout = zb;
    for (int r = 0; r < R; ++r) {
      if (launch_block_f32(g, w, r, zin, zout, S, r == R - 1, s) != cudaSuccess) return NRX_ECUDA;
      float* t = zin;
      zin = zout;
      zout = t;
    }
  }
  ReadoutWeightsF32 rw{};
  rw.ro1_t[0] = W + o_ro1;
  rw.ro1_b[0] = W + o_ro1b;
  rw.ro2[0] = W + o_ro2;
  rw.ro2_b[0] = W + o_ro2b;
  if (launch_readout_f32(g, tab, rw, S, llr, s) != cudaSuccess)
    return NRX_ECUDA;
  return NRX_OK;
}
