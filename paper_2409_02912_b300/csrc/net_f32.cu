// FP32 CUDA-core kernels of the CGNN iterations and the LLR read-out
// (Sec. II-A).  This is the reference-precision path: plain FMAs, no tensor
// cores, FP32 activations [slot][user][symbol][subcarrier][C].
#include "common.cuh"
#include "kernels.h"

namespace {

constexpr int kThreads = 256;

// acc[i][j] += sum_k A[row_i][k] * WT[k][c0 + j], rows row0 + i * rstep.
// A in shared memory with leading dimension lda; WT [K][C] in global (L1).
template <int C, int RPT>
__device__ __forceinline__ void gemm_rows(float (&acc)[RPT][4], const float* A, int lda, int row0, int rstep,
                                          const float* __restrict__ WT, int K, int c0) {
  for (int k = 0; k < K; ++k) {
    const float4 w = __ldg(reinterpret_cast<const float4*>(WT + (size_t)k * C + c0));
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      const float a = A[(row0 + i * rstep) * lda + k];
      acc[i][0] = fmaf(a, w.x, acc[i][0]);
      acc[i][1] = fmaf(a, w.y, acc[i][1]);
      acc[i][2] = fmaf(a, w.z, acc[i][2]);
      acc[i][3] = fmaf(a, w.w, acc[i][3]);
    }
  }
}

template <int RPT>
__device__ __forceinline__ void init_bias(float (&acc)[RPT][4], const float* __restrict__ b, int c0) {
  const float4 bv = __ldg(reinterpret_cast<const float4*>(b + c0));
#pragma unroll
  for (int i = 0; i < RPT; ++i) {
    acc[i][0] = bv.x;
    acc[i][1] = bv.y;
    acc[i][2] = bv.z;
    acc[i][3] = bv.w;
  }
}

// ---------------------------------------------------------------------------
// Message passing + CNN-update input layer of one CGNN iteration.
// Per RE: m_u = mp2(ReLU(mp1(S_u))), a_u = sum_{v != u} m_v over active users,
// z_u = in([S_u, a_u, PE_u]).  One CTA holds kRE REs of all users.
// ---------------------------------------------------------------------------
template <int C>
struct MpCfg {
  static constexpr int kRE = 32;
  static constexpr int CG = C / 4;
  static constexpr int RG = kThreads / CG;
  static constexpr int ROWS = NRX_MAX_USERS * kRE;
  static constexpr int RPT = ROWS / RG;
  static constexpr int LD = C + 1;
};

template <int C>
__global__ void __launch_bounds__(kThreads) k_mp_f32(Geometry g, IterWeightsF32 w, const float* __restrict__ state,
                                                      float* __restrict__ z) {
  using Cf = MpCfg<C>;
  extern __shared__ __align__(16) float sm[];
  float* sa = sm;                 // [ROWS][LD] states
  float* sb = sm + Cf::ROWS * Cf::LD;  // [ROWS][LD] hidden, then messages, then aggregates
  const int sl = blockIdx.y;
  const int re0 = blockIdx.x * Cf::kRE;
  const int n_re = NRX_SYMBOLS * g.S;
  const int U = g.U;
  for (int i = threadIdx.x; i < Cf::ROWS * C; i += kThreads) {
    const int c = i % C, row = i / C;
    const int u = row / Cf::kRE, re = re0 + row % Cf::kRE;
    float v = 0.f;
    const size_t si = (((size_t)sl * U + u) * n_re + re) * C + c;
    if (u < U && re < n_re && NRX_IN(si, (size_t)g.n_slots * U * n_re * C, 201)) v = __ldg(state + si);
    if (NRX_IN(row * Cf::LD + c, Cf::ROWS * Cf::LD, 202)) sa[row * Cf::LD + c] = v;
  }
  __syncthreads();
  const int cg = threadIdx.x % Cf::CG, rg = threadIdx.x / Cf::CG;
  const int c0 = cg * 4;
  float acc[Cf::RPT][4];
  // hidden = ReLU(mp1 S + b1)
  init_bias(acc, w.mp1_b, c0);
  gemm_rows<C, Cf::RPT>(acc, sa, Cf::LD, rg, Cf::RG, w.mp1_t, C, c0);
#pragma unroll
  for (int i = 0; i < Cf::RPT; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) sb[(rg + i * Cf::RG) * Cf::LD + c0 + j] = fmaxf(acc[i][j], 0.f);
  __syncthreads();
  // messages = mp2 hidden + b2 (in place after a barrier)
  init_bias(acc, w.mp2_b, c0);
  gemm_rows<C, Cf::RPT>(acc, sb, Cf::LD, rg, Cf::RG, w.mp2_t, C, c0);
  __syncthreads();
#pragma unroll
  for (int i = 0; i < Cf::RPT; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) sb[(rg + i * Cf::RG) * Cf::LD + c0 + j] = acc[i][j];
  __syncthreads();
  // aggregate over the other active users
  for (int i = threadIdx.x; i < Cf::kRE * C; i += kThreads) {
    const int c = i % C, j = i / C;
    float m[NRX_MAX_USERS];
#pragma unroll
    for (int u = 0; u < NRX_MAX_USERS; ++u) m[u] = sb[(u * Cf::kRE + j) * Cf::LD + c];
#pragma unroll
    for (int u = 0; u < NRX_MAX_USERS; ++u) {
      float a = 0.f;
#pragma unroll
      for (int v = 0; v < NRX_MAX_USERS; ++v)
        if (v != u && v < U) a += m[v];
      sb[(u * Cf::kRE + j) * Cf::LD + c] = a;
    }
  }
  __syncthreads();
  // z = in([S, a, PE]) + b
  init_bias(acc, w.in_b, c0);
  gemm_rows<C, Cf::RPT>(acc, sa, Cf::LD, rg, Cf::RG, w.in_t, C, c0);
  gemm_rows<C, Cf::RPT>(acc, sb, Cf::LD, rg, Cf::RG, w.in_t + (size_t)C * C, C, c0);
  const float4 wt = __ldg(reinterpret_cast<const float4*>(w.in_t + (size_t)2 * C * C + c0));
  const float4 wf = __ldg(reinterpret_cast<const float4*>(w.in_t + (size_t)(2 * C + 1) * C + c0));
#pragma unroll
  for (int i = 0; i < Cf::RPT; ++i) {
    const int row = rg + i * Cf::RG;
    const int u = row / Cf::kRE, re = re0 + row % Cf::kRE;
    if (u >= U || re >= n_re) continue;
    const int t = re / g.S, s = re % g.S;
    const float pt = pe_time(g, t), pf = pe_freq(u, s);
    float4 o;
    o.x = fmaf(pf, wf.x, fmaf(pt, wt.x, acc[i][0]));
    o.y = fmaf(pf, wf.y, fmaf(pt, wt.y, acc[i][1]));
    o.z = fmaf(pf, wf.z, fmaf(pt, wt.z, acc[i][2]));
    o.w = fmaf(pf, wf.w, fmaf(pt, wt.w, acc[i][3]));
    const size_t zi = (((size_t)sl * U + u) * n_re + re) * C + c0;
    if (NRX_IN(zi + 3, (size_t)g.n_slots * U * n_re * C, 203)) *reinterpret_cast<float4*>(z + zi) = o;
  }
}

// ---------------------------------------------------------------------------
// One residual block z <- z + pw2(ReLU(dw2(ReLU(pw1(dw1(z)))))) on a tile of
// kTW subcarriers x 14 symbols of one (slot, user); the input tile carries a
// two-subcarrier halo.  With `last`, the block output is added to the state
// instead (S <- S + z, the end of the CNN update).
// ---------------------------------------------------------------------------
template <int C>
struct BlkCfg {
  static constexpr int kTW = 12;
  static constexpr int IW = kTW + 4;  // input columns
  static constexpr int MW = kTW + 2;  // dw1 / pw1 columns
  static constexpr int CG = C / 4;
  static constexpr int RG = kThreads / CG;
  static constexpr int R1 = NRX_SYMBOLS * MW;
  static constexpr int R2 = NRX_SYMBOLS * kTW;
  static constexpr int RPT1 = (R1 + RG - 1) / RG;
  static constexpr int RPT2 = (R2 + RG - 1) / RG;
  static constexpr int LD = C + 1;
  static constexpr size_t smem_floats = (size_t)(NRX_SYMBOLS * IW + RPT1 * RG + RPT2 * RG) * LD + 18 * C;
};

template <int C>
__global__ void __launch_bounds__(kThreads) k_block_f32(Geometry g, const float* __restrict__ dw1,
                                                         const float* __restrict__ pw1_t,
                                                         const float* __restrict__ pw1_b,
                                                         const float* __restrict__ dw2,
                                                         const float* __restrict__ pw2_t,
                                                         const float* __restrict__ pw2_b,
                                                         const float* __restrict__ z_in, float* __restrict__ z_out,
                                                         float* __restrict__ state, int last) {
  using Cf = BlkCfg<C>;
  extern __shared__ __align__(16) float sm[];
  float* zin = sm;                                   // [14][IW][LD]
  float* d1 = zin + NRX_SYMBOLS * Cf::IW * Cf::LD;   // [RPT1*RG][LD]
  float* d2 = d1 + Cf::RPT1 * Cf::RG * Cf::LD;       // [RPT2*RG][LD]
  float* k1 = d2 + Cf::RPT2 * Cf::RG * Cf::LD;       // [C][9]
  float* k2 = k1 + 9 * C;
  const int tile = blockIdx.x, u = blockIdx.y, sl = blockIdx.z;
  const int S = g.S;
  const int s0 = tile * Cf::kTW;
  const size_t base = ((size_t)sl * g.U + u) * NRX_SYMBOLS * S;
  for (int i = threadIdx.x; i < 9 * C; i += kThreads) {
    k1[i] = __ldg(dw1 + i);
    k2[i] = __ldg(dw2 + i);
  }
  for (int i = threadIdx.x; i < NRX_SYMBOLS * Cf::IW * C; i += kThreads) {
    const int c = i % C, e = (i / C) % Cf::IW, t = i / (C * Cf::IW);
    const int s = s0 - 2 + e;
    float v = 0.f;
    const size_t act = (size_t)g.n_slots * g.U * NRX_SYMBOLS * S * C;
    if (s >= 0 && s < S && NRX_IN((base + (size_t)t * S + s) * C + c, act, 204))
      v = __ldg(z_in + (base + (size_t)t * S + s) * C + c);
    zin[(t * Cf::IW + e) * Cf::LD + c] = v;
  }
  __syncthreads();
  // dw1 on MW columns (s = s0 - 1 + e)
  for (int i = threadIdx.x; i < Cf::R1 * C; i += kThreads) {
    const int c = i % C, row = i / C;
    const int t = row / Cf::MW, e = row % Cf::MW;
    float acc = 0.f;
#pragma unroll
    for (int dt = -1; dt <= 1; ++dt) {
      const int tt = t + dt;
      if (tt < 0 || tt >= NRX_SYMBOLS) continue;
#pragma unroll
      for (int ds = -1; ds <= 1; ++ds)
        acc = fmaf(k1[c * 9 + (dt + 1) * 3 + ds + 1], zin[(tt * Cf::IW + e + 1 + ds) * Cf::LD + c], acc);
    }
    d1[row * Cf::LD + c] = acc;
  }
  __syncthreads();
  const int cg = threadIdx.x % Cf::CG, rg = threadIdx.x / Cf::CG;
  const int c0 = cg * 4;
  {
    float acc[Cf::RPT1][4];
    init_bias(acc, pw1_b, c0);
    gemm_rows<C, Cf::RPT1>(acc, d1, Cf::LD, rg, Cf::RG, pw1_t, C, c0);
    __syncthreads();
#pragma unroll
    for (int i = 0; i < Cf::RPT1; ++i) {
      const int row = rg + i * Cf::RG;
      const int s = s0 - 1 + row % Cf::MW;
      const bool inside = row < Cf::R1 && s >= 0 && s < S;
#pragma unroll
      for (int j = 0; j < 4; ++j) d1[row * Cf::LD + c0 + j] = inside ? fmaxf(acc[i][j], 0.f) : 0.f;
    }
  }
  __syncthreads();
  // dw2 + ReLU on the kTW output columns
  for (int i = threadIdx.x; i < Cf::R2 * C; i += kThreads) {
    const int c = i % C, row = i / C;
    const int t = row / Cf::kTW, x = row % Cf::kTW;
    float acc = 0.f;
#pragma unroll
    for (int dt = -1; dt <= 1; ++dt) {
      const int tt = t + dt;
      if (tt < 0 || tt >= NRX_SYMBOLS) continue;
#pragma unroll
      for (int ds = -1; ds <= 1; ++ds)
        acc = fmaf(k2[c * 9 + (dt + 1) * 3 + ds + 1], d1[(tt * Cf::MW + x + 1 + ds) * Cf::LD + c], acc);
    }
    d2[row * Cf::LD + c] = fmaxf(acc, 0.f);
  }
  __syncthreads();
  {
    float acc[Cf::RPT2][4];
    init_bias(acc, pw2_b, c0);
    gemm_rows<C, Cf::RPT2>(acc, d2, Cf::LD, rg, Cf::RG, pw2_t, C, c0);
#pragma unroll
    for (int i = 0; i < Cf::RPT2; ++i) {
      const int row = rg + i * Cf::RG;
      if (row >= Cf::R2) continue;
      const int t = row / Cf::kTW, x = row % Cf::kTW, s = s0 + x;
      if (s >= S) continue;
      const float* res = zin + (t * Cf::IW + x + 2) * Cf::LD + c0;
      float4 o = make_float4(acc[i][0] + res[0], acc[i][1] + res[1], acc[i][2] + res[2], acc[i][3] + res[3]);
      const size_t off = (base + (size_t)t * S + s) * C + c0;
      if (!NRX_IN(off + 3, (size_t)g.n_slots * g.U * NRX_SYMBOLS * S * C, 205)) continue;
      if (last) {
        float4 sv = *reinterpret_cast<const float4*>(state + off);
        sv.x += o.x;
        sv.y += o.y;
        sv.z += o.z;
        sv.w += o.w;
        *reinterpret_cast<float4*>(state + off) = sv;
      } else {
        *reinterpret_cast<float4*>(z_out + off) = o;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// ReadoutLLRs + masking: l = ro2(ReLU(ro1(S))) on the data REs, user u keeps
// its first m_u outputs, stored packed.
// ---------------------------------------------------------------------------
template <int C>
struct RoCfg {
  static constexpr int kRows = 64;
  static constexpr int CG = C / 4;
  static constexpr int RG = kThreads / CG;
  static constexpr int RPT = kRows / RG;
  static constexpr int LD = C + 1;
};

template <int C>
__global__ void __launch_bounds__(kThreads) k_readout_f32(Geometry g, SlotTable tab, ReadoutWeightsF32 w,
                                                           const float* __restrict__ state, float* __restrict__ llr) {
  using Cf = RoCfg<C>;
  extern __shared__ __align__(16) float sm[];
  float* sa = sm;
  float* sb = sm + Cf::kRows * Cf::LD;
  const int u = blockIdx.y, sl = blockIdx.z;
  const int head = tab.head[sl][u];  // Var-IO head of this user's modulation order
  const float* __restrict__ ro1_t = pick_head(w.ro1_t, head);
  const float* __restrict__ ro1_b = pick_head(w.ro1_b, head);
  const float* __restrict__ ro2 = pick_head(w.ro2, head);  // [m_max][C]
  const float* __restrict__ ro2_b = pick_head(w.ro2_b, head);
  const int r0 = blockIdx.x * Cf::kRows;
  const int S = g.S;
  const size_t base = ((size_t)sl * g.U + u) * NRX_SYMBOLS * S;
  for (int i = threadIdx.x; i < Cf::kRows * C; i += kThreads) {
    const int c = i % C, j = i / C, r = r0 + j;
    float v = 0.f;
    if (r < g.n_data) {
      const int t = g.data_t[r / S], s = r % S;
      if (NRX_IN((base + (size_t)t * S + s) * C + c, (size_t)g.n_slots * g.U * NRX_SYMBOLS * S * C, 206))
        v = __ldg(state + (base + (size_t)t * S + s) * C + c);
    }
    sa[j * Cf::LD + c] = v;
  }
  __syncthreads();
  const int cg = threadIdx.x % Cf::CG, rg = threadIdx.x / Cf::CG;
  const int c0 = cg * 4;
  float acc[Cf::RPT][4];
  init_bias(acc, ro1_b, c0);
  gemm_rows<C, Cf::RPT>(acc, sa, Cf::LD, rg, Cf::RG, ro1_t, C, c0);
#pragma unroll
  for (int i = 0; i < Cf::RPT; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) sb[(rg + i * Cf::RG) * Cf::LD + c0 + j] = fmaxf(acc[i][j], 0.f);
  __syncthreads();
  const int m = tab.bits[sl][u];
  float* dst = llr + tab.llr_off[sl][u];
  for (int i = threadIdx.x; i < Cf::kRows * m; i += kThreads) {
    const int j = i / m, o = i % m, r = r0 + j;
    if (r >= g.n_data) continue;
    float a = __ldg(ro2_b + o);
    const float* wr = ro2 + o * C;
    for (int k = 0; k < C; ++k) a = fmaf(__ldg(wr + k), sb[j * Cf::LD + k], a);
    if (NRX_IN(tab.llr_off[sl][u] + (long long)r * m + o, tab.llr_total, 207)) dst[(size_t)r * m + o] = a;
  }
}


}  // namespace

cudaError_t launch_mp_f32(const Geometry& g, const IterWeightsF32& w, const float* state, float* z, cudaStream_t st) {
  const int n_re = NRX_SYMBOLS * g.S;
  if (g.C == 64) {
    using Cf = MpCfg<64>;
    const size_t smem = sizeof(float) * 2 * Cf::ROWS * Cf::LD;
    ensure_smem<k_mp_f32<64>>((int)smem);
    k_mp_f32<64><<<dim3((n_re + Cf::kRE - 1) / Cf::kRE, g.n_slots), kThreads, smem, st>>>(g, w, state, z);
  } else if (g.C == 32) {
    using Cf = MpCfg<32>;
    const size_t smem = sizeof(float) * 2 * Cf::ROWS * Cf::LD;
    ensure_smem<k_mp_f32<32>>((int)smem);
    k_mp_f32<32><<<dim3((n_re + Cf::kRE - 1) / Cf::kRE, g.n_slots), kThreads, smem, st>>>(g, w, state, z);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_block_f32(const Geometry& g, const IterWeightsF32& w, int r, const float* z_in, float* z_out,
                             float* state, bool last, cudaStream_t st) {
  if (g.C == 64) {
    using Cf = BlkCfg<64>;
    const size_t smem = sizeof(float) * Cf::smem_floats;
    ensure_smem<k_block_f32<64>>((int)smem);
    k_block_f32<64><<<dim3((g.S + Cf::kTW - 1) / Cf::kTW, g.U, g.n_slots), kThreads, smem, st>>>(
        g, w.dw1[r], w.pw1_t[r], w.pw1_b[r], w.dw2[r], w.pw2_t[r], w.pw2_b[r], z_in, z_out, state, last ? 1 : 0);
  } else if (g.C == 32) {
    using Cf = BlkCfg<32>;
    const size_t smem = sizeof(float) * Cf::smem_floats;
    ensure_smem<k_block_f32<32>>((int)smem);
    k_block_f32<32><<<dim3((g.S + Cf::kTW - 1) / Cf::kTW, g.U, g.n_slots), kThreads, smem, st>>>(
        g, w.dw1[r], w.pw1_t[r], w.pw1_b[r], w.dw2[r], w.pw2_t[r], w.pw2_b[r], z_in, z_out, state, last ? 1 : 0);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_readout_f32(const Geometry& g, const SlotTable& tab, const ReadoutWeightsF32& w,
                               const float* state, float* llr, cudaStream_t st) {
  if (g.C == 64) {
    using Cf = RoCfg<64>;
    const size_t smem = sizeof(float) * 2 * Cf::kRows * Cf::LD;
    k_readout_f32<64><<<dim3((g.n_data + Cf::kRows - 1) / Cf::kRows, g.U, g.n_slots), kThreads, smem, st>>>(
        g, tab, w, state, llr);
  } else if (g.C == 32) {
    using Cf = RoCfg<32>;
    const size_t smem = sizeof(float) * 2 * Cf::kRows * Cf::LD;
    k_readout_f32<32><<<dim3((g.n_data + Cf::kRows - 1) / Cf::kRows, g.U, g.n_slots), kThreads, smem, st>>>(
        g, tab, w, state, llr);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

NRX_DEBUG_READER(debug_read_net_f32)
