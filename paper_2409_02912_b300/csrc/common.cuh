// Device-side definitions shared by the NRX / LMMSE kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "debug.cuh"

#define NRX_MAX_USERS 4
#define NRX_MAX_RX 8
#define NRX_MAX_LAUNCH_SLOTS 64
#define NRX_SYMBOLS 14

// Geometry shared by every slot of one launch.
struct Geometry {
  int n_slots;    // slots in this launch
  int S;          // subcarriers
  int U;          // active users
  int B;          // Rx antennas
  int C;          // state depth
  int F;          // input features 4B+2
  int m_max;      // LLR head width
  int n_dmrs;     // 1 or 2
  int td0, td1;   // DMRS symbols (td1 == td0 when n_dmrs == 1)
  int n_data;     // data REs per slot = (14 - n_dmrs) * S
  int8_t data_t[NRX_SYMBOLS];  // data symbol index -> symbol t
};

// Per-slot table, passed by value in kernel parameters (no per-call copies).
struct SlotTable {
  const float2* dmrs[NRX_MAX_LAUNCH_SLOTS];        // [n_dmrs][S/2] per slot
  float noise_var[NRX_MAX_LAUNCH_SLOTS];
  int8_t bits[NRX_MAX_LAUNCH_SLOTS][NRX_MAX_USERS];  // m_u per slot and user
  int32_t llr_off[NRX_MAX_LAUNCH_SLOTS][NRX_MAX_USERS];  // float offset of user u's LLRs
  int8_t head[NRX_MAX_LAUNCH_SLOTS][NRX_MAX_USERS];  // Var-IO head of the user's modulation order (0 otherwise)
  long long llr_total;  // floats of the call's packed LLR vector (bounds-checked build)
};

// ---------------------------------------------------------------------------
// DMRS LS estimate and linear interpolation (Sec. II-A front end)
// ---------------------------------------------------------------------------

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // a * conj(b)
  return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

// True when the other port of user u's CDM group is active (OCC de-spread).
__device__ __forceinline__ bool occ_shared(int u, int U) { return (u ^ 1) < U; }

// LS on comb position m of user u on DMRS symbol index d:
//   y(2m+g) * conj(p) / |p|^2,  p = w_u(m) r(m).
__device__ __forceinline__ float2 ls_pilot(const float2* __restrict__ y_bt,  // y[b][t][:S]
                                           const float2* __restrict__ r,     // r of this DMRS symbol, [S/2]
                                           int u, int m, int S) {
  const int g = u >> 1;
  if (!NRX_IN(m, S / 2, 1) || !NRX_IN(2 * m + g, S, 2)) return make_float2(0.f, 0.f);
  float2 p = __ldg(r + m);
  if ((u & 1) && (m & 1)) p = make_float2(-p.x, -p.y);
  const float inv = 1.0f / (p.x * p.x + p.y * p.y);
  float2 z = cmulc(__ldg(y_bt + 2 * m + g), p);
  return make_float2(z.x * inv, z.y * inv);
}

// Estimate number n of user u (after OCC de-spread when the group is shared).
__device__ __forceinline__ float2 ls_estimate(const float2* __restrict__ y_bt, const float2* __restrict__ r,
                                              int u, int U, int n, int S) {
  if (occ_shared(u, U)) {
    float2 a = ls_pilot(y_bt, r, u, 2 * n, S), b = ls_pilot(y_bt, r, u, 2 * n + 1, S);
    return make_float2(0.5f * (a.x + b.x), 0.5f * (a.y + b.y));
  }
  return ls_pilot(y_bt, r, u, n, S);
}

// Frequency-interpolated estimate of user u at subcarrier s on one DMRS symbol,
// holding the edge estimates outside the first / last estimate position.
__device__ __forceinline__ float2 ls_interp_freq(const float2* __restrict__ y_bt, const float2* __restrict__ r,
                                                 int u, int U, int S, int s) {
  const bool sh = occ_shared(u, U);
  const int spacing = sh ? 4 : 2;
  const int off = sh ? 1 + (u >> 1) : (u >> 1);
  const int N = sh ? S / 4 : S / 2;
  if (s <= off) return ls_estimate(y_bt, r, u, U, 0, S);
  const int last = off + spacing * (N - 1);
  if (s >= last) return ls_estimate(y_bt, r, u, U, N - 1, S);
  const int n = (s - off) / spacing;
  const float a = (float)(s - (off + spacing * n)) / (float)spacing;
  float2 e0 = ls_estimate(y_bt, r, u, U, n, S), e1 = ls_estimate(y_bt, r, u, U, n + 1, S);
  return make_float2(e0.x + a * (e1.x - e0.x), e0.y + a * (e1.y - e0.y));
}

// Time interpolation between the DMRS symbols (hold outside).
__device__ __forceinline__ float2 interp_time(const Geometry& g, int t, float2 h0, float2 h1) {
  if (g.n_dmrs == 1 || t <= g.td0) return h0;
  if (t >= g.td1) return h1;
  const float a = (float)(t - g.td0) / (float)(g.td1 - g.td0);
  return make_float2(h0.x + a * (h1.x - h0.x), h0.y + a * (h1.y - h0.y));
}

// Positional encoding (distance to the nearest pilot, ties to the lower index).
__device__ __forceinline__ float pe_time(const Geometry& g, int t) {
  int near = g.td0;
  if (g.n_dmrs == 2 && abs(t - g.td1) < abs(t - g.td0)) near = g.td1;
  return (float)(t - near) / 7.0f;
}
__device__ __forceinline__ float pe_freq(int u, int s) {
  const int grp = u >> 1;
  if (((s - grp) & 1) == 0) return 0.0f;
  return s < grp ? -0.5f : 0.5f;
}

__device__ __forceinline__ int ceil_div(int a, int b) { return (a + b - 1) / b; }
