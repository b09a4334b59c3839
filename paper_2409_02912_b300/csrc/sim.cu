// Link simulator for NRX training on the GPU: bits -> Gray QAM (TS 38.211
// Sec. 5.1), QPSK DMRS on the type-1 comb with OCC, tapped-delay-line channel
// with a Clarke sum-of-sinusoids Doppler process (or static CN(0,1) gains),
// ULA steering, AWGN (system model, Eq. 1).  Every random number comes from
// the Philox4x32-10 counter-based generator (Salmon et al., SC'11) with the
// stream and index assignment documented in include/nrx_train.h, so a batch
// is a pure function of (seed, batch index, slot parameters).
#include <cuda_runtime.h>

#include <cstring>

#include "../../include/nrx_train.h"
#include "common.cuh"

namespace {

constexpr int kMaxTaps = 32;
constexpr int kSinusoids = 16;
constexpr uint32_t kStreamBits = 1, kStreamDmrs = 2, kStreamNoise = 3, kStreamGain = 4, kStreamAoa = 9;
constexpr float kPi = 3.14159265358979323846f;
constexpr float kSlotS = 0.5e-3f, kScsHz = 30e3f;

struct SimParams {
  int n, U, B, S, nd, m_max, n_data, max_taps;
  int td[2];
  int8_t data_t[NRX_SYMBOLS];
  uint32_t key0, key1, batch;
  nrx_sim_slot slot[NRX_MAX_LAUNCH_SLOTS];
};

__device__ __forceinline__ uint4 philox(unsigned long long index, uint32_t batch, uint32_t stream, uint32_t k0,
                                        uint32_t k1) {
  uint32_t c0 = (uint32_t)index, c1 = (uint32_t)(index >> 32), c2 = batch, c3 = stream;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  return make_uint4(c0, c1, c2, c3);
}

__device__ __forceinline__ float uniform24(uint32_t x) { return (float)(x >> 8) * 5.9604644775390625e-8f; }

__device__ __forceinline__ float2 box_muller(uint32_t x0, uint32_t x1) {
  const float u1 = ((float)(x0 >> 8) + 1.f) * 5.9604644775390625e-8f;
  const float r = sqrtf(-2.f * logf(u1));
  float s, c;
  sincospif(2.f * uniform24(x1), &s, &c);
  return make_float2(r * c, r * s);
}

__global__ void k_sim_dmrs(SimParams p, float2* __restrict__ dmrs) {
  const int total = p.n * p.nd * (p.S / 2);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const uint32_t w = philox((unsigned long long)i, p.batch, kStreamDmrs, p.key0, p.key1).x;
    const float a = 0.70710678118654752f;
    dmrs[i] = make_float2((1.f - 2.f * (float)(w & 1u)) * a, (1.f - 2.f * (float)((w >> 1) & 1u)) * a);
  }
}

// taps[((slot U + u) max_taps + l) B + b][t]: tap l's gain on antenna b at symbol t.
__global__ void k_sim_taps(SimParams p, float2* __restrict__ taps) {
  const int total = p.n * p.U * p.max_taps * p.B;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int bd = i % p.B;
    const int l = (i / p.B) % p.max_taps;
    const int su = i / (p.B * p.max_taps);
    const int sl = su / p.U;
    const nrx_sim_slot& sp = p.slot[sl];
    const int L = sp.num_taps;
    const int Bd = sp.ula ? 1 : p.B;
    if (l >= L || bd >= Bd) continue;
    // normalised exponential power-delay profile
    const float step = L > 1 ? 4.f / (float)(L - 1) : 0.f;  // tau_l / DS
    float psum = 0.f;
    for (int k = 0; k < L; ++k) psum += expf(-(float)k * step);
    const float amp = sqrtf(expf(-(float)l * step) / psum);
    const unsigned long long gidx = ((unsigned long long)su * L + l) * Bd + bd;
    float2 a[NRX_SYMBOLS];
    const uint4 w0 = philox(gidx, p.batch, kStreamGain, p.key0, p.key1);
    if (sp.doppler_hz == 0.f) {
      const float2 g = box_muller(w0.x, w0.y);
      const float s = 0.70710678118654752f * amp;
#pragma unroll
      for (int t = 0; t < NRX_SYMBOLS; ++t) a[t] = make_float2(g.x * s, g.y * s);
    } else {
      const float theta = (2.f * uniform24(w0.x) - 1.f) * kPi;
#pragma unroll
      for (int t = 0; t < NRX_SYMBOLS; ++t) a[t] = make_float2(0.f, 0.f);
      for (int k = 0; k < 4; ++k) {
        const uint4 wp = philox(gidx, p.batch, kStreamGain + 1 + k, p.key0, p.key1);
        const uint32_t ws[4] = {wp.x, wp.y, wp.z, wp.w};
        for (int q = 0; q < 4; ++q) {
          const int m = 4 * k + q + 1;  // sinusoid 1..16
          const float phi = 2.f * kPi * uniform24(ws[q]);
          const float alpha = (2.f * kPi * (float)m - kPi + theta) / (float)kSinusoids;
          const float fd = sp.doppler_hz * cosf(alpha);
#pragma unroll
          for (int t = 0; t < NRX_SYMBOLS; ++t) {
            float sn, cs;
            sincosf(2.f * kPi * fd * ((float)t * (kSlotS / NRX_SYMBOLS)) + phi, &sn, &cs);
            a[t].x += cs;
            a[t].y += sn;
          }
        }
      }
      const float s = amp * 0.25f;  // 1 / sqrt(16)
#pragma unroll
      for (int t = 0; t < NRX_SYMBOLS; ++t) a[t] = make_float2(a[t].x * s, a[t].y * s);
    }
    if (sp.ula) {
      const uint32_t wa = philox((unsigned long long)su * L + l, p.batch, kStreamAoa, p.key0, p.key1).x;
      const float aoa = (2.f * uniform24(wa) - 1.f) * (kPi / 3.f);
      const float sa = sinf(aoa);
      for (int b = 0; b < p.B; ++b) {
        float sn, cs;
        sincospif((float)b * sa, &sn, &cs);
        float2* o = taps + (((size_t)su * p.max_taps + l) * p.B + b) * NRX_SYMBOLS;
#pragma unroll
        for (int t = 0; t < NRX_SYMBOLS; ++t)
          o[t] = make_float2(a[t].x * cs - a[t].y * sn, a[t].x * sn + a[t].y * cs);
      }
    } else {
      float2* o = taps + (((size_t)su * p.max_taps + l) * p.B + bd) * NRX_SYMBOLS;
#pragma unroll
      for (int t = 0; t < NRX_SYMBOLS; ++t) o[t] = a[t];
    }
  }
}

__device__ __forceinline__ float2 qam(uint32_t w, int m) {
  const float b0 = 1.f - 2.f * (float)(w & 1u), b1 = 1.f - 2.f * (float)((w >> 1) & 1u);
  if (m == 2) return make_float2(b0 * 0.70710678118654752f, b1 * 0.70710678118654752f);
  const float b2 = 1.f - 2.f * (float)((w >> 2) & 1u), b3 = 1.f - 2.f * (float)((w >> 3) & 1u);
  if (m == 4) {
    const float s = 0.31622776601683794f;  // 1 / sqrt(10)
    return make_float2(b0 * (2.f - b2) * s, b1 * (2.f - b3) * s);
  }
  const float b4 = 1.f - 2.f * (float)((w >> 4) & 1u), b5 = 1.f - 2.f * (float)((w >> 5) & 1u);
  const float s = 0.15430334996209191f;  // 1 / sqrt(42)
  return make_float2(b0 * (4.f - b2 * (2.f - b4)) * s, b1 * (4.f - b3 * (2.f - b5)) * s);
}

// One thread per (slot, t, s): transmitted symbols of every user, channel of
// every (user, antenna), received value of every antenna.
__global__ void k_sim_rx(SimParams p, const float2* __restrict__ taps, const float2* __restrict__ dmrs,
                         float2* __restrict__ y, uint8_t* __restrict__ bits, int32_t* __restrict__ m_u,
                         float* __restrict__ h) {
  const int total = p.n * NRX_SYMBOLS * p.S;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int s = i % p.S;
    const int t = (i / p.S) % NRX_SYMBOLS;
    const int sl = i / (p.S * NRX_SYMBOLS);
    const nrx_sim_slot& sp = p.slot[sl];
    const int L = sp.num_taps;
    const float tau_step = L > 1 ? 4.f * sp.delay_spread_s / (float)(L - 1) : 0.f;
    const float fs = ((float)s - 0.5f * (float)p.S) * kScsHz;
    int d = -1, di = -1;
    for (int k = 0; k < p.nd; ++k)
      if (p.td[k] == t) d = k;
    for (int k = 0; k < NRX_SYMBOLS - p.nd; ++k)
      if (p.data_t[k] == t) di = k;
    float2 acc[NRX_MAX_RX];
    for (int b = 0; b < p.B; ++b) acc[b] = make_float2(0.f, 0.f);
    for (int u = 0; u < p.U; ++u) {
      const int m = sp.bits_per_symbol[u];
      float2 x = make_float2(0.f, 0.f);
      const size_t su = (size_t)sl * p.U + u;
      if (d >= 0) {
        if ((s & 1) == (u >> 1)) {
          const int mm = s >> 1;
          x = dmrs[((size_t)sl * p.nd + d) * (p.S / 2) + mm];
          if ((u & 1) && (mm & 1)) x = make_float2(-x.x, -x.y);
        }
      } else {
        const int re = di * p.S + s;
        const uint32_t w = philox(su * p.n_data + re, p.batch, kStreamBits, p.key0, p.key1).x;
        uint8_t* bo = bits + (su * p.n_data + re) * p.m_max;
        for (int j = 0; j < p.m_max; ++j) bo[j] = j < m ? (uint8_t)((w >> j) & 1u) : (uint8_t)0;
        x = qam(w, m);
      }
      if (t == 0 && s == 0) m_u[su] = m;
      float* ho = h + ((su * NRX_SYMBOLS + t) * p.S + s) * (2 * p.B);
      for (int b = 0; b < p.B; ++b) {
        float2 H = make_float2(0.f, 0.f);
        for (int l = 0; l < L; ++l) {
          float sn, cs;
          sincospif(-2.f * fs * ((float)l * tau_step), &sn, &cs);
          const float2 a = taps[((su * p.max_taps + l) * p.B + b) * NRX_SYMBOLS + t];
          H.x += a.x * cs - a.y * sn;
          H.y += a.x * sn + a.y * cs;
        }
        ho[2 * b] = H.x;
        ho[2 * b + 1] = H.y;
        acc[b].x += H.x * x.x - H.y * x.y;
        acc[b].y += H.x * x.y + H.y * x.x;
      }
    }
    const float sn0 = sqrtf(0.5f * sp.noise_var);
    for (int b = 0; b < p.B; ++b) {
      const uint4 w = philox((((unsigned long long)sl * p.B + b) * NRX_SYMBOLS + t) * p.S + s, p.batch,
                             kStreamNoise, p.key0, p.key1);
      const float2 z = box_muller(w.x, w.y);
      y[(((size_t)sl * p.B + b) * NRX_SYMBOLS + t) * p.S + s] =
          make_float2(acc[b].x + sn0 * z.x, acc[b].y + sn0 * z.y);
    }
  }
}

int blocks_for(size_t n) {
  const size_t b = (n + 255) / 256;
  return (int)(b < 148 * 16 ? (b ? b : 1) : 148 * 16);
}

}  // namespace

extern "C" {

size_t nrx_train_sim_scratch_bytes(int32_t n_slots, int32_t num_users, int32_t num_rx_ant, int32_t max_taps) {
  if (n_slots < 1 || num_users < 1 || num_rx_ant < 1 || max_taps < 1) return 0;
  return (size_t)n_slots * num_users * max_taps * num_rx_ant * NRX_SYMBOLS * sizeof(float2);
}

nrx_status nrx_train_simulate(int32_t n_slots, const nrx_sim_slot* slots, int32_t num_users, int32_t num_rx_ant,
                              int32_t num_prb, int32_t num_dmrs_symbols, const int32_t* dmrs_symbols, int32_t m_max,
                              uint64_t seed, uint32_t batch, void* scratch, void* y, void* dmrs, uint8_t* bits,
                              int32_t* bits_per_symbol_dev, float* h, void* stream) {
  if (n_slots < 1 || n_slots > NRX_MAX_LAUNCH_SLOTS || !slots || num_users < 1 || num_users > NRX_MAX_USERS ||
      num_rx_ant < 1 || num_rx_ant > NRX_MAX_RX || num_prb < 1 || num_prb > 275 ||
      (num_dmrs_symbols != 1 && num_dmrs_symbols != 2) || !dmrs_symbols || m_max < 2 || m_max > 8 || !scratch ||
      !y || !dmrs || !bits || !bits_per_symbol_dev || !h)
    return NRX_EINVAL;
  SimParams p;
  memset(&p, 0, sizeof(p));
  p.n = n_slots;
  p.U = num_users;
  p.B = num_rx_ant;
  p.S = 12 * num_prb;
  p.nd = num_dmrs_symbols;
  p.m_max = m_max;
  p.n_data = (NRX_SYMBOLS - num_dmrs_symbols) * p.S;
  p.key0 = (uint32_t)seed;
  p.key1 = (uint32_t)(seed >> 32);
  p.batch = batch;
  for (int k = 0; k < num_dmrs_symbols; ++k) {
    if (dmrs_symbols[k] < 0 || dmrs_symbols[k] > 13 || (k == 1 && dmrs_symbols[1] <= dmrs_symbols[0]))
      return NRX_EINVAL;
    p.td[k] = dmrs_symbols[k];
  }
  for (int t = 0, di = 0; t < NRX_SYMBOLS; ++t)
    if (t != p.td[0] && (num_dmrs_symbols == 1 || t != p.td[1])) p.data_t[di++] = (int8_t)t;
  for (int i = 0; i < n_slots; ++i) {
    const nrx_sim_slot& sp = slots[i];
    if (sp.num_taps < 1 || sp.num_taps > kMaxTaps || !(sp.delay_spread_s > 0.f) || !(sp.noise_var >= 0.f) ||
        sp.doppler_hz < 0.f)
      return NRX_EINVAL;
    for (int u = 0; u < num_users; ++u) {
      const int m = sp.bits_per_symbol[u];
      if ((m != 2 && m != 4 && m != 6) || m > m_max) return NRX_EINVAL;
    }
    p.slot[i] = sp;
    if (sp.num_taps > p.max_taps) p.max_taps = sp.num_taps;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  float2* taps = static_cast<float2*>(scratch);
  k_sim_dmrs<<<blocks_for((size_t)p.n * p.nd * (p.S / 2)), 256, 0, st>>>(p, static_cast<float2*>(dmrs));
  k_sim_taps<<<blocks_for((size_t)p.n * p.U * p.max_taps * p.B), 256, 0, st>>>(p, taps);
  k_sim_rx<<<blocks_for((size_t)p.n * NRX_SYMBOLS * p.S), 256, 0, st>>>(p, taps, static_cast<const float2*>(dmrs),
                                                                     static_cast<float2*>(y), bits,
                                                                     bits_per_symbol_dev, h);
  return cudaGetLastError() == cudaSuccess ? NRX_OK : NRX_ECUDA;
}

}  // extern "C"
