// Training kernels (FP32, CUDA cores): the NRX layers of Sec. II-A one at a
// time, with their backward passes, for the BCE training scheme of Sec. II-B.
// Composed into forward / backward by the Python binding (torch autograd
// supplies only the bookkeeping; every arithmetic step runs here).
#include <cuda_runtime.h>

#include <cstring>

#include "../../include/nrx_train.h"
#include "common.cuh"

namespace {

constexpr int kThreads = 256;

// ---------------------------------------------------------------------------
// Network input features x [n][U][14][S][4B+2] (Sec. II-A): received grid,
// interpolated LS estimate of the user, positional encoding.
// ---------------------------------------------------------------------------
__global__ void k_features(Geometry g, SlotTable tab, const float2* __restrict__ y, float* __restrict__ x) {
  const size_t total = (size_t)g.n_slots * g.U * NRX_SYMBOLS * g.S;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int s = (int)(i % g.S);
    const int t = (int)((i / g.S) % NRX_SYMBOLS);
    const int u = (int)((i / ((size_t)g.S * NRX_SYMBOLS)) % g.U);
    const int sl = (int)(i / ((size_t)g.S * NRX_SYMBOLS * g.U));
    const float2* ys = y + (size_t)sl * g.B * NRX_SYMBOLS * g.S;
    float* f = x + i * g.F;
    for (int b = 0; b < g.B; ++b) {
      const float2 v = ys[((size_t)b * NRX_SYMBOLS + t) * g.S + s];
      f[2 * b] = v.x;
      f[2 * b + 1] = v.y;
      const float2 h0 = ls_interp_freq(ys + ((size_t)b * NRX_SYMBOLS + g.td0) * g.S, tab.dmrs[sl], u, g.U, g.S, s);
      float2 h1 = h0;
      if (g.n_dmrs == 2)
        h1 = ls_interp_freq(ys + ((size_t)b * NRX_SYMBOLS + g.td1) * g.S, tab.dmrs[sl] + g.S / 2, u, g.U, g.S, s);
      const float2 hv = interp_time(g, t, h0, h1);
      f[2 * g.B + 2 * b] = hv.x;
      f[2 * g.B + 2 * b + 1] = hv.y;
    }
    f[4 * g.B] = pe_time(g, t);
    f[4 * g.B + 1] = pe_freq(u, s);
  }
}

// ---------------------------------------------------------------------------
// Strided GEMM: C[m][n] (+)= act(sum_k A(m,k) B(k,n) + bias[n] + R[m][n]),
// A(m,k) = A[m*sam + k*sak], B(k,n) = B[k*sbk + n*sbn].  64x64 output tiles,
// K in chunks of 16 through shared memory, 4x4 outputs per thread.  With
// `atomic` the tile is added to C with atomics instead (gradient accumulation);
// gridDim.z > 1 then splits the K range across CTAs (weight gradients, where K
// is the number of REs).
// ---------------------------------------------------------------------------
// R may alias C (in-place accumulation): each element is read, then written,
// by the same thread.
__global__ void __launch_bounds__(kThreads) k_gemm(int M, int N, int K, const float* __restrict__ A, long long sam,
                                                   long long sak, const float* __restrict__ B, long long sbk,
                                                   long long sbn, const float* __restrict__ bias, const float* R,
                                                   long long ldr, float* C, long long ldc, int relu, int atomic) {
  __shared__ float As[16][64 + 4];
  __shared__ float Bs[16][64 + 4];
  const int m0 = blockIdx.x * 64, n0 = blockIdx.y * 64;
  const int kchunk = (K + gridDim.z - 1) / gridDim.z;
  const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  float acc[4][4] = {};
  for (int k0 = kb; k0 < ke; k0 += 16) {
    // Consecutive threads walk the operand's unit-stride index (coalesced).
    for (int i = threadIdx.x; i < 16 * 64; i += kThreads) {
      int kk = i / 64, mm = i % 64;
      if (sak == 1) kk = i % 16, mm = i / 16;
      const int m = m0 + mm, k = k0 + kk;
      As[kk][mm] = (m < M && k < ke) ? A[(long long)m * sam + (long long)k * sak] : 0.f;
    }
    for (int i = threadIdx.x; i < 16 * 64; i += kThreads) {
      int kk = i / 64, nn = i % 64;
      if (sbk == 1) kk = i % 16, nn = i / 16;
      const int n = n0 + nn, k = k0 + kk;
      Bs[kk][nn] = (n < N && k < ke) ? B[(long long)k * sbk + (long long)n * sbn] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        a[i] = As[kk][ty * 4 + i];
        b[i] = Bs[kk][tx * 4 + i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty * 4 + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx * 4 + j;
      if (n >= N) continue;
      if (atomic) {
        atomicAdd(C + (long long)m * ldc + n, acc[i][j]);
      } else {
        float v = acc[i][j];
        if (bias) v += bias[n];
        if (R) v += R[(long long)m * ldr + n];
        if (relu) v = fmaxf(v, 0.f);
        C[(long long)m * ldc + n] = v;
      }
    }
  }
}

// out[n] += sum_m X[m][n] (bias gradients).  256 threads: 64 columns x 4 row
// groups, four independent partial sums per thread, a shared-memory reduction
// over the row groups, one atomic per column and CTA.
__global__ void __launch_bounds__(256) k_colsum(int M, int N, const float* __restrict__ X, long long ldx,
                                                float* __restrict__ out) {
  __shared__ float red[4][64];
  const int cn = threadIdx.x & 63, rg = threadIdx.x >> 6;
  const long long step = (long long)gridDim.x * 4;
  for (int n0 = 0; n0 < N; n0 += 64) {
    const int n = n0 + cn;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    if (n < N) {
      long long m = (long long)blockIdx.x * 4 + rg;
      for (; m + 3 * step < M; m += 4 * step) {
        a0 += X[m * ldx + n];
        a1 += X[(m + step) * ldx + n];
        a2 += X[(m + 2 * step) * ldx + n];
        a3 += X[(m + 3 * step) * ldx + n];
      }
      for (; m < M; m += step) a0 += X[m * ldx + n];
    }
    red[rg][cn] = (a0 + a1) + (a2 + a3);
    __syncthreads();
    if (rg == 0 && n < N) atomicAdd(out + n, (red[0][cn] + red[1][cn]) + (red[2][cn] + red[3][cn]));
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Depthwise 3x3 over [planes][14][S][C], zero padding:
//   Y[t,s,c] = act(sum_{i,j} k[c][i][j] X[t+i-1, s+j-1, c]); with flip the taps
//   are read as k[c][2-i][2-j] (the adjoint, used for the input gradient).
// One thread per (plane, s, c) slides down the 14 symbols with a window of
// three input rows x three subcarriers (each input value is loaded once per
// thread, consecutive threads read consecutive channels).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void dw_load_row(const float* __restrict__ xp, int t, int s, int S, int C, int c,
                                            float (&r)[3]) {
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const int ss = s + j - 1;
    r[j] = (t >= 0 && t < NRX_SYMBOLS && ss >= 0 && ss < S) ? xp[((size_t)t * S + ss) * C + c] : 0.f;
  }
}

__global__ void k_dw3(int planes, int S, int C, const float* __restrict__ X, const float* __restrict__ k, int flip,
                      int relu, float* __restrict__ Y) {
  const size_t total = (size_t)planes * S * C;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const int s = (int)((i / C) % S);
    const size_t plane = i / ((size_t)C * S);
    const float* xp = X + plane * NRX_SYMBOLS * S * C;
    float* yp = Y + plane * NRX_SYMBOLS * S * C;
    float kk[9];
#pragma unroll
    for (int j = 0; j < 9; ++j) kk[j] = k[c * 9 + (flip ? 8 - j : j)];
    float r0[3], r1[3], r2[3];
    dw_load_row(xp, -1, s, S, C, c, r0);
    dw_load_row(xp, 0, s, S, C, c, r1);
    dw_load_row(xp, 1, s, S, C, c, r2);
    for (int t = 0; t < NRX_SYMBOLS; ++t) {
      float acc = 0.f;
#pragma unroll
      for (int j = 0; j < 3; ++j) acc = fmaf(kk[j], r0[j], acc);
#pragma unroll
      for (int j = 0; j < 3; ++j) acc = fmaf(kk[3 + j], r1[j], acc);
#pragma unroll
      for (int j = 0; j < 3; ++j) acc = fmaf(kk[6 + j], r2[j], acc);
      yp[((size_t)t * S + s) * C + c] = relu ? fmaxf(acc, 0.f) : acc;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        r0[j] = r1[j];
        r1[j] = r2[j];
      }
      dw_load_row(xp, t + 2, s, S, C, c, r2);
    }
  }
}

// gk[c][i][j] += sum_{plane,t,s} G[t,s,c] X[t+i-1, s+j-1, c]: one thread per
// (plane, s, c) sliding down the symbols, partial sums reduced per channel in
// shared memory, then one atomic per (channel, tap) and CTA.
__global__ void __launch_bounds__(256) k_dw3_wgrad(int planes, int S, int C, const float* __restrict__ X,
                                                   const float* __restrict__ G, float* __restrict__ gk) {
  extern __shared__ float red[];  // [C][9]
  for (int i = threadIdx.x; i < 9 * C; i += blockDim.x) red[i] = 0.f;
  __syncthreads();
  const size_t total = (size_t)planes * S * C;
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < total) {
    const int c = (int)(i % C);
    const int s = (int)((i / C) % S);
    const size_t plane = i / ((size_t)C * S);
    const float* xp = X + plane * NRX_SYMBOLS * S * C;
    const float* gp = G + plane * NRX_SYMBOLS * S * C;
    float acc[9] = {};
    float r0[3], r1[3], r2[3];
    dw_load_row(xp, -1, s, S, C, c, r0);
    dw_load_row(xp, 0, s, S, C, c, r1);
    dw_load_row(xp, 1, s, S, C, c, r2);
    for (int t = 0; t < NRX_SYMBOLS; ++t) {
      const float gv = gp[((size_t)t * S + s) * C + c];
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        acc[j] = fmaf(gv, r0[j], acc[j]);
        acc[3 + j] = fmaf(gv, r1[j], acc[3 + j]);
        acc[6 + j] = fmaf(gv, r2[j], acc[6 + j]);
      }
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        r0[j] = r1[j];
        r1[j] = r2[j];
      }
      dw_load_row(xp, t + 2, s, S, C, c, r2);
    }
#pragma unroll
    for (int j = 0; j < 9; ++j) atomicAdd(red + c * 9 + j, acc[j]);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < 9 * C; j += blockDim.x)
    if (red[j] != 0.f) atomicAdd(gk + j, red[j]);
}

// G <- G * (Y > 0)
__global__ void k_relu_mask(size_t n, float* __restrict__ G, const float* __restrict__ Y) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    if (!(Y[i] > 0.f)) G[i] = 0.f;
}

// a[sl][u][r][c] = sum_{v != u, v < U} m[sl][v][r][c]  (its own adjoint)
__global__ void k_aggregate(int n_slots, int U, size_t per_user, const float* __restrict__ m, float* __restrict__ a) {
  const size_t total = (size_t)n_slots * per_user;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t sl = i / per_user, e = i % per_user;
    float v[NRX_MAX_USERS];
    for (int u = 0; u < U; ++u) v[u] = m[(sl * U + u) * per_user + e];
    for (int u = 0; u < U; ++u) {
      float acc = 0.f;
      for (int w = 0; w < U; ++w)
        if (w != u) acc += v[w];
      a[(sl * U + u) * per_user + e] = acc;
    }
  }
}

__global__ void k_axpy(size_t n, float alpha, const float* __restrict__ x, float* __restrict__ y) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = fmaf(alpha, x[i], y[i]);
}

// Masked BCE on the logits of Eq. 2 (Sec. II-B): data REs, first m_u bits,
// normalised by the number of counted bits n_bits = n_data * sum m_u:
//   loss += weight/n_bits * (softplus(l) - b l); grad = weight/n_bits * (sigmoid(l) - b).
// l, grad: [n][U][14][S][m_max]; bits: [n][U][n_data][m_max]; m: [n][U].
__global__ void k_bce(Geometry g, const float* __restrict__ l, const uint8_t* __restrict__ bits,
                      const int32_t* __restrict__ m_u, float weight, float* __restrict__ grad,
                      double* __restrict__ loss) {
  __shared__ float s_scale;
  if (threadIdx.x == 0) {
    long long sum_m = 0;
    for (int i = 0; i < g.n_slots * g.U; ++i) sum_m += m_u[i];
    s_scale = sum_m > 0 ? (float)((double)weight / ((double)g.n_data * (double)sum_m)) : 0.f;
  }
  __syncthreads();
  const float scale = s_scale;
  const size_t total = (size_t)g.n_slots * g.U * NRX_SYMBOLS * g.S * g.m_max;
  double part = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(i % g.m_max);
    const size_t re = i / g.m_max;
    const int s = (int)(re % g.S);
    const int t = (int)((re / g.S) % NRX_SYMBOLS);
    const size_t su = re / ((size_t)g.S * NRX_SYMBOLS);
    int di = -1;
    for (int d = 0; d < NRX_SYMBOLS - g.n_dmrs; ++d)
      if (g.data_t[d] == t) di = d;
    float gr = 0.f;
    if (di >= 0 && j < m_u[su]) {
      const float x = l[i];
      const float b = (float)bits[((su * g.n_data) + (size_t)di * g.S + s) * g.m_max + j];
      const float sp = x > 0.f ? x + log1pf(expf(-x)) : log1pf(expf(x));
      part += (double)scale * ((double)sp - (double)b * x);
      gr = scale * (1.f / (1.f + expf(-x)) - b);
    }
    grad[i] = gr;
  }
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, part);
}

// Channel-estimate MSE of the second read-out (Sec. II-B, weighted by gamma):
//   loss += scale * sum (h_hat - h)^2;  grad = 2 scale (h_hat - h).
__global__ void k_mse(size_t n, const float* __restrict__ h_hat, const float* __restrict__ h, float scale,
                      float* __restrict__ grad, double* __restrict__ loss) {
  double part = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float d = h_hat[i] - h[i];
    part += (double)scale * (double)d * (double)d;
    grad[i] = 2.f * scale * d;
  }
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, part);
}

// Var-IO plane selection: rows of the planes (slot, user) whose modulation
// order is m_head take src (first `width` columns), other planes 0 (or stay
// unchanged with accumulate).
__global__ void k_plane_mask(long long planes, long long rows_per_plane, int width, long long ld_src,
                             long long ld_dst, const int32_t* __restrict__ m_u, int m_head,
                             const float* __restrict__ src, float* __restrict__ dst, int accumulate) {
  const long long total = planes * rows_per_plane * width;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % width);
    const long long row = i / width;
    const bool sel = m_u[row / rows_per_plane] == m_head;
    const float v = sel ? src[row * ld_src + c] : 0.f;
    float* d = dst + row * ld_dst + c;
    if (accumulate) {
      if (sel) *d += v;
    } else {
      *d = v;
    }
  }
}

// Adam on FP32 master weights (bias-corrected step sizes passed in).
__global__ void k_adam(size_t n, float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m1,
                       float* __restrict__ m2, const float* __restrict__ lr_t_dev, float b1, float b2, float eps) {
  const float lr_t = *lr_t_dev;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.f - b1) * gi;
    const float b = b2 * m2[i] + (1.f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = b;
    w[i] -= lr_t * a / (sqrtf(b) + eps);
  }
}

int blocks_for(size_t n) {
  size_t b = (n + kThreads - 1) / kThreads;
  return (int)(b < 148 * 32 ? (b ? b : 1) : 148 * 32);
}

nrx_status to_status(cudaError_t e) { return e == cudaSuccess ? NRX_OK : NRX_ECUDA; }

}  // namespace

extern "C" {

nrx_status nrx_train_features(int32_t n_slots, int32_t num_rx_ant, const void* y, const nrx_slot_cfg* cfgs,
                              float* x, void* stream) {
  if (!y || !cfgs || !x || n_slots < 1 || n_slots > NRX_MAX_LAUNCH_SLOTS || num_rx_ant < 1 ||
      num_rx_ant > NRX_MAX_RX)
    return NRX_EINVAL;
  const nrx_slot_cfg& c0 = cfgs[0];
  if (c0.num_prb < 1 || c0.num_users < 1 || c0.num_users > NRX_MAX_USERS ||
      (c0.num_dmrs_symbols != 1 && c0.num_dmrs_symbols != 2))
    return NRX_EINVAL;
  Geometry g;
  SlotTable tab;
  memset(&g, 0, sizeof(g));
  memset(&tab, 0, sizeof(tab));
  g.n_slots = n_slots;
  g.S = 12 * c0.num_prb;
  g.U = c0.num_users;
  g.B = num_rx_ant;
  g.F = 4 * num_rx_ant + 2;
  g.n_dmrs = c0.num_dmrs_symbols;
  g.td0 = c0.dmrs_symbols[0];
  g.td1 = g.n_dmrs == 2 ? c0.dmrs_symbols[1] : g.td0;
  for (int i = 0; i < n_slots; ++i) {
    if (!cfgs[i].dmrs_seq || cfgs[i].num_prb != c0.num_prb || cfgs[i].num_users != c0.num_users) return NRX_EINVAL;
    tab.dmrs[i] = static_cast<const float2*>(cfgs[i].dmrs_seq);
  }
  const size_t n = (size_t)n_slots * g.U * NRX_SYMBOLS * g.S;
  k_features<<<blocks_for(n), kThreads, 0, static_cast<cudaStream_t>(stream)>>>(g, tab, static_cast<const float2*>(y),
                                                                               x);
  return to_status(cudaGetLastError());
}

nrx_status nrx_train_gemm(int32_t M, int32_t N, int32_t K, const float* A, int64_t sam, int64_t sak, const float* B,
                          int64_t sbk, int64_t sbn, const float* bias, const float* R, int64_t ldr, float* C,
                          int64_t ldc, int32_t relu, int32_t accumulate, int32_t split_k, void* stream) {
  if (M < 1 || N < 1 || K < 1 || !A || !B || !C || split_k < 1 || split_k > 65535) return NRX_EINVAL;
  if ((split_k > 1 && !accumulate) || (accumulate && (bias || R || relu))) return NRX_EINVAL;
  dim3 grid((M + 63) / 64, (N + 63) / 64, split_k);
  k_gemm<<<grid, kThreads, 0, static_cast<cudaStream_t>(stream)>>>(M, N, K, A, sam, sak, B, sbk, sbn, bias, R, ldr, C,
                                                                  ldc, relu, accumulate ? 1 : 0);
  return to_status(cudaGetLastError());
}

nrx_status nrx_train_colsum(int32_t M, int32_t N, const float* X, int64_t ldx, float* out, void* stream) {
  if (M < 1 || N < 1 || !X || !out) return NRX_EINVAL;
  const int blocks = (M + 63) / 64 < 592 ? (M + 63) / 64 : 592;
  k_colsum<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(M, N, X, ldx, out);
  return to_status(cudaGetLastError());
}

nrx_status nrx_train_dw3(int32_t planes, int32_t S, int32_t C, const float* X, const float* k, int32_t flip,
                         int32_t relu, float* Y, void* stream) {
  if (planes < 1 || S < 1 || C < 1 || !X || !k || !Y) return NRX_EINVAL;
  const size_t n = (size_t)planes * S * C;  // one thread per (plane, subcarrier, channel)
  k_dw3<<<blocks_for(n), kThreads, 0, static_cast<cudaStream_t>(stream)>>>(planes, S, C, X, k, flip, relu, Y);
  return to_status(cudaGetLastError());
}

nrx_status nrx_train_dw3_wgrad(int32_t planes, int32_t S, int32_t C, const float* X, const float* G, float* gk,
                               void* stream) {
  if (planes < 1 || S < 1 || C < 1 || C > 1024 || !X || !G || !gk) return NRX_EINVAL;
  const size_t n = (size_t)planes * S * C;  // one thread per (plane, subcarrier, channel)
  const size_t blocks = (n + 255) / 256;
  if (blocks > 0x7fffffff) return NRX_EINVAL;
  k_dw3_wgrad<<<(unsigned)blocks, 256, 9 * C * sizeof(float), static_cast<cudaStream_t>(stream)>>>(planes, S, C, X,
                                                                                                   G, gk);
  return to_status(cudaGetLastError());
}

nrx_status nrx_train_relu_mask(int64_t n, float* G, const float* Y, void* stream) {
  if (n < 1 || !G || !Y) return NRX_EINVAL;
  k_relu_mask<<<blocks_for((size_t)n), kThreads, 0, static_cast<cudaStream_t>(stream)>>>((size_t)n, G, Y);
  return to_status(cudaGetLastError());
}

nrx_status nrx_train_aggregate(int32_t n_slots, int32_t num_users, int64_t per_user, const float* m, float* a,
                               void* stream) {
  if (n_slots < 1 || num_users < 1 || num_users > NRX_MAX_USERS || per_user < 1 || !m || !a || m == a)
    return NRX_EINVAL;
  const size_t n = (size_t)n_slots * per_user;
  k_aggregate<<<blocks_for(n), kThreads, 0, static_cast<cudaStream_t>(stream)>>>(n_slots, num_users, (size_t)per_user,
                                                                                m, a);
  return to_status(cudaGetLastError());
}

nrx_status nrx_train_axpy(int64_t n, float alpha, const float* x, float* y, void* stream) {
  if (n < 1 || !x || !y) return NRX_EINVAL;
  k_axpy<<<blocks_for((size_t)n), kThreads, 0, static_cast<cudaStream_t>(stream)>>>((size_t)n, alpha, x, y);
  return to_status(cudaGetLastError());
}

nrx_status nrx_train_bce(int32_t n_slots, const nrx_slot_cfg* cfg, int32_t m_max, const float* llr,
                         const uint8_t* bits, const int32_t* bits_per_symbol_dev, float weight, float* grad,
                         double* loss, void* stream) {
  if (n_slots < 1 || !cfg || m_max < 2 || m_max > 8 || !llr || !bits || !bits_per_symbol_dev || !grad || !loss)
    return NRX_EINVAL;
  Geometry g;
  memset(&g, 0, sizeof(g));
  g.n_slots = n_slots;
  g.S = 12 * cfg->num_prb;
  g.U = cfg->num_users;
  g.m_max = m_max;
  g.n_dmrs = cfg->num_dmrs_symbols;
  g.td0 = cfg->dmrs_symbols[0];
  g.td1 = g.n_dmrs == 2 ? cfg->dmrs_symbols[1] : g.td0;
  g.n_data = (NRX_SYMBOLS - g.n_dmrs) * g.S;
  for (int t = 0, di = 0; t < NRX_SYMBOLS; ++t)
    if (t != g.td0 && t != g.td1) g.data_t[di++] = (int8_t)t;
  const size_t n = (size_t)n_slots * g.U * NRX_SYMBOLS * g.S * m_max;
  k_bce<<<blocks_for(n), kThreads, 0, static_cast<cudaStream_t>(stream)>>>(g, llr, bits, bits_per_symbol_dev, weight,
                                                                          grad, loss);
  return to_status(cudaGetLastError());
}

nrx_status nrx_train_mse(int64_t n, const float* h_hat, const float* h, float scale, float* grad, double* loss,
                         void* stream) {
  if (n < 1 || !h_hat || !h || !grad || !loss) return NRX_EINVAL;
  k_mse<<<blocks_for((size_t)n), kThreads, 0, static_cast<cudaStream_t>(stream)>>>((size_t)n, h_hat, h, scale, grad,
                                                                                  loss);
  return to_status(cudaGetLastError());
}

nrx_status nrx_train_plane_mask(int64_t planes, int64_t rows_per_plane, int32_t width, int64_t ld_src, int64_t ld_dst,
                                const int32_t* bits_per_symbol_dev, int32_t m_head, const float* src, float* dst,
                                int32_t accumulate, void* stream) {
  if (planes < 1 || rows_per_plane < 1 || width < 1 || ld_src < width || ld_dst < width || !bits_per_symbol_dev ||
      !src || !dst)
    return NRX_EINVAL;
  const size_t n = (size_t)planes * rows_per_plane * width;
  k_plane_mask<<<blocks_for(n), kThreads, 0, static_cast<cudaStream_t>(stream)>>>(
      planes, rows_per_plane, width, ld_src, ld_dst, bits_per_symbol_dev, m_head, src, dst, accumulate ? 1 : 0);
  return to_status(cudaGetLastError());
}

nrx_status nrx_train_zero(int64_t bytes, void* ptr, void* stream) {
  if (bytes < 0 || (bytes > 0 && !ptr)) return NRX_EINVAL;
  if (bytes == 0) return NRX_OK;
  return to_status(cudaMemsetAsync(ptr, 0, (size_t)bytes, static_cast<cudaStream_t>(stream)));
}

nrx_status nrx_train_copy(int64_t bytes, void* dst, const void* src, void* stream) {
  if (bytes < 0 || (bytes > 0 && (!dst || !src))) return NRX_EINVAL;
  if (bytes == 0) return NRX_OK;
  return to_status(cudaMemcpyAsync(dst, src, (size_t)bytes, cudaMemcpyDefault, static_cast<cudaStream_t>(stream)));
}

nrx_status nrx_train_adam(int64_t n, float* w, const float* g, float* m1, float* m2, const float* lr_t,
                          float beta1, float beta2, float eps, void* stream) {
  if (n < 1 || !w || !g || !m1 || !m2 || !lr_t) return NRX_EINVAL;
  k_adam<<<blocks_for((size_t)n), kThreads, 0, static_cast<cudaStream_t>(stream)>>>((size_t)n, w, g, m1, m2, lr_t,
                                                                                   beta1, beta2, eps);
  return to_status(cudaGetLastError());
}

}  // extern "C"

NRX_DEBUG_READER(debug_read_train)
