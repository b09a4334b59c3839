// Front end of both receivers: DMRS LS estimation, linear interpolation and
// positional encoding, fused into (a) the NRX StateInit kernel and (b) the
// per-RE LMMSE + max-log kernel (the "LS + LMMSE" baseline of Fig. 3).
#include "common.cuh"
#include "kernels.h"
#include "tc.cuh"

// ---------------------------------------------------------------------------
// StateInit (Sec. II-A): S0 = ReLU(DW(PW(x_u))), x_u = [y, h_u, PE].
// Persistent CTAs (as many per SM as registers and shared memory allow:
// three with the register bound of 80) loop over tiles of TW subcarriers of
// one (slot, user), all 14 symbols.  The PW output is formed on the tile plus
// a one-subcarrier halo (zero outside the grid, i.e. the depthwise input's
// zero padding), then the 3x3 depthwise and ReLU produce the tile.  FP32
// CUDA-core arithmetic (each thread computes the input layer of one RE, four
// channels at a time; the depthwise slides over the symbols for one channel
// pair); output FP32, BF16 or FP16.
// ---------------------------------------------------------------------------
template <typename OutT>
__device__ __forceinline__ void store_pair(OutT* p, float a, float b);
template <>
__device__ __forceinline__ void store_pair<float>(float* p, float a, float b) {
  *reinterpret_cast<float2*>(p) = make_float2(a, b);
}
template <>
__device__ __forceinline__ void store_pair<__nv_bfloat16>(__nv_bfloat16* p, float a, float b) {
  *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(a, b);
}
template <>
__device__ __forceinline__ void store_pair<__half>(__half* p, float a, float b) {
  *reinterpret_cast<__half2*>(p) = __floats2half2_rn(a, b);
}

template <int C, int B, typename OutT>
__global__ void __launch_bounds__(256, 3) k_state_init(Geometry g, SlotTable tab, const float2* __restrict__ y,
                                                    InitWeights wts, OutT* __restrict__ s_out) {
  constexpr int F = 4 * B + 2;
  constexpr int TW = kStateInitTile;
  constexpr int EW = TW + 2;
  constexpr int NRE = NRX_SYMBOLS * EW;  // REs of the extended tile, index t * EW + e (<= 256)
  constexpr int NQ = C / 4;               // channel quads
  constexpr int CP = C / 2, NG = 256 / CP;  // DW: channel pairs x column groups
  static_assert(NRE <= 256, "one RE per thread");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* hf = reinterpret_cast<float2*>(smem_raw);  // [2][B][EW]
  float* wt = reinterpret_cast<float*>(hf + 2 * B * EW);  // [F][C]
  float* kd = wt + F * C;                                // [C][9]
  float* bias = kd + 9 * C;                              // [C]
  // [NRE][C]: float4 chunk q of row r = t * EW + e stored at q ^ (e & (NQ - 1)), so a
  // depthwise column's addresses step by a constant over the symbols
  float* h = bias + C;

  const int tid = threadIdx.x;
  int loaded = -1;  // head whose weights are in shared memory
  const int S = g.S;
  const int tps = (S + TW - 1) / TW;
  const int n_tiles = g.n_slots * g.U * tps;
  tc::pdl_launch_dependents();
  tc::pdl_wait();  // the previous kernel may still read the state this kernel writes
  for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int su = tile / tps, u = su % g.U, sl = su / g.U;
    const int s0 = (tile % tps) * TW - 1;
    const float2* ys = y + (size_t)sl * B * NRX_SYMBOLS * S;
    __syncthreads();  // previous tile's readers of hf, h and the weights are done
    const int head = tab.head[sl][u];
    if (head != loaded) {  // uniform over the CTA
      const float* w_pw = pick_head(wts.w_pw, head);
      const float* k_dw = pick_head(wts.k_dw, head);
      const float* b_pw = pick_head(wts.b_pw, head);
      for (int i = tid; i < F * C; i += 256) {
        const int c = i % C, f = i / C;
        wt[f * C + c] = __ldg(w_pw + c * F + f);
      }
      for (int i = tid; i < 9 * C; i += 256) kd[i] = __ldg(k_dw + i);
      for (int i = tid; i < C; i += 256) bias[i] = __ldg(b_pw + i);
      loaded = head;
    }
    for (int i = tid; i < g.n_dmrs * B * EW; i += 256) {
      const int e = i % EW, b = (i / EW) % B, d = i / (EW * B);
      const int s = s0 + e;
      float2 v = make_float2(0.f, 0.f);
      if (s >= 0 && s < S) {
        const int td = d == 0 ? g.td0 : g.td1;
        v = ls_interp_freq(ys + ((size_t)b * NRX_SYMBOLS + td) * S, tab.dmrs[sl] + (size_t)d * (S / 2), u, g.U, S, s);
      }
      if (NRX_IN((d * B + b) * EW + e, 2 * B * EW, 101)) hf[(d * B + b) * EW + e] = v;
    }
    __syncthreads();
    // features of RE tid (registers) and the input layer, channel quad by quad
    if (tid < NRE) {
      const int t = tid / EW, e = tid % EW, s = s0 + e;
      float4* hrow = reinterpret_cast<float4*>(h + tid * C);
      if (s < 0 || s >= S) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) hrow[q] = make_float4(0.f, 0.f, 0.f, 0.f);
      } else {
        float x[F];
#pragma unroll
        for (int b = 0; b < B; ++b) {
          const size_t yi = ((size_t)b * NRX_SYMBOLS + t) * S + s;
          const float2 v = NRX_IN(yi, (size_t)B * NRX_SYMBOLS * S, 102) ? __ldg(ys + yi) : make_float2(0.f, 0.f);
          x[2 * b] = v.x;
          x[2 * b + 1] = v.y;
        }
#pragma unroll
        for (int b = 0; b < B; ++b) {
          const int i1 = ((g.n_dmrs - 1) * B + b) * EW + e;
          if (!NRX_IN(b * EW + e, 2 * B * EW, 103) || !NRX_IN(i1, 2 * B * EW, 103)) continue;
          const float2 hv = interp_time(g, t, hf[b * EW + e], hf[i1]);
          x[2 * B + 2 * b] = hv.x;
          x[2 * B + 2 * b + 1] = hv.y;
        }
        x[4 * B] = pe_time(g, t);
        x[4 * B + 1] = pe_freq(u, s);
#pragma unroll 4
        for (int q = 0; q < NQ; ++q) {
          const float4 b4 = *reinterpret_cast<const float4*>(bias + 4 * q);
          float2 a01 = make_float2(b4.x, b4.y), a23 = make_float2(b4.z, b4.w);
#pragma unroll
          for (int k = 0; k < F; ++k) {  // packed FP32 FMAs, two channels each
            const float4 w = *reinterpret_cast<const float4*>(wt + k * C + 4 * q);  // same for all lanes
            const float2 xk = make_float2(x[k], x[k]);
            a01 = tc::ffma2(make_float2(w.x, w.y), xk, a01);
            a23 = tc::ffma2(make_float2(w.z, w.w), xk, a23);
          }
          hrow[q ^ (e & (NQ - 1))] = make_float4(a01.x, a01.y, a23.x, a23.y);
        }
      }
    }
    __syncthreads();
    // DW + ReLU: thread = channel pair cp, output columns x = cg, cg + NG, ...
    {
      const int cp = tid % CP, cg = tid / CP;
      float2 kk[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) kk[i] = make_float2(kd[(2 * cp) * 9 + i], kd[(2 * cp + 1) * 9 + i]);
      OutT* out_base = s_out + (size_t)su * NRX_SYMBOLS * S * C;
      const int sx0 = (tile % tps) * TW;
      for (int xc = cg; xc < TW; xc += NG) {
        const int s = sx0 + xc;
        if (s >= S) continue;
        tc::dw_column(
            kk,
            [&](int ti, int k) {
              const int r = ti * EW + xc + k;
              const int hi = r * C + (((cp >> 1) ^ ((xc + k) & (NQ - 1))) << 2) + (cp & 1) * 2;
              return NRX_IN(hi + 1, NRE * C, 104) ? *reinterpret_cast<const float2*>(h + hi) : make_float2(0.f, 0.f);
            },
            [&](int t, float2 v) {
              const size_t oi = ((size_t)t * S + s) * C + 2 * cp;
              if (NRX_IN(oi + 1, (size_t)NRX_SYMBOLS * S * C, 105) &&
                  NRX_IN(su, (long long)g.n_slots * g.U, 106))
                store_pair<OutT>(out_base + oi, fmaxf(v.x, 0.f), fmaxf(v.y, 0.f));
            });
      }
    }
  }
}

size_t state_init_smem_bytes(int C, int B) {
  constexpr int EW = kStateInitTile + 2;
  const int F = 4 * B + 2;
  return sizeof(float2) * 2 * B * EW + sizeof(float) * ((size_t)F * C + 9 * C + C) +
         sizeof(float) * NRX_SYMBOLS * EW * C;
}

namespace {
int sm_count() {
  static const int n = [] {  // thread-safe one-time initialisation (serving calls from several threads)
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 148;
  }();
  return n;
}

template <int C, int B, typename OutT>
cudaError_t launch_si(const Geometry& g, const SlotTable& tab, const float2* y, const InitWeights& w, OutT* s_out,
                      cudaStream_t st) {
  const size_t smem = state_init_smem_bytes(C, B);
  ensure_smem<k_state_init<C, B, OutT>>((int)smem);
  // resident CTAs per SM (registers and shared memory), so that the grid is one wave
  static const int per_sm = [smem] {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_state_init<C, B, OutT>, 256, smem) != cudaSuccess ||
        n < 1)
      n = 1;
    return n;
  }();
  const int tiles = g.n_slots * g.U * ((g.S + kStateInitTile - 1) / kStateInitTile);
  const int grid = tiles < per_sm * sm_count() ? tiles : per_sm * sm_count();
  return launch_pdl(k_state_init<C, B, OutT>, grid, 256, smem, st, g, tab, y, w, s_out);
}

template <int C, typename OutT>
cudaError_t launch_si_b(const Geometry& g, const SlotTable& tab, const float2* y, const InitWeights& w, OutT* s_out,
                        cudaStream_t st) {
  switch (g.B) {
    case 1: return launch_si<C, 1, OutT>(g, tab, y, w, s_out, st);
    case 2: return launch_si<C, 2, OutT>(g, tab, y, w, s_out, st);
    case 4: return launch_si<C, 4, OutT>(g, tab, y, w, s_out, st);
    case 8: return launch_si<C, 8, OutT>(g, tab, y, w, s_out, st);
  }
  return cudaErrorInvalidValue;
}
}  // namespace

template <typename OutT>
cudaError_t launch_state_init(const Geometry& g, const SlotTable& tab, const float2* y, const InitWeights& w,
                              OutT* s_out, cudaStream_t st) {
  if (g.C == 64) return launch_si_b<64, OutT>(g, tab, y, w, s_out, st);
  if (g.C == 32) return launch_si_b<32, OutT>(g, tab, y, w, s_out, st);
  return cudaErrorInvalidValue;
}
template cudaError_t launch_state_init<float>(const Geometry&, const SlotTable&, const float2*, const InitWeights&,
                                              float*, cudaStream_t);
template cudaError_t launch_state_init<__nv_bfloat16>(const Geometry&, const SlotTable&, const float2*,
                                                      const InitWeights&, __nv_bfloat16*, cudaStream_t);
template cudaError_t launch_state_init<__half>(const Geometry&, const SlotTable&, const float2*, const InitWeights&,
                                               __half*, cudaStream_t);

// ---------------------------------------------------------------------------
// LS + LMMSE + max-log.  Per data RE: H = interpolated LS estimates [B x U],
// G = H^H H + N0 I, Cholesky G = L L^H, xhat = G^-1 H^H y,
// d_u = [G^-1 H^H H]_uu, xt_u = xhat_u / d_u, var_u = 1/d_u - 1, then max-log
// over the user's Gray QAM (per I/Q PAM dimension).  FP32, with the solve
// taken in FP64 for every RE of a slot whose SNR 10 log10(1/N0) exceeds
// 20 dB (N0 < kLmmseF64NoiseVar), and for any RE whose FP32 Cholesky pivots
// spread by more than 1e6 (or is not positive definite).  The REs solved in
// FP64 are counted in *f64_count.
// ---------------------------------------------------------------------------
constexpr float kLmmseF64NoiseVar = 0.01f;  // 10 log10(1/N0) > 20 dB
template <typename T>
struct Cx {
  T re, im;
};
template <typename T>
__device__ __forceinline__ Cx<T> cx_mul(Cx<T> a, Cx<T> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename T>
__device__ __forceinline__ Cx<T> cx_mulc(Cx<T> a, Cx<T> b) {  // conj(a) * b
  return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}

// Per-RE LMMSE solve for U users and B antennas (compile-time).  Returns false
// if a Cholesky pivot is not positive or the pivots spread by more than 1e6.
// Outputs xhat = G^-1 H^H y, d_u = Re [G^-1 H^H H]_uu and e_u = N0 [G^-1]_uu;
// since G^-1 H^H H = I - N0 G^-1, the post-equalisation variance 1/d_u - 1
// equals e_u / d_u, which callers use to avoid the cancellation of 1/d - 1
// near d = 1 (high SNR).
template <typename T, int U, int B>
__device__ __forceinline__ bool lmmse_solve(const Cx<T> (&H)[U][B], const Cx<T> (&yv)[B], T n0, Cx<T> (&xhat)[U],
                                            T (&d)[U], T (&e)[U]) {
  Cx<T> A[U][U], rhs[U];
#pragma unroll
  for (int i = 0; i < U; ++i) {
    rhs[i] = {0, 0};
#pragma unroll
    for (int j = 0; j < U; ++j) A[i][j] = {0, 0};
  }
#pragma unroll
  for (int b = 0; b < B; ++b) {
#pragma unroll
    for (int i = 0; i < U; ++i) {
      const Cx<T> c = cx_mulc(H[i][b], yv[b]);
      rhs[i].re += c.re;
      rhs[i].im += c.im;
#pragma unroll
      for (int j = 0; j <= i; ++j) {
        const Cx<T> a = cx_mulc(H[i][b], H[j][b]);
        A[i][j].re += a.re;
        A[i][j].im += a.im;
      }
    }
  }
#pragma unroll
  for (int i = 0; i < U; ++i)
#pragma unroll
    for (int j = i + 1; j < U; ++j) A[i][j] = {A[j][i].re, -A[j][i].im};
  // Cholesky of G = A + n0 I (lower, real diagonal)
  Cx<T> L[U][U];
  T piv_min = (T)1e30, piv_max = (T)0;
  bool ok = true;
#pragma unroll
  for (int i = 0; i < U; ++i) {
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      Cx<T> s = A[i][j];
      if (i == j) s.re += n0;
#pragma unroll
      for (int k = 0; k < j; ++k) {
        s.re -= L[i][k].re * L[j][k].re + L[i][k].im * L[j][k].im;  // L[i][k] conj(L[j][k])
        s.im -= L[i][k].im * L[j][k].re - L[i][k].re * L[j][k].im;
      }
      if (i == j) {
        if (!(s.re > (T)0)) ok = false;
        piv_min = s.re < piv_min ? s.re : piv_min;
        piv_max = s.re > piv_max ? s.re : piv_max;
        L[i][i] = {sqrt(s.re > (T)0 ? s.re : (T)1), (T)0};
      } else {
        const T inv = (T)1 / L[j][j].re;
        L[i][j] = {s.re * inv, s.im * inv};
      }
    }
  }
  if (!ok || piv_min < (T)1e-6 * piv_max) ok = false;
  // Li = L^-1 (lower triangular)
  Cx<T> Li[U][U];
#pragma unroll
  for (int j = 0; j < U; ++j) {
    Li[j][j] = {(T)1 / L[j][j].re, (T)0};
#pragma unroll
    for (int i = j + 1; i < U; ++i) {
      Cx<T> s = {0, 0};
#pragma unroll
      for (int k = j; k < i; ++k) {
        const Cx<T> p = cx_mul(L[i][k], Li[k][j]);
        s.re += p.re;
        s.im += p.im;
      }
      const T inv = -(T)1 / L[i][i].re;
      Li[i][j] = {s.re * inv, s.im * inv};
    }
  }
  // Ginv = Li^H Li ; xhat = Ginv rhs ; d_u = Re (Ginv A)_uu
#pragma unroll
  for (int a = 0; a < U; ++a) {
    Cx<T> xs = {0, 0};
    T dd = 0;
#pragma unroll
    for (int b = 0; b < U; ++b) {
      Cx<T> gi = {0, 0};
#pragma unroll
      for (int k = (a > b ? a : b); k < U; ++k) {
        const Cx<T> p = cx_mulc(Li[k][a], Li[k][b]);
        gi.re += p.re;
        gi.im += p.im;
      }
      const Cx<T> p = cx_mul(gi, rhs[b]);
      xs.re += p.re;
      xs.im += p.im;
      dd += gi.re * A[b][a].re - gi.im * A[b][a].im;
      if (b == a) e[a] = n0 * gi.re;
    }
    xhat[a] = xs;
    d[a] = dd;
  }
  return ok;
}

// FP64 redo of one RE (taken when the FP32 Cholesky is ill-conditioned).
template <int U, int B>
__device__ __noinline__ void lmmse_solve_f64(const Cx<float> (&H)[U][B], const Cx<float> (&yv)[B], float n0,
                                             float (&xr)[U], float (&xi)[U], float (&iv)[U]) {
  Cx<double> Hd[U][B], yd[B], xd[U];
  double dd[U], ed[U];
#pragma unroll
  for (int b = 0; b < B; ++b) {
    yd[b] = {(double)yv[b].re, (double)yv[b].im};
#pragma unroll
    for (int u = 0; u < U; ++u) Hd[u][b] = {(double)H[u][b].re, (double)H[u][b].im};
  }
  lmmse_solve<double, U, B>(Hd, yd, (double)n0, xd, dd, ed);
#pragma unroll
  for (int u = 0; u < U; ++u) {
    xr[u] = (float)(xd[u].re / dd[u]);
    xi[u] = (float)(xd[u].im / dd[u]);
    iv[u] = (float)(dd[u] / ed[u]);
  }
}

// Gray PAM level of label l with K bits (bit j of the label = (l >> (K-1-j)) & 1,
// j = 0 the sign bit): level = (1-2c0) * mag, mag built from the innermost bit out,
// mag <- 2^(K-j) - (1-2c_j) mag for j = K-1 .. 1, starting from 1.
template <int K>
__device__ __forceinline__ float pam_level(int l) {
  float mag = 1.f;
#pragma unroll
  for (int j = K - 1; j >= 1; --j) {
    const int c = (l >> (K - 1 - j)) & 1;
    mag = (float)(1 << (K - j)) - (1.f - 2.f * c) * mag;
  }
  const int c0 = (l >> (K - 1)) & 1;
  return (1.f - 2.f * c0) * mag;
}

// Max-log LLRs of the I component xr and Q component xi for 2K-bit Gray QAM;
// QAM bit 2j is I-PAM bit j, bit 2j+1 is Q-PAM bit j.  Stores 2K floats.
template <int K>
__device__ __forceinline__ void qam_maxlog_store(float xr, float xi, float inv_var, float* __restrict__ dst) {
  const float scale = rsqrtf(2.f * (float)((1 << (2 * K)) - 1) / 3.f);
  float o[2 * K];
#pragma unroll
  for (int dim = 0; dim < 2; ++dim) {
    const float x = dim == 0 ? xr : xi;
    float d0[K], d1[K];
#pragma unroll
    for (int j = 0; j < K; ++j) d0[j] = d1[j] = 1e30f;
#pragma unroll
    for (int l = 0; l < (1 << K); ++l) {
      const float e = x - pam_level<K>(l) * scale;
      const float dist = e * e;
#pragma unroll
      for (int j = 0; j < K; ++j) {
        if ((l >> (K - 1 - j)) & 1)
          d1[j] = fminf(d1[j], dist);
        else
          d0[j] = fminf(d0[j], dist);
      }
    }
#pragma unroll
    for (int j = 0; j < K; ++j) o[2 * j + dim] = (d0[j] - d1[j]) * inv_var;
  }
#pragma unroll
  for (int j = 0; j < 2 * K; ++j) dst[j] = o[j];
}

template <int TW, int U, int B>
__global__ void __launch_bounds__(256) k_lmmse(Geometry g, SlotTable tab, const float2* __restrict__ y,
                                               float* __restrict__ llr, unsigned long long* __restrict__ f64_count) {
  __shared__ float2 hf[U][2][B][TW];
  const int tile = blockIdx.x, sl = blockIdx.y;
  const int S = g.S;
  const float2* ys = y + (size_t)sl * B * NRX_SYMBOLS * S;
  for (int i = threadIdx.x; i < U * g.n_dmrs * B * TW; i += blockDim.x) {
    const int e = i % TW, b = (i / TW) % B, d = (i / (TW * B)) % g.n_dmrs, u = i / (TW * B * g.n_dmrs);
    const int s = tile * TW + e;
    float2 v = make_float2(0.f, 0.f);
    if (s < S) {
      const int td = d == 0 ? g.td0 : g.td1;
      v = ls_interp_freq(ys + ((size_t)b * NRX_SYMBOLS + td) * S, tab.dmrs[sl] + (size_t)d * (S / 2), u, U, S, s);
    }
    if (NRX_IN(((u * 2 + d) * B + b) * TW + e, U * 2 * B * TW, 107)) hf[u][d][b][e] = v;
  }
  __syncthreads();
  const float n0 = tab.noise_var[sl];
  const bool high_snr = n0 < kLmmseF64NoiseVar;  // uniform over the CTA: no divergence
  const int n_data_sym = NRX_SYMBOLS - g.n_dmrs;
  const int dl = g.n_dmrs - 1;
  unsigned n_f64 = 0;
  for (int i = threadIdx.x; i < n_data_sym * TW; i += blockDim.x) {
    const int e = i % TW, di = i / TW;
    const int s = tile * TW + e;
    if (s >= S) continue;
    const int t = g.data_t[di];
    Cx<float> H[U][B], yv[B];
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const size_t yi = ((size_t)b * NRX_SYMBOLS + t) * S + s;
      const float2 v = NRX_IN(yi, (size_t)B * NRX_SYMBOLS * S, 108) ? __ldg(ys + yi) : make_float2(0.f, 0.f);
      yv[b] = {v.x, v.y};
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const float2 hv = interp_time(g, t, hf[u][0][b][e], hf[u][dl][b][e]);
        H[u][b] = {hv.x, hv.y};
      }
    }
    Cx<float> xh[U];
    float dd[U], ee[U], xr[U], xi[U], iv[U];
    if (!high_snr && lmmse_solve<float, U, B>(H, yv, n0, xh, dd, ee)) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const float inv_d = 1.f / dd[u];
        xr[u] = xh[u].re * inv_d;
        xi[u] = xh[u].im * inv_d;
        iv[u] = dd[u] / ee[u];  // 1 / var, var = 1/d - 1 = e/d
      }
    } else {
      lmmse_solve_f64<U, B>(H, yv, n0, xr, xi, iv);
      ++n_f64;
    }
    const int r = di * S + s;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int m = tab.bits[sl][u];
      float* dst = llr + tab.llr_off[sl][u] + (size_t)r * m;
      if (!NRX_IN(tab.llr_off[sl][u] + (long long)r * m + m - 1, tab.llr_total, 109)) continue;
      if (m == 2)
        qam_maxlog_store<1>(xr[u], xi[u], iv[u], dst);
      else if (m == 4)
        qam_maxlog_store<2>(xr[u], xi[u], iv[u], dst);
      else
        qam_maxlog_store<3>(xr[u], xi[u], iv[u], dst);
    }
  }
  // every thread leaves the loop above, so the whole warp takes part
  n_f64 = __reduce_add_sync(0xffffffffu, n_f64);
  if (f64_count && (threadIdx.x & 31) == 0 && n_f64) atomicAdd(f64_count, (unsigned long long)n_f64);
}

template <int U, int B>
static cudaError_t launch_lmmse_ub(const Geometry& g, const SlotTable& tab, const float2* y, float* llr,
                                   unsigned long long* f64_count, cudaStream_t st) {
  constexpr int TW = 32;
  dim3 grid((g.S + TW - 1) / TW, g.n_slots);
  k_lmmse<TW, U, B><<<grid, 256, 0, st>>>(g, tab, y, llr, f64_count);
  return cudaGetLastError();
}

template <int B>
static cudaError_t launch_lmmse_b(const Geometry& g, const SlotTable& tab, const float2* y, float* llr,
                                  unsigned long long* f64_count, cudaStream_t st) {
  switch (g.U) {
    case 1: return launch_lmmse_ub<1, B>(g, tab, y, llr, f64_count, st);
    case 2: return launch_lmmse_ub<2, B>(g, tab, y, llr, f64_count, st);
    case 3: return launch_lmmse_ub<3, B>(g, tab, y, llr, f64_count, st);
    case 4: return launch_lmmse_ub<4, B>(g, tab, y, llr, f64_count, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_lmmse(const Geometry& g, const SlotTable& tab, const float2* y, float* llr,
                         unsigned long long* f64_count, cudaStream_t st) {
  switch (g.B) {
    case 1: return launch_lmmse_b<1>(g, tab, y, llr, f64_count, st);
    case 2: return launch_lmmse_b<2>(g, tab, y, llr, f64_count, st);
    case 4: return launch_lmmse_b<4>(g, tab, y, llr, f64_count, st);
    case 8: return launch_lmmse_b<8>(g, tab, y, llr, f64_count, st);
  }
  return cudaErrorInvalidValue;
}

NRX_DEBUG_READER(debug_read_frontend)
