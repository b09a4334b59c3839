// C ABI of the NRX library (declared in include/nrx.h): context life cycle,
// weight-blob parsing, argument validation and the kernel launch sequence.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/nrx.h"
#include "common.cuh"
#include "kernels.h"
#include "net_tc.h"
#include "tc.cuh"

namespace {

constexpr int32_t kMagic = 0x5758524E;
constexpr int32_t kVersion = 1;
constexpr int32_t kVersionVarIO = 2;  // modulation-specific StateInit / ReadoutLLRs heads (Sec. III)

}  // namespace

struct nrx_ctx {
  int B = 0, C = 0, R = 0, N_it = 0, m_max = 0;
  int max_users = 0, max_prb = 0, max_slots = 0;
  nrx_precision prec = NRX_FP32;
  int device = 0;
  // device weights (one allocation per precision)
  float* w_f32 = nullptr;
  void* w_tc = nullptr;
  InitWeights init{};        // StateInit per Var-IO head (entry 0 for a single-head net)
  std::vector<IterWeightsF32> it32;
  std::vector<IterWeightsTC> it16;
  ReadoutWeightsF32 ro32{};  // ReadoutLLRs per Var-IO head
  ReadoutWeightsTC ro_tc{};
  int n_heads = 1;
  int8_t head_of_bits[9] = {};  // modulation order -> head
  int* d_err = nullptr;  // device word set by a bounded wait that gave up (tensor-core path)
  unsigned long long* d_f64 = nullptr;  // LMMSE: REs solved in FP64 since the last reset
  // workspaces [max_slots][max_users][14][S_max][C]
  void* state = nullptr;
  void* z_a = nullptr;
  void* z_b = nullptr;
  size_t act_elems = 0;
  // staging for the host-buffer entry point
  float2* y_stage = nullptr;
  float* llr_stage = nullptr;
  float2* dmrs_stage = nullptr;
  size_t y_stage_bytes = 0, llr_stage_bytes = 0, dmrs_stage_bytes = 0;
  // pipelined host-buffer calls: a second staging set, upload / compute /
  // download streams and per-set events (created on the first such call)
  float2* y_stage2 = nullptr;
  float* llr_stage2 = nullptr;
  float2* dmrs_stage2 = nullptr;
  cudaStream_t h2d_st = nullptr, cmp_st = nullptr, d2h_st = nullptr;
  cudaEvent_t ev_in[2] = {}, ev_cmp[2] = {}, ev_out[2] = {};
  int64_t host_calls = 0;
  bool host_inflight = false;
  bool pipeline_ready = false;  // all of the above created
  // per-kernel event timing
  bool profiling = false;
  std::vector<cudaEvent_t> ev_free;
  struct Rec {
    int kind;
    cudaEvent_t a, b;
  };
  std::vector<Rec> ev_pending;
  double prof_ms[NRX_KERNEL_KINDS] = {};
  int64_t prof_n[NRX_KERNEL_KINDS] = {};
  // last call
  Geometry last_geo{};
  bool have_state = false;
  int32_t last_launches = 0;
  std::string err;
};

namespace {

nrx_status fail(nrx_ctx* ctx, nrx_status st, const char* fmt, ...) {
  if (ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    ctx->err = buf;
  }
  return st;
}

nrx_status cuda_fail(nrx_ctx* ctx, cudaError_t e, const char* what) {
  return fail(ctx, NRX_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

size_t align4(size_t n) { return (n + 3) & ~size_t(3); }

const char* const kKindNames[NRX_KERNEL_KINDS] = {"state_init", "message_passing", "residual_block", "readout",
                                                  "lmmse"};
enum { K_INIT = 0, K_MP = 1, K_BLOCK = 2, K_READOUT = 3, K_LMMSE = 4 };

cudaEvent_t take_event(nrx_ctx* ctx) {
  if (!ctx->ev_free.empty()) {
    cudaEvent_t e = ctx->ev_free.back();
    ctx->ev_free.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Brackets one kernel launch with events when profiling is on.
struct KernelTimer {
  nrx_ctx* ctx;
  int kind;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  KernelTimer(nrx_ctx* c, int k, cudaStream_t s) : ctx(c), kind(k), st(s) {
    if (ctx->profiling) {
      a = take_event(ctx);
      cudaEventRecord(a, st);
    }
  }
  ~KernelTimer() {
    if (a) {
      cudaEvent_t b = take_event(ctx);
      cudaEventRecord(b, st);
      ctx->ev_pending.push_back({kind, a, b});
    }
  }
};

// Validate the per-slot configurations of one call; fill geometry and table.
nrx_status prepare(nrx_ctx* ctx, int32_t n_slots, const nrx_slot_cfg* cfgs, const int32_t* bits, bool need_dmrs,
                   bool lmmse, Geometry* g, SlotTable* tab, int* iterations, size_t* llr_total) {
  if (!ctx) return NRX_EINVAL;
  if (!cfgs || !bits) return fail(ctx, NRX_EINVAL, "null cfgs or bits_per_symbol");
  if (n_slots < 1 || n_slots > ctx->max_slots)
    return fail(ctx, NRX_EINVAL, "n_slots %d outside [1, %d]", n_slots, ctx->max_slots);
  const nrx_slot_cfg& c0 = cfgs[0];
  if (c0.num_prb < 1 || c0.num_prb > ctx->max_prb)
    return fail(ctx, NRX_EINVAL, "num_prb %d outside [1, %d]", c0.num_prb, ctx->max_prb);
  if (c0.num_users < 1 || c0.num_users > ctx->max_users)
    return fail(ctx, NRX_EINVAL, "num_users %d outside [1, %d]", c0.num_users, ctx->max_users);
  if (c0.num_dmrs_symbols != 1 && c0.num_dmrs_symbols != 2)
    return fail(ctx, NRX_EINVAL, "num_dmrs_symbols must be 1 or 2");
  for (int d = 0; d < c0.num_dmrs_symbols; ++d)
    if (c0.dmrs_symbols[d] < 0 || c0.dmrs_symbols[d] >= NRX_SYMBOLS)
      return fail(ctx, NRX_EINVAL, "dmrs symbol %d out of range", c0.dmrs_symbols[d]);
  if (c0.num_dmrs_symbols == 2 && c0.dmrs_symbols[1] <= c0.dmrs_symbols[0])
    return fail(ctx, NRX_EINVAL, "dmrs symbols must be ascending");
  const int its = c0.iterations == 0 ? ctx->N_it : c0.iterations;
  if (!lmmse && (its < 1 || its > ctx->N_it))
    return fail(ctx, NRX_EINVAL, "iterations %d outside [1, %d]", c0.iterations, ctx->N_it);
  memset(g, 0, sizeof(*g));
  memset(tab, 0, sizeof(*tab));
  g->n_slots = n_slots;
  g->S = 12 * c0.num_prb;
  g->U = c0.num_users;
  g->B = ctx->B;
  g->C = ctx->C;
  g->F = 4 * ctx->B + 2;
  g->m_max = ctx->m_max;
  g->n_dmrs = c0.num_dmrs_symbols;
  g->td0 = c0.dmrs_symbols[0];
  g->td1 = c0.num_dmrs_symbols == 2 ? c0.dmrs_symbols[1] : c0.dmrs_symbols[0];
  g->n_data = (NRX_SYMBOLS - g->n_dmrs) * g->S;
  int di = 0;
  for (int t = 0; t < NRX_SYMBOLS; ++t)
    if (t != g->td0 && t != g->td1) g->data_t[di++] = (int8_t)t;
  size_t off = 0;
  for (int i = 0; i < n_slots; ++i) {
    const nrx_slot_cfg& c = cfgs[i];
    if (c.num_prb != c0.num_prb || c.num_users != c0.num_users || c.num_dmrs_symbols != c0.num_dmrs_symbols ||
        c.dmrs_symbols[0] != c0.dmrs_symbols[0] ||
        (c0.num_dmrs_symbols == 2 && c.dmrs_symbols[1] != c0.dmrs_symbols[1]) || c.iterations != c0.iterations)
      return fail(ctx, NRX_EINVAL, "slot %d geometry differs from slot 0", i);
    if (need_dmrs && (!c.dmrs_seq || (reinterpret_cast<uintptr_t>(c.dmrs_seq) & 7)))
      return fail(ctx, NRX_EINVAL, "slot %d: dmrs_seq null or not 8-byte aligned", i);
    if (lmmse && !(c.noise_var > 0.f)) return fail(ctx, NRX_EINVAL, "slot %d: noise_var must be > 0", i);
    tab->dmrs[i] = static_cast<const float2*>(c.dmrs_seq);
    tab->noise_var[i] = c.noise_var;
    for (int u = 0; u < g->U; ++u) {
      const int m = bits[i * g->U + u];
      if (m != 2 && m != 4 && m != 6) return fail(ctx, NRX_EINVAL, "slot %d user %d: bits %d not in {2,4,6}", i, u, m);
      if (!lmmse && m > ctx->m_max)
        return fail(ctx, NRX_EINVAL, "slot %d user %d: bits %d > m_max %d", i, u, m, ctx->m_max);
      tab->bits[i][u] = (int8_t)m;
      tab->head[i][u] = ctx->head_of_bits[m];
      if (off > (size_t)INT32_MAX) return fail(ctx, NRX_EINVAL, "LLR output too large");
      tab->llr_off[i][u] = (int32_t)off;
      off += (size_t)g->n_data * m;
    }
  }
  *iterations = its;
  *llr_total = off;
  tab->llr_total = (long long)off;
  return NRX_OK;
}

template <typename P>
nrx_status run_tc(nrx_ctx* ctx, const Geometry& g, const SlotTable& tab, int its, const float2* y, float* llr,
                  cudaStream_t st, int* launches) {
  using T = typename P::T;
  cudaError_t e;
  T* S = static_cast<T*>(ctx->state);
  T* za = static_cast<T*>(ctx->z_a);
  T* zb = static_cast<T*>(ctx->z_b);
  {
    KernelTimer kt(ctx, K_INIT, st);
    e = launch_state_init<T>(g, tab, y, ctx->init, S, st);
  }
  if (e != cudaSuccess) return cuda_fail(ctx, e, "state_init");
  ++*launches;
  for (int k = 0; k < its; ++k) {
    const IterWeightsTC& w = ctx->it16[k];
    {
      KernelTimer kt(ctx, K_MP, st);
      e = launch_mp_tc<P>(g, w, S, za, st);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "message_passing");
    ++*launches;
    T* zin = za;
    T* zout = zb;
    for (int r = 0; r < ctx->R; ++r) {
      const bool last = r == ctx->R - 1;
      {
        KernelTimer kt(ctx, K_BLOCK, st);
        e = launch_block_tc<P>(g, w, r, zin, zout, S, last, st);
      }
      if (e != cudaSuccess) return cuda_fail(ctx, e, "residual_block");
      ++*launches;
      T* tmp = zin;
      zin = zout;
      zout = tmp;
    }
  }
  {
    KernelTimer kt(ctx, K_READOUT, st);
    e = launch_readout_tc<P>(g, tab, ctx->ro_tc, S, llr, st);
  }
  if (e != cudaSuccess) return cuda_fail(ctx, e, "readout");
  ++*launches;
  return NRX_OK;
}

nrx_status run_nrx(nrx_ctx* ctx, const Geometry& g, const SlotTable& tab, int its, const float2* y, float* llr,
                   cudaStream_t st) {
  cudaError_t e;
  int launches = 0;
  if (ctx->prec == NRX_FP32) {
    float* S = static_cast<float*>(ctx->state);
    float* za = static_cast<float*>(ctx->z_a);
    float* zb = static_cast<float*>(ctx->z_b);
    {
      KernelTimer kt(ctx, K_INIT, st);
      e = launch_state_init<float>(g, tab, y, ctx->init, S, st);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "state_init");
    ++launches;
    for (int k = 0; k < its; ++k) {
      const IterWeightsF32& w = ctx->it32[k];
      {
        KernelTimer kt(ctx, K_MP, st);
        e = launch_mp_f32(g, w, S, za, st);
      }
      if (e != cudaSuccess) return cuda_fail(ctx, e, "mp_f32");
      ++launches;
      float* zin = za;
      float* zout = zb;
      for (int r = 0; r < ctx->R; ++r) {
        const bool last = r == ctx->R - 1;
        {
          KernelTimer kt(ctx, K_BLOCK, st);
          e = launch_block_f32(g, w, r, zin, zout, S, last, st);
        }
        if (e != cudaSuccess) return cuda_fail(ctx, e, "block_f32");
        ++launches;
        float* tmp = zin;
        zin = zout;
        zout = tmp;
      }
    }
    {
      KernelTimer kt(ctx, K_READOUT, st);
      e = launch_readout_f32(g, tab, ctx->ro32, S, llr, st);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "readout_f32");
    ++launches;
  } else if (ctx->prec == NRX_BF16) {
    if (run_tc<PolBF16>(ctx, g, tab, its, y, llr, st, &launches) != NRX_OK) return NRX_ECUDA;
  } else if (ctx->prec == NRX_FP16) {
    if (run_tc<PolFP16>(ctx, g, tab, its, y, llr, st, &launches) != NRX_OK) return NRX_ECUDA;
  } else {
    if (run_tc<PolFP8>(ctx, g, tab, its, y, llr, st, &launches) != NRX_OK) return NRX_ECUDA;
  }
  ctx->last_geo = g;
  ctx->have_state = true;
  ctx->last_launches = launches;
  return NRX_OK;
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

}  // namespace

extern "C" {

const char* nrx_status_string(nrx_status s) {
  switch (s) {
    case NRX_OK: return "NRX_OK";
    case NRX_EINVAL: return "NRX_EINVAL";
    case NRX_ENOMEM: return "NRX_ENOMEM";
    case NRX_ECUDA: return "NRX_ECUDA";
    case NRX_ETIMEDOUT: return "NRX_ETIMEDOUT";
    case NRX_EUNSUPPORTED: return "NRX_EUNSUPPORTED";
  }
  return "NRX_UNKNOWN";
}

const char* nrx_last_error(const nrx_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int32_t nrx_last_launch_count(const nrx_ctx* ctx) { return ctx ? ctx->last_launches : 0; }

nrx_status nrx_host_drain(nrx_ctx* ctx) {
  if (!ctx) return NRX_EINVAL;
  if (!ctx->host_inflight) return NRX_OK;
  ctx->host_inflight = false;
  // the download stream ends every completed call; the others matter after a
  // call that failed part-way
  const cudaError_t a = cudaStreamSynchronize(ctx->h2d_st);
  const cudaError_t b = cudaStreamSynchronize(ctx->cmp_st);
  if (a != cudaSuccess) return cuda_fail(ctx, a, "upload stream");
  if (b != cudaSuccess) return cuda_fail(ctx, b, "compute stream");
  return nrx_check(ctx, ctx->d2h_st);
}

nrx_status nrx_check(nrx_ctx* ctx, void* stream) {
  if (!ctx) return NRX_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "stream");
  if (ctx->d_err) {
    int v = 0;
    e = cudaMemcpy(&v, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "read device status");
    if (v) {
      cudaMemset(ctx->d_err, 0, sizeof(int));
      return fail(ctx, NRX_ETIMEDOUT, "a kernel's bounded wait for its tensor-core work gave up");
    }
  }
  return NRX_OK;
}

}  // extern "C"

namespace {
// One bounded wait that cannot succeed: nothing arrives on the barrier.
__global__ void k_expire_wait(uint64_t limit_ns, int* err) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    tc::fence_mbar_init();
    if (!tc::mbar_wait(&bar, 0, limit_ns)) atomicExch(err, 1);
  }
}
}  // namespace

extern "C" {

nrx_status nrx_expire_wait(nrx_ctx* ctx, int32_t limit_us, void* stream) {
  if (!ctx || limit_us < 1 || limit_us > 1000000) return NRX_EINVAL;
  if (!ctx->d_err) return fail(ctx, NRX_EUNSUPPORTED, "no device status word in an FP32 context");
  k_expire_wait<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>((uint64_t)limit_us * 1000ull, ctx->d_err);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? NRX_OK : cuda_fail(ctx, e, "k_expire_wait");
}

nrx_status nrx_profile(nrx_ctx* ctx, int32_t enable) {
  if (!ctx) return NRX_EINVAL;
  ctx->profiling = enable != 0;
  return NRX_OK;
}

nrx_status nrx_profile_read(nrx_ctx* ctx, int32_t kind, const char** name, double* total_ms, int64_t* launches,
                            int32_t reset) {
  if (!ctx || kind < 0 || kind >= NRX_KERNEL_KINDS) return NRX_EINVAL;
  for (auto& r : ctx->ev_pending) {
    float ms = 0.f;
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.a, r.b);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "profile events");
    ctx->prof_ms[r.kind] += ms;
    ctx->prof_n[r.kind] += 1;
    ctx->ev_free.push_back(r.a);
    ctx->ev_free.push_back(r.b);
  }
  ctx->ev_pending.clear();
  if (name) *name = kKindNames[kind];
  if (total_ms) *total_ms = ctx->prof_ms[kind];
  if (launches) *launches = ctx->prof_n[kind];
  if (reset) {
    for (int k = 0; k < NRX_KERNEL_KINDS; ++k) {
      ctx->prof_ms[k] = 0;
      ctx->prof_n[k] = 0;
    }
  }
  return NRX_OK;
}

nrx_status nrx_get_net(const nrx_ctx* ctx, int32_t* B, int32_t* C, int32_t* R, int32_t* N_it, int32_t* m_max) {
  if (!ctx) return NRX_EINVAL;
  if (B) *B = ctx->B;
  if (C) *C = ctx->C;
  if (R) *R = ctx->R;
  if (N_it) *N_it = ctx->N_it;
  if (m_max) *m_max = ctx->m_max;
  return NRX_OK;
}

size_t nrx_llr_count(const nrx_slot_cfg* cfg, const int32_t* bits) {
  if (!cfg || !bits || cfg->num_prb < 1 || cfg->num_users < 1 || cfg->num_users > NRX_MAX_USERS ||
      (cfg->num_dmrs_symbols != 1 && cfg->num_dmrs_symbols != 2))
    return 0;
  size_t m = 0;
  for (int u = 0; u < cfg->num_users; ++u) {
    if (bits[u] != 2 && bits[u] != 4 && bits[u] != 6) return 0;
    m += (size_t)bits[u];
  }
  return (size_t)(NRX_SYMBOLS - cfg->num_dmrs_symbols) * 12 * (size_t)cfg->num_prb * m;
}

void nrx_destroy(nrx_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  for (int b = 0; b < 2; ++b) {
    if (ctx->ev_in[b]) cudaEventDestroy(ctx->ev_in[b]);
    if (ctx->ev_cmp[b]) cudaEventDestroy(ctx->ev_cmp[b]);
    if (ctx->ev_out[b]) cudaEventDestroy(ctx->ev_out[b]);
  }
  for (cudaStream_t s : {ctx->h2d_st, ctx->cmp_st, ctx->d2h_st})
    if (s) cudaStreamDestroy(s);
  cudaFree(ctx->y_stage2);
  cudaFree(ctx->llr_stage2);
  cudaFree(ctx->dmrs_stage2);
  cudaFree(ctx->w_f32);
  cudaFree(ctx->w_tc);
  cudaFree(ctx->state);
  cudaFree(ctx->z_a);
  cudaFree(ctx->z_b);
  cudaFree(ctx->y_stage);
  cudaFree(ctx->llr_stage);
  cudaFree(ctx->dmrs_stage);
  cudaFree(ctx->d_f64);
  for (auto& r : ctx->ev_pending) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : ctx->ev_free) cudaEventDestroy(e);
  delete ctx;
}

nrx_status nrx_create(const void* weights, size_t weights_bytes, int32_t num_rx_ant, int32_t max_users,
                      int32_t max_prb, int32_t max_slots, nrx_precision precision, nrx_ctx** out) {
  if (!out) return NRX_EINVAL;
  *out = nullptr;
  if (!weights || weights_bytes < 32) return NRX_EINVAL;
  if ((num_rx_ant != 1 && num_rx_ant != 2 && num_rx_ant != 4 && num_rx_ant != 8) || max_users < 1 || max_users > NRX_MAX_USERS || max_prb < 1 ||
      max_prb > 275 || max_slots < 1 || max_slots > NRX_MAX_LAUNCH_SLOTS)
    return NRX_EINVAL;
  if (precision != NRX_FP32 && precision != NRX_BF16 && precision != NRX_FP16 && precision != NRX_FP8)
    return NRX_EINVAL;
  int32_t hdr[8];
  memcpy(hdr, weights, sizeof(hdr));
  const int B = hdr[2], C = hdr[3], R = hdr[4], N_it = hdr[5], m_max = hdr[6];
  const int64_t n_floats = hdr[7];
  if (hdr[0] != kMagic || (hdr[1] != kVersion && hdr[1] != kVersionVarIO) || B != num_rx_ant ||
      (C != 32 && C != 64) || R < 1 || R > 4 || N_it < 1 || N_it > 16 || m_max < 2 || m_max > 8)
    return NRX_EINVAL;
  const int F = 4 * B + 2;
  // Heads: one shared head (version 1), or one per modulation order 2, 4, 6
  // up to m_max (Var-IO, version 2), each with m_h outputs.
  std::vector<int> head_m;
  if (hdr[1] == kVersion) {
    head_m.push_back(m_max);
  } else {
    for (int m = 2; m <= 6 && m <= m_max; m += 2) head_m.push_back(m);
  }
  int64_t expect = (int64_t)N_it * (2 * ((int64_t)C * C + C) + (int64_t)C * (2 * C + 2) + C +
                                    (int64_t)R * (2 * (9 * C + (int64_t)C * C + C)));
  for (int m : head_m) expect += (int64_t)C * F + C + 9 * C + (int64_t)C * C + C + (int64_t)m * C + m;
  if (n_floats != expect || weights_bytes != 32 + (size_t)n_floats * 4) return NRX_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return NRX_ECUDA;

  nrx_ctx* ctx = new nrx_ctx();
  cudaGetDevice(&ctx->device);
  ctx->B = B;
  ctx->C = C;
  ctx->R = R;
  ctx->N_it = N_it;
  ctx->m_max = m_max;
  ctx->max_users = max_users;
  ctx->n_heads = (int)head_m.size();
  for (int h = 0; h < (int)head_m.size(); ++h)
    for (int m = 0; m <= 8; ++m)
      if (hdr[1] == kVersion || m == head_m[h]) ctx->head_of_bits[m] = hdr[1] == kVersion ? 0 : (int8_t)h;
  ctx->max_prb = max_prb;
  ctx->max_slots = max_slots;
  ctx->prec = precision;

  // Host copy of the blob in blob order, then the device layout.
  const float* src = reinterpret_cast<const float*>(static_cast<const char*>(weights) + 32);
  std::vector<float> dev;
  auto put = [&](const float* p, size_t n) {
    const size_t at = dev.size();
    dev.insert(dev.end(), p, p + n);
    dev.resize(align4(dev.size()), 0.f);
    return at;
  };
  auto put_t = [&](const float* w, int n_out, int n_in) {  // [out][in] -> [in][out]
    std::vector<float> t((size_t)n_out * n_in);
    for (int o = 0; o < n_out; ++o)
      for (int i = 0; i < n_in; ++i) t[(size_t)i * n_out + o] = w[(size_t)o * n_in + i];
    return put(t.data(), t.size());
  };
  struct Off {
    size_t init_w[kMaxHeads], init_b[kMaxHeads], init_dw[kMaxHeads];
    size_t ro1_t[kMaxHeads], ro1_b[kMaxHeads], ro2[kMaxHeads], ro2_b[kMaxHeads];
    std::vector<size_t> f;
  } o{};
  const float* p = src;
  auto take = [&](size_t n) {
    const float* q = p;
    p += n;
    return q;
  };
  const int n_heads = (int)head_m.size();
  for (int h = 0; h < n_heads; ++h) {
    o.init_w[h] = put(take((size_t)C * F), (size_t)C * F);
    o.init_b[h] = put(take(C), C);
    o.init_dw[h] = put(take(9 * C), 9 * C);
  }
  std::vector<const float*> blob_it;  // per iteration raw pointers, for the BF16 packer
  for (int k = 0; k < N_it; ++k) {
    const float* mp1w = take((size_t)C * C);
    const float* mp1b = take(C);
    const float* mp2w = take((size_t)C * C);
    const float* mp2b = take(C);
    const float* inw = take((size_t)C * (2 * C + 2));
    const float* inb = take(C);
    blob_it.insert(blob_it.end(), {mp1w, mp1b, mp2w, mp2b, inw, inb});
    o.f.push_back(put_t(mp1w, C, C));
    o.f.push_back(put(mp1b, C));
    o.f.push_back(put_t(mp2w, C, C));
    o.f.push_back(put(mp2b, C));
    o.f.push_back(put_t(inw, C, 2 * C + 2));
    o.f.push_back(put(inb, C));
    for (int r = 0; r < R; ++r) {
      const float* dw1 = take(9 * C);
      const float* pw1w = take((size_t)C * C);
      const float* pw1b = take(C);
      const float* dw2 = take(9 * C);
      const float* pw2w = take((size_t)C * C);
      const float* pw2b = take(C);
      blob_it.insert(blob_it.end(), {dw1, pw1w, pw1b, dw2, pw2w, pw2b});
      o.f.push_back(put(dw1, 9 * C));
      o.f.push_back(put_t(pw1w, C, C));
      o.f.push_back(put(pw1b, C));
      o.f.push_back(put(dw2, 9 * C));
      o.f.push_back(put_t(pw2w, C, C));
      o.f.push_back(put(pw2b, C));
    }
  }
  std::vector<const float*> ro1w_heads;
  for (int h = 0; h < n_heads; ++h) {
    const int m = head_m[h];
    const float* ro1w = take((size_t)C * C);
    const float* ro1b = take(C);
    std::vector<float> ro2w((size_t)m_max * C, 0.f), ro2b(m_max, 0.f);  // rows beyond m stay zero
    memcpy(ro2w.data(), take((size_t)m * C), sizeof(float) * (size_t)m * C);
    memcpy(ro2b.data(), take(m), sizeof(float) * m);
    ro1w_heads.push_back(ro1w);
    o.ro1_t[h] = put_t(ro1w, C, C);
    o.ro1_b[h] = put(ro1b, C);
    o.ro2[h] = put(ro2w.data(), ro2w.size());
    o.ro2_b[h] = put(ro2b.data(), ro2b.size());
  }

  cudaError_t e = cudaMalloc(&ctx->w_f32, dev.size() * sizeof(float));
  if (e != cudaSuccess) {
    nrx_destroy(ctx);
    return NRX_ENOMEM;
  }
  e = cudaMemcpy(ctx->w_f32, dev.data(), dev.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    nrx_destroy(ctx);
    return NRX_ECUDA;
  }
  const float* W = ctx->w_f32;
  for (int h = 0; h < n_heads; ++h) {
    ctx->init.w_pw[h] = W + o.init_w[h];
    ctx->init.b_pw[h] = W + o.init_b[h];
    ctx->init.k_dw[h] = W + o.init_dw[h];
    ctx->ro32.ro1_t[h] = W + o.ro1_t[h];
    ctx->ro32.ro1_b[h] = W + o.ro1_b[h];
    ctx->ro32.ro2[h] = W + o.ro2[h];
    ctx->ro32.ro2_b[h] = W + o.ro2_b[h];
  }
  ctx->it32.resize(N_it);
  size_t fi = 0;
  for (int k = 0; k < N_it; ++k) {
    IterWeightsF32& w = ctx->it32[k];
    memset(&w, 0, sizeof(w));
    w.mp1_t = W + o.f[fi++];
    w.mp1_b = W + o.f[fi++];
    w.mp2_t = W + o.f[fi++];
    w.mp2_b = W + o.f[fi++];
    w.in_t = W + o.f[fi++];
    w.in_b = W + o.f[fi++];
    for (int r = 0; r < R; ++r) {
      w.dw1[r] = W + o.f[fi++];
      w.pw1_t[r] = W + o.f[fi++];
      w.pw1_b[r] = W + o.f[fi++];
      w.dw2[r] = W + o.f[fi++];
      w.pw2_t[r] = W + o.f[fi++];
      w.pw2_b[r] = W + o.f[fi++];
    }
  }
  if (precision != NRX_FP32) {
    const int mode = precision == NRX_BF16 ? 1 : precision == NRX_FP8 ? 2 : 0;
    nrx_status st = upload_tc_weights(mode, C, R, N_it, blob_it, ro1w_heads, ctx->it32, ctx->ro32, &ctx->it16,
                                      &ctx->w_tc, &ctx->ro_tc, &ctx->d_err);
    if (st != NRX_OK) {
      nrx_destroy(ctx);
      return st;
    }
  }

  const size_t S_max = 12 * (size_t)max_prb;
  ctx->act_elems = (size_t)max_slots * max_users * NRX_SYMBOLS * S_max * C;
  const size_t act_bytes = ctx->act_elems * (precision == NRX_FP32 ? 4 : 2);
  const size_t y_bytes = (size_t)max_slots * B * NRX_SYMBOLS * S_max * sizeof(float2);
  const size_t llr_bytes = (size_t)max_slots * max_users * NRX_SYMBOLS * S_max * 6 * sizeof(float);
  const size_t dmrs_bytes = (size_t)max_slots * 2 * (S_max / 2) * sizeof(float2);
  if (cudaMalloc(&ctx->state, act_bytes) != cudaSuccess || cudaMalloc(&ctx->z_a, act_bytes) != cudaSuccess ||
      cudaMalloc(&ctx->z_b, act_bytes) != cudaSuccess || cudaMalloc(&ctx->y_stage, y_bytes) != cudaSuccess ||
      cudaMalloc(&ctx->llr_stage, llr_bytes) != cudaSuccess ||
      cudaMalloc(&ctx->dmrs_stage, dmrs_bytes) != cudaSuccess ||
      cudaMalloc(&ctx->d_f64, sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    nrx_destroy(ctx);
    return NRX_ENOMEM;
  }
  if (cudaMemset(ctx->d_f64, 0, sizeof(unsigned long long)) != cudaSuccess) {
    nrx_destroy(ctx);
    return NRX_ECUDA;
  }
  ctx->y_stage_bytes = y_bytes;
  ctx->llr_stage_bytes = llr_bytes;
  ctx->dmrs_stage_bytes = dmrs_bytes;
  *out = ctx;
  return NRX_OK;
}

nrx_status nrx_detect_batch(nrx_ctx* ctx, int32_t n_slots, const void* y, const nrx_slot_cfg* cfgs,
                            const int32_t* bits, float* llr, void* stream) {
  if (!ctx) return NRX_EINVAL;
  if (ctx->host_inflight) {  // pipelined host calls share the scratch: finish them first
    const nrx_status d = nrx_host_drain(ctx);
    if (d != NRX_OK) return d;
  }
  ctx->last_launches = 0;
  if (!y || !llr || !aligned(y, 16) || !aligned(llr, 4))
    return fail(ctx, NRX_EINVAL, "y must be 16-byte aligned and llr 4-byte aligned (non-null)");
  Geometry g;
  SlotTable tab;
  int its = 0;
  size_t total = 0;
  nrx_status st = prepare(ctx, n_slots, cfgs, bits, true, false, &g, &tab, &its, &total);
  if (st != NRX_OK) return st;
  return run_nrx(ctx, g, tab, its, static_cast<const float2*>(y), llr, static_cast<cudaStream_t>(stream));
}

nrx_status nrx_detect(nrx_ctx* ctx, const void* y, const nrx_slot_cfg* cfg, const int32_t* bits, float* llr,
                      void* stream) {
  return nrx_detect_batch(ctx, 1, y, cfg, bits, llr, stream);
}

nrx_status lmmse_detect_batch(nrx_ctx* ctx, int32_t n_slots, const void* y, const nrx_slot_cfg* cfgs,
                              const int32_t* bits, float* llr, void* stream) {
  if (ctx && ctx->host_inflight) {
    const nrx_status d = nrx_host_drain(ctx);
    if (d != NRX_OK) return d;
  }
  if (!ctx) return NRX_EINVAL;
  ctx->last_launches = 0;
  if (!y || !llr || !aligned(y, 16) || !aligned(llr, 4))
    return fail(ctx, NRX_EINVAL, "y must be 16-byte aligned and llr 4-byte aligned (non-null)");
  Geometry g;
  SlotTable tab;
  int its = 0;
  size_t total = 0;
  nrx_status st = prepare(ctx, n_slots, cfgs, bits, true, true, &g, &tab, &its, &total);
  if (st != NRX_OK) return st;
  cudaError_t e;
  {
    KernelTimer kt(ctx, K_LMMSE, static_cast<cudaStream_t>(stream));
    e = launch_lmmse(g, tab, static_cast<const float2*>(y), llr, ctx->d_f64, static_cast<cudaStream_t>(stream));
  }
  if (e != cudaSuccess) return cuda_fail(ctx, e, "lmmse");
  ctx->last_launches = 1;
  return NRX_OK;
}

nrx_status lmmse_detect(nrx_ctx* ctx, const void* y, const nrx_slot_cfg* cfg, const int32_t* bits, float* llr,
                        void* stream) {
  return lmmse_detect_batch(ctx, 1, y, cfg, bits, llr, stream);
}

nrx_status nrx_debug_counters(int64_t* violations, int32_t* first_site, int64_t* first_index,
                              int64_t* first_extent, int32_t reset) {
#ifndef NRX_DEBUG
  (void)violations;
  (void)first_site;
  (void)first_index;
  (void)first_extent;
  (void)reset;
  return NRX_EUNSUPPORTED;
#else
  if (!violations) return NRX_EINVAL;
  cudaError_t (*const readers[])(unsigned long long*, bool) = {debug_read_frontend, debug_read_net_f32,
                                                               debug_read_net_tc,   debug_read_block_tc,
                                                               debug_read_mp_tc,    debug_read_ldpc,
                                                               debug_read_train};
  int64_t total = 0;
  bool have_first = false;
  for (auto rd : readers) {
    unsigned long long rec[4];
    if (rd(rec, reset != 0) != cudaSuccess) return NRX_ECUDA;
    total += (int64_t)rec[0];
    if (rec[0] && !have_first) {
      have_first = true;
      if (first_site) *first_site = (int32_t)rec[1];
      if (first_index) *first_index = (int64_t)rec[2];
      if (first_extent) *first_extent = (int64_t)rec[3];
    }
  }
  if (!have_first) {
    if (first_site) *first_site = 0;
    if (first_index) *first_index = 0;
    if (first_extent) *first_extent = 0;
  }
  *violations = total;
  return NRX_OK;
#endif
}

nrx_status lmmse_fp64_count(nrx_ctx* ctx, int64_t* count, int32_t reset, void* stream) {
  if (!ctx || !count) return NRX_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "stream");
  unsigned long long v = 0;
  e = cudaMemcpy(&v, ctx->d_f64, sizeof(v), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "read FP64 RE count");
  *count = (int64_t)v;
  if (reset) {
    e = cudaMemset(ctx->d_f64, 0, sizeof(v));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "reset FP64 RE count");
  }
  return NRX_OK;
}

nrx_status nrx_detect_batch_host(nrx_ctx* ctx, int32_t n_slots, const void* y_host, const nrx_slot_cfg* cfgs,
                                 const int32_t* bits, float* llr_host, void* stream) {
  if (!ctx) return NRX_EINVAL;
  if (ctx->host_inflight) {  // pipelined host calls share the scratch: finish them first
    const nrx_status d = nrx_host_drain(ctx);
    if (d != NRX_OK) return d;
  }
  ctx->last_launches = 0;
  if (!y_host || !llr_host) return fail(ctx, NRX_EINVAL, "null host buffer");
  Geometry g;
  SlotTable tab;
  int its = 0;
  size_t total = 0;
  nrx_status st = prepare(ctx, n_slots, cfgs, bits, true, false, &g, &tab, &its, &total);
  if (st != NRX_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t y_bytes = (size_t)n_slots * g.B * NRX_SYMBOLS * g.S * sizeof(float2);
  cudaError_t e = cudaMemcpyAsync(ctx->y_stage, y_host, y_bytes, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "copy y");
  const size_t per = (size_t)g.n_dmrs * (g.S / 2);
  for (int i = 0; i < n_slots; ++i) {
    e = cudaMemcpyAsync(ctx->dmrs_stage + i * per, cfgs[i].dmrs_seq, per * sizeof(float2), cudaMemcpyHostToDevice,
                        s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "copy dmrs");
    tab.dmrs[i] = ctx->dmrs_stage + i * per;
  }
  st = run_nrx(ctx, g, tab, its, ctx->y_stage, ctx->llr_stage, s);
  if (st != NRX_OK) return st;
  e = cudaMemcpyAsync(llr_host, ctx->llr_stage, total * sizeof(float), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "copy llr");
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "synchronize");
  return NRX_OK;
}

nrx_status nrx_detect_batch_host_async(nrx_ctx* ctx, int32_t n_slots, const void* y_host, const nrx_slot_cfg* cfgs,
                                       const int32_t* bits, float* llr_host) {
  if (!ctx) return NRX_EINVAL;
  ctx->last_launches = 0;
  if (!y_host || !llr_host) return fail(ctx, NRX_EINVAL, "null host buffer");
  Geometry g;
  SlotTable tab;
  int its = 0;
  size_t total = 0;
  nrx_status st = prepare(ctx, n_slots, cfgs, bits, true, false, &g, &tab, &its, &total);
  if (st != NRX_OK) return st;
  cudaError_t e = cudaSuccess;
  if (!ctx->pipeline_ready) {  // first pipelined call: streams, events, second staging set (all or nothing)
    for (cudaStream_t* s : {&ctx->h2d_st, &ctx->cmp_st, &ctx->d2h_st})
      if (e == cudaSuccess && !*s) e = cudaStreamCreateWithFlags(s, cudaStreamNonBlocking);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b)
      for (cudaEvent_t* ev : {&ctx->ev_in[b], &ctx->ev_cmp[b], &ctx->ev_out[b]})
        if (e == cudaSuccess && !*ev) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (e == cudaSuccess && !ctx->y_stage2) e = cudaMalloc(&ctx->y_stage2, ctx->y_stage_bytes);
    if (e == cudaSuccess && !ctx->llr_stage2) e = cudaMalloc(&ctx->llr_stage2, ctx->llr_stage_bytes);
    if (e == cudaSuccess && !ctx->dmrs_stage2) e = cudaMalloc(&ctx->dmrs_stage2, ctx->dmrs_stage_bytes);
    if (e != cudaSuccess) {  // what was created is kept (nrx_destroy releases it); the next call retries the rest
      cudaGetLastError();
      return e == cudaErrorMemoryAllocation ? fail(ctx, NRX_ENOMEM, "pipeline staging")
                                            : cuda_fail(ctx, e, "pipeline set-up");
    }
    ctx->pipeline_ready = true;
  }
  // call k uses staging set k % 2; the set is free once call k - 2 has downloaded
  const int b = (int)(ctx->host_calls & 1);
  float2* ys = b ? ctx->y_stage2 : ctx->y_stage;
  float2* ds = b ? ctx->dmrs_stage2 : ctx->dmrs_stage;
  float* ls = b ? ctx->llr_stage2 : ctx->llr_stage;
  if (ctx->host_calls >= 2) e = cudaStreamWaitEvent(ctx->h2d_st, ctx->ev_out[b], 0);
  const size_t y_bytes = (size_t)n_slots * g.B * NRX_SYMBOLS * g.S * sizeof(float2);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ys, y_host, y_bytes, cudaMemcpyHostToDevice, ctx->h2d_st);
  const size_t per = (size_t)g.n_dmrs * (g.S / 2);
  for (int i = 0; i < n_slots && e == cudaSuccess; ++i) {
    e = cudaMemcpyAsync(ds + i * per, cfgs[i].dmrs_seq, per * sizeof(float2), cudaMemcpyHostToDevice, ctx->h2d_st);
    tab.dmrs[i] = ds + i * per;
  }
  if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_in[b], ctx->h2d_st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->cmp_st, ctx->ev_in[b], 0);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "pipelined upload");
  ctx->host_inflight = true;
  st = run_nrx(ctx, g, tab, its, ys, ls, ctx->cmp_st);
  if (st != NRX_OK) return st;
  e = cudaEventRecord(ctx->ev_cmp[b], ctx->cmp_st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->d2h_st, ctx->ev_cmp[b], 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(llr_host, ls, total * sizeof(float), cudaMemcpyDeviceToHost, ctx->d2h_st);
  if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_out[b], ctx->d2h_st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "pipelined download");
  ctx->host_calls++;
  return NRX_OK;
}

nrx_status nrx_copy_state(nrx_ctx* ctx, int32_t slot, float* out, void* stream) {
  if (ctx && ctx->host_inflight) {
    const nrx_status d = nrx_host_drain(ctx);
    if (d != NRX_OK) return d;
  }
  if (!ctx) return NRX_EINVAL;
  if (!ctx->have_state) return fail(ctx, NRX_EINVAL, "no nrx_detect call yet");
  const Geometry& g = ctx->last_geo;
  if (slot < 0 || slot >= g.n_slots || !out) return fail(ctx, NRX_EINVAL, "slot out of range or null output");
  const size_t n = (size_t)g.U * NRX_SYMBOLS * g.S * g.C;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (ctx->prec == NRX_FP32) {
    e = cudaMemcpyAsync(out, static_cast<float*>(ctx->state) + slot * n, n * sizeof(float), cudaMemcpyDeviceToDevice,
                        s);
  } else {
    if (ctx->prec == NRX_BF16)
      e = launch_to_f32<__nv_bfloat16>(static_cast<const __nv_bfloat16*>(ctx->state) + slot * n, out, n, s);
    else
      e = launch_to_f32<__half>(static_cast<const __half*>(ctx->state) + slot * n, out, n, s);
  }
  if (e != cudaSuccess) return cuda_fail(ctx, e, "copy state");
  return NRX_OK;
}

}  // extern "C"
