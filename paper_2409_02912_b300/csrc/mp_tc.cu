// Message passing + CNN-update input layer of one CGNN iteration (Sec. II-A)
// on the tensor cores, 16-bit operands: S and the products with it in the
// activation type (BF16 with split hi + lo weights, or FP16); g and the G part
// of GEMM2 in FP16 in both modes (FP16 g and weights are more precise than
// BF16 ones, and one MMA pass).
// One M tile = 128 rows = nre REs x U users (row = u nre + j):
//   GEMM1: h = ReLU(S W1^T + b1)
//   g_u = sum over the other active users v of h_v (FP32, through shared memory)
//   GEMM2: z = S Win_S^T + g (Win_a W2)^T + b_in + (U-1) Win_a b2 + PE Win_pe^T
// (the message output layer W2 folded into the input layer: a_u = W2 g_u +
// (U-1) b2 since the layer is affine).
//
// Warp-specialised: eight worker warps run the epilogues and the cross-user
// sum, and one issuer warp (its lane 0) runs the bulk tensor copies and the
// MMAs, one tile ahead where the data allow: GEMM1 and the S part of GEMM2 of
// tile j + 1 are issued while the workers finish tile j (TMEM holds two sets
// of accumulators), so the workers wait only for the G part of GEMM2.  The
// two 16 KB operand buffers swap roles every tile: tile j's S buffer takes
// its 16-bit z staging once GEMM2 has read S, and tile j + 1's G after the
// bulk tensor store has read that staging; tile j + 1's S is loaded into
// tile j's G buffer once GEMM2 has read G.  Workers and issuer meet on
// mbarriers; every wait is bounded, and on a timeout the context's error
// word is set and both sides stop.
#include <cuda_runtime.h>

#include <cstring>

#include <cudaTypedefs.h>

#include "net_tc.h"
#include "tc.cuh"

namespace {

constexpr int kWorkers = 256;                 // 8 worker warps
constexpr int kThreads = kWorkers + 32;       // + the issuer warp
constexpr int kTile = 16384;                  // 128 x 64 16-bit operand tile
constexpr uint64_t kWaitNs = 1000000000ull;   // limit of every wait
constexpr uint64_t kDrainNs = 100000000ull;   // teardown wait for work in flight

template <typename T>
struct MpOps;
template <>
struct MpOps<__nv_bfloat16> {
  static constexpr uint32_t fmt = 1;
  static constexpr bool split = true;  // two-pass weights
  __device__ static __forceinline__ uint32_t pack(float a, float b) { return tc::pack_bf16x2(a, b); }
};
template <>
struct MpOps<__half> {
  static constexpr uint32_t fmt = 0;
  static constexpr bool split = false;
  __device__ static __forceinline__ uint32_t pack(float a, float b) {
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
  }
};

template <typename T>
constexpr uint32_t mp_idesc() {  // kind::f16, M = 128, N = 64, FP32 accumulate, K-major A and B
  return (1u << 4) | (MpOps<T>::fmt << 7) | (MpOps<T>::fmt << 10) | ((uint32_t)(64 >> 3) << 17) |
         ((uint32_t)(128 >> 4) << 24);
}

// Shared-memory layout (offsets from the 1024-byte-aligned base): the FP32
// exchange of h holds whole rows (32 KB); W1 and WS are packed in the
// activation type (hi + lo for BF16), WC in FP16.
template <typename T>
struct MpLay {
  static constexpr int WB = MpOps<T>::split ? 2 * 8192 : 8192;  // W1, WS: one packed 64 x 64 weight (hi [+ lo])
  static constexpr int BUF = 0;                                  // two operand buffers (S / G / z staging)
  static constexpr int XCH = BUF + 2 * kTile;
  static constexpr int W1 = XCH + 32768;
  static constexpr int WS = W1 + WB;
  static constexpr int WC = WS + WB;     // FP16 image (8 KB)
  static constexpr int VEC = WC + 8192;  // b1, b_in + (U-1) Win_a b2, PE weights (t, f): 4 x 64 FP32
  static constexpr int BAR = VEC + 1024; // 8 mbarriers; TMEM slot at +64
  static constexpr int TOTAL = BAR + 128;
  static constexpr int DYN = TOTAL + 1024;
};
static_assert(2 * (MpLay<__nv_bfloat16>::DYN + 1024) <= 233472, "two CTAs per SM");
static_assert(2 * (MpLay<__half>::DYN + 1024) <= 233472, "two CTAs per SM");

enum MpBar { kSFull = 0, kHFull, kGReady, kZFull, kStaged, kGFree, kNumBars };

template <typename T>
__device__ __forceinline__ void mp_gemm(uint32_t d, uint32_t a, uint32_t w, bool acc) {
  tc::mma_k64(d, a, w, mp_idesc<T>(), acc);
  if constexpr (MpOps<T>::split) tc::mma_k64(d, a, w + 8192, mp_idesc<T>(), true);
}

__device__ __forceinline__ void workers_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(kWorkers) : "memory");
}
// OR of `v` over the 256 worker threads (a barrier as well).
__device__ __forceinline__ bool workers_any(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred pi, po;\n\t"
      "setp.ne.u32 pi, %1, 0;\n\t"
      "bar.red.or.pred po, 1, %2, pi;\n\t"
      "selp.u32 %0, 1, 0, po;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(kWorkers)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void mbar_arrive1(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}
// Bounded wait for the phase of `parity`, sleeping in hardware between tries.
__device__ __forceinline__ bool mp_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns = kWaitNs) {
  auto try_wait = [&]() {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(tc::smem_u32(bar)), "r"(parity), "r"(20000u)
        : "memory");
    return ok != 0;
  };
  if (try_wait()) return true;
  const uint64_t t0 = tc::globaltimer();
  for (uint32_t i = 1; i < (1u << 24); ++i) {
    if (try_wait()) return true;
    if (tc::globaltimer() - t0 > limit_ns) return false;
  }
  return false;
}

template <typename T>
__device__ __forceinline__ uint4 mp_pack8(const float* v) {
  return make_uint4(MpOps<T>::pack(v[0], v[1]), MpOps<T>::pack(v[2], v[3]), MpOps<T>::pack(v[4], v[5]),
                    MpOps<T>::pack(v[6], v[7]));
}

template <typename T>
__global__ void __launch_bounds__(kThreads, 2)
    k_mp_ws(Geometry g, IterWeightsTC w, int nre, int tiles_per_slot, const __grid_constant__ CUtensorMap smap,
            const __grid_constant__ CUtensorMap zmap) {
  using L = MpLay<T>;
  tc::pdl_launch_dependents();
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                       ~uintptr_t(1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int U = g.U, S = g.S;
  // ---- prologue: weights, vectors, barriers, TMEM (two sets of h and z accumulators) ----
  {
    uint4* d1 = reinterpret_cast<uint4*>(sm + L::W1);
    uint4* ds = reinterpret_cast<uint4*>(sm + L::WS);
    uint4* dc = reinterpret_cast<uint4*>(sm + L::WC);
    for (int i = tid; i < L::WB / 16; i += kThreads) {
      d1[i] = __ldg(w.mp1 + i);
      ds[i] = __ldg(w.in_s + i);
    }
    for (int i = tid; i < 8192 / 16; i += kThreads) dc[i] = __ldg(w.in_c + i);
    float* vec = reinterpret_cast<float*>(sm + L::VEC);
    if (tid < 64) {
      vec[tid] = __ldg(w.mp1_b + tid);
      vec[64 + tid] = __ldg(w.in_b + tid) + (float)(U - 1) * __ldg(w.cb2 + tid);
      vec[128 + tid] = __ldg(w.in_pe + tid);
      vec[192 + tid] = __ldg(w.in_pe + 64 + tid);
    }
  }
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + L::BAR);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L::BAR + 64);
  if (tid == 0) {
    for (int i = 0; i < kNumBars; ++i) tc::mbar_init(bars + i, 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(tslot, 256);
  tc::fence_async_smem();  // the weights are MMA operands
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tslot;  // set p (tile parity): h at [128 p, 128 p + 64), z at + 64
  const float* vec = reinterpret_cast<const float*>(sm + L::VEC);
  const int n_re = NRX_SYMBOLS * S;
  const int n_tiles = g.n_slots * tiles_per_slot;
  const uint32_t buf_s = tc::smem_u32(sm + L::BUF);
  tc::pdl_wait();  // from here on the previous kernel's output is read

  if (warp == kWorkers / 32) {
    // ---------------- issuer (lane 0) ----------------
    if (lane == 0) {
      const uint32_t w1_s = tc::smem_u32(sm + L::W1), ws_s = tc::smem_u32(sm + L::WS),
                     wc_s = tc::smem_u32(sm + L::WC);
      uint32_t ph_s = 0, ph_g = 0, ph_z = 0, ph_st = 0;
      bool s_pending = false, mma_pending = false, ok = true;
      auto load_s = [&](int t, int buf) {
        NRX_IN((t % tiles_per_slot) * nre, n_re, 501);
        NRX_IN((t / tiles_per_slot) * U, g.n_slots * U, 502);
        tc::mbar_arrive_expect_tx(bars + kSFull, (uint32_t)(U * nre * 128));
        tc::tma_load_3d(sm + L::BUF + buf * kTile, &smap, 0, (t % tiles_per_slot) * nre, (t / tiles_per_slot) * U,
                        bars + kSFull);
        s_pending = true;
      };
      // GEMM1 and the S part of GEMM2 of the tile whose S rows land in buffer `buf`
      auto front = [&](int parity, int buf) {
        ok = mp_wait(bars + kSFull, ph_s);
        if (!ok) return;  // ph_s keeps the pending phase for the teardown drain
        ph_s ^= 1u;
        s_pending = false;
        tc::tc_fence_after();
        const uint32_t d = tmem + 128 * parity, a = buf_s + buf * kTile;
        mp_gemm<T>(d, a, w1_s, false);
        tc::mma_commit(bars + kHFull);
        mp_gemm<T>(d + 64, a, ws_s, false);
        mma_pending = true;
      };
      int k = 0, sb = 0;  // tile counter of this CTA, S buffer of tile k
      if ((int)blockIdx.x < n_tiles) {
        load_s(blockIdx.x, 0);
        front(0, 0);
      }
      for (int tile = blockIdx.x; ok && tile < n_tiles; tile += gridDim.x, ++k, sb ^= 1) {
        const int p = k & 1, gb = sb ^ 1;
        ok = mp_wait(bars + kGReady, ph_g);  // the workers have written G into buffer gb
        ph_g ^= 1u;
        if (!ok) break;
        tc::tc_fence_after();
        mp_gemm<__half>(tmem + 128 * p + 64, buf_s + gb * kTile, wc_s, true);  // G part: FP16
        tc::mma_commit(bars + kZFull);
        ok = mp_wait(bars + kZFull, ph_z);  // GEMM2 has read S and G
        ph_z ^= 1u;
        if (!ok) break;
        mma_pending = false;
        const int nt = tile + gridDim.x;
        if (nt < n_tiles) {  // the next tile's S into this tile's G buffer, its GEMM1 and S part of GEMM2
          load_s(nt, gb);
          front(p ^ 1, gb);
          if (!ok) break;
        }
        ok = mp_wait(bars + kStaged, ph_st);  // z staging written into this tile's S buffer
        ph_st ^= 1u;
        if (!ok) break;
        const int sl = tile / tiles_per_slot, re0 = (tile % tiles_per_slot) * nre;
        NRX_IN(re0, n_re, 503);
        NRX_IN(sl * U, g.n_slots * U, 503);
        tc::tma_store_3d(&zmap, 0, re0, sl * U, sm + L::BUF + sb * kTile);
        tc::bulk_commit();
        tc::bulk_wait_read_all();  // the staging has been read: the buffer may take the next G
        mbar_arrive1(bars + kGFree);
      }
      if (!ok) atomicExch(w.err, 1);
      if (s_pending) mp_wait(bars + kSFull, ph_s, kDrainNs);
      if (mma_pending) {  // let issued MMAs land (a commit that tracks them)
        tc::mma_commit(bars + kZFull);
        mp_wait(bars + kZFull, ph_z, kDrainNs);
      }
      tc::bulk_wait_all();
    }
  } else {
    // ---------------- workers ----------------
    const int q = warp & 3, hc = warp >> 2;  // TMEM lane quarter, column half
    const int r = q * 32 + lane;             // epilogue row of this thread
    const uint32_t tlane = (uint32_t)(q * 32) << 16;
    float* xch = reinterpret_cast<float*>(sm + L::XCH);
    uint32_t ph_h = 0, ph_z = 0, ph_free = 0;
    int k = 0, sb = 0;
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++k, sb ^= 1) {
      const int p = k & 1;
      const int sl = tile / tiles_per_slot;
      const int re0 = (tile % tiles_per_slot) * nre;
      unsigned char* const s_buf = sm + L::BUF + sb * kTile;
      unsigned char* const g_buf = sm + L::BUF + (sb ^ 1) * kTile;
      (void)sl;
      {
        bool ok = true;
        if (tid == 0) ok = mp_wait(bars + kHFull, ph_h);
        ph_h ^= 1u;
        if (workers_any(!ok)) {
          if (tid == 0) atomicExch(w.err, 1);
          break;
        }
      }
      tc::tc_fence_after();
      const uint32_t dh = tmem + 128 * p + tlane;
      // g_u = sum over the other active users of the exchanged h -> G (SW128),
      // items (RE j, channel quad): `xw` floats per exchange row, quads [q0, q0 + nq)
      auto aggregate = [&](int xw, int q0, int nq) {
        for (int i = tid; i < nre * nq; i += kWorkers) {
          const int j = i / nq, cql = i % nq, cq = q0 + cql;
          float4 hv[NRX_MAX_USERS];
#pragma unroll
          for (int u = 0; u < NRX_MAX_USERS; ++u) {
            const int rw = u * nre + j;
            hv[u] = u < U ? *reinterpret_cast<const float4*>(xch + rw * xw + ((cql ^ (rw & 7)) << 2))
                          : make_float4(0.f, 0.f, 0.f, 0.f);
          }
#pragma unroll
          for (int u = 0; u < NRX_MAX_USERS; ++u) {
            if (u >= U) break;
            float4 s4 = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int v = 0; v < NRX_MAX_USERS; ++v)
              if (v != u && v < U) {
                s4.x += hv[v].x;
                s4.y += hv[v].y;
                s4.z += hv[v].z;
                s4.w += hv[v].w;
              }
            const int row = u * nre + j;
            *reinterpret_cast<uint2*>(g_buf + tc::sw128_offset(row, 4 * cq)) =
                make_uint2(MpOps<__half>::pack(s4.x, s4.y), MpOps<__half>::pack(s4.z, s4.w));
          }
        }
      };
      // the previous tile's store has read g_buf (its z staging) before G is written
      auto wait_free = [&]() {
        bool ok = true;
        if (k > 0) {
          if (tid == 0) ok = mp_wait(bars + kGFree, ph_free);
          ph_free ^= 1u;
        }
        return workers_any(!ok);  // also the barrier after the exchange writes
      };
      // h = ReLU(acc + b1) of row r, columns [32 hc, 32 hc + 32), into the exchange
      // (float4 chunk k of a row at k ^ (r & 7)), then g_u
      {
        uint32_t a[16], b[16];
        tc::tmem_ld16(dh + 32 * hc, a);
        tc::tmem_ld16(dh + 32 * hc + 16, b);
        tc::tmem_wait16(a);
        tc::tmem_wait16(b);
        const float* b1 = vec + 32 * hc;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const uint32_t* src = c < 4 ? a + 4 * c : b + 4 * (c - 4);
          const int kk = 8 * hc + c;
          *reinterpret_cast<float4*>(xch + r * 64 + ((kk ^ (r & 7)) << 2)) =
              make_float4(fmaxf(__uint_as_float(src[0]) + b1[4 * c], 0.f),
                          fmaxf(__uint_as_float(src[1]) + b1[4 * c + 1], 0.f),
                          fmaxf(__uint_as_float(src[2]) + b1[4 * c + 2], 0.f),
                          fmaxf(__uint_as_float(src[3]) + b1[4 * c + 3], 0.f));
        }
      }
      tc::tc_fence_before();
      if (wait_free()) {
        if (tid == 0) atomicExch(w.err, 1);
        break;
      }
      aggregate(64, 0, 16);
      // rows of G not covered by (u < U, j < nre) only feed rows that are never stored
      tc::fence_async_smem();
      workers_sync();
      if (tid == 0) mbar_arrive1(bars + kGReady);
      // PE of this thread's row, computed while the G part of GEMM2 runs
      float pt = 0.f, pf = 0.f;
      {
        const int u = r / nre, j = r % nre, re = re0 + j;
        if (u < U && re < n_re) {
          pt = pe_time(g, re / S);
          pf = pe_freq(u, re % S);
        }
      }
      {
        bool ok = true;
        if (tid == 0) ok = mp_wait(bars + kZFull, ph_z);
        ph_z ^= 1u;
        if (workers_any(!ok)) {
          if (tid == 0) atomicExch(w.err, 1);
          break;
        }
      }
      tc::tc_fence_after();
      // z = acc + b + PE terms -> 16-bit staging [128][128 B] in this tile's S
      // buffer (GEMM2 has read it); 16-byte chunk c of a row stored at c ^ (r & 7)
      {
        uint32_t a[16], b[16];
        const uint32_t dz = tmem + 128 * p + 64 + tlane;
        tc::tmem_ld16(dz + 32 * hc, a);
        tc::tmem_ld16(dz + 32 * hc + 16, b);
        tc::tmem_wait16(a);
        tc::tmem_wait16(b);
        float acc[32];
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          acc[e] = __uint_as_float(a[e]);
          acc[16 + e] = __uint_as_float(b[e]);
        }
        const float* bb = vec + 64 + 32 * hc;
        const float* wt = vec + 128 + 32 * hc;
        const float* wf = vec + 192 + 32 * hc;
        unsigned char* rowp = s_buf + r * 128;
        const float2 pt2 = make_float2(pt, pt), pf2 = make_float2(pf, pf);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          float o[8];
#pragma unroll
          for (int e = 0; e < 8; e += 2) {  // packed: (acc + b) + pt w_t + pf w_f per channel pair
            const int cc = 8 * c + e;
            float2 x = tc::fadd2(make_float2(acc[cc], acc[cc + 1]), make_float2(bb[cc], bb[cc + 1]));
            x = tc::ffma2(pt2, make_float2(wt[cc], wt[cc + 1]), x);
            x = tc::ffma2(pf2, make_float2(wf[cc], wf[cc + 1]), x);
            o[e] = x.x;
            o[e + 1] = x.y;
          }
          const int kk = 4 * hc + c;
          *reinterpret_cast<uint4*>(rowp + ((kk ^ (r & 7)) << 4)) = mp_pack8<T>(o);
        }
      }
      tc::tc_fence_before();
      tc::fence_async_smem();
      workers_sync();
      if (tid == 0) mbar_arrive1(bars + kStaged);
    }
  }
  // ---- teardown: TMEM is freed once every warp is done with it ----
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, 256);
  }
}

}  // namespace

template <typename T>
cudaError_t state_rows_map(CUtensorMap* map, const T* base, int planes, int n_re, int nre, int U);

template <typename T>
cudaError_t launch_mp16_tc(const Geometry& g, const IterWeightsTC& w, const T* state, T* z, cudaStream_t st) {
  if (g.C != 64) return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(state) | reinterpret_cast<uintptr_t>(z)) & 15)
    return cudaErrorInvalidValue;  // TMA global address alignment
  const int nre = g.U == 4 ? 32 : g.U == 3 ? 40 : g.U == 2 ? 64 : 128;
  const int tps = (NRX_SYMBOLS * g.S + nre - 1) / nre;
  const int tiles = g.n_slots * tps;
  if (tiles == 0) return cudaSuccess;
  const int smem = MpLay<T>::DYN;
  cudaError_t e = ensure_smem<k_mp_ws<T>>(smem);
  if (e != cudaSuccess) return e;
  CUtensorMap smap, zmap;
  memset(&smap, 0, sizeof(smap));
  memset(&zmap, 0, sizeof(zmap));
  e = state_rows_map(&smap, state, g.n_slots * g.U, NRX_SYMBOLS * g.S, nre, g.U);
  if (e == cudaSuccess)
    e = state_rows_map(&zmap, static_cast<const T*>(z), g.n_slots * g.U, NRX_SYMBOLS * g.S, nre, g.U);
  if (e != cudaSuccess) return e;
  const int grid = tiles < 2 * block_sms() ? tiles : 2 * block_sms();
  return launch_pdl(k_mp_ws<T>, grid, kThreads, smem, st, g, w, nre, tps, smap, zmap);
}

template cudaError_t launch_mp16_tc<__nv_bfloat16>(const Geometry&, const IterWeightsTC&, const __nv_bfloat16*,
                                                  __nv_bfloat16*, cudaStream_t);
template cudaError_t launch_mp16_tc<__half>(const Geometry&, const IterWeightsTC&, const __half*, __half*,
                                           cudaStream_t);

NRX_DEBUG_READER(debug_read_mp_tc)
