// Residual block of the CNN update (Sec. II-A) on the tensor cores, 16-bit
// activations (BF16 or FP16) in and out:
//   z_out = z_in + PW2(ReLU(DW2(ReLU(PW1(DW1(z_in))))))     (+ S, last block)
// with 3x3 depthwise taps DW on the CUDA cores and the 1x1 layers PW as
// tcgen05 MMAs with FP32 accumulators in TMEM.  The block's intermediates
// (the depthwise outputs, which are the PW operands, and P1) are FP16, the
// taps run as packed FP16 FMAs and the PW weights are FP16 in both modes:
// FP16 carries three more mantissa bits than BF16, so the BF16 mode needs no
// split (hi + lo) weights here; the input, the residual, the biases and the
// output stay in the activation type.
//
// Tiles: 12 subcarriers x 14 symbols of one (slot, user); since S = 12 N_PRB
// no tile is ragged.  Every operand tile has 224 rows, row = t * 16 + c, over
// the 16 input columns c (subcarrier s0 - 2 + c, a halo of two on each side),
// in the 128-byte-swizzle K-major layout of the MMA; the MMAs cover it as two
// M = 128 tiles starting at rows 0 and 96.  Per tile:
//   1. TMA: input box [14][16][64] -> IN (zero outside the grid), loaded
//      during the previous tile (three buffers rotate through the roles IN,
//      A and free; the last block of an iteration, whose third buffer holds
//      the state tile ST, keeps fixed roles).
//   2. DW1 (columns 1..14) from IN -> A, while the leader issues
//      D2 = IN x I + 1 b2^T (identity weights: the residual lands in the PW2
//      accumulator exactly, since I is exact in 16 bits) and D1 = 1 b1^T.
//   3. MMA: D1 += A W1^T on both M tiles.
//   4. Epilogue 1: P1 = ReLU(D1), zero outside the grid, over IN.
//   5. DW2 + ReLU (columns 2..13) from P1 -> A.  MMA: D2 += A W2^T (+ ST x I:
//      the state tile, last block).
//   6. Epilogue 2: D2 -> OUT (in A; rows t * 12 + c - 2) -> TMA store.
// The biases enter the accumulators through one K = 16 MMA of an all-ones
// tile with a tile holding [b_hi, b_lo], b_hi the 16-bit rounding of b and
// b_lo that of the remainder.
// A CTA of 16 warps holds one copy of the weights and runs two 8-warp tile
// pipelines (own buffers, barriers and 256 TMEM columns each) whose
// depthwise phases take turns: while one group runs its taps on the CUDA
// cores, the other waits for its MMAs and runs its epilogues and copies.
// All waits are bounded (the waiting thread sleeps in hardware); on a timeout
// the context's error word is set and the group stops working but keeps
// taking its turns, and the CTA drains its asynchronous work and exits.
#include <cuda_runtime.h>

#include <cstring>
#include <type_traits>

#include <cudaTypedefs.h>

#include "net_tc.h"
#include "tc.cuh"

namespace {

constexpr int kTW = 12;                       // output subcarriers per tile
constexpr int kIW = kTW + 4;                  // input columns
constexpr int kRows = NRX_SYMBOLS * kIW;      // 224 operand rows
constexpr int kBuf = kRows * 128;             // 28 KB operand tile
constexpr int kM1Row = 96;                    // first row of the second M tile
constexpr int kGroupThreads = 256;
constexpr int kThreads = 2 * kGroupThreads;
constexpr uint32_t kInBytes = kBuf;           // bytes of one [14][16][64] 16-bit box
constexpr uint64_t kWaitNs = 1000000000ull;   // limit of every wait
constexpr uint64_t kDrainNs = 100000000ull;   // teardown wait for work in flight

template <typename T>
struct Ops;
template <>
struct Ops<__nv_bfloat16> {
  static constexpr uint32_t fmt = 1;
  static constexpr uint16_t one = 0x3F80;
  __device__ static __forceinline__ uint32_t pack(float a, float b) { return tc::pack_bf16x2(a, b); }
  __device__ static __forceinline__ uint32_t pack_relu(float a, float b) { return tc::pack_relu_bf16x2(a, b); }
};
template <>
struct Ops<__half> {
  static constexpr uint32_t fmt = 0;
  static constexpr uint16_t one = 0x3C00;
  __device__ static __forceinline__ uint32_t pack(float a, float b) {
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
  }
  __device__ static __forceinline__ uint32_t pack_relu(float a, float b) { return tc::pack_relu_f16x2(a, b); }
};

template <typename T>
constexpr uint32_t idesc16() {  // kind::f16, M = 128, N = 64, FP32 accumulate, K-major A and B
  return (1u << 4) | (Ops<T>::fmt << 7) | (Ops<T>::fmt << 10) | ((uint32_t)(64 >> 3) << 17) |
         ((uint32_t)(128 >> 4) << 24);
}

// Shared-memory layout (offsets from the 1024-byte-aligned base).
template <typename T>
struct Lay {
  static constexpr int WB = 8192;             // one packed 64 x 64 FP16 weight (both modes)
  static constexpr int W1 = 0;
  static constexpr int W2 = W1 + WB;
  static constexpr int ID = W2 + WB;          // 64 x 64 identity, SW128
  static constexpr int ONES = ID + 8192;      // 128 x 16 all-ones A tile (k = 0, 1), no swizzle
  static constexpr int BI1 = ONES + 4096;     // 64 x 16 bias B tiles [b_hi, b_lo], no swizzle
  static constexpr int BI2 = BI1 + 2048;
  static constexpr int K1 = BI2 + 2048;       // DW1 taps [64][9] FP32
  static constexpr int K2 = K1 + 64 * 9 * 4;
  static constexpr int BAR = K2 + 64 * 9 * 4; // per group: six mbarriers (48 B); TMEM slot at +96
  static constexpr int GRP = ((BAR + 128 + 1023) / 1024) * 1024;
  static constexpr int GSTRIDE = 3 * kBuf;    // per group: IN/P1, A, ST/OUT
  static constexpr int TOTAL = GRP + 2 * GSTRIDE;
  static constexpr int DYN = TOTAL + 1024;
};
static_assert(Lay<__nv_bfloat16>::DYN <= 232448, "shared memory per CTA");
static_assert(kBuf % 1024 == 0 && (kM1Row * 128) % 1024 == 0, "SW128 atoms stay 1024-byte aligned");
static_assert(kM1Row + 128 == kRows, "the two M tiles cover the operand rows");

extern __shared__ unsigned char nrx_dyn_smem[];  // the kernel's dynamic shared memory (same base)
// Bounds-checked build: is [a, a + bytes) inside the dynamic shared memory?
__device__ __forceinline__ bool smem_ok(uint32_t a, uint32_t bytes, int site) {
#ifdef NRX_DEBUG
  uint32_t size;
  asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(size));
  const uint32_t lo = tc::smem_u32(nrx_dyn_smem);
  return NRX_IN((long long)a - lo + bytes - 1, size, site) && NRX_IN((long long)a - lo, size, site);
#else
  (void)a;
  (void)bytes;
  (void)site;
  return true;
#endif
}
__device__ __forceinline__ uint32_t lds32(uint32_t a) {
  uint32_t v = 0;
  if (smem_ok(a, 4, 401)) asm volatile("ld.shared.b32 %0, [%1];" : "=r"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ void sts32c(uint32_t a, uint32_t v) {
  if (smem_ok(a, 4, 402)) tc::sts32(a, v);
}
__device__ __forceinline__ void sts128(uint32_t a, uint32_t x, uint32_t y, uint32_t z, uint32_t w) {
  if (smem_ok(a, 16, 403))
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(x), "r"(y), "r"(z), "r"(w));
}

// try_wait with a suspend-time hint: a thread whose phase is not complete
// sleeps in hardware (up to hint_ns) instead of spinning on issue slots that
// the working warps need, and wakes when the phase completes.
__device__ __forceinline__ bool try_wait_sleep(uint64_t* bar, uint32_t parity, uint32_t hint_ns) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(tc::smem_u32(bar)), "r"(parity), "r"(hint_ns)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void group_sync(uint32_t id) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "n"(kGroupThreads) : "memory");
}
// OR of `v` over the group's 256 threads (a barrier as well).
__device__ __forceinline__ bool group_any(uint32_t id, bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred pi, po;\n\t"
      "setp.ne.u32 pi, %1, 0;\n\t"
      "bar.red.or.pred po, %2, %3, pi;\n\t"
      "selp.u32 %0, 1, 0, po;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(id), "n"(kGroupThreads)
      : "memory");
  return r != 0;
}
// Bounded wait for the phase of `parity` by one thread, sleeping in hardware.
__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t parity, uint64_t limit_ns = kWaitNs) {
  if (try_wait_sleep(bar, parity, 20000)) return true;
  const uint64_t t0 = tc::globaltimer();
  for (uint32_t i = 1; i < (1u << 24); ++i) {
    if (try_wait_sleep(bar, parity, 20000)) return true;
    if (tc::globaltimer() - t0 > limit_ns) return false;
  }
  return false;
}

// Sliding 3x3 depthwise over the 14 symbols for two adjacent output columns
// of one channel pair (2 cp, 2 cp + 1), packed FP16 FMAs with FP16 taps.
// in_addr[k] (k < 4) addresses this lane's word of input column k on symbol 0
// (one symbol = 16 rows = 2048 bytes further); out_addr[o] likewise for
// output column o.  Inputs Tin (a BF16 pair is rounded to an FP16 pair on
// load), FP16 outputs; zero padding in time; kRelu applies max(., 0).  The
// words of symbol ti + 2 are requested before symbol ti is computed.  Symbols
// 0..11 run as a loop over blocks of three (the period of the register
// window), 12 and 13 after it: a small loop body keeps the kernel's code
// within the instruction caches.
template <typename Tin, bool kRelu>
__device__ __forceinline__ void dw_pair(const float* __restrict__ taps, int cp, const uint32_t (&in_addr)[4],
                                        const uint32_t (&out_addr)[2]) {
  __half2 kk[9];  // (channel 2 cp, channel 2 cp + 1)
#pragma unroll
  for (int i = 0; i < 9; ++i) kk[i] = __floats2half2_rn(taps[(2 * cp) * 9 + i], taps[(2 * cp + 1) * 9 + i]);
  const __half2 zero = __float2half2_rn(0.f);
  __half2 am[2], a0[2], ap[2];  // per output column: outputs of symbols ti - 1, ti, ti + 1
#pragma unroll
  for (int j = 0; j < 2; ++j) am[j] = a0[j] = ap[j] = zero;
  uint32_t w0[4], w1[4], w2[4];  // words of symbols ti, ti + 1, ti + 2
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    w0[k] = lds32(in_addr[k]);
    w1[k] = lds32(in_addr[k] + 2048);
  }
  auto put = [&](int t, int o) {
    __half2 v = am[o];
    if (kRelu) v = __hmax2(v, zero);
    sts32c(out_addr[o] + t * 2048, *reinterpret_cast<uint32_t*>(&v));
  };
  auto step = [&](int ti, bool prefetch) {
    if (prefetch)
#pragma unroll
      for (int k = 0; k < 4; ++k) w2[k] = lds32(in_addr[k] + (ti + 2) * 2048);
    __half2 x[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if constexpr (std::is_same<Tin, __nv_bfloat16>::value)
        x[k] = __floats2half2_rn(__uint_as_float(w0[k] << 16), __uint_as_float(w0[k] & 0xFFFF0000u));
      else
        x[k] = *reinterpret_cast<const __half2*>(&w0[k]);
    }
#pragma unroll
    for (int o = 0; o < 2; ++o)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        am[o] = __hfma2(kk[6 + k], x[o + k], am[o]);
        a0[o] = __hfma2(kk[3 + k], x[o + k], a0[o]);
        ap[o] = __hfma2(kk[k], x[o + k], ap[o]);
      }
    if (ti >= 1) {
      put(ti - 1, 0);
      put(ti - 1, 1);
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      am[j] = a0[j];
      a0[j] = ap[j];
      ap[j] = zero;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      w0[k] = w1[k];
      w1[k] = w2[k];
    }
  };
#pragma unroll 1
  for (int tb = 0; tb < 12; tb += 3) {
    step(tb, true);
    step(tb + 1, true);
    step(tb + 2, true);
  }
  step(12, false);
  step(13, false);
  put(NRX_SYMBOLS - 1, 0);
  put(NRX_SYMBOLS - 1, 1);
}

// This lane's word (channel pair cp) of operand column c on symbol 0 of the
// SW128 tile at `base`: row c, 16-byte chunk (cp / 4) ^ (row & 7), and
// (row & 7) == (c & 7) for every symbol since a symbol spans 16 rows.
__device__ __forceinline__ uint32_t col_word(uint32_t base, int c, int cp) {
  return base + c * 128 + ((((cp >> 2) ^ (c & 7)) << 4) | ((cp & 3) << 2));
}

// 64 FP32 values -> 8 packed 16-byte chunks of one SW128 row (zeros if `zero`).
template <typename T, bool kRelu>
__device__ __forceinline__ void store_row(uint32_t row_addr, int row, const float (&v)[64], bool zero) {
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    uint32_t w[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float a = v[8 * k + 2 * j], b = v[8 * k + 2 * j + 1];
      w[j] = kRelu ? Ops<T>::pack_relu(a, b) : Ops<T>::pack(a, b);
    }
    if (zero) w[0] = w[1] = w[2] = w[3] = 0u;
    sts128(row_addr + ((k ^ (row & 7)) << 4), w[0], w[1], w[2], w[3]);
  }
}

// K = 64 product of one M tile with a packed 64 x 64 weight.
template <typename T>
__device__ __forceinline__ void mma_w(uint32_t d, uint32_t a, uint32_t w, bool acc) {
  tc::mma_k64(d, a, w, idesc16<T>(), acc);
}

// Shared-memory descriptor of a K-major tile without swizzle: 8-row x 16-byte
// core matrices, `lbo` bytes apart along K, `sbo` bytes apart along M / N.
__device__ __forceinline__ uint64_t desc_plain(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version; layout type 0 (no swizzle)
  return d;
}
// Byte offset of element (row r, k) of such a tile with lbo = 128, sbo = 256.
__host__ __device__ constexpr uint32_t plain_offset(int r, int k) {
  return (uint32_t)((r >> 3) * 256 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}
// D (+)= 1 [b_hi b_lo]^T: one K = 16 MMA of the all-ones tile with a bias tile.
template <typename T>
__device__ __forceinline__ void mma_bias(uint32_t d, uint32_t ones, uint32_t bias, bool acc) {
  tc::mma_bf16(d, desc_plain(ones, 128, 256), desc_plain(bias, 128, 256), idesc16<T>(), acc ? 1u : 0u);
}

template <typename T>
__global__ void __launch_bounds__(kThreads, 1)
    k_block2(int n_tiles, int tps, int S, const uint4* __restrict__ w1p, const uint4* __restrict__ w2p,
             const float* __restrict__ b1, const float* __restrict__ b2, const float* __restrict__ k1g,
             const float* __restrict__ k2g, int last, int* err, const __grid_constant__ CUtensorMap in_map,
             const __grid_constant__ CUtensorMap st_map, const __grid_constant__ CUtensorMap out_map) {
  using L = Lay<T>;
  // Inside the block the depthwise outputs (PW operands) and P1 are FP16, the taps
  // packed FP16 FMAs and the PW weights FP16 in both modes; the input, the residual,
  // the biases and the output keep T.
  using TI = __half;
  tc::pdl_launch_dependents();
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                       ~uintptr_t(1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // ---- prologue: weights, identity, ones and bias tiles, taps, barriers, TMEM ----
  {
    uint4* d1 = reinterpret_cast<uint4*>(sm + L::W1);
    uint4* d2 = reinterpret_cast<uint4*>(sm + L::W2);
    for (int i = tid; i < L::WB / 16; i += kThreads) {
      d1[i] = __ldg(w1p + i);
      d2[i] = __ldg(w2p + i);
    }
    uint4* z = reinterpret_cast<uint4*>(sm + L::ID);
    for (int i = tid; i < (8192 + 4096 + 2048 + 2048) / 16; i += kThreads) z[i] = make_uint4(0, 0, 0, 0);
    float* k1 = reinterpret_cast<float*>(sm + L::K1);
    float* k2 = reinterpret_cast<float*>(sm + L::K2);
    for (int i = tid; i < 64 * 9; i += kThreads) {
      k1[i] = __ldg(k1g + i);
      k2[i] = __ldg(k2g + i);
    }
  }
  __syncthreads();  // identity, ones and bias tiles zeroed before their entries are written
  if (tid < 64) {
    *reinterpret_cast<uint16_t*>(sm + L::ID + tc::sw128_offset(tid, tid)) = Ops<T>::one;
    // bias tiles: row n = [b_hi, b_lo, 0 ...], b_hi = T(b), b_lo = T(b - b_hi)
    const float bias[2] = {__ldg(b1 + tid), __ldg(b2 + tid)};
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      const uint32_t hl = Ops<T>::pack(bias[l], 0.f) & 0xFFFFu;
      const float hi = std::is_same<T, __half>::value ? __half2float(__ushort_as_half((unsigned short)hl))
                                                      : __bfloat162float(__ushort_as_bfloat16((unsigned short)hl));
      const uint32_t lo = Ops<T>::pack(bias[l] - hi, 0.f) & 0xFFFFu;
      unsigned char* t = sm + (l ? L::BI2 : L::BI1);
      *reinterpret_cast<uint16_t*>(t + plain_offset(tid, 0)) = (uint16_t)hl;
      *reinterpret_cast<uint16_t*>(t + plain_offset(tid, 1)) = (uint16_t)lo;
    }
  }
  if (tid < 128) {  // all-ones tile: A[m][0] = A[m][1] = 1
    *reinterpret_cast<uint16_t*>(sm + L::ONES + plain_offset(tid, 0)) = Ops<T>::one;
    *reinterpret_cast<uint16_t*>(sm + L::ONES + plain_offset(tid, 1)) = Ops<T>::one;
  }
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L::BAR + 96);
  if (tid == 0) {
    // per group (48 bytes): copies into buffers 0..2, MMA commits (two slots unused)
    for (int i = 0; i < 12; ++i) tc::mbar_init(reinterpret_cast<uint64_t*>(sm + L::BAR + i * 8), 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(tslot, 512);
  tc::fence_async_smem();  // weights, identity, ones and bias tiles are MMA operands
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tslot;

  // ---- this group's pipeline ----
  const int grp = warp >> 3, gw = warp & 7, gtid = tid & (kGroupThreads - 1);
  const uint32_t bar_id = 1 + grp;
  // the group's leader (TMA, MMA issue, waits) is lane 0 of warp 7, which has no depthwise
  // columns in DW1: it issues the residual and bias MMAs while the other warps run DW1
  const bool leader = gtid == 7 * 32;
  uint64_t* in_bar = reinterpret_cast<uint64_t*>(sm + L::BAR + grp * 48);  // [i]: copy into buffer i
  uint64_t* mma_bar = in_bar + 3;
  unsigned char* g_buf0 = sm + L::GRP + grp * L::GSTRIDE;  // three operand buffers of kBuf bytes
  const uint32_t buf0_s = tc::smem_u32(g_buf0), st_s = buf0_s + 2 * kBuf;
  const uint32_t w1_s = tc::smem_u32(sm + L::W1), w2_s = tc::smem_u32(sm + L::W2), id_s = tc::smem_u32(sm + L::ID),
                 ones_s = tc::smem_u32(sm + L::ONES), bi1_s = tc::smem_u32(sm + L::BI1),
                 bi2_s = tc::smem_u32(sm + L::BI2);
  const uint32_t d1 = tmem + grp * 256, d2 = d1 + 128;  // + 64 for the second M tile
  const float* sk1 = reinterpret_cast<const float*>(sm + L::K1);
  const float* sk2 = reinterpret_cast<const float*>(sm + L::K2);
  const int cp = lane;
  // epilogue row of this thread: TMEM lane quadrant gw & 3 of M tile gw >> 2;
  // warp 4 would repeat rows 96..127 of the first M tile and stays idle
  const int e_mt = gw >> 2, e_row = (gw & 3) * 32 + lane;
  const int e_r = e_mt ? kM1Row + e_row : e_row;
  const int e_c = e_r & 15, e_t = e_r >> 4;
  const uint32_t e_lane = (uint32_t)((gw & 3) * 32) << 16;
  // Buffer roles.  The last block of an iteration: IN = 0, A = 1, ST = 2; the
  // next tile's input is loaded into buffer 0 once DW2 is done with P1, and
  // DW1 waits until the previous tile's store has read OUT (in A).  The other
  // blocks rotate the three buffers: tile j has IN = j % 3 and A = (j + 2) % 3,
  // which was the IN of tile j - 1 (P1 no longer read), so DW1 never waits for
  // a store; tile j + 1's input is loaded during tile j's PW1 into buffer
  // (j + 1) % 3, the A of tile j - 1, once that tile's store has read it.
  const bool rot = !last;

  uint32_t in_ph = 0, in_pending = 0;  // bit i: parity / copy in flight of buffer i
  uint32_t st_ph = 0, mma_ph = 0;
  bool st_pending = false, mma_pending = false;
  const int vt0 = blockIdx.x * 2 + grp, vstride = gridDim.x * 2;
  // both groups run the same number of iterations, so that the turns below pair up
  const int n_grp0 = blockIdx.x * 2 < n_tiles ? (n_tiles - blockIdx.x * 2 + vstride - 1) / vstride : 0;
  const int n_grp1 = blockIdx.x * 2 + 1 < n_tiles ? (n_tiles - blockIdx.x * 2 - 1 + vstride - 1) / vstride : 0;
  const int n_iter = n_grp0 > n_grp1 ? n_grp0 : n_grp1;
  tc::pdl_wait();  // from here on the previous kernel's output is read
  if (leader && vt0 < n_tiles) {
    NRX_IN(vt0 / tps, n_tiles / tps, 404);
    tc::mbar_arrive_expect_tx(in_bar, kInBytes);
    tc::tma_load_3d(g_buf0, &in_map, 0, (vt0 % tps) * kTW - 2, (vt0 / tps) * NRX_SYMBOLS, in_bar);
    in_pending = 1u;
  }
  // The depthwise phases of the two groups take turns (group 0 first): while
  // one group runs its depthwise taps on the CUDA cores, the other waits for
  // its MMAs, runs its epilogues and copies.  Named barrier 3 + g is group g's
  // turn: the group syncs on it before a depthwise phase, and the other group
  // arrives on it after each of its own (group 1 skips its very last arrival,
  // which no phase of group 0 would consume).
  const uint32_t my_turn = 3 + grp, other_turn = 4 - grp;
  auto take_turn = [&]() { asm volatile("bar.sync %0, %1;" ::"r"(my_turn), "n"(kThreads) : "memory"); };
  auto pass_turn = [&](bool final_phase) {
    if (!(grp == 1 && final_phase)) asm volatile("bar.arrive %0, %1;" ::"r"(other_turn), "n"(kThreads) : "memory");
  };
  if (grp == 1 && n_iter > 0) pass_turn(false);
  bool dead = false;  // a wait gave up: the group only keeps taking and passing its turns
  int b = 0;           // IN buffer of this tile
  for (int it = 0; it < n_iter; ++it) {
    const int tile = vt0 + it * vstride;
    const bool final_it = it + 1 == n_iter;
    bool work = !dead && tile < n_tiles;
    const int ba = rot ? (b == 0 ? 2 : b - 1) : 1;  // A buffer
    const int bn = rot ? (b == 2 ? 0 : b + 1) : 0;  // next tile's IN buffer
    const uint32_t in_s = buf0_s + b * kBuf, a_s = buf0_s + ba * kBuf;
    const int su = tile / tps, s0 = (tile % tps) * kTW;
    // 1: input tile; OUT (in A) read by the previous store
    if (work) {
      bool ok = true;
      if (leader) {
        ok = wait_bar(in_bar + b, (in_ph >> b) & 1u);
        if (ok) {
          in_pending &= ~(1u << b);
          if (!rot) tc::bulk_wait_read_all();  // OUT (in A) read by the previous store
        }
      }
      if (ok) in_ph ^= 1u << b;  // after a failed wait the bit keeps the pending phase (teardown drain)
      if (group_any(bar_id, !ok)) {
        if (leader) atomicExch(err, 1);
        dead = true;
        work = false;
      }
    }
    // 2-3: DW1, output columns 1..14 (warp gw: columns 2 gw + 1, 2 gw + 2); meanwhile the
    // leader issues D2 = IN x I + 1 b2^T (the residual, exact: I is exact in 16 bits) and
    // D1 = 1 b1^T, which the PW1 commit below covers
    take_turn();
    if (work && gw < 7) {
      uint32_t ia[4], oa[2];
#pragma unroll
      for (int k = 0; k < 4; ++k) ia[k] = col_word(in_s, 2 * gw + k, cp);
#pragma unroll
      for (int o = 0; o < 2; ++o) oa[o] = col_word(a_s, 2 * gw + 1 + o, cp);
      dw_pair<T, false>(sk1, cp, ia, oa);
    } else if (work && leader) {
      tc::tc_fence_after();
      tc::mma_k64(d2, in_s, id_s, idesc16<T>(), false);
      tc::mma_k64(d2 + 64, in_s + kM1Row * 128, id_s, idesc16<T>(), false);
      mma_bias<T>(d2, ones_s, bi2_s, true);
      mma_bias<T>(d2 + 64, ones_s, bi2_s, true);
      mma_bias<T>(d1, ones_s, bi1_s, false);
      mma_bias<T>(d1 + 64, ones_s, bi1_s, false);
    }
    pass_turn(false);
    if (work) {
      tc::fence_async_smem();
      if (leader && last) {  // state tile for the last block (buffer 2: its previous tile's MMAs are done)
        tc::mbar_arrive_expect_tx(in_bar + 2, kInBytes);
        NRX_IN(s0 + kTW - 1, S, 405);
        tc::tma_load_3d(g_buf0 + 2 * kBuf, &st_map, 0, s0 - 2, su * NRX_SYMBOLS, in_bar + 2);
        st_pending = true;
      }
      group_sync(bar_id);
      bool ok = true;
      if (leader) {
        tc::tc_fence_after();
        mma_w<TI>(d1, a_s, w1_s, true);
        mma_w<TI>(d1 + 64, a_s + kM1Row * 128, w1_s, true);
        tc::mma_commit(mma_bar);
        mma_pending = true;
        const int nt = tile + vstride;
        if (rot && nt < n_tiles) {  // next tile's input into the previous tile's A, once its store has read it
          tc::bulk_wait_read_all();
          NRX_IN(nt / tps, n_tiles / tps, 406);
          tc::mbar_arrive_expect_tx(in_bar + bn, kInBytes);
          tc::tma_load_3d(g_buf0 + bn * kBuf, &in_map, 0, (nt % tps) * kTW - 2, (nt / tps) * NRX_SYMBOLS,
                          in_bar + bn);
          in_pending |= 1u << bn;
        }
        ok = wait_bar(mma_bar, mma_ph);
        if (ok) mma_pending = false;
      }
      if (!mma_pending) mma_ph ^= 1u;
      if (group_any(bar_id, !ok)) {
        if (leader) atomicExch(err, 1);
        dead = true;
        work = false;
      }
    }
    if (work) {
      tc::tc_fence_after();
      // 4: epilogue 1 -> P1 (over IN: the residual MMA and DW1 are done with it)
      if (gw != 4) {
        float v[64];
        tc::tmem_row64(d1 + e_mt * 64 + e_lane, v);
        if (e_c >= 1 && e_c <= 14) {
          const int s = s0 - 2 + e_c;
          store_row<TI, true>(in_s + e_r * 128, e_r, v, s < 0 || s >= S);
        }
      }
      tc::tc_fence_before();
      group_sync(bar_id);
    }
    // 5: DW2 + ReLU, output columns 2..13 (warp gw: columns 2 gw + 2, 2 gw + 3)
    take_turn();
    if (work && gw < 6) {
      uint32_t ia[4], oa[2];
#pragma unroll
      for (int k = 0; k < 4; ++k) ia[k] = col_word(in_s, 2 * gw + 1 + k, cp);
#pragma unroll
      for (int o = 0; o < 2; ++o) oa[o] = col_word(a_s, 2 * gw + 2 + o, cp);
      dw_pair<TI, true>(sk2, cp, ia, oa);
    }
    pass_turn(final_it);
    if (work) {
      tc::fence_async_smem();
      group_sync(bar_id);
      bool ok = true;
      if (leader) {
        if (last) {
          ok = wait_bar(in_bar + 2, st_ph);
          if (ok) st_pending = false;
        }
        if (ok) {
          tc::tc_fence_after();
          mma_w<TI>(d2, a_s, w2_s, true);
          mma_w<TI>(d2 + 64, a_s + kM1Row * 128, w2_s, true);
          if (last) {
            tc::mma_k64(d2, st_s, id_s, idesc16<T>(), true);
            tc::mma_k64(d2 + 64, st_s + kM1Row * 128, id_s, idesc16<T>(), true);
          }
          tc::mma_commit(mma_bar);
          mma_pending = true;
          // last block: the next tile's input into IN, whose P1 DW2 no longer reads
          const int nt = tile + vstride;
          if (!rot && nt < n_tiles) {
            NRX_IN(nt / tps, n_tiles / tps, 406);
            tc::mbar_arrive_expect_tx(in_bar, kInBytes);
            tc::tma_load_3d(g_buf0, &in_map, 0, (nt % tps) * kTW - 2, (nt / tps) * NRX_SYMBOLS, in_bar);
            in_pending |= 1u;
          }
          ok = wait_bar(mma_bar, mma_ph);
          if (ok) mma_pending = false;
        }
      }
      if (last && !st_pending) st_ph ^= 1u;
      if (!mma_pending) mma_ph ^= 1u;
      if (group_any(bar_id, !ok)) {
        if (leader) atomicExch(err, 1);
        dead = true;
        work = false;
      }
    }
    if (work) {
      tc::tc_fence_after();
      // 6: epilogue 2 -> OUT (in A, whose A2 rows the PW2 MMAs have read), rows t * 12 + c - 2,
      // then one bulk tensor store
      if (gw != 4) {
        float v[64];
        tc::tmem_row64(d2 + e_mt * 64 + e_lane, v);
        if (e_c >= 2 && e_c <= 13) {
          const int ro = e_t * kTW + e_c - 2;
          store_row<T, false>(a_s + ro * 128, ro, v, false);
        }
      }
      tc::fence_async_smem();
      tc::tc_fence_before();
      group_sync(bar_id);
      if (leader && NRX_IN(s0 + kTW - 1, S, 407) && NRX_IN(su, n_tiles / tps, 407)) {
        tc::tma_store_3d(&out_map, 0, s0, su * NRX_SYMBOLS, g_buf0 + ba * kBuf);
        tc::bulk_commit();
      }
    }
    b = bn;
  }
  // ---- teardown: let asynchronous work in flight land, then free TMEM (a phase
  // variable advances only past a successful wait, so it names the pending phase) ----
  if (leader) {
    for (int j = 0; j < 3; ++j)
      if ((in_pending >> j) & 1u) wait_bar(in_bar + j, (in_ph >> j) & 1u, kDrainNs);
    if (st_pending) wait_bar(in_bar + 2, st_ph, kDrainNs);
    if (mma_pending) wait_bar(mma_bar, mma_ph, kDrainNs);
    tc::bulk_wait_all();
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, 512);
  }
}

// 3-D map of a 16-bit activation tensor [planes x 14][S][64] with a
// [14 symbols][box_s subcarriers][64 channels] box in the 128-byte swizzle
// (the MMA operand layout), zero fill outside the tensor.
template <typename T>
cudaError_t swizzled_map(CUtensorMap* map, const T* base, int planes, int S, int box_s) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return cudaErrorNotSupported;
  const cuuint64_t dims[3] = {64, (cuuint64_t)S, (cuuint64_t)planes * NRX_SYMBOLS};
  const cuuint64_t strides[2] = {64 * sizeof(T), (cuuint64_t)S * 64 * sizeof(T)};
  const cuuint32_t box[3] = {64, (cuuint32_t)box_s, NRX_SYMBOLS};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUtensorMapDataType dt =
      std::is_same<T, __half>::value ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  const CUresult r = enc(map, dt, 3, const_cast<T*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

int block_sms() {
  static const int n = [] {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 148;
  }();
  return n;
}

template <typename T>
cudaError_t launch_block16_tc(const Geometry& g, const IterWeightsTC& w, int r, const T* z_in, T* z_out, T* state,
                             bool last, cudaStream_t st) {
  if (g.C != 64 || g.S % kTW != 0) return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(z_in) | reinterpret_cast<uintptr_t>(z_out) |
       reinterpret_cast<uintptr_t>(state)) & 15)
    return cudaErrorInvalidValue;  // TMA global address alignment
  const int tps = g.S / kTW;
  const int tiles = g.n_slots * g.U * tps;
  if (tiles == 0) return cudaSuccess;
  const int smem = Lay<T>::DYN;
  cudaError_t e = ensure_smem<k_block2<T>>(smem);
  if (e != cudaSuccess) return e;
  const int planes = g.n_slots * g.U;
  CUtensorMap in_map, st_map, out_map;
  memset(&st_map, 0, sizeof(st_map));
  e = swizzled_map(&in_map, z_in, planes, g.S, kIW);
  if (e == cudaSuccess && last) e = swizzled_map(&st_map, static_cast<const T*>(state), planes, g.S, kIW);
  if (e == cudaSuccess) e = swizzled_map(&out_map, static_cast<const T*>(last ? state : z_out), planes, g.S, kTW);
  if (e != cudaSuccess) return e;
  const int want = (tiles + 1) / 2;
  const int grid = want < block_sms() ? want : block_sms();
  return launch_pdl(k_block2<T>, grid, kThreads, smem, st, tiles, tps, g.S, w.pw1[r], w.pw2[r], w.pw1_b[r],
                    w.pw2_b[r], w.dw1[r], w.dw2[r], last ? 1 : 0, w.err, in_map, st_map, out_map);
}

template cudaError_t launch_block16_tc<__nv_bfloat16>(const Geometry&, const IterWeightsTC&, int, const __nv_bfloat16*,
                                                     __nv_bfloat16*, __nv_bfloat16*, bool, cudaStream_t);
template cudaError_t launch_block16_tc<__half>(const Geometry&, const IterWeightsTC&, int, const __half*, __half*,
                                              __half*, bool, cudaStream_t);

NRX_DEBUG_READER(debug_read_block_tc)
