// Inline-PTX helpers for the Blackwell tensor-core path (sm_100a family):
// tcgen05 MMA with FP32 accumulators in tensor memory (TMEM), shared-memory
// matrix descriptors in the 128-byte-swizzle K-major layout, mbarriers with
// bounded waits.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// ---------------------------------------------------------------------------
// mbarrier
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Non-blocking probe of the phase of `parity`.
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase of `parity` to complete (try_wait suspends the thread in
// hardware until the phase flips or a short system limit); gives up after
// ~`limit_ns` (or 2^28 polls).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns = 1000000000ull) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  for (uint32_t i = 1; i < (1u << 28); ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 15) == 0 && globaltimer() - t0 > limit_ns) return false;
  }
  return false;
}

// Arrive on `bar` and add `bytes` to the transaction count it waits for (the
// bytes of the bulk tensor copies that complete on it).
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// TMA: copy the box at coordinates (x, y, z) of the 3-D tensor `map` into
// shared memory at dst; completion is signalled on `bar` (complete_tx).  x
// must be a multiple of 16 bytes / element size; y and z may lie outside the
// tensor (the fill value, zero, is read there).
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
          "r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// ---------------------------------------------------------------------------
// Fences
// ---------------------------------------------------------------------------
// Make generic-proxy shared-memory writes visible to the async proxy (MMA operand reads).
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// ---------------------------------------------------------------------------
// TMEM allocation (one full warp executes these)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t* slot_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot_smem)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// ---------------------------------------------------------------------------
// Descriptors
// ---------------------------------------------------------------------------
// Shared-memory matrix descriptor, K-major operand with 128-byte swizzle:
// rows of 64 BF16 (128 B), 8-row atoms of 1024 B stacked with a 1024 B stride
// (SBO); the atom base must be 1024-byte aligned.  Advancing K by 16 elements
// inside the atom adds 32 B to the start address.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address [0,14)
  d |= (uint64_t)1 << 16;                     // leading byte offset (unused for this layout)
  d |= (uint64_t)(1024 >> 4) << 32;           // stride byte offset [32,46)
  d |= (uint64_t)1 << 46;                     // descriptor version
  d |= (uint64_t)2 << 61;                     // 128-byte swizzle
  return d;
}

// Instruction descriptor of kind::f16: BF16 A and B (K-major), FP32 D.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Byte offset of element pair (row r, column c even) in a K-major SW128 tile
// with 64 BF16 columns per row.
__host__ __device__ __forceinline__ uint32_t sw128_offset(int r, int c) {
  const int chunk = c >> 3;  // 16-byte chunk (8 BF16)
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((chunk ^ (r & 7)) << 4) + ((c & 7) << 1));
}

// ---------------------------------------------------------------------------
// MMA: D[tmem] (+)= A[smem] * B[smem]^T, M=128, N, K=16, issued by one thread.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// D[tmem] (+)= A * B^T with 8-bit operands (kind::f8f6f4), M=128, N, K=32.
__device__ __forceinline__ void mma_f8(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Instruction descriptor of kind::f8f6f4: E4M3 A and B (K-major), FP32 D.
__host__ __device__ constexpr uint32_t idesc_e4m3_f32(int M, int N) {
  return (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// K = 64 GEMM tile of 8-bit operands stored in the first 64 bytes of each
// 128-byte swizzled row: 2 MMAs of K = 32 stepping 32 B inside the atom.
__device__ __forceinline__ void mma_k64_f8(uint32_t d_tmem, uint32_t a_saddr, uint32_t b_saddr, bool accumulate_first) {
#pragma unroll
  for (int k = 0; k < 2; ++k)
    mma_f8(d_tmem, desc_sw128(a_saddr + 32 * k), desc_sw128(b_saddr + 32 * k), idesc_e4m3_f32(128, 64),
           (k > 0 || accumulate_first) ? 1u : 0u);
}

// Arrive on `bar` once all previously issued MMAs of this thread complete.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// K = 64 GEMM tile: 4 MMAs of K = 16 stepping 32 B inside the swizzle atom.
__device__ __forceinline__ void mma_k64(uint32_t d_tmem, uint32_t a_saddr, uint32_t b_saddr, uint32_t idesc,
                                        bool accumulate_first) {
#pragma unroll
  for (int k = 0; k < 4; ++k)
    mma_bf16(d_tmem, desc_sw128(a_saddr + 32 * k), desc_sw128(b_saddr + 32 * k), idesc,
             (k > 0 || accumulate_first) ? 1u : 0u);
}

// ---------------------------------------------------------------------------
// TMEM -> registers: this warp's 32 lanes, 16 consecutive FP32 columns.  The
// values are valid only after tmem_wait16 on the same registers (the "+r"
// operands keep the compiler from using them before the wait).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait16(uint32_t (&r)[16]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                 "+r"(r[15])
               :
               : "memory");
}

// 32 FP32 columns of this thread's lane (row) into v.
__device__ __forceinline__ void tmem_row32(uint32_t taddr, float (&v)[32]) {
  uint32_t a[16], b[16];
  tmem_ld16(taddr, a);
  tmem_ld16(taddr + 16, b);
  tmem_wait16(a);
  tmem_wait16(b);
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    v[i] = __uint_as_float(a[i]);
    v[16 + i] = __uint_as_float(b[i]);
  }
}

// 64 FP32 columns of this thread's lane (row) into v.
__device__ __forceinline__ void tmem_row64(uint32_t taddr, float (&v)[64]) {
  uint32_t a[16], b[16], c[16], d[16];
  tmem_ld16(taddr, a);
  tmem_ld16(taddr + 16, b);
  tmem_ld16(taddr + 32, c);
  tmem_ld16(taddr + 48, d);
  tmem_wait16(a);
  tmem_wait16(b);
  tmem_wait16(c);
  tmem_wait16(d);
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    v[i] = __uint_as_float(a[i]);
    v[16 + i] = __uint_as_float(b[i]);
    v[32 + i] = __uint_as_float(c[i]);
    v[48 + i] = __uint_as_float(d[i]);
  }
}

// Bring the line holding p into L2 (no register result, no ordering).
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// d = a * b + c on both FP32 lanes (one packed instruction).
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;"
      : "=l"(d)
      : "l"(*reinterpret_cast<unsigned long long*>(&a)), "l"(*reinterpret_cast<unsigned long long*>(&b)),
        "l"(*reinterpret_cast<unsigned long long*>(&c)));
  return *reinterpret_cast<float2*>(&d);
}

// Sliding 3x3 depthwise over the 14 symbols of one column for one channel
// pair: in(ti, k) returns the input of symbol ti, column offset k in {0,1,2};
// out(t, v) receives the output of symbol t.  Zero padding in time.
template <typename In, typename Out>
__device__ __forceinline__ void dw_column(const float2 (&kk)[9], In in, Out out) {
  float2 am = make_float2(0.f, 0.f), a0 = am, ap = am;
#pragma unroll
  for (int ti = 0; ti < 14; ++ti) {
    float2 x[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) x[k] = in(ti, k);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      am = ffma2(kk[6 + k], x[k], am);  // contributes to output ti-1 (tap row +1)
      a0 = ffma2(kk[3 + k], x[k], a0);  // output ti (tap row 0)
      ap = ffma2(kk[k], x[k], ap);      // output ti+1 (tap row -1)
    }
    if (ti >= 1) out(ti - 1, am);
    am = a0;
    a0 = ap;
    ap = make_float2(0.f, 0.f);
  }
  out(14 - 1, am);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&h);
}
__device__ __forceinline__ float2 unpack_bf16x2(uint32_t w) {
  return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xFFFF0000u));
}
// max(x, 0) of a pair, rounded to nearest into one packed bf16x2 / f16x2 word
// (low half = lo) by a single conversion.
__device__ __forceinline__ uint32_t pack_relu_bf16x2(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}
__device__ __forceinline__ uint32_t pack_relu_f16x2(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.relu.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}
// 32-bit store to a shared-memory address (state space known: no address
// conversion, and the caller's precomputed address + constant folds).
__device__ __forceinline__ void sts32(uint32_t addr, uint32_t v) {
  asm volatile("st.shared.b32 [%0], %1;" ::"r"(addr), "r"(v));
}
// TMA: store the box at coordinates (x, y, z) of `map` from shared memory at
// src as one bulk async-group operation (coordinates not negative; elements
// outside the tensor are not written).
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, int x, int y, int z, const void* src) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(y), "r"(z), "r"(smem_u32(src))
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// Wait until the committed bulk stores have read their shared-memory source /
// have completed.
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// Programmatic dependent launch: let the next kernel on the stream start its
// prologue now / wait until the previous kernel's writes are visible.
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// a + b on a pair (one packed FP32 instruction; a * 1 + b rounds once, like an add).
__device__ __forceinline__ float2 fadd2(float2 a, float2 b) { return ffma2(a, make_float2(1.f, 1.f), b); }

}  // namespace tc
