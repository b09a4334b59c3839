/*
 * nrx.h - C ABI of the B300 neural receiver (NRX) and LS+LMMSE receiver.
 *
 * The library computes, for one or more 5G NR PUSCH slots, per-bit LLRs of
 * every co-scheduled user from the received resource grid (system model,
 * Eq. 1, Sec. II), in two ways:
 *
 *   nrx_detect*   the convolutional-and-graph neural receiver of Sec. II-A:
 *                 DMRS LS estimate + linear interpolation + positional
 *                 encoding -> StateInit -> N_it CGNN iterations (per-RE
 *                 message passing over the other users, then a CNN update of
 *                 depthwise-separable residual blocks) -> ReadoutLLRs, masked
 *                 to each user's modulation order (Sec. III, masking).
 *   lmmse_detect* the classical "LS + LMMSE" baseline of Fig. 3: the same LS
 *                 estimate and interpolation, per-RE LMMSE equalisation with
 *                 unbiased scaling, max-log demapping over the user's Gray QAM.
 *
 * LLR sign (Eq. 2): llr = ln P(b=1 | y) / P(b=0 | y); positive means bit 1.
 *
 * All compute runs in CUDA kernels on the caller's stream; calls return once
 * the work is enqueued.  There is no CPU fallback: a context cannot be created
 * without a CUDA device.
 *
 * ------------------------------------------------------------------------
 * Data layouts (all little-endian, row-major, innermost index last)
 * ------------------------------------------------------------------------
 * y        complex64 (interleaved float re, im) [n_slots][B][14][S],
 *          S = 12 * num_prb, B = num_rx_ant of the context.
 * dmrs_seq complex64 [num_dmrs_symbols][S/2]: the DMRS base sequence r(m) of
 *          each DMRS symbol (non-zero values; normally unit-modulus QPSK).
 *          DMRS type 1: user/port u in {0,1,2,3} occupies CDM group g = u/2,
 *          i.e. subcarriers 2m+g, and sends w_u(m) r(m) with the frequency
 *          OCC w_u(m) = 1 for even u and (-1)^m for odd u.  DMRS symbols carry
 *          no data.
 * llr      float32, per slot the users' LLRs concatenated in user order; user
 *          u occupies n_data * m_u floats laid out [n_data][m_u], where the
 *          n_data = (14 - num_dmrs_symbols) * S data REs are ordered by
 *          symbol (ascending, DMRS symbols skipped) then subcarrier.  Slots
 *          follow each other without gaps (see nrx_llr_count).
 *
 * Weight blob (nrx_create): 32-byte header of eight int32
 *   {magic 0x5758524E, version 1, B, C, R, N_it, m_max, n_floats}
 * then n_floats float32 in this order (dense W is [out][in], y = W x + b;
 * depthwise k is [C][3][3] indexed [channel][symbol offset+1][subcarrier
 * offset+1], zero padding at the grid edges, no bias):
 *   init.pw.w [C][4B+2], init.pw.b [C], init.dw [C][3][3]
 *   for each iteration k < N_it:
 *     mp1.w [C][C], mp1.b [C], mp2.w [C][C], mp2.b [C],
 *     in.w [C][2C+2], in.b [C]                     (input order [S, a, PE])
 *     for each residual block r < R:
 *       dw1 [C][3][3], pw1.w [C][C], pw1.b [C], dw2 [C][3][3], pw2.w [C][C], pw2.b [C]
 *   ro1.w [C][C], ro1.b [C], ro2.w [m_max][C], ro2.b [m_max]
 * Network (Sec. II-A, this library's depthwise-separable layout):
 *   x_u   = [Re/Im y_b (b<B), Re/Im h_u,b (b<B), dt, df]   (4B+2 features)
 *           h_u = interpolated LS estimate; dt = (t - nearest DMRS symbol)/7,
 *           df = (s - nearest pilot subcarrier of u's CDM group)/2, ties to
 *           the lower index.
 *   S0    = ReLU(DW_init(PW_init(x_u)))
 *   per iteration: m_u = mp2(ReLU(mp1(S_u)));  a_u = sum_{v != u, active} m_v
 *           z = in([S_u, a_u, PE_u]);  R times z += pw2(ReLU(dw2(ReLU(pw1(dw1(z))))))
 *           S_u += z
 *   llr_u = ro2(ReLU(ro1(S_u)))[:m_u]
 *
 * Ownership: the caller owns y, dmrs_seq and llr buffers; the context owns
 * the device weights and every workspace, all allocated in nrx_create, so the
 * detect calls allocate nothing.
 * Thread safety: one context per host thread, or external locking.  Calls on
 * one context must not overlap on the GPU (they share the workspaces): issue
 * them on one stream, or order them.
 */
#ifndef NRX_H_
#define NRX_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nrx_ctx nrx_ctx;

typedef enum {
  NRX_OK = 0,
  NRX_EINVAL = 1,        /* bad argument; nothing was launched */
  NRX_ENOMEM = 2,        /* device allocation failed (nrx_create, first pipelined host call) */
  NRX_ECUDA = 3,         /* a CUDA call failed; see nrx_last_error */
  NRX_ETIMEDOUT = 4,     /* a bounded device-side wait gave up */
  NRX_EUNSUPPORTED = 5   /* valid but not supported by this build/context */
} nrx_status;

typedef enum {
  NRX_FP32 = 0,  /* CUDA-core FP32 arithmetic and FP32 activations */
  NRX_BF16 = 1,  /* tensor-core GEMMs (tcgen05) on BF16 operands with FP32
                    accumulation, BF16 activations; each weight matrix is split
                    into two BF16 parts (hi + lo, two MMA passes) */
  NRX_FP16 = 2,  /* tensor-core GEMMs on FP16 operands with FP32 accumulation,
                    FP16 activations (the paper's deployment precision, Sec. IV-A) */
  NRX_FP8 = 3    /* tensor-core GEMMs on E4M3 operands (per-row activation scales,
                    per-output-channel weight scales), FP32 accumulation, FP16
                    activations and depthwise; error reported, not bounded */
} nrx_precision;
/* The tensor-core modes need C = 64 (NRX_EUNSUPPORTED otherwise).  In every
 * mode depthwise taps, biases, ReLU, the cross-user sum, residual adds and
 * the last read-out layer are FP32 CUDA-core arithmetic. */

/* Per-slot configuration.  A host struct copied at call time. */
typedef struct {
  int32_t num_prb;            /* S = 12 * num_prb subcarriers; 1 <= num_prb <= max_prb */
  int32_t num_users;          /* U active users, ports 0..U-1; 1 <= U <= max_users (<= 4) */
  int32_t num_dmrs_symbols;   /* 1 or 2 */
  int32_t dmrs_symbols[2];    /* ascending symbol indices in [0, 13] */
  int32_t iterations;         /* CGNN iterations to run, 1..N_it; 0 means N_it
                                 (early exit of a multi-loss-trained net, Sec. IV-B) */
  float noise_var;            /* N0 (LMMSE only; the NRX has no N0 input) */
  const void* dmrs_seq;       /* device complex64 [num_dmrs_symbols][6*num_prb] */
} nrx_slot_cfg;

/*
 * Create a context: parse and upload the weight blob (host memory, see the
 * layout above), allocate every workspace for up to max_slots slots of up to
 * max_users users and max_prb PRBs.  precision selects the arithmetic of the
 * network layers.  On success *out receives the context.
 * Errors: NRX_EINVAL (blob header/size mismatch, B != num_rx_ant, limits out of
 * range: num_rx_ant in {1, 2, 4, 8}, 1<=max_users<=4, 1<=max_prb<=275,
 * 1<=max_slots<=64, C in {32, 64}), NRX_ENOMEM, NRX_ECUDA (no device).
 */
nrx_status nrx_create(const void* weights, size_t weights_bytes, int32_t num_rx_ant,
                      int32_t max_users, int32_t max_prb, int32_t max_slots,
                      nrx_precision precision, nrx_ctx** out);

/* Release the context and its device memory (synchronises the device first). */
void nrx_destroy(nrx_ctx* ctx);

/* Number of LLR floats one slot produces: (14 - num_dmrs_symbols) * 12 *
 * num_prb * sum_u bits_per_symbol[u]; 0 if the arguments are invalid. */
size_t nrx_llr_count(const nrx_slot_cfg* cfg, const int32_t* bits_per_symbol);

/*
 * NRX forward over n_slots slots of the same geometry (num_prb, num_users,
 * DMRS symbols and iterations equal; dmrs_seq and noise_var may differ).
 *   y               device, see layout; n_slots consecutive slots
 *   cfgs            host array [n_slots]
 *   bits_per_symbol host int32 [n_slots][num_users], each 2, 4 or 6 and <= m_max
 *   llr             device float32, slots back to back
 *   stream          cudaStream_t (NULL = legacy default stream)
 * Errors: NRX_EINVAL (n_slots > max_slots, geometry mismatch or beyond the
 * context limits, bad modulation order, misaligned pointer), NRX_ECUDA.
 */
nrx_status nrx_detect_batch(nrx_ctx* ctx, int32_t n_slots, const void* y, const nrx_slot_cfg* cfgs,
                            const int32_t* bits_per_symbol, float* llr, void* stream);

/* Single slot: nrx_detect_batch with n_slots = 1. */
nrx_status nrx_detect(nrx_ctx* ctx, const void* y, const nrx_slot_cfg* cfg,
                      const int32_t* bits_per_symbol, float* llr, void* stream);

/* LS + linear interpolation + LMMSE + max-log over n_slots slots, same
 * arguments and output layout as nrx_detect_batch (iterations is ignored). */
nrx_status lmmse_detect_batch(nrx_ctx* ctx, int32_t n_slots, const void* y, const nrx_slot_cfg* cfgs,
                              const int32_t* bits_per_symbol, float* llr, void* stream);

/* Single slot: lmmse_detect_batch with n_slots = 1. */
nrx_status lmmse_detect(nrx_ctx* ctx, const void* y, const nrx_slot_cfg* cfg,
                        const int32_t* bits_per_symbol, float* llr, void* stream);

/*
 * Number of REs whose LMMSE solve (lmmse_detect*) ran in FP64 on this
 * context since it was created or last reset.  The per-RE solve of the
 * LS + LMMSE receiver is FP32 except (a) every RE of a slot whose SNR
 * 10 log10(1/N0) exceeds 20 dB (noise_var < 0.01), and (b) any RE whose FP32
 * Cholesky factor of G = H^H H + N0 I has a non-positive pivot or pivots
 * that spread by more than 1e6; those are solved in FP64 (the channel
 * estimates and the demapper stay FP32).  Synchronises `stream`, copies the
 * counter into *count and, if `reset` is non-zero, sets it to zero.
 * NRX_EINVAL for a null argument, NRX_ECUDA on a CUDA error.
 */
nrx_status lmmse_fp64_count(nrx_ctx* ctx, int64_t* count, int32_t reset, void* stream);

/*
 * Bounds-checked build (the library compiled with -DNRX_DEBUG, e.g.
 * libnrx_debug.so from the package's build script): every instrumented
 * shared-memory and global index of the kernels is checked against the
 * extent of the array it addresses, and an index outside it is counted and
 * its access skipped (no device assertion, no fault).  Returns the number of
 * such indices since the last reset (all kernels, all devices' records read
 * on the current device) and the site number, index and extent of the first;
 * clears the records if `reset` is non-zero.  Call with no kernel running.
 * NRX_EUNSUPPORTED from the regular build, NRX_EINVAL for a null
 * `violations`, NRX_ECUDA on a CUDA error.
 */
nrx_status nrx_debug_counters(int64_t* violations, int32_t* first_site, int64_t* first_index,
                              int64_t* first_extent, int32_t reset);

/*
 * End-to-end variant of nrx_detect_batch on HOST buffers: y_host (complex64,
 * same layout), each cfgs[i].dmrs_seq a HOST pointer, llr_host float32.
 * Copies the inputs into context-owned device staging buffers, runs the NRX,
 * copies the LLRs back and synchronises the stream before returning.
 * Host buffers should be pinned for full copy bandwidth.
 */
nrx_status nrx_detect_batch_host(nrx_ctx* ctx, int32_t n_slots, const void* y_host,
                                 const nrx_slot_cfg* cfgs, const int32_t* bits_per_symbol,
                                 float* llr_host, void* stream);

/*
 * Pipelined form of nrx_detect_batch_host for a stream of batches: enqueue the
 * upload of y_host and of the pilots, the NRX, and the download of the LLRs
 * into llr_host, and return without waiting.  The context runs uploads,
 * compute and downloads on three internal streams with two staging sets, so
 * consecutive calls overlap: call k + 1 uploads while call k computes, and
 * call k downloads while call k + 1 computes.  Calls complete in order.
 * Arguments as nrx_detect_batch_host; cfgs and bits are read before the call
 * returns, but y_host, the pilots (cfgs[i].dmrs_seq) and llr_host must stay
 * valid and unmodified until nrx_host_drain returns.  Host buffers should be
 * pinned.  The first call creates the context's streams and a second staging
 * set (NRX_ENOMEM if that does not fit; a later call retries).  Every other
 * entry point drains the pipeline before it runs; device
 * calls issued on a stream of their own must have completed before a
 * pipelined call is made (the context's scratch is shared).
 */
nrx_status nrx_detect_batch_host_async(nrx_ctx* ctx, int32_t n_slots, const void* y_host,
                                       const nrx_slot_cfg* cfgs, const int32_t* bits_per_symbol,
                                       float* llr_host);

/* Wait for every pipelined call of the context; report device-side failures
 * as nrx_check does (NRX_ETIMEDOUT, NRX_ECUDA), else NRX_OK. */
nrx_status nrx_host_drain(nrx_ctx* ctx);

/*
 * Copy the CGNN state S (after the iterations run by the last nrx_detect*
 * call on this context) of batch slot `slot` into state_out: device float32
 * [num_users][14][S][C].  Ordered on `stream` after that call.
 */
nrx_status nrx_copy_state(nrx_ctx* ctx, int32_t slot, float* state_out, void* stream);

/*
 * NRX forward pass (FP32 arithmetic) over ONE slot that allocates no device
 * memory and needs no context.  The paper has no counterpart: this entry point
 * exists for callers that cannot call cudaMalloc, such as code running while a
 * stream is captured into a CUDA graph, real-time pipelines that fix their
 * device memory at start-up, or plug-ins whose host framework owns every GPU
 * allocation.
 *   weights_header  host: the blob's 32-byte header (layout above)
 *   weights_dev     device float32: the blob's n_floats payload, 16-byte aligned
 *   y, cfg, bits_per_symbol, llr, stream: as nrx_detect (y device, llr device)
 * The activation scratch is one static device array of 16 MiB per GPU that
 * loads the library (held until the process exits); its first MiB holds the
 * weights in kernel layout, the rest three FP32 activation tensors of
 * num_users * 14 * 12*num_prb * C floats each.  Larger slots are rejected with
 * NRX_EINVAL (e.g. C=64: up to 4 users x 27 PRB, 2 users x 55 PRB, 1 user x
 * 110 PRB).  The network must fit too: at most 121 layer tensors in its
 * iterations (N_it * (6 + 6 R) <= 121) and at most 1 MiB of weights in kernel
 * layout (C=64, R=2: N_it <= 7); larger nets get NRX_EINVAL from the header
 * alone, before anything is launched.  Every call re-lays the weights into
 * the array (one extra launch, up to 1 MiB of traffic).  The first call on
 * each device looks up the array's device address (cudaGetSymbolAddress) and
 * keeps it for the life of the process; make that first call before any
 * stream capture, and do not use this entry point across a cudaDeviceReset
 * (the kept address would be stale).
 * Every call shares the array and keeps the last call's contents (each kernel
 * writes scratch before reading it, so nothing needs clearing); calls whose
 * executions overlap on the GPU race on it and must be ordered.
 * Errors: NRX_EINVAL (bad header, net or slot beyond the limits, alignment),
 * NRX_ECUDA.
 */
nrx_status nrx_detect_noalloc(const void* weights_header, const float* weights_dev, const void* y,
                              const nrx_slot_cfg* cfg, const int32_t* bits_per_symbol, float* llr,
                              void* stream);

/*
 * PUSCH DMRS base sequences per TS 38.211 (the standard-compliant pilots of
 * Sec. II): for each slot i and DMRS symbol l,
 *   c_init = (2^17 (14 n_s + l + 1)(2 N_ID + 1) + 2 N_ID + n_SCID) mod 2^31
 *   (Sec. 6.4.1.1.1.1, transform precoding disabled, CDM groups 0 and 1),
 *   c(n) the length-31 Gold sequence of Sec. 5.2.1 (Nc = 1600),
 *   r(m) = ((1 - 2 c(2m)) + j (1 - 2 c(2m+1))) / sqrt(2),  m < 6 num_prb,
 * with the allocation starting at common resource block 0 (comb position m
 * carries r(m)).  Output: device complex64 [n_slots][num_dmrs_symbols][6 num_prb],
 * the dmrs_seq layout of nrx_slot_cfg.
 *   slot_numbers  host int32 [n_slots], each 0..159 (n_s within the frame)
 *   dmrs_symbols  host int32 [num_dmrs_symbols], each 0..13
 * 1 <= n_slots <= 64, 0 <= n_id <= 65535, n_scid in {0, 1}, 1 <= num_prb <= 275.
 * Errors: NRX_EINVAL, NRX_ECUDA.
 */
nrx_status nrx_dmrs_gold(int32_t n_slots, const int32_t* slot_numbers, int32_t n_id, int32_t n_scid,
                         int32_t num_prb, int32_t num_dmrs_symbols, const int32_t* dmrs_symbols, void* out,
                         void* stream);

/*
 * Synchronise `stream` and report device-side failures of the previous calls:
 * NRX_ETIMEDOUT if a kernel's bounded wait for its tensor-core work gave up
 * (the kernel then skipped its remaining tiles; the word is cleared), NRX_ECUDA
 * on a CUDA error, else NRX_OK.
 */
nrx_status nrx_check(nrx_ctx* ctx, void* stream);

/*
 * Failure-path diagnostic (no fault, no hang): enqueue on `stream` one CTA
 * whose thread 0 waits, with the same bounded mbarrier wait the tensor-core
 * kernels use, on a barrier that no thread arrives on.  After `limit_us`
 * microseconds (1..1,000,000) the wait gives up and the kernel sets the
 * context's device status word exactly as a real timeout does, so the next
 * nrx_check returns NRX_ETIMEDOUT (and clears it) and the context stays
 * usable.  NRX_EUNSUPPORTED for an FP32 context (it has no status word),
 * NRX_EINVAL for a bad limit.
 */
nrx_status nrx_expire_wait(nrx_ctx* ctx, int32_t limit_us, void* stream);

/* Network hyper-parameters of the context: B, C, R, N_it, m_max. */
nrx_status nrx_get_net(const nrx_ctx* ctx, int32_t* num_rx_ant, int32_t* channels,
                       int32_t* res_blocks, int32_t* iterations, int32_t* m_max);

/*
 * Per-kernel device timing.  While enabled, every kernel launch of the detect
 * calls is bracketed by two CUDA events on the launch stream (a few device
 * timestamps, no synchronisation).  Kernel kinds, in order:
 *   0 state_init, 1 message_passing, 2 residual_block, 3 readout, 4 lmmse.
 * nrx_profile_read waits for the recorded events, returns the kind's name,
 * summed duration in ms and launch count since the last reset, and clears all
 * kinds if reset != 0.  NRX_EINVAL for an unknown kind.
 */
#define NRX_KERNEL_KINDS 5
/* Turn the per-kernel event timing on (enable != 0) or off. */
nrx_status nrx_profile(nrx_ctx* ctx, int32_t enable);
/* Totals of kernel kind `kind` (name: static string owned by the library). */
nrx_status nrx_profile_read(nrx_ctx* ctx, int32_t kind, const char** name, double* total_ms,
                            int64_t* launches, int32_t reset);

/* Number of kernels the last nrx_detect* / lmmse_detect* call launched. */
int32_t nrx_last_launch_count(const nrx_ctx* ctx);

/* Human-readable message of the last error on this context ("" if none). */
const char* nrx_last_error(const nrx_ctx* ctx);

/* Static name of a status code. */
const char* nrx_status_string(nrx_status status);

#ifdef __cplusplus
}
#endif

#endif /* NRX_H_ */
