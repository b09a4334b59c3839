/*
 * nrx_eval.h - BLER evaluation support (same library, libnrx.so).
 *
 * The paper compares receivers by transport-block error rate with the 5G NR
 * LDPC code (Sec. IV).  This library measures block error rates with the
 * textbook rate-1/2, constraint-length-7 convolutional code (generators 133
 * and 171 octal, zero-tail terminated), so that receivers' LLRs can be
 * compared at matched BLER.  The decoder is the soft-input Viterbi algorithm
 * over the 64-state trellis.  The paper has no counterpart of this code.
 * It also decodes a 5G-structured quasi-cyclic LDPC code (nrx_ldpc_decode)
 * for transport-block error rates closer to the paper's (Fig. 3).
 *
 * Trellis conventions (shared with the transmitter in synth.py):
 *   state = the six most recent inputs, newest in bit 5; input u moves state
 *   s to (u << 5) | (s >> 1); output j of a transition is the parity of
 *   ((u << 6) | s) & g_j; the two outputs of step t are coded bits 2t, 2t+1.
 * Metric: LLR sign of Eq. 2 (l = ln P(c=1)/P(c=0)); a path's metric is the
 * sum of the LLRs of its 1-bits; FP32 add-compare-select in the order
 *   (PM[s] + (c0 ? l0 : 0)) + (c1 ? l1 : 0), the b = 1 predecessor
 * (((s' << 1) & 63) | 1) winning only when strictly larger, and the metric of
 * state 0 subtracted from every state after each step.  Start and end state 0.
 */
#ifndef NRX_EVAL_H_
#define NRX_EVAL_H_

#include <stddef.h>
#include <stdint.h>

#include "nrx.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Decode n_blocks code blocks of n_info information bits each
 * (2 (n_info + 6) coded bits per block).
 *   llr           device float32: coded bit i of block b is read at
 *                 llr[block_offset[b] + (perm ? perm[i] : i)]
 *   block_offset  device int64 [n_blocks]
 *   perm          device int32 [2 (n_info + 6)] (the interleaver: coded bit i
 *                 was sent at position perm[i] of the block), or NULL
 *   info_bits     device uint8 [n_blocks][n_info]: decoded bits (0/1)
 * 1 <= n_info <= 4096.  One warp decodes one block (trellis decisions in
 * shared memory, 8 bytes per step).  NRX_EINVAL on bad arguments.
 */
nrx_status nrx_conv_decode(int32_t n_blocks, int32_t n_info, const float* llr, const int64_t* block_offset,
                           const int32_t* perm, uint8_t* info_bits, void* stream);

/*
 * Layered normalised min-sum decoding of n_blocks code blocks of a
 * quasi-cyclic LDPC code with the TS 38.212 Sec. 5.3.2 structure (the
 * transport-block code the paper's receiver feeds, Sec. II; base graph given
 * by the caller), including the rate recovery of TS 38.212 Sec. 5.4.2.
 *   llr           device float32: block b's E received LLRs (Eq. 2 sign,
 *                 ln P(c=1)/P(c=0)) in transmission order start at
 *                 llr[block_offset[b]]
 *   block_offset  device int64 [n_blocks]
 *   E, qm         bits per block (a multiple of qm) and bits per modulation
 *                 symbol of the qm-row bit interleaver (1..8)
 *   Z, kb, mb     lifting size (1..384), systematic base columns, base rows
 *                 (1..64); nb = kb + mb codeword columns, the first 2 Z
 *                 codeword bits punctured, the circular buffer the other
 *                 (nb - 2) Z bits, read from its start (redundancy version 0)
 *   row_ptr, col, shift   HOST int32 edge lists of the base graph in row-major
 *                 order (row r's edges row_ptr[r] .. row_ptr[r+1]-1; column
 *                 in [0, nb); circulant shift >= 0, reduced mod Z): check
 *                 r Z + i meets variable col Z + ((i + shift) mod Z); at most
 *                 320 edges, 1..16 per row
 *   iterations    1..100 full passes over the rows in order; with stop_early
 *                 non-zero, decoding stops after a pass whose hard decisions
 *                 satisfy every check
 *   alpha         > 0, the min-sum normalisation (e.g. 0.75)
 *   c2v           device float32 scratch of n_blocks * nnz * Z values
 *                 (caller-owned; contents on return unspecified)
 *   info_bits     device uint8 [n_blocks][kb Z]: decoded systematic bits
 * One CTA of Z threads per block; the block's nb Z posteriors in shared
 * memory.  NRX_EINVAL on bad arguments (nothing launched), NRX_ECUDA on a
 * launch error.
 */
nrx_status nrx_ldpc_decode(int32_t n_blocks, const float* llr, const int64_t* block_offset, int32_t E, int32_t qm,
                           int32_t Z, int32_t kb, int32_t mb, const int32_t* row_ptr, const int32_t* col,
                           const int32_t* shift, int32_t iterations, float alpha, int32_t stop_early, float* c2v,
                           uint8_t* info_bits, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* NRX_EVAL_H_ */
