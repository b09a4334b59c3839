/*
 * nrx_eval.h - BLER evaluation support (same library, libnrx.so).
 *
 * The paper compares receivers by transport-block error rate with the 5G NR
 * LDPC code (Sec. IV).  This library measures block error rates with the
 * textbook rate-1/2, constraint-length-7 convolutional code (generators 133
 * and 171 octal, zero-tail terminated), so that receivers' LLRs can be
 * compared at matched BLER.  The decoder is the soft-input Viterbi algorithm
 * over the 64-state trellis.  The paper has no counterpart of this code.
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

#ifdef __cplusplus
}
#endif

#endif /* NRX_EVAL_H_ */
