/*
 * nrx_train.h - C ABI of the NRX training kernels (same library, libnrx.so).
 *
 * Training scheme (Sec. II-B): empirical risk minimisation of the binary
 * cross-entropy between the LLRs of ReadoutLLRs and the transmitted bits,
 * plus gamma times the mean-squared error of a second read-out head
 * (ReadoutChEst) against the true channel ("double read-out"), with the
 * read-outs applied after every CGNN iteration and the losses summed
 * (multi-loss, Sec. II-B), Var-MCS masking of the LLR outputs (Sec. III) and
 * per-sample random MCS-to-user association with SNR offsets (Sec. IV-A).
 * Weights are updated with Adam.
 *
 * These are the layer-level building blocks of that scheme: each call runs
 * one forward or backward step of one layer kind over a batch of REs on the
 * caller's stream (FP32 CUDA-core arithmetic, FP32 activations).  The caller
 * composes them into the network's forward pass with saved activations and
 * the reverse pass (see the Python trainer), and owns every buffer.
 *
 * Common conventions
 *   - All pointers are device pointers unless stated; float32 unless stated.
 *   - Activations of one layer are row-major matrices [rows][width]; a row is
 *     one RE of one user of one slot, rows ordered [slot][user][symbol t (14)]
 *     [subcarrier s] — so a "plane" (slot, user) is a 14 x S grid.
 *   - stream is a cudaStream_t (NULL = legacy default stream).
 *   - Calls return once the work is enqueued.  NRX_EINVAL: bad argument,
 *     nothing launched.  NRX_ECUDA: the launch failed.
 *   - No call allocates memory.
 */
#ifndef NRX_TRAIN_H_
#define NRX_TRAIN_H_

#include <stddef.h>
#include <stdint.h>

#include "nrx.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Network input features (Sec. II-A) of every user of n_slots slots of one
 * geometry: x [n_slots][U][14][S][4B+2] with the feature order of nrx.h
 * (Re/Im y per antenna, Re/Im interpolated LS estimate per antenna, dt, df).
 *   y     complex64 [n_slots][B][14][S]
 *   cfgs  host array [n_slots]; num_prb, num_users and DMRS symbols taken from
 *         cfgs[0] (all slots must agree), dmrs_seq per slot (device).
 * 1 <= n_slots <= 64, 1 <= num_rx_ant <= 8.
 */
nrx_status nrx_train_features(int32_t n_slots, int32_t num_rx_ant, const void* y, const nrx_slot_cfg* cfgs,
                              float* x, void* stream);

/*
 * Strided matrix product with epilogue:
 *   C[m][n] = act(sum_k A(m,k) B(k,n) + bias[n] + R[m][n])       (accumulate = 0)
 *   C[m][n] += sum_k A(m,k) B(k,n)                                (accumulate != 0)
 * with A(m,k) = A[m*sam + k*sak], B(k,n) = B[k*sbk + n*sbn], C row stride ldc,
 * R row stride ldr.  act is ReLU when relu != 0.  bias and R may be NULL; R may
 * equal C (in-place residual add).  One call covers a dense layer y = W x + b
 * (B(k,n) = W[n][k]), its input gradient dx = dy W (B(k,n) = W[k][n]) and its
 * weight gradient dW += dy^T x (A(m,k) = dy[k][m], accumulate = 1).
 * split_k (>= 1) splits the K range over CTAs; split_k > 1 requires
 * accumulate.  Accumulation uses float atomics (summation order varies).
 */
nrx_status nrx_train_gemm(int32_t M, int32_t N, int32_t K, const float* A, int64_t sam, int64_t sak, const float* B,
                          int64_t sbk, int64_t sbn, const float* bias, const float* R, int64_t ldr, float* C,
                          int64_t ldc, int32_t relu, int32_t accumulate, int32_t split_k, void* stream);

/*
 * nrx_train_gemm with BF16 tensor-core compute (tcgen05, kind::f16): the same
 * arguments, layouts, epilogues and errors; A and B are rounded to BF16
 * (round to nearest even) as they are staged, products accumulate in FP32.
 * One CTA per 128 x 64 output tile and K range (split_k ranges, each a whole
 * number of 64-wide chunks).  A bounded wait for the tensor cores that gives
 * up sets a device flag (nrx_train_check) and leaves the tile unwritten.
 */
nrx_status nrx_train_gemm_bf16(int32_t M, int32_t N, int32_t K, const float* A, int64_t sam, int64_t sak,
                               const float* B, int64_t sbk, int64_t sbn, const float* bias, const float* R,
                               int64_t ldr, float* C, int64_t ldc, int32_t relu, int32_t accumulate, int32_t split_k,
                               void* stream);

/* Synchronise `stream`; NRX_ETIMEDOUT (and clear the flag) if a tensor-core
 * training GEMM gave up waiting since the last check, NRX_ECUDA on a CUDA
 * error, else NRX_OK. */
nrx_status nrx_train_check(void* stream);

/* out[n] += sum_m X[m*ldx + n], n < N (bias gradients). */
nrx_status nrx_train_colsum(int32_t M, int32_t N, const float* X, int64_t ldx, float* out, void* stream);

/*
 * Depthwise 3x3 layer over `planes` grids of 14 x S with C channels,
 * X, Y [planes][14][S][C], taps k [C][3][3], zero "same" padding:
 *   Y[t][s][c] = act(sum_{i,j} k[c][i][j] X[t+i-1][s+j-1][c])
 * flip != 0 reads the taps as k[c][2-i][2-j] (the adjoint: with flip, the call
 * maps an output gradient to the input gradient).  act is ReLU when relu != 0.
 * X and Y must not overlap.
 */
nrx_status nrx_train_dw3(int32_t planes, int32_t S, int32_t C, const float* X, const float* k, int32_t flip,
                         int32_t relu, float* Y, void* stream);

/* Tap gradient of nrx_train_dw3: gk[c][i][j] += sum G[t][s][c] X[t+i-1][s+j-1][c]
 * over all planes, t, s (zero padding).  Float atomics.  1 <= C <= 1024. */
nrx_status nrx_train_dw3_wgrad(int32_t planes, int32_t S, int32_t C, const float* X, const float* G, float* gk,
                               void* stream);

/* ReLU backward, in place: G[i] = 0 where Y[i] <= 0 (Y the ReLU output). */
nrx_status nrx_train_relu_mask(int64_t n, float* G, const float* Y, void* stream);

/*
 * Message aggregation of the CGNN (Sec. II-A): for m, a [n_slots][U][per_user],
 *   a[sl][u][e] = sum_{v != u} m[sl][v][e].
 * The map is symmetric, so the same call maps the gradient of a to the
 * gradient of m.  1 <= U <= 4; m and a must differ.
 */
nrx_status nrx_train_aggregate(int32_t n_slots, int32_t num_users, int64_t per_user, const float* m, float* a,
                               void* stream);

/* y[i] += alpha * x[i], i < n. */
nrx_status nrx_train_axpy(int64_t n, float alpha, const float* x, float* y, void* stream);

/*
 * Masked BCE of one LLR read-out (Sec. II-B; LLR sign of Eq. 2, so
 * P(b=1) = sigmoid(l)), as a mean over the counted bits:
 *   *loss += weight / n_bits * sum (softplus(l) - b l)     (FP64 accumulation)
 *   grad   = weight / n_bits * (sigmoid(l) - b)             on counted entries, else 0
 * over the data REs (DMRS symbols of cfg skipped) and the first m_u outputs of
 * each user (Var-MCS masking, Sec. III); n_bits = n_data * sum of m_u over the
 * batch, computed on the device from bits_per_symbol_dev (so a captured graph
 * stays valid when the modulation orders of the batch change).
 *   llr, grad             [n_slots][U][14][S][m_max]
 *   bits                  uint8 [n_slots][U][n_data][m_max], n_data REs in the
 *                         order symbol (DMRS skipped) then subcarrier; entries
 *                         at j >= m_u are ignored
 *   bits_per_symbol_dev   device int32 [n_slots][U] (m_u)
 *   cfg                   host; num_prb, num_users, DMRS symbols of the batch
 * 2 <= m_max <= 8.
 */
nrx_status nrx_train_bce(int32_t n_slots, const nrx_slot_cfg* cfg, int32_t m_max, const float* llr,
                         const uint8_t* bits, const int32_t* bits_per_symbol_dev, float weight, float* grad,
                         double* loss, void* stream);

/*
 * Squared error of the channel-estimate read-out (Sec. II-B, double read-out):
 *   *loss += scale * sum_i (h_hat[i] - h[i])^2;  grad[i] = 2 scale (h_hat[i] - h[i]).
 */
nrx_status nrx_train_mse(int64_t n, const float* h_hat, const float* h, float scale, float* grad, double* loss,
                         void* stream);

/*
 * GPU link simulator for training data (system model, Eq. 1): per slot the
 * users' bits -> Gray QAM (TS 38.211 Sec. 5.1), QPSK DMRS on the type-1 comb
 * with the frequency OCC (DMRS symbols carry no data), a tapped delay line per
 * user (L taps at l 4 DS/(L-1), exponential power-delay profile normalised to
 * one; a Clarke sum of 16 sinusoids per tap for Doppler > 0, CN(0, 1) static
 * gains otherwise; a half-wavelength ULA with one arrival angle in
 * [-60, 60] degrees per tap, or independent gains per antenna), AWGN of
 * variance noise_var.  Subcarrier s sits at (s - S/2) 30 kHz, symbol t at
 * t 0.5 ms / 14.
 * Random numbers: Philox4x32-10 (Salmon et al., SC'11), key = (seed low,
 * seed high), counter = (index low, index high, batch, stream); stream 1 bits
 * (index (slot U + u) n_data + re, bit j of word 0), 2 DMRS (index
 * (slot n_dmrs + d) S/2 + m, bits 0 and 1 of word 0 are the QPSK signs of Re
 * and Im), 3 noise (index ((slot B + b) 14 + t) S + s, Box-Muller of words 0
 * and 1), 4-8 tap gains (index ((slot U + u) L + l) Bd + bd, Bd = 1 for a ULA
 * else B; stream 4 word 0 the arrival rotation, or words 0 and 1 a Box-Muller
 * static gain; streams 5-8 words 0-3 the 16 sinusoid phases), 9 arrival
 * angles (index (slot U + u) L + l).  Uniform u(x) = (x >> 8) 2^-24;
 * Box-Muller u1 = ((x0 >> 8) + 1) 2^-24, u2 = u(x1).
 * Outputs, in the layouts of nrx_train_features / nrx_train_bce /
 * nrx_train_mse: y complex64 [n][B][14][S], dmrs complex64 [n][n_dmrs][S/2],
 * bits uint8 [n][U][n_data][m_max] (zero beyond m_u), bits_per_symbol_dev
 * int32 [n][U], h float32 [n][U][14][S][2B] (the true channel).
 * scratch: device memory of nrx_train_sim_scratch_bytes(n, U, B, max taps).
 * 1 <= n <= 64, 1 <= U <= 4, 1 <= B <= 8, 1 <= num_prb <= 275, taps 1..32.
 */
typedef struct {
  float noise_var;           /* N0 (unit average symbol energy and channel power) */
  float delay_spread_s;      /* DS > 0 */
  float doppler_hz;          /* maximum Doppler, >= 0 (0: static channel) */
  int32_t num_taps;          /* L, 1..32 */
  int32_t ula;               /* 1: half-wavelength ULA, 0: independent antennas */
  int32_t bits_per_symbol[4];
} nrx_sim_slot;

/* Bytes of device scratch nrx_train_simulate needs for n_slots slots of
 * num_users users, num_rx_ant antennas and up to max_taps taps (0 for
 * arguments out of range). */
size_t nrx_train_sim_scratch_bytes(int32_t n_slots, int32_t num_users, int32_t num_rx_ant, int32_t max_taps);

/* Draw one training batch on `stream` as described above: per-slot
 * parameters in slots[n_slots] (host), batch index `batch` and `seed` select
 * the Philox counters; outputs in device memory (layouts above).  NRX_EINVAL
 * for out-of-range arguments, NRX_ECUDA on a launch failure. */
nrx_status nrx_train_simulate(int32_t n_slots, const nrx_sim_slot* slots, int32_t num_users, int32_t num_rx_ant,
                              int32_t num_prb, int32_t num_dmrs_symbols, const int32_t* dmrs_symbols, int32_t m_max,
                              uint64_t seed, uint32_t batch, void* scratch, void* y, void* dmrs, uint8_t* bits,
                              int32_t* bits_per_symbol_dev, float* h, void* stream);

/*
 * Var-IO head selection (Sec. III): activations [planes][rows_per_plane][*]
 * (a plane is one (slot, user)); for the planes whose modulation order
 * bits_per_symbol_dev[plane] equals m_head, dst[row][c] = src[row][c] (or +=
 * with accumulate), c < width; other planes get dst = 0 (unchanged with
 * accumulate).  Row strides ld_src, ld_dst >= width.  Used to assemble the
 * per-user StateInit and read-out of the matching head in the forward pass
 * and to route the gradient to that head in the reverse pass.
 */
nrx_status nrx_train_plane_mask(int64_t planes, int64_t rows_per_plane, int32_t width, int64_t ld_src, int64_t ld_dst,
                                const int32_t* bits_per_symbol_dev, int32_t m_head, const float* src, float* dst,
                                int32_t accumulate, void* stream);

/* Asynchronous zero fill of `bytes` bytes at ptr (gradient and loss reset). */
nrx_status nrx_train_zero(int64_t bytes, void* ptr, void* stream);

/* Asynchronous copy of `bytes` bytes between any two of device, pinned-host or
 * pageable-host memory (direction inferred from the unified address space;
 * pageable host memory makes the copy synchronous).  src and dst must not
 * overlap.  Used for the gradient-path copies and the batch uploads. */
nrx_status nrx_train_copy(int64_t bytes, void* dst, const void* src, void* stream);

/*
 * One Adam step on n FP32 weights, in place:
 *   m1 = b1 m1 + (1-b1) g;  m2 = b2 m2 + (1-b2) g^2;  w -= lr_t m1 / (sqrt(m2) + eps)
 * lr_t points to one float in device memory: the caller's bias-corrected step
 * size lr sqrt(1-b2^t) / (1-b1^t), read when the kernel runs (so a captured
 * CUDA graph of the training step picks up each step's value).
 */
nrx_status nrx_train_adam(int64_t n, float* w, const float* g, float* m1, float* m2, const float* lr_t,
                          float beta1, float beta2, float eps, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* NRX_TRAIN_H_ */
