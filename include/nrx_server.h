/*
 * nrx_server.h - Real-time serving loop for the NRX (same library, libnrx.so).
 *
 * The paper's deployment constraint (Sec. IV-A) is a per-slot latency budget
 * under real-time operation with intra-frame parallelism only.  This server
 * takes PUSCH slots as they arrive (several cells, each slot with its own PRB
 * count and user count), groups pending slots of equal geometry into batches
 * on the fly (continuous batching), and runs each batch through the NRX, or,
 * when the NRX cannot finish a slot before its deadline, through the LS+LMMSE
 * receiver of Fig. 3 (fallback).  The paper has no counterpart of this loop.
 *
 * Design:
 *   - one NRX context (nrx.h) per PRB bucket and two lanes, each a CUDA stream
 *     with its own staging buffers: the NRX lane and the fallback lane
 *     (LS+LMMSE), so that a fallback never waits behind an NRX batch; batches
 *     of one lane run in order, lanes and buckets run concurrently;
 *   - admission by device-memory budget: at creation each bucket gets the
 *     largest batch capacity (<= max_batch, halving) whose context and
 *     staging fit in what remains of hbm_budget_bytes; at run time a request
 *     whose bucket queue is full is rejected (backpressure);
 *   - a worker thread per bucket moves every queued slot that the NRX lane cannot
 *     finish before its deadline, even alone once the lane is free, to the
 *     fallback lane; each idle NRX lane takes the pending slots of one user
 *     count, earliest deadline first, as many as the measured execution time
 *     allows before the earliest deadline; each idle fallback lane takes up
 *     to a batch of its queue;
 *   - an NRX batch runs as a CUDA graph: the receiver's launch sequence is
 *     captured once per (bucket, user count, batch size, modulation orders)
 *     on the lane's fixed staging buffers and replayed after (up to 256
 *     graphs per bucket; the uploads and downloads, whose host addresses
 *     change, are issued around it);
 *   - execution times per (bucket, users, batch size, receiver) are measured
 *     at creation (calibration launches) and tracked with an exponential
 *     moving average of the CUDA-event times of served batches;
 *   - completion times come from CUDA events (converted to the host's
 *     steady clock through a reference event), not from polling.
 * A slot's LLRs do not depend on which other slots share its batch (every
 * kernel works per slot), so serving is batch-invariant bit for bit.
 *
 * Threading: submit, poll and stats may be called from any one host thread
 * at a time while the worker runs; the server owns its CUDA streams.
 */
#ifndef NRX_SERVER_H_
#define NRX_SERVER_H_

#include <stddef.h>
#include <stdint.h>

#include "nrx.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nrx_server nrx_server;

#define NRX_SERVER_MAX_BUCKETS 8

typedef struct {
  int32_t num_buckets;                          /* 1..8 */
  int32_t bucket_prb[NRX_SERVER_MAX_BUCKETS];   /* the PRB counts served (each 1..275) */
  int32_t max_users;                            /* 1..4 */
  int32_t max_batch;                            /* slots per launch, 1..64 */
  int32_t queue_capacity;                       /* pending slots per bucket before rejection, >= 1 */
  int32_t num_dmrs_symbols;                     /* 1 or 2 */
  int32_t dmrs_symbols[2];
  int32_t precision;                            /* nrx_precision of the NRX contexts */
  double deadline_us;                           /* latency budget of a slot from its arrival */
  size_t hbm_budget_bytes;                      /* device memory the server may take */
} nrx_server_cfg;

typedef struct {
  int32_t num_prb;              /* must equal one bucket_prb */
  int32_t num_users;            /* 1..max_users */
  int32_t bits_per_symbol[4];   /* m_u of users 0..num_users-1 (2, 4 or 6, <= m_max) */
  float noise_var;              /* N0 (used by the LMMSE fallback) */
  const void* y_host;           /* pinned host complex64 [B][14][12 num_prb] */
  const void* dmrs_host;        /* pinned host complex64 [n_dmrs][6 num_prb], or NULL: the server
                                   generates the cell's TS 38.211 pilots on the device from
                                   n_id and slot_number (nrx_dmrs_gold, n_SCID = 0) */
  float* llr_host;              /* pinned host float32, nrx_llr_count floats (written on completion) */
  int64_t arrival_ns;           /* arrival time on the steady clock (nrx_server_now_ns); 0 = now */
  int32_t n_id;                 /* DMRS scrambling identity of the cell (0..65535; with dmrs_host NULL) */
  int32_t slot_number;          /* slot index within the frame (0..159; with dmrs_host NULL) */
} nrx_request;

typedef struct {
  uint64_t ticket;
  int32_t receiver;             /* 0 NRX, 1 LS+LMMSE fallback, -1 rejected (queue full) */
  int32_t status;               /* nrx_status of the batch */
  int32_t batch_size;           /* slots in the launch that served it */
  int32_t bucket;
  int64_t arrival_ns;
  int64_t done_ns;              /* LLRs in llr_host (D2H copy complete) */
} nrx_completion;

typedef struct {
  int64_t submitted, served_nrx, served_lmmse, rejected, launches;
  int32_t bucket_batch_capacity[NRX_SERVER_MAX_BUCKETS];  /* after admission */
  size_t device_bytes;          /* device memory taken by the server */
  int64_t graph_launches;       /* NRX batches run by replaying a captured CUDA graph */
  int64_t graphs_captured;
  int64_t direct_launches;      /* NRX batches launched kernel by kernel (composition not captured yet) */
  int64_t enqueue_ns_graph;     /* host time spent enqueueing the NRX on each path (sums) */
  int64_t enqueue_ns_direct;
} nrx_server_stats;

/* Create the server: contexts per bucket (weights blob as nrx_create),
 * admission against hbm_budget_bytes, calibration launches, worker thread.
 * Errors: NRX_EINVAL (bad config or blob), NRX_ENOMEM (not even batch 1 of a
 * bucket fits the budget or the device), NRX_ECUDA. */
nrx_status nrx_server_create(const void* weights, size_t weights_bytes, int32_t num_rx_ant,
                             const nrx_server_cfg* cfg, nrx_server** out);

/* Stop the worker after the in-flight batches finish and free everything. */
void nrx_server_destroy(nrx_server* srv);

/* The server's clock (steady clock, ns) for nrx_request.arrival_ns. */
int64_t nrx_server_now_ns(void);

/* Queue one slot; *ticket identifies its completion.  A full bucket queue
 * produces a completion with receiver = -1 instead.  NRX_EINVAL for a
 * request that matches no bucket or is malformed (nothing queued). */
nrx_status nrx_server_submit(nrx_server* srv, const nrx_request* req, uint64_t* ticket);

/* Trace replay (load generation without host-language timing jitter): submit
 * reqs[0..n) in order, each when the steady clock reaches its arrival_ns
 * (spinning in the calling thread; requests whose time has passed are
 * submitted at once).  Returns after the last submission; tickets[i] (if not
 * NULL) receives request i's ticket and *max_late_ns the largest delay
 * between a request's arrival_ns and its submission. */
nrx_status nrx_server_replay(nrx_server* srv, int32_t n, const nrx_request* reqs, uint64_t* tickets,
                             int64_t* max_late_ns);

/* Move up to max_out completions into out (oldest first); *n receives the count. */
nrx_status nrx_server_poll(nrx_server* srv, nrx_completion* out, int32_t max_out, int32_t* n);

/* Block until every submitted slot has completed (or timeout_ms passed:
 * NRX_ETIMEDOUT). */
nrx_status nrx_server_drain(nrx_server* srv, int32_t timeout_ms);

/* Copy the server's counters (nrx_server_stats: served / fallback / rejected
 * slots, launches, graph replays, admitted batch capacities, device bytes)
 * into *out.  NRX_EINVAL for null arguments. */
nrx_status nrx_server_get_stats(const nrx_server* srv, nrx_server_stats* out);

#ifdef __cplusplus
}
#endif

#endif /* NRX_SERVER_H_ */
