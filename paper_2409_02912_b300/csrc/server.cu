// Real-time serving loop: continuous batching of arriving slots per PRB
// bucket, deadline-aware dispatch with an LS+LMMSE fallback, admission by a
// device-memory budget (see include/nrx_server.h).  Host code; the compute is
// the nrx_detect_batch / lmmse_detect_batch calls of nrx_api.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <cstddef>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/nrx_server.h"

namespace {

constexpr int kSymbols = 14;
constexpr int kMaxUsers = 4;
constexpr int kRcvNrx = 0, kRcvLmmse = 1;
constexpr size_t kMaxGraphs = 256;  // captured NRX launch sequences per bucket
static_assert(sizeof(nrx_request) == 72 && offsetof(nrx_request, slot_number) == 68, "nrx_request layout");
static_assert(sizeof(nrx_completion) == 40 && sizeof(nrx_server_stats) == 120, "serving ABI layout");

int64_t steady_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct Pending {
  uint64_t ticket;
  nrx_request req;
  int64_t deadline_ns;
};

struct Inflight {
  bool active = false;
  int users = 0, n = 0;
  std::vector<Pending> reqs;
  cudaEvent_t start = nullptr, done = nullptr;
};

// One execution lane of a bucket: a stream with its own staging buffers.
// Lane 0 runs the NRX, lane 1 the LS+LMMSE fallback, so that a fallback
// never waits behind an NRX batch.
struct Lane {
  cudaStream_t st = nullptr;
  float2* y = nullptr;
  float2* dmrs = nullptr;
  float* llr = nullptr;
  Inflight cur;
  cudaEvent_t ref = nullptr;
  int64_t ref_ns = 0;
  int64_t busy_until_ns = 0;  // predicted end of the in-flight batch
};

struct Bucket {
  int prb = 0, S = 0, cap = 0;
  nrx_ctx* ctx = nullptr;
  Lane lane[2];
  std::deque<Pending> inbox;  // submitted, not yet seen by the bucket's worker (guarded by the server mutex)
  std::deque<Pending> q[2][kMaxUsers + 1];  // [lane][users], arrival (= deadline) order
  int queued = 0;
  std::vector<double> est_us[2][kMaxUsers + 1];  // [lane][users][n], n <= cap
  // (users, n, m_u...) -> captured NRX launch sequence; nullptr while the
  // composition waits in `to_capture` for an idle moment of the worker
  std::map<std::vector<int32_t>, cudaGraphExec_t> graphs;
  std::deque<std::vector<int32_t>> to_capture;
  cudaStream_t capture_st = nullptr;
};

}  // namespace

struct nrx_server {
  nrx_server_cfg cfg{};
  int B = 0, m_max = 0, device = 0;
  std::vector<Bucket> buckets;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<nrx_completion> done;
  std::atomic<bool> stop{false};
  std::atomic<bool> abandon{false};  // stop without waiting for in-flight batches (drain timed out)
  std::atomic<int64_t> outstanding{0};
  std::vector<std::thread> workers;  // one per bucket
  nrx_server_stats stats{};
  uint64_t next_ticket = 1;
};

namespace {

void complete(nrx_server* s, const Pending& p, int receiver, int status, int batch, int bucket, int64_t done_ns) {
  nrx_completion c{};
  c.ticket = p.ticket;
  c.receiver = receiver;
  c.status = status;
  c.batch_size = batch;
  c.bucket = bucket;
  c.arrival_ns = p.req.arrival_ns;
  c.done_ns = done_ns;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->done.push_back(c);
    if (receiver == kRcvNrx) s->stats.served_nrx++;
    if (receiver == kRcvLmmse) s->stats.served_lmmse++;
    if (receiver < 0) s->stats.rejected++;
  }
  s->outstanding.fetch_sub(1);
}

size_t slot_llr_floats(int S, int n_dmrs, int users, int m_max) {
  return (size_t)(kSymbols - n_dmrs) * S * users * m_max;
}

std::vector<nrx_slot_cfg> slot_cfgs(const nrx_server* s, const Bucket& b, const Lane& L, int n, int users,
                                    const std::vector<Pending>* reqs) {
  const nrx_server_cfg& c = s->cfg;
  const size_t d_per = (size_t)c.num_dmrs_symbols * (b.S / 2);
  std::vector<nrx_slot_cfg> cfgs(n);
  for (int i = 0; i < n; ++i) {
    nrx_slot_cfg& sc = cfgs[i];
    memset(&sc, 0, sizeof(sc));
    sc.num_prb = b.prb;
    sc.num_users = users;
    sc.num_dmrs_symbols = c.num_dmrs_symbols;
    sc.dmrs_symbols[0] = c.dmrs_symbols[0];
    sc.dmrs_symbols[1] = c.dmrs_symbols[c.num_dmrs_symbols - 1];
    sc.iterations = 0;
    sc.noise_var = reqs ? (*reqs)[i].req.noise_var : 0.1f;
    sc.dmrs_seq = L.dmrs + i * d_per;
  }
  return cfgs;
}

// The NRX launch sequence of a batch composition: replayed from its captured
// CUDA graph when there is one, else launched directly and the composition
// queued for capture (capture and instantiation cost host time, so they run
// only when the bucket's worker is idle, never in front of a waiting batch).
nrx_status run_nrx_batch(nrx_server* s, Bucket& b, Lane& L, int n, const nrx_slot_cfg* cfgs, const int32_t* bits,
                         int users) {
  const int64_t t0 = steady_ns();
  std::vector<int32_t> key = {users, n};
  key.insert(key.end(), bits, bits + (size_t)n * users);
  auto it = b.graphs.find(key);
  if (it != b.graphs.end() && it->second) {
    if (cudaGraphLaunch(it->second, L.st) != cudaSuccess) return NRX_ECUDA;
    const int64_t dt = steady_ns() - t0;
    std::lock_guard<std::mutex> lk(s->mu);
    s->stats.graph_launches++;
    s->stats.enqueue_ns_graph += dt;
    return NRX_OK;
  }
  if (it == b.graphs.end() && b.graphs.size() < kMaxGraphs) {
    b.to_capture.push_back(key);
    b.graphs.emplace(std::move(key), nullptr);
  }
  const nrx_status st = nrx_detect_batch(b.ctx, n, L.y, cfgs, bits, L.llr, L.st);
  const int64_t dt = steady_ns() - t0;
  std::lock_guard<std::mutex> lk(s->mu);
  s->stats.direct_launches++;
  s->stats.enqueue_ns_direct += dt;
  return st;
}

// Capture one queued composition on the bucket's capture stream (nothing
// executes) and instantiate it.  A failed capture leaves the composition on
// direct launches.
void capture_one(nrx_server* s, Bucket& b) {
  const std::vector<int32_t> key = b.to_capture.front();
  b.to_capture.pop_front();
  const int users = key[0], n = key[1];
  Lane& L = b.lane[kRcvNrx];
  std::vector<nrx_slot_cfg> cfgs = slot_cfgs(s, b, L, n, users, nullptr);
  if (cudaStreamBeginCapture(b.capture_st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  const nrx_status st = nrx_detect_batch(b.ctx, n, L.y, cfgs.data(), key.data() + 2, L.llr, b.capture_st);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(b.capture_st, &g);
  cudaGraphExec_t exec = nullptr;
  const bool ok = st == NRX_OK && e == cudaSuccess && g && cudaGraphInstantiate(&exec, g, 0) == cudaSuccess;
  if (g) cudaGraphDestroy(g);
  cudaGetLastError();
  if (!ok) {
    if (exec) cudaGraphExecDestroy(exec);
    return;
  }
  b.graphs[key] = exec;
  std::lock_guard<std::mutex> lk(s->mu);
  s->stats.graphs_captured++;
}

// Enqueue one batch on lane `li` of bucket b: uploads (or device-generated
// pilots), receiver, LLR downloads.
nrx_status launch(nrx_server* s, Bucket& b, int li, const std::vector<Pending>& reqs, int users) {
  Lane& L = b.lane[li];
  const int n = (int)reqs.size();
  const size_t y_per = (size_t)s->B * kSymbols * b.S;
  const size_t d_per = (size_t)s->cfg.num_dmrs_symbols * (b.S / 2);
  std::vector<nrx_slot_cfg> cfgs = slot_cfgs(s, b, L, n, users, &reqs);
  std::vector<int32_t> bits((size_t)n * users);
  for (int i = 0; i < n; ++i) {
    const nrx_request& r = reqs[i].req;
    if (cudaMemcpyAsync(L.y + i * y_per, r.y_host, y_per * sizeof(float2), cudaMemcpyHostToDevice, L.st) !=
        cudaSuccess)
      return NRX_ECUDA;
    if (r.dmrs_host) {
      if (cudaMemcpyAsync(L.dmrs + i * d_per, r.dmrs_host, d_per * sizeof(float2), cudaMemcpyHostToDevice, L.st) !=
          cudaSuccess)
        return NRX_ECUDA;
    } else {
      const nrx_status st = nrx_dmrs_gold(1, &r.slot_number, r.n_id, 0, b.prb, s->cfg.num_dmrs_symbols,
                                          s->cfg.dmrs_symbols, L.dmrs + i * d_per, L.st);
      if (st != NRX_OK) return st;
    }
    for (int u = 0; u < users; ++u) bits[(size_t)i * users + u] = r.bits_per_symbol[u];
  }
  nrx_status st = li == kRcvNrx ? run_nrx_batch(s, b, L, n, cfgs.data(), bits.data(), users)
                                : lmmse_detect_batch(b.ctx, n, L.y, cfgs.data(), bits.data(), L.llr, L.st);
  if (st != NRX_OK) return st;
  size_t off = 0;
  for (int i = 0; i < n; ++i) {
    const size_t cnt = nrx_llr_count(&cfgs[i], bits.data() + (size_t)i * users);
    if (reqs[i].req.llr_host &&
        cudaMemcpyAsync(reqs[i].req.llr_host, L.llr + off, cnt * sizeof(float), cudaMemcpyDeviceToHost, L.st) !=
            cudaSuccess)
      return NRX_ECUDA;
    off += cnt;
  }
  return NRX_OK;
}

double est(const Bucket& b, int li, int users, int n) {
  const std::vector<double>& v = b.est_us[li][users];
  if (v.empty()) return 0.0;
  return v[std::min<size_t>((size_t)n, v.size() - 1)];
}

void finish(nrx_server* s, int bi, int li) {
  Bucket& b = s->buckets[bi];
  Lane& L = b.lane[li];
  Inflight& f = L.cur;
  float ms_done = 0.f, ms_exec = 0.f;
  cudaEventElapsedTime(&ms_done, L.ref, f.done);
  cudaEventElapsedTime(&ms_exec, f.start, f.done);
  const int64_t done_ns = L.ref_ns + (int64_t)(ms_done * 1e6);
  std::vector<double>& v = b.est_us[li][f.users];
  if ((size_t)f.n < v.size()) v[f.n] = 0.8 * v[f.n] + 0.2 * (double)ms_exec * 1e3;
  for (const Pending& p : f.reqs) complete(s, p, li, NRX_OK, f.n, bi, done_ns);
  f.reqs.clear();
  f.active = false;
}

// Users whose queue head on lane li has the earliest deadline (-1: empty).
int earliest_users(const nrx_server* s, const Bucket& b, int li) {
  int users = -1;
  int64_t best = INT64_MAX;
  for (int u = 1; u <= s->cfg.max_users; ++u)
    if (!b.q[li][u].empty() && b.q[li][u].front().deadline_ns < best) best = b.q[li][u].front().deadline_ns, users = u;
  return users;
}

// Move to the fallback lane every NRX-queued slot that the NRX lane cannot
// finish in time even alone, once the lane is free.
void triage(nrx_server* s, Bucket& b, int64_t now) {
  const int64_t free_at = std::max(now, b.lane[kRcvNrx].cur.active ? b.lane[kRcvNrx].busy_until_ns : now);
  for (int u = 1; u <= s->cfg.max_users; ++u) {
    std::deque<Pending>& Q = b.q[kRcvNrx][u];
    const int64_t nrx1 = free_at + (int64_t)(est(b, kRcvNrx, u, 1) * 1e3);
    while (!Q.empty() && Q.front().deadline_ns < nrx1) {
      b.q[kRcvLmmse][u].push_back(Q.front());
      Q.pop_front();
    }
  }
}

void dispatch(nrx_server* s, int bi, int li, int64_t now) {
  Bucket& b = s->buckets[bi];
  const int users = earliest_users(s, b, li);
  if (users < 0) return;
  std::deque<Pending>& Q = b.q[li][users];
  int n = std::min<int>(b.cap, (int)Q.size());
  if (li == kRcvNrx)  // the largest batch that still meets the earliest deadline
    while (n > 1 && now + (int64_t)(est(b, li, users, n) * 1e3) > Q.front().deadline_ns) --n;
  Lane& L = b.lane[li];
  Inflight& f = L.cur;
  f.reqs.assign(Q.begin(), Q.begin() + n);
  Q.erase(Q.begin(), Q.begin() + n);
  b.queued -= n;
  f.users = users;
  f.n = n;
  L.busy_until_ns = now + (int64_t)(est(b, li, users, n) * 1e3);
  cudaEventRecord(f.start, L.st);
  const nrx_status st = launch(s, b, li, f.reqs, users);
  cudaEventRecord(f.done, L.st);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stats.launches++;
  }
  if (st != NRX_OK) {
    cudaStreamSynchronize(L.st);
    const int64_t t = steady_ns();
    for (const Pending& p : f.reqs) complete(s, p, li, st, n, bi, t);
    f.reqs.clear();
    return;
  }
  f.active = true;
}

// Worker of one bucket: ingest its submissions, retire finished batches,
// triage, dispatch.  One thread per bucket keeps the host-side launch work of
// the buckets in parallel.
void worker_main(nrx_server* s, int bi) {
  cudaSetDevice(s->device);
  Bucket& b = s->buckets[bi];
  std::vector<Pending> incoming;
  for (;;) {
    bool idle = false;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      const bool busy = b.lane[0].cur.active || b.lane[1].cur.active || b.queued > 0;
      if (s->abandon.load()) break;
      idle = !busy && b.inbox.empty();
      if (idle && s->stop.load()) break;
      if (idle && b.to_capture.empty()) s->cv.wait_for(lk, std::chrono::microseconds(200));
      incoming.assign(b.inbox.begin(), b.inbox.end());
      b.inbox.clear();
    }
    if (idle && incoming.empty() && !b.to_capture.empty()) {
      capture_one(s, b);
      continue;
    }
    for (const Pending& p : incoming) {
      if (b.queued >= s->cfg.queue_capacity) {
        complete(s, p, -1, NRX_OK, 0, bi, steady_ns());
        continue;
      }
      b.q[kRcvNrx][p.req.num_users].push_back(p);
      b.queued++;
    }
    for (int li = 0; li < 2; ++li) {
      Lane& L = b.lane[li];
      if (L.cur.active && cudaEventQuery(L.cur.done) == cudaSuccess) finish(s, bi, li);
    }
    if (b.queued > 0) {
      const int64_t now = steady_ns();
      triage(s, b, now);
      for (int li = 0; li < 2; ++li)
        if (!b.lane[li].cur.active) dispatch(s, bi, li, now);
    }
    std::this_thread::yield();
  }
}

// Median CUDA-event time (us) of a lane's receiver on zero inputs (unit pilots).
double time_batch(nrx_server* s, Bucket& b, int li, int users, int n) {
  Lane& L = b.lane[li];
  std::vector<nrx_slot_cfg> cfgs = slot_cfgs(s, b, L, n, users, nullptr);
  std::vector<int32_t> bits((size_t)n * users, std::min(6, s->m_max - (s->m_max & 1)));
  std::vector<float> t;
  for (int r = 0; r < 4; ++r) {
    cudaEventRecord(L.cur.start, L.st);
    nrx_status st = li == kRcvNrx ? nrx_detect_batch(b.ctx, n, L.y, cfgs.data(), bits.data(), L.llr, L.st)
                                  : lmmse_detect_batch(b.ctx, n, L.y, cfgs.data(), bits.data(), L.llr, L.st);
    cudaEventRecord(L.cur.done, L.st);
    if (st != NRX_OK || cudaEventSynchronize(L.cur.done) != cudaSuccess) return -1.0;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, L.cur.start, L.cur.done);
    if (r > 0) t.push_back(ms);
  }
  std::sort(t.begin(), t.end());
  return 1e3 * t[t.size() / 2];
}

__global__ void k_fill_unit(float2* p, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    p[i] = make_float2(1.f, 0.f);
}

nrx_status calibrate(nrx_server* s, Bucket& b) {
  const size_t d_n = (size_t)b.cap * s->cfg.num_dmrs_symbols * (b.S / 2);
  for (int li = 0; li < 2; ++li) {
    Lane& L = b.lane[li];
    if (cudaMemsetAsync(L.y, 0, (size_t)b.cap * s->B * kSymbols * b.S * sizeof(float2), L.st) != cudaSuccess)
      return NRX_ECUDA;
    k_fill_unit<<<64, 256, 0, L.st>>>(L.dmrs, d_n);
    for (int u = 1; u <= s->cfg.max_users; ++u) {
      std::vector<double>& v = b.est_us[li][u];
      v.assign((size_t)b.cap + 1, 0.0);
      std::vector<int> sizes;
      for (int n = 1; n < b.cap; n *= 2) sizes.push_back(n);
      sizes.push_back(b.cap);
      std::vector<double> ts;
      for (int n : sizes) {
        const double us = time_batch(s, b, li, u, n);
        if (us < 0) return NRX_ECUDA;
        ts.push_back(us);
      }
      for (int n = 1; n <= b.cap; ++n) {  // piecewise-linear in n between measured sizes
        size_t k = 0;
        while (k + 1 < sizes.size() && sizes[k + 1] < n) ++k;
        if (k + 1 >= sizes.size() || sizes[k] >= n) {
          v[n] = ts[std::min(k, ts.size() - 1)];
        } else {
          const double a = (double)(n - sizes[k]) / (double)(sizes[k + 1] - sizes[k]);
          v[n] = ts[k] + a * (ts[k + 1] - ts[k]);
        }
      }
      v[0] = v[1];
    }
  }
  return NRX_OK;
}

void free_bucket(Bucket& b) {
  for (auto& kv : b.graphs)
    if (kv.second) cudaGraphExecDestroy(kv.second);
  b.graphs.clear();
  if (b.capture_st) cudaStreamDestroy(b.capture_st);
  if (b.ctx) nrx_destroy(b.ctx);
  for (Lane& L : b.lane) {
    if (L.y) cudaFree(L.y);
    if (L.dmrs) cudaFree(L.dmrs);
    if (L.llr) cudaFree(L.llr);
    if (L.cur.start) cudaEventDestroy(L.cur.start);
    if (L.cur.done) cudaEventDestroy(L.cur.done);
    if (L.ref) cudaEventDestroy(L.ref);
    if (L.st) cudaStreamDestroy(L.st);
  }
  b = Bucket();
}

// Context + both lanes' staging at batch capacity `cap`; bytes taken in *used.
nrx_status make_bucket(nrx_server* s, const void* w, size_t wb, Bucket& b, int prb, int cap, size_t* used) {
  size_t free0 = 0, total = 0, free1 = 0;
  cudaMemGetInfo(&free0, &total);
  b.prb = prb;
  b.S = 12 * prb;
  b.cap = cap;
  nrx_status st = nrx_create(w, wb, s->B, s->cfg.max_users, prb, cap, (nrx_precision)s->cfg.precision, &b.ctx);
  if (st != NRX_OK) return st;
  const size_t y_n = (size_t)cap * s->B * kSymbols * b.S;
  const size_t d_n = (size_t)cap * s->cfg.num_dmrs_symbols * (b.S / 2);
  const size_t l_n = (size_t)cap * slot_llr_floats(b.S, s->cfg.num_dmrs_symbols, s->cfg.max_users, s->m_max);
  for (Lane& L : b.lane) {
    if (cudaMalloc(&L.y, y_n * sizeof(float2)) != cudaSuccess ||
        cudaMalloc(&L.dmrs, d_n * sizeof(float2)) != cudaSuccess || cudaMalloc(&L.llr, l_n * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      return NRX_ENOMEM;
    }
    if (cudaStreamCreateWithFlags(&L.st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&L.cur.start) != cudaSuccess || cudaEventCreate(&L.cur.done) != cudaSuccess ||
        cudaEventCreate(&L.ref) != cudaSuccess)
      return NRX_ECUDA;
  }
  if (cudaStreamCreateWithFlags(&b.capture_st, cudaStreamNonBlocking) != cudaSuccess) return NRX_ECUDA;
  cudaMemGetInfo(&free1, &total);
  *used = free0 > free1 ? free0 - free1 : 0;
  return NRX_OK;
}

}  // namespace

extern "C" {

int64_t nrx_server_now_ns(void) { return steady_ns(); }

nrx_status nrx_server_create(const void* weights, size_t weights_bytes, int32_t num_rx_ant, const nrx_server_cfg* cfg,
                             nrx_server** out) {
  if (!weights || weights_bytes < 32 || !cfg || !out) return NRX_EINVAL;
  const nrx_server_cfg& c = *cfg;
  if (c.num_buckets < 1 || c.num_buckets > NRX_SERVER_MAX_BUCKETS || c.max_users < 1 ||
      c.max_users > kMaxUsers || c.max_batch < 1 || c.max_batch > 64 || c.queue_capacity < 1 ||
      (c.num_dmrs_symbols != 1 && c.num_dmrs_symbols != 2) || c.deadline_us <= 0.0)
    return NRX_EINVAL;
  for (int i = 0; i < c.num_buckets; ++i) {
    if (c.bucket_prb[i] < 1 || c.bucket_prb[i] > 275) return NRX_EINVAL;
    for (int j = 0; j < i; ++j)
      if (c.bucket_prb[j] == c.bucket_prb[i]) return NRX_EINVAL;
  }
  int32_t hdr[8];
  memcpy(hdr, weights, sizeof(hdr));
  nrx_server* s = new nrx_server();
  s->cfg = c;
  s->B = num_rx_ant;
  s->m_max = hdr[6];
  cudaGetDevice(&s->device);
  size_t used_total = 0;
  for (int i = 0; i < c.num_buckets; ++i) {
    Bucket b;
    int cap = c.max_batch;
    nrx_status st = NRX_ENOMEM;
    for (; cap >= 1; cap /= 2) {
      size_t used = 0;
      st = make_bucket(s, weights, weights_bytes, b, c.bucket_prb[i], cap, &used);
      if (st == NRX_OK && used_total + used <= c.hbm_budget_bytes) {
        used_total += used;
        break;
      }
      free_bucket(b);
      if (st != NRX_OK && st != NRX_ENOMEM) break;
      st = NRX_ENOMEM;
    }
    if (st != NRX_OK || cap < 1) {
      for (Bucket& o : s->buckets) free_bucket(o);
      delete s;
      return st == NRX_OK ? NRX_ENOMEM : st;
    }
    s->buckets.push_back(b);
    s->stats.bucket_batch_capacity[i] = cap;
  }
  s->stats.device_bytes = used_total;
  for (Bucket& b : s->buckets) {
    nrx_status st = calibrate(s, b);
    for (Lane& L : b.lane) {
      if (st != NRX_OK) break;
      cudaEventRecord(L.ref, L.st);
      if (cudaEventSynchronize(L.ref) != cudaSuccess) st = NRX_ECUDA;
      L.ref_ns = steady_ns();
    }
    if (st != NRX_OK) {
      for (Bucket& o : s->buckets) free_bucket(o);
      delete s;
      return st;
    }
  }
  for (int bi = 0; bi < (int)s->buckets.size(); ++bi) s->workers.emplace_back(worker_main, s, bi);
  *out = s;
  return NRX_OK;
}

void nrx_server_destroy(nrx_server* s) {
  if (!s) return;
  if (nrx_server_drain(s, 10000) != NRX_OK) s->abandon.store(true);
  s->stop.store(true);
  s->cv.notify_all();
  for (std::thread& t : s->workers)
    if (t.joinable()) t.join();
  for (Bucket& b : s->buckets) {
    for (Lane& L : b.lane)
      if (L.st) cudaStreamSynchronize(L.st);
    free_bucket(b);
  }
  delete s;
}

nrx_status nrx_server_submit(nrx_server* s, const nrx_request* r, uint64_t* ticket) {
  if (!s || !r || !r->y_host) return NRX_EINVAL;
  if (!r->dmrs_host && (r->n_id < 0 || r->n_id > 65535 || r->slot_number < 0 || r->slot_number > 159))
    return NRX_EINVAL;
  int bi = -1;
  for (int i = 0; i < (int)s->buckets.size(); ++i)
    if (s->buckets[i].prb == r->num_prb) bi = i;
  if (bi < 0 || r->num_users < 1 || r->num_users > s->cfg.max_users) return NRX_EINVAL;
  for (int u = 0; u < r->num_users; ++u) {
    const int m = r->bits_per_symbol[u];
    if ((m != 2 && m != 4 && m != 6) || m > s->m_max) return NRX_EINVAL;
  }
  Pending p;
  p.req = *r;
  if (p.req.arrival_ns == 0) p.req.arrival_ns = steady_ns();
  p.deadline_ns = p.req.arrival_ns + (int64_t)(s->cfg.deadline_us * 1e3);
  s->outstanding.fetch_add(1);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    p.ticket = s->next_ticket++;
    s->buckets[bi].inbox.push_back(p);
    s->stats.submitted++;
  }
  s->cv.notify_all();
  if (ticket) *ticket = p.ticket;
  return NRX_OK;
}

nrx_status nrx_server_replay(nrx_server* s, int32_t n, const nrx_request* reqs, uint64_t* tickets,
                             int64_t* max_late_ns) {
  if (!s || n < 0 || (n > 0 && !reqs)) return NRX_EINVAL;
  int64_t late = 0;
  for (int32_t i = 0; i < n; ++i) {
    while (steady_ns() < reqs[i].arrival_ns) {
    }
    late = std::max(late, steady_ns() - reqs[i].arrival_ns);
    const nrx_status st = nrx_server_submit(s, &reqs[i], tickets ? tickets + i : nullptr);
    if (st != NRX_OK) return st;
  }
  if (max_late_ns) *max_late_ns = late;
  return NRX_OK;
}

nrx_status nrx_server_poll(nrx_server* s, nrx_completion* out, int32_t max_out, int32_t* n) {
  if (!s || !n || max_out < 0 || (max_out > 0 && !out)) return NRX_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  int k = 0;
  while (k < max_out && !s->done.empty()) {
    out[k++] = s->done.front();
    s->done.pop_front();
  }
  *n = k;
  return NRX_OK;
}

nrx_status nrx_server_drain(nrx_server* s, int32_t timeout_ms) {
  if (!s) return NRX_EINVAL;
  const int64_t end = steady_ns() + (int64_t)timeout_ms * 1000000;
  while (s->outstanding.load() > 0) {
    if (steady_ns() > end) return NRX_ETIMEDOUT;
    std::this_thread::sleep_for(std::chrono::microseconds(100));
  }
  return NRX_OK;
}

nrx_status nrx_server_get_stats(const nrx_server* s, nrx_server_stats* out) {
  if (!s || !out) return NRX_EINVAL;
  std::lock_guard<std::mutex> lk(const_cast<nrx_server*>(s)->mu);
  *out = s->stats;
  return NRX_OK;
}

}  // extern "C"
