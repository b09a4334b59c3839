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
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/nrx_server.h"

namespace {

constexpr int kSymbols = 14;
constexpr int kMaxUsers = 4;
constexpr int kRcvNrx = 0, kRcvLmmse = 1;

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
  int receiver = 0, users = 0, n = 0;
  std::vector<Pending> reqs;
  cudaEvent_t start = nullptr, done = nullptr;
};

struct Bucket {
  int prb = 0, S = 0, cap = 0;
  nrx_ctx* ctx = nullptr;
  cudaStream_t st = nullptr;
  float2* y = nullptr;
  float2* dmrs = nullptr;
  float* llr = nullptr;
  std::deque<Pending> q[kMaxUsers + 1];
  int queued = 0;
  Inflight cur;
  cudaEvent_t ref = nullptr;
  int64_t ref_ns = 0;
  std::vector<double> est_us[2][kMaxUsers + 1];  // [receiver][users][n], n <= cap
};

}  // namespace

struct nrx_server {
  nrx_server_cfg cfg{};
  int B = 0, m_max = 0, device = 0;
  std::vector<Bucket> buckets;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Pending> inbox;
  std::deque<nrx_completion> done;
  std::atomic<bool> stop{false};
  std::atomic<int64_t> outstanding{0};
  std::thread worker;
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

// Launch one batch of `reqs` on bucket b with the chosen receiver (async).
nrx_status launch(nrx_server* s, Bucket& b, const std::vector<Pending>& reqs, int receiver, int users) {
  const nrx_server_cfg& c = s->cfg;
  const int n = (int)reqs.size();
  const size_t y_per = (size_t)s->B * kSymbols * b.S;
  const size_t d_per = (size_t)c.num_dmrs_symbols * (b.S / 2);
  std::vector<nrx_slot_cfg> cfgs(n);
  std::vector<int32_t> bits((size_t)n * users);
  for (int i = 0; i < n; ++i) {
    const nrx_request& r = reqs[i].req;
    if (cudaMemcpyAsync(b.y + i * y_per, r.y_host, y_per * sizeof(float2), cudaMemcpyHostToDevice, b.st) !=
            cudaSuccess ||
        cudaMemcpyAsync(b.dmrs + i * d_per, r.dmrs_host, d_per * sizeof(float2), cudaMemcpyHostToDevice, b.st) !=
            cudaSuccess)
      return NRX_ECUDA;
    nrx_slot_cfg& sc = cfgs[i];
    memset(&sc, 0, sizeof(sc));
    sc.num_prb = b.prb;
    sc.num_users = users;
    sc.num_dmrs_symbols = c.num_dmrs_symbols;
    sc.dmrs_symbols[0] = c.dmrs_symbols[0];
    sc.dmrs_symbols[1] = c.dmrs_symbols[c.num_dmrs_symbols - 1];
    sc.iterations = 0;
    sc.noise_var = r.noise_var;
    sc.dmrs_seq = b.dmrs + i * d_per;
    for (int u = 0; u < users; ++u) bits[(size_t)i * users + u] = r.bits_per_symbol[u];
  }
  nrx_status st = receiver == kRcvNrx
                      ? nrx_detect_batch(b.ctx, n, b.y, cfgs.data(), bits.data(), b.llr, b.st)
                      : lmmse_detect_batch(b.ctx, n, b.y, cfgs.data(), bits.data(), b.llr, b.st);
  if (st != NRX_OK) return st;
  size_t off = 0;
  for (int i = 0; i < n; ++i) {
    const size_t cnt = nrx_llr_count(&cfgs[i], bits.data() + (size_t)i * users);
    if (reqs[i].req.llr_host &&
        cudaMemcpyAsync(reqs[i].req.llr_host, b.llr + off, cnt * sizeof(float), cudaMemcpyDeviceToHost, b.st) !=
            cudaSuccess)
      return NRX_ECUDA;
    off += cnt;
  }
  return NRX_OK;
}

double est(const Bucket& b, int rcv, int users, int n) {
  const std::vector<double>& v = b.est_us[rcv][users];
  if (v.empty()) return 0.0;
  return v[std::min<size_t>((size_t)n, v.size() - 1)];
}

void finish(nrx_server* s, int bi) {
  Bucket& b = s->buckets[bi];
  Inflight& f = b.cur;
  float ms_done = 0.f, ms_exec = 0.f;
  cudaEventElapsedTime(&ms_done, b.ref, f.done);
  cudaEventElapsedTime(&ms_exec, f.start, f.done);
  const int64_t done_ns = b.ref_ns + (int64_t)(ms_done * 1e6);
  std::vector<double>& v = b.est_us[f.receiver][f.users];
  if ((size_t)f.n < v.size()) v[f.n] = 0.8 * v[f.n] + 0.2 * (double)ms_exec * 1e3;
  for (const Pending& p : f.reqs) complete(s, p, f.receiver, NRX_OK, f.n, bi, done_ns);
  f.reqs.clear();
  f.active = false;
}

void dispatch(nrx_server* s, int bi) {
  Bucket& b = s->buckets[bi];
  int users = -1;
  int64_t best = INT64_MAX;
  for (int u = 1; u <= s->cfg.max_users; ++u)
    if (!b.q[u].empty() && b.q[u].front().deadline_ns < best) best = b.q[u].front().deadline_ns, users = u;
  if (users < 0) return;
  std::deque<Pending>& Q = b.q[users];
  const int64_t now = steady_ns();
  int n = std::min<int>(b.cap, (int)Q.size());
  // largest NRX batch that still finishes before the earliest deadline
  while (n > 1 && now + (int64_t)(est(b, kRcvNrx, users, n) * 1e3) > Q.front().deadline_ns) --n;
  int rcv = kRcvNrx;
  if (now + (int64_t)(est(b, kRcvNrx, users, n) * 1e3) > Q.front().deadline_ns) {
    // the NRX misses even alone: LS+LMMSE for every queued slot that would miss
    rcv = kRcvLmmse;
    const int64_t nrx1 = now + (int64_t)(est(b, kRcvNrx, users, 1) * 1e3);
    n = 0;
    while (n < (int)Q.size() && n < b.cap && Q[n].deadline_ns < nrx1) ++n;
    if (n == 0) n = 1;
  }
  Inflight& f = b.cur;
  f.reqs.assign(Q.begin(), Q.begin() + n);
  Q.erase(Q.begin(), Q.begin() + n);
  b.queued -= n;
  f.receiver = rcv;
  f.users = users;
  f.n = n;
  cudaEventRecord(f.start, b.st);
  const nrx_status st = launch(s, b, f.reqs, rcv, users);
  cudaEventRecord(f.done, b.st);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stats.launches++;
  }
  if (st != NRX_OK) {
    cudaStreamSynchronize(b.st);
    const int64_t t = steady_ns();
    for (const Pending& p : f.reqs) complete(s, p, rcv, st, n, bi, t);
    f.reqs.clear();
    return;
  }
  f.active = true;
}

void worker_main(nrx_server* s) {
  cudaSetDevice(s->device);
  std::vector<Pending> incoming;
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(s->mu);
      bool busy = false;
      for (const Bucket& b : s->buckets) busy = busy || b.cur.active || b.queued > 0;
      if (!busy && s->inbox.empty()) {
        if (s->stop.load()) break;
        s->cv.wait_for(lk, std::chrono::microseconds(200));
      }
      incoming.assign(s->inbox.begin(), s->inbox.end());
      s->inbox.clear();
    }
    for (const Pending& p : incoming) {
      int bi = 0;
      while (s->buckets[bi].prb != p.req.num_prb) ++bi;
      Bucket& b = s->buckets[bi];
      if (b.queued >= s->cfg.queue_capacity) {
        complete(s, p, -1, NRX_OK, 0, bi, steady_ns());
        continue;
      }
      b.q[p.req.num_users].push_back(p);
      b.queued++;
    }
    for (size_t bi = 0; bi < s->buckets.size(); ++bi)
      if (s->buckets[bi].cur.active && cudaEventQuery(s->buckets[bi].cur.done) == cudaSuccess) finish(s, (int)bi);
    for (size_t bi = 0; bi < s->buckets.size(); ++bi)
      if (!s->buckets[bi].cur.active && s->buckets[bi].queued > 0) dispatch(s, (int)bi);
    std::this_thread::yield();
  }
}

// Median CUDA-event time (us) of a receiver on zero inputs (unit pilots).
double time_batch(nrx_server* s, Bucket& b, int rcv, int users, int n) {
  const nrx_server_cfg& c = s->cfg;
  std::vector<nrx_slot_cfg> cfgs(n);
  std::vector<int32_t> bits((size_t)n * users, std::min(6, s->m_max - (s->m_max & 1)));
  const size_t d_per = (size_t)c.num_dmrs_symbols * (b.S / 2);
  for (int i = 0; i < n; ++i) {
    nrx_slot_cfg& sc = cfgs[i];
    memset(&sc, 0, sizeof(sc));
    sc.num_prb = b.prb;
    sc.num_users = users;
    sc.num_dmrs_symbols = c.num_dmrs_symbols;
    sc.dmrs_symbols[0] = c.dmrs_symbols[0];
    sc.dmrs_symbols[1] = c.dmrs_symbols[c.num_dmrs_symbols - 1];
    sc.noise_var = 0.1f;
    sc.dmrs_seq = b.dmrs + i * d_per;
  }
  std::vector<float> t;
  for (int r = 0; r < 4; ++r) {
    cudaEventRecord(b.cur.start, b.st);
    nrx_status st = rcv == kRcvNrx ? nrx_detect_batch(b.ctx, n, b.y, cfgs.data(), bits.data(), b.llr, b.st)
                                   : lmmse_detect_batch(b.ctx, n, b.y, cfgs.data(), bits.data(), b.llr, b.st);
    cudaEventRecord(b.cur.done, b.st);
    if (st != NRX_OK || cudaEventSynchronize(b.cur.done) != cudaSuccess) return -1.0;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, b.cur.start, b.cur.done);
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
  if (cudaMemsetAsync(b.y, 0, (size_t)b.cap * s->B * kSymbols * b.S * sizeof(float2), b.st) != cudaSuccess)
    return NRX_ECUDA;
  k_fill_unit<<<64, 256, 0, b.st>>>(b.dmrs, d_n);
  for (int rcv = 0; rcv < 2; ++rcv)
    for (int u = 1; u <= s->cfg.max_users; ++u) {
      std::vector<double>& v = b.est_us[rcv][u];
      v.assign((size_t)b.cap + 1, 0.0);
      std::vector<int> sizes;
      for (int n = 1; n < b.cap; n *= 2) sizes.push_back(n);
      sizes.push_back(b.cap);
      std::vector<double> ts;
      for (int n : sizes) {
        const double us = time_batch(s, b, rcv, u, n);
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
  return NRX_OK;
}

void free_bucket(Bucket& b) {
  if (b.ctx) nrx_destroy(b.ctx);
  if (b.y) cudaFree(b.y);
  if (b.dmrs) cudaFree(b.dmrs);
  if (b.llr) cudaFree(b.llr);
  if (b.cur.start) cudaEventDestroy(b.cur.start);
  if (b.cur.done) cudaEventDestroy(b.cur.done);
  if (b.ref) cudaEventDestroy(b.ref);
  if (b.st) cudaStreamDestroy(b.st);
  b = Bucket();
}

// Context + staging of one bucket at batch capacity `cap`; bytes taken in *used.
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
  if (cudaMalloc(&b.y, y_n * sizeof(float2)) != cudaSuccess || cudaMalloc(&b.dmrs, d_n * sizeof(float2)) != cudaSuccess ||
      cudaMalloc(&b.llr, l_n * sizeof(float)) != cudaSuccess)
    return NRX_ENOMEM;
  if (cudaStreamCreateWithFlags(&b.st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&b.cur.start) != cudaSuccess || cudaEventCreate(&b.cur.done) != cudaSuccess ||
      cudaEventCreate(&b.ref) != cudaSuccess)
    return NRX_ECUDA;
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
    if (st == NRX_OK) {
      cudaEventRecord(b.ref, b.st);
      if (cudaEventSynchronize(b.ref) != cudaSuccess) st = NRX_ECUDA;
      b.ref_ns = steady_ns();
    }
    if (st != NRX_OK) {
      for (Bucket& o : s->buckets) free_bucket(o);
      delete s;
      return st;
    }
  }
  s->worker = std::thread(worker_main, s);
  *out = s;
  return NRX_OK;
}

void nrx_server_destroy(nrx_server* s) {
  if (!s) return;
  nrx_server_drain(s, 10000);
  s->stop.store(true);
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (Bucket& b : s->buckets) {
    if (b.st) cudaStreamSynchronize(b.st);
    free_bucket(b);
  }
  delete s;
}

nrx_status nrx_server_submit(nrx_server* s, const nrx_request* r, uint64_t* ticket) {
  if (!s || !r || !r->y_host || !r->dmrs_host) return NRX_EINVAL;
  bool found = false;
  for (const Bucket& b : s->buckets) found = found || b.prb == r->num_prb;
  if (!found || r->num_users < 1 || r->num_users > s->cfg.max_users) return NRX_EINVAL;
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
    s->inbox.push_back(p);
    s->stats.submitted++;
  }
  s->cv.notify_one();
  if (ticket) *ticket = p.ticket;
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
