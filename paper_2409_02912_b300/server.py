"""Python binding of the serving loop (``include/nrx_server.h``) and a
load generator: Poisson slot arrivals from several cells, each cell with its
own PRB count, per-slot user counts and modulation orders drawn at random.

The binding marshals arguments only; batching, dispatch, fallback and timing
run in the library's worker thread and CUDA kernels.
"""
from __future__ import annotations

import ctypes
import dataclasses
from typing import Dict, List, Sequence

import numpy as np

from . import nrx, synth

SERVER_EXPORTED = ("nrx_server_create", "nrx_server_destroy", "nrx_server_now_ns", "nrx_server_submit",
                   "nrx_server_replay", "nrx_server_poll", "nrx_server_drain", "nrx_server_get_stats")
MAX_BUCKETS = 8
RECEIVER_NAMES = {0: "nrx", 1: "lmmse", -1: "rejected"}


class nrx_server_cfg(ctypes.Structure):
    _fields_ = [("num_buckets", ctypes.c_int32), ("bucket_prb", ctypes.c_int32 * MAX_BUCKETS),
                ("max_users", ctypes.c_int32), ("max_batch", ctypes.c_int32), ("queue_capacity", ctypes.c_int32),
                ("num_dmrs_symbols", ctypes.c_int32), ("dmrs_symbols", ctypes.c_int32 * 2),
                ("precision", ctypes.c_int32), ("deadline_us", ctypes.c_double),
                ("hbm_budget_bytes", ctypes.c_size_t)]


class nrx_request(ctypes.Structure):
    _fields_ = [("num_prb", ctypes.c_int32), ("num_users", ctypes.c_int32),
                ("bits_per_symbol", ctypes.c_int32 * 4), ("noise_var", ctypes.c_float),
                ("y_host", ctypes.c_void_p), ("dmrs_host", ctypes.c_void_p), ("llr_host", ctypes.c_void_p),
                ("arrival_ns", ctypes.c_int64), ("n_id", ctypes.c_int32), ("slot_number", ctypes.c_int32)]


class nrx_completion(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("receiver", ctypes.c_int32), ("status", ctypes.c_int32),
                ("batch_size", ctypes.c_int32), ("bucket", ctypes.c_int32), ("arrival_ns", ctypes.c_int64),
                ("done_ns", ctypes.c_int64)]


class nrx_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("served_nrx", ctypes.c_int64), ("served_lmmse", ctypes.c_int64),
                ("rejected", ctypes.c_int64), ("launches", ctypes.c_int64),
                ("bucket_batch_capacity", ctypes.c_int32 * MAX_BUCKETS), ("device_bytes", ctypes.c_size_t),
                ("graph_launches", ctypes.c_int64), ("graphs_captured", ctypes.c_int64),
                ("direct_launches", ctypes.c_int64), ("enqueue_ns_graph", ctypes.c_int64),
                ("enqueue_ns_direct", ctypes.c_int64)]


_configured = False


def load():
    global _configured
    lib = nrx.load()
    if not _configured:
        P, I32 = ctypes.c_void_p, ctypes.c_int32
        lib.nrx_server_create.argtypes = [P, ctypes.c_size_t, I32, ctypes.POINTER(nrx_server_cfg), ctypes.POINTER(P)]
        lib.nrx_server_create.restype = ctypes.c_int
        lib.nrx_server_destroy.argtypes = [P]
        lib.nrx_server_destroy.restype = None
        lib.nrx_server_now_ns.argtypes = []
        lib.nrx_server_now_ns.restype = ctypes.c_int64
        lib.nrx_server_submit.argtypes = [P, ctypes.POINTER(nrx_request), ctypes.POINTER(ctypes.c_uint64)]
        lib.nrx_server_submit.restype = ctypes.c_int
        lib.nrx_server_replay.argtypes = [P, I32, ctypes.POINTER(nrx_request), ctypes.POINTER(ctypes.c_uint64),
                                          ctypes.POINTER(ctypes.c_int64)]
        lib.nrx_server_replay.restype = ctypes.c_int
        lib.nrx_server_poll.argtypes = [P, ctypes.POINTER(nrx_completion), I32, ctypes.POINTER(I32)]
        lib.nrx_server_poll.restype = ctypes.c_int
        lib.nrx_server_drain.argtypes = [P, I32]
        lib.nrx_server_drain.restype = ctypes.c_int
        lib.nrx_server_get_stats.argtypes = [P, ctypes.POINTER(nrx_server_stats)]
        lib.nrx_server_get_stats.restype = ctypes.c_int
        _configured = True
    return lib


class Server:
    """``nrx_server_create`` and the calls on it."""

    def __init__(self, weights_blob: bytes, num_rx_ant: int, bucket_prb: Sequence[int], max_users: int = 4,
                 max_batch: int = 8, queue_capacity: int = 256, dmrs_symbols=(2, 11), precision: str = "bf16",
                 deadline_us: float = 500.0, hbm_budget_bytes: int = 16 << 30):
        lib = load()
        self._lib = lib
        c = nrx_server_cfg()
        c.num_buckets = len(bucket_prb)
        for i, p in enumerate(bucket_prb):
            c.bucket_prb[i] = p
        c.max_users, c.max_batch, c.queue_capacity = max_users, max_batch, queue_capacity
        c.num_dmrs_symbols = len(dmrs_symbols)
        c.dmrs_symbols[0] = dmrs_symbols[0]
        c.dmrs_symbols[1] = dmrs_symbols[-1]
        c.precision = nrx.PRECISIONS[precision]
        c.deadline_us = deadline_us
        c.hbm_budget_bytes = hbm_budget_bytes
        self.cfg = c
        self._blob = ctypes.create_string_buffer(weights_blob, len(weights_blob))
        h = ctypes.c_void_p()
        st = lib.nrx_server_create(self._blob, len(weights_blob), num_rx_ant, ctypes.byref(c), ctypes.byref(h))
        if st != nrx.NRX_OK:
            raise nrx.NrxError(st, "nrx_server_create")
        self.h = h
        self.bucket_prb = list(bucket_prb)

    def close(self):
        if getattr(self, "h", None):
            self._lib.nrx_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def now_ns(self) -> int:
        return int(self._lib.nrx_server_now_ns())

    def submit(self, req: nrx_request) -> int:
        t = ctypes.c_uint64()
        st = self._lib.nrx_server_submit(self.h, ctypes.byref(req), ctypes.byref(t))
        if st != nrx.NRX_OK:
            raise nrx.NrxError(st, "nrx_server_submit")
        return t.value

    def replay(self, reqs) -> tuple:
        """Submit a ctypes array of requests at their arrival times (native
        spin-wait); returns (tickets, max lateness in ns)."""
        n = len(reqs)
        tickets = (ctypes.c_uint64 * n)()
        late = ctypes.c_int64()
        st = self._lib.nrx_server_replay(self.h, n, reqs, tickets, ctypes.byref(late))
        if st != nrx.NRX_OK:
            raise nrx.NrxError(st, "nrx_server_replay")
        return list(tickets), late.value

    def poll(self, max_out: int = 4096) -> List[nrx_completion]:
        buf = (nrx_completion * max_out)()
        n = ctypes.c_int32()
        st = self._lib.nrx_server_poll(self.h, buf, max_out, ctypes.byref(n))
        if st != nrx.NRX_OK:
            raise nrx.NrxError(st, "nrx_server_poll")
        return [buf[i] for i in range(n.value)]

    def drain(self, timeout_ms: int = 30000):
        st = self._lib.nrx_server_drain(self.h, timeout_ms)
        if st != nrx.NRX_OK:
            raise nrx.NrxError(st, "nrx_server_drain")

    def stats(self) -> dict:
        s = nrx_server_stats()
        self._lib.nrx_server_get_stats(self.h, ctypes.byref(s))
        return {"submitted": s.submitted, "served_nrx": s.served_nrx, "served_lmmse": s.served_lmmse,
                "rejected": s.rejected, "launches": s.launches,
                "bucket_batch_capacity": list(s.bucket_batch_capacity)[:len(self.bucket_prb)],
                "device_bytes": int(s.device_bytes), "graph_launches": s.graph_launches,
                "graphs_captured": s.graphs_captured, "direct_launches": s.direct_launches,
                "enqueue_us_graph_mean": s.enqueue_ns_graph / max(s.graph_launches, 1) / 1e3,
                "enqueue_us_direct_mean": s.enqueue_ns_direct / max(s.direct_launches, 1) / 1e3}


def make_request(sl: synth.Slot, y_pin, dmrs_pin, llr_pin, arrival_ns: int = 0) -> nrx_request:
    """Request for one slot whose grid / pilots are in the pinned host tensors
    ``y_pin`` / ``dmrs_pin`` and whose LLRs go to ``llr_pin``.  With
    ``dmrs_pin`` None the server generates the cell's TS 38.211 pilots on the
    device from the slot's ``n_id`` and ``slot_number``."""
    r = nrx_request()
    r.num_prb = sl.cfg.num_prb
    r.num_users = sl.cfg.num_users
    for u, m in enumerate(sl.cfg.bits_per_symbol):
        r.bits_per_symbol[u] = m
    r.noise_var = sl.cfg.noise_var
    r.y_host = y_pin.data_ptr()
    r.dmrs_host = dmrs_pin.data_ptr() if dmrs_pin is not None else None
    r.n_id = sl.cfg.n_id
    r.slot_number = sl.cfg.slot_number
    r.llr_host = llr_pin.data_ptr() if llr_pin is not None else None
    r.arrival_ns = arrival_ns
    return r


@dataclasses.dataclass
class LoadSpec:
    """Offered load: ``cells`` cells, each with one PRB count from
    ``prb_choices`` (assigned round-robin), Poisson slot arrivals at
    ``slots_per_s_per_cell``, users uniform in ``users`` per slot, modulation
    orders uniform in ``mcs`` per user."""

    cells: int = 16
    prb_choices: tuple = (24, 51, 106, 273)
    users: tuple = (1, 2, 3, 4)
    mcs: tuple = (2, 4, 6)
    slots_per_s_per_cell: float = 2000.0
    seconds: float = 2.0
    num_rx_ant: int = 4
    dmrs_symbols: tuple = (2, 11)
    pool_per_key: int = 4
    seed: int = 77


def run_load(srv: Server, spec: LoadSpec) -> Dict[str, object]:
    """Offer ``spec`` to the server in real time (arrivals paced on the
    server's clock; host jitter counts as queueing) and summarise the
    completions: latency percentiles per receiver, deadline misses, fallback
    and rejection rates, served REs/s."""
    import torch
    rng = np.random.Generator(np.random.PCG64(spec.seed))
    cell_prb = [spec.prb_choices[c % len(spec.prb_choices)] for c in range(spec.cells)]
    # pinned pools of received slots per (prb, users)
    pools: Dict[tuple, list] = {}
    for prb in sorted(set(cell_prb)):
        for U in spec.users:
            entries = []
            for i in range(spec.pool_per_key):
                prng = np.random.Generator(np.random.PCG64(spec.seed * 7919 + prb * 31 + U * 7 + i))
                cfg = synth.SlotConfig(num_prb=prb, num_users=U, num_rx_ant=spec.num_rx_ant,
                                       dmrs_symbols=spec.dmrs_symbols,
                                       bits_per_symbol=tuple(int(prng.choice(spec.mcs)) for _ in range(U)),
                                       snr_db=float(prng.uniform(0, 20)), num_taps=12,
                                       delay_spread_s=float(prng.uniform(10e-9, 300e-9)),
                                       doppler_hz=float(prng.uniform(0, 400)), ula=True)
                sl = synth.make_slot(cfg, prng)
                y = torch.from_numpy(sl.y).pin_memory()
                d = torch.from_numpy(sl.dmrs).pin_memory()
                n_llr = cfg.num_data_symbols * cfg.num_subcarriers * sum(cfg.bits_per_symbol)
                entries.append((sl, y, d, torch.empty(n_llr, dtype=torch.float32).pin_memory()))
            pools[(prb, U)] = entries
    # arrival schedule
    events = []
    for c in range(spec.cells):
        t = float(rng.exponential(1.0 / spec.slots_per_s_per_cell))
        while t < spec.seconds:
            events.append((t, c))
            t += float(rng.exponential(1.0 / spec.slots_per_s_per_cell))
    events.sort()
    picks = [(cell_prb[c], int(rng.choice(spec.users)), int(rng.integers(0, spec.pool_per_key))) for _, c in events]
    reqs = (nrx_request * len(events))()
    for i, ((t, _), (prb, U, k)) in enumerate(zip(events, picks)):
        sl, y, d, l = pools[(prb, U)][k]
        reqs[i] = make_request(sl, y, d, l)
    res_per_req = [14 * 12 * prb for (prb, _, _) in picks]
    t0 = srv.now_ns() + 50_000_000
    for i, (t, _) in enumerate(events):
        reqs[i].arrival_ns = t0 + int(t * 1e9)
    tickets, max_late = srv.replay(reqs)
    res_of: Dict[int, int] = dict(zip(tickets, res_per_req))
    comps: List[nrx_completion] = []
    srv.drain(60000)
    comps.extend(srv.poll(max(4096, len(reqs))))
    lat = {0: [], 1: []}
    served_res = {0: 0, 1: 0}
    deadline_ns = srv.cfg.deadline_us * 1e3
    misses = 0
    batches = []
    for c in comps:
        res = res_of.get(c.ticket)
        if res is None:
            continue
        if c.receiver in (0, 1):
            lt = c.done_ns - c.arrival_ns
            lat[c.receiver].append(lt / 1e3)
            served_res[c.receiver] += res
            misses += lt > deadline_ns
            batches.append(c.batch_size)
    all_lat = lat[0] + lat[1]
    pct = lambda v, q: float(np.percentile(v, q)) if v else None  # noqa: E731
    n = len(reqs)
    return {
        "offered_slots": n, "offered_slots_per_s": n / spec.seconds,
        "offered_res_per_s": float(sum(res_per_req)) / spec.seconds,
        "served_nrx": len(lat[0]), "served_lmmse": len(lat[1]), "rejected": n - len(all_lat),
        "lmmse_fallback_rate": len(lat[1]) / max(n, 1), "deadline_us": srv.cfg.deadline_us,
        "deadline_miss_rate": misses / max(n, 1),
        "latency_us": {"all_p50": pct(all_lat, 50), "all_p99": pct(all_lat, 99),
                       "nrx_p50": pct(lat[0], 50), "nrx_p99": pct(lat[0], 99),
                       "lmmse_p50": pct(lat[1], 50), "lmmse_p99": pct(lat[1], 99)},
        "nrx_res_per_s": served_res[0] / spec.seconds, "mean_batch": float(np.mean(batches)) if batches else 0.0,
        "max_submit_late_us": max_late / 1e3,
        "stats": srv.stats(),
    }
