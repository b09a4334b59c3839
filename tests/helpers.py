"""Shared test helpers: seeded slots on the device, oracle references, and the
per-(slot, user) error metric max|gpu - ref| / max|ref|."""
from __future__ import annotations

import numpy as np

from oracle import nrx_oracle as O
from paper_2409_02912_b300 import synth


def slots_for(workload: str, n=None, start=0):
    w = synth.WORKLOADS[workload]
    return w, synth.workload_slots(w, n, start)


def weights64(net):
    return {k: v.astype(np.float64) for k, v in synth.make_weights(net).items()}


def device_inputs(slots):
    import torch
    y = torch.from_numpy(synth.stack_batch(slots)).cuda()
    dmrs = torch.from_numpy(np.stack([s.dmrs for s in slots]).astype(np.complex64)).cuda()
    bits = [list(s.cfg.bits_per_symbol) for s in slots]
    nv = [s.cfg.noise_var for s in slots]
    return y, dmrs, bits, nv


def oracle_nrx(slots, W, net, iterations=None):
    its = net.iterations if iterations is None else iterations
    out = []
    for s in slots:
        c = s.cfg
        out.append(O.nrx_forward(s.y, s.dmrs, c.num_users, c.dmrs_symbols, c.bits_per_symbol, W, its,
                                 net.res_blocks))
    return out


def oracle_lmmse(slots):
    return [O.lmmse_receiver(s.y, s.dmrs, s.cfg.num_users, s.cfg.dmrs_symbols, s.cfg.bits_per_symbol,
                             s.cfg.noise_var) for s in slots]


def split(llr_flat, slots):
    """Split a batch's packed LLRs into per-slot, per-user arrays."""
    out, off = [], 0
    for s in slots:
        per = []
        n_data = s.cfg.num_data_symbols * s.cfg.num_subcarriers
        for m in s.cfg.bits_per_symbol:
            per.append(llr_flat[off:off + n_data * m])
            off += n_data * m
        out.append(per)
    return out, off


def rel_errors(gpu_flat, refs, slots):
    """List of max|gpu-ref|/max|ref| per (slot, user)."""
    g, total = split(np.asarray(gpu_flat, dtype=np.float64), slots)
    assert total == len(gpu_flat)
    errs = []
    for gs, ref, s in zip(g, refs, slots):
        r, _ = split(ref, [s])
        for gu, ru in zip(gs, r[0]):
            errs.append(float(np.max(np.abs(gu - ru)) / max(np.max(np.abs(ru)), 1e-30)))
    return errs
