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


def elementwise_rel(gpu_flat, refs, slots):
    """Elementwise relative error |gpu - ref| / max(|ref|, 1) over every LLR of
    the batch (the floor of 1.0 keeps it defined near llr = 0); returns
    (median, 99th percentile)."""
    ref = np.concatenate([np.asarray(r, dtype=np.float64).ravel() for r in refs])
    g = np.asarray(gpu_flat, dtype=np.float64)[:ref.size]
    rel = np.abs(g - ref) / np.maximum(np.abs(ref), 1.0)
    return float(np.median(rel)), float(np.percentile(rel, 99))


def _slot_from_channel(cfg, dmrs, h, rng, noisy_pilots=True):
    """Received grid of ``cfg`` over channel h [U, B, 14, S] with the given
    DMRS base sequence; with ``noisy_pilots`` False the DMRS symbols are
    received noise-free (their values then stay exact in FP32)."""
    S = cfg.num_subcarriers
    n_data = cfg.num_data_symbols * S
    bits = [rng.integers(0, 2, size=(n_data, m), dtype=np.uint8) for m in cfg.bits_per_symbol]
    x = synth.transmit_grid(cfg, dmrs, bits)
    n0 = cfg.noise_var
    noise = np.sqrt(n0 / 2.0) * (rng.standard_normal((cfg.num_rx_ant, 14, S))
                                + 1j * rng.standard_normal((cfg.num_rx_ant, 14, S)))
    if not noisy_pilots:
        noise[:, list(cfg.dmrs_symbols), :] = 0.0
    y = np.einsum("ubts,uts->bts", h, x) + noise
    return synth.Slot(cfg=cfg, y=y.astype(np.complex64), dmrs=np.asarray(dmrs, dtype=np.complex64), bits=bits,
                      h=h, x=x)


def collinear_slot(num_users, num_prb, snr_db, eps, seed, num_rx_ant=4):
    """Users whose channels share one steering vector up to a perturbation of
    relative size ``eps`` (flat in time and frequency), seeded QPSK pilots on
    DMRS symbols {2, 11}: an ill-conditioned U x U LMMSE system on every RE."""
    rng = np.random.Generator(np.random.PCG64(seed))
    cfg = synth.SlotConfig(num_prb=num_prb, num_users=num_users, num_rx_ant=num_rx_ant, dmrs_symbols=(2, 11),
                           bits_per_symbol=tuple([2, 4, 6, 4][:num_users]), snr_db=snr_db, num_taps=1,
                           delay_spread_s=0.0, doppler_hz=0.0, ula=False)
    a = np.exp(1j * np.pi * np.arange(num_rx_ant) * np.sin(0.3))
    h = np.zeros((num_users, num_rx_ant, 14, cfg.num_subcarriers), dtype=np.complex128)
    for u in range(num_users):
        gain = (rng.standard_normal() + 1j * rng.standard_normal()) / np.sqrt(2.0)
        pert = eps * (rng.standard_normal(num_rx_ant) + 1j * rng.standard_normal(num_rx_ant)) / np.sqrt(2.0)
        h[u] = (gain * a + pert)[:, None, None]
    return _slot_from_channel(cfg, synth.slot_dmrs(cfg, rng), h, rng)


def exact_pivot_slot(num_users, num_prb, snr_db, seed, num_rx_ant=4, scale=128.0, delta=1.0 / 64.0):
    """A slot whose U x U LMMSE system is ill-conditioned through a strong,
    nearly collinear channel while the LS + interpolation front end is exact
    in FP32: DMRS base sequence r(m) = 1 on one DMRS symbol, noise-free DMRS
    symbol, and a channel flat in time and frequency whose entries are short
    dyadic numbers (user u: scale * e^{j pi b / 2} on antenna b, plus delta on
    antenna u mod B).  The Gram matrix then has a largest eigenvalue of about
    U * B * scale^2 and pivots that spread far beyond 1e6 at SNR <= 20 dB."""
    rng = np.random.Generator(np.random.PCG64(seed))
    cfg = synth.SlotConfig(num_prb=num_prb, num_users=num_users, num_rx_ant=num_rx_ant, dmrs_symbols=(2,),
                           bits_per_symbol=tuple([2, 4, 6, 4][:num_users]), snr_db=snr_db, num_taps=1,
                           delay_spread_s=0.0, doppler_hz=0.0, ula=False)
    base = scale * np.array([1j ** b for b in range(num_rx_ant)], dtype=np.complex128)
    h = np.zeros((num_users, num_rx_ant, 14, cfg.num_subcarriers), dtype=np.complex128)
    for u in range(num_users):
        v = base.copy()
        v[u % num_rx_ant] += delta
        h[u] = v[:, None, None]
    dmrs = np.ones((1, cfg.num_subcarriers // 2), dtype=np.complex64)
    return _slot_from_channel(cfg, dmrs, h, rng, noisy_pilots=False)
