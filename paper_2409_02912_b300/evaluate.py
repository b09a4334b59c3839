"""Matched-BLER comparison of the receivers (NRX in each precision, LS+LMMSE)
on coded synthetic slots: BLER over an SNR grid and the SNR at 10% BLER,
the operating point at which the paper compares receivers (Sec. IV).

Every step runs in ``libnrx.so`` (detection, Viterbi and LDPC decoding);
this module draws the slots (``synth``), calls the receivers and counts
errors.
"""
from __future__ import annotations

import dataclasses
import os
from typing import Dict, Optional, Sequence

import numpy as np

from . import bler, nrx, synth

WEIGHTS_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights")
# Trained by ``python -m paper_2409_02912_b300.train`` on 2-user, 4-Rx slots
# with QPSK / 16-QAM (the mu2_4rx_24prb network: C=64, R=2, N_it=2, m_max=4).
TRAINED_MU2 = os.path.join(WEIGHTS_DIR, "nrx_mu2_4rx_c64_r2_it2.bin")
# The same network with modulation-specific StateInit / ReadoutLLRs heads
# (Var-IO, Sec. III; blob version 2), initialised from the masked network's
# checkpoint and trained 135 k further steps on the GPU simulator.
TRAINED_MU2_VAR_IO = os.path.join(WEIGHTS_DIR, "nrx_mu2_4rx_c64_r2_it2_varIO.bin")
# The benchmarked network (mu4_4rx_273prb: C=64, R=2, N_it=2, m_max=6), trained
# at config 4's shape: 51-PRB slots, up to four users with the number of active
# users drawn per batch, QPSK / 16-QAM / 64-QAM, batches of 64, BF16 GEMMs with
# FP32 master weights, on the GPU simulator; started from TRAINED_MU2 with its
# read-out widened to six outputs.
TRAINED_MU4 = os.path.join(WEIGHTS_DIR, "nrx_mu4_4rx_c64_r2_it2.bin")


@dataclasses.dataclass(frozen=True)
class Sweep:
    """Coded-slot SNR sweep: by default the geometry of the mu2_4rx_24prb
    workload with one modulation order for both users; ``mcs`` draws each
    user's order per slot instead (the mixed-MCS 273-PRB 4-user workload);
    config-2 channel distributions."""

    num_prb: int = 24
    num_users: int = 2
    num_rx_ant: int = 4
    dmrs_symbols: tuple = (2, 11)
    bits: int = 4
    snrs: tuple = (2.0, 4.0, 6.0, 8.0, 10.0, 12.0, 14.0)
    slots_per_point: int = 32
    n_info: int = 1024
    seed: int = 900
    ldpc_rate: float = 0.5
    mcs: tuple = ()              # if given, each user's modulation order is drawn from it per slot
    ldpc_slots_per_point: int = 0  # slots per point of the LDPC sweep (0: slots_per_point)


# Coded sweep of the benchmarked workload: 273 PRB, four users, modulation order
# drawn per user and slot; 4 slots (~1300 convolutional code blocks) per SNR
# point, 32 slots (128 transport blocks, ~3000 LDPC code blocks) per point for
# the LDPC curve.
MU4_SWEEP = Sweep(num_prb=273, num_users=4, mcs=(2, 4, 6), snrs=(4.0, 8.0, 12.0, 16.0, 20.0, 24.0),
                  slots_per_point=4, ldpc_slots_per_point=32)


def _slot_cfg(sw: Sweep, snr: float, rng: np.random.Generator) -> synth.SlotConfig:
    bits = tuple(int(rng.choice(sw.mcs)) for _ in range(sw.num_users)) if sw.mcs else (sw.bits,) * sw.num_users
    return synth.SlotConfig(num_prb=sw.num_prb, num_users=sw.num_users, num_rx_ant=sw.num_rx_ant,
                            dmrs_symbols=sw.dmrs_symbols, bits_per_symbol=bits, snr_db=float(snr), num_taps=12,
                            delay_spread_s=float(rng.uniform(10e-9, 300e-9)),
                            doppler_hz=float(rng.uniform(0.0, 400.0)), ula=True)


def sweep_batches(sw: Sweep):
    out = []
    for k, snr in enumerate(sw.snrs):
        cfgs, seeds = [], []
        for i in range(sw.slots_per_point):
            seed = sw.seed * 100_000 + k * 1_000 + i
            rng = np.random.Generator(np.random.PCG64(seed))
            cfgs.append(_slot_cfg(sw, snr, rng))
            seeds.append(seed + 7)
        out.append(bler.coded_batch(cfgs, seeds, n_info=sw.n_info))
    return out


def ldpc_sweep_batches(sw: Sweep, bg=None):
    """The sweep's slot draws (different seeds from the convolutional-code
    slots) carrying LDPC transport blocks at rate ``sw.ldpc_rate``."""
    bg = synth.ldpc_base_graph() if bg is None else bg
    out = []
    for k, snr in enumerate(sw.snrs):
        cfgs, seeds = [], []
        for i in range(sw.ldpc_slots_per_point or sw.slots_per_point):
            seed = sw.seed * 100_000 + 50_000 + k * 1_000 + i
            rng = np.random.Generator(np.random.PCG64(seed))
            cfgs.append(_slot_cfg(sw, snr, rng))
            seeds.append(seed + 7)
        out.append(bler.ldpc_batch(cfgs, seeds, bg, sw.ldpc_rate))
    return out


def compare(blob: bytes, precisions: Sequence[str] = ("fp32", "bf16", "fp16", "fp8"), sw: Sweep = Sweep(),
            batches=None, untrained_blob: Optional[bytes] = None, early_exit: bool = True,
            ldpc: bool = True, ldpc_batches=None) -> Dict[str, dict]:
    """BLER curves and SNR at 10% BLER of the NRX (each precision) and of
    LS+LMMSE on the same coded slots; with ``early_exit`` also the FP32 NRX
    stopped after each number of CGNN iterations below N_it (the multi-loss
    read-outs, Sec. II-B and Sec. IV-B).  With ``ldpc``, each receiver also
    gets a transport-block error rate curve with the LDPC code ("tbler_ldpc"
    and "snr_at_10pct_tbler_ldpc"), on slots of its own."""
    import torch
    batches = sweep_batches(sw) if batches is None else batches
    if ldpc and ldpc_batches is None:
        ldpc_batches = ldpc_sweep_batches(sw)
    n = max(sw.slots_per_point, sw.ldpc_slots_per_point if ldpc else 0)
    dev = [(torch.from_numpy(synth.stack_batch(b.slots)).cuda(),
            torch.from_numpy(np.stack([s.dmrs for s in b.slots])).cuda()) for b in batches]
    ldev = [] if not ldpc else [(torch.from_numpy(synth.stack_batch(b.slots)).cuda(),
                                 torch.from_numpy(np.stack([s.dmrs for s in b.slots])).cuda()) for b in ldpc_batches]
    res: Dict[str, dict] = {}

    def run(name, rx, fn):
        curve = []
        for b, (y, dm) in zip(batches, dev):
            llr = fn(rx, b, y, dm)
            e, nb, _, _ = bler.block_errors(llr, b)
            curve.append(e / max(nb, 1))
        res[name] = {"bler": curve, "snr_at_10pct": bler.snr_at_bler(sw.snrs, curve, 0.1)}
        if ldpc:
            tcurve = []
            for b, (y, dm) in zip(ldpc_batches, ldev):
                e, nt = bler.tb_errors(fn(rx, b, y, dm), b)
                tcurve.append(e / max(nt, 1))
            res[name]["tbler_ldpc"] = tcurve
            res[name]["snr_at_10pct_tbler_ldpc"] = bler.snr_at_bler(sw.snrs, tcurve, 0.1)

    def nrx_fn(rx, b, y, dm):
        return rx.nrx_detect_batch(y, dm, sw.dmrs_symbols, b.bits)

    def lmmse_fn(rx, b, y, dm):
        return rx.lmmse_detect_batch(y, dm, sw.dmrs_symbols, b.bits, b.noise_vars)

    for p in precisions:
        rx = nrx.Receiver(blob, sw.num_rx_ant, sw.num_users, sw.num_prb, max_slots=n, precision=p)
        run(f"nrx_{p}", rx, nrx_fn)
        if p == precisions[0]:
            run("lmmse", rx, lmmse_fn)
        if early_exit and p == "fp32":
            for its in range(1, rx.iterations):
                run(f"nrx_fp32_it{its}", rx,
                    lambda r, b, y, dm, its=its: r.nrx_detect_batch(y, dm, sw.dmrs_symbols, b.bits, iterations=its))
        rx.close()
    if untrained_blob is not None:
        rx = nrx.Receiver(untrained_blob, sw.num_rx_ant, sw.num_users, sw.num_prb, max_slots=n, precision="fp32")
        run("nrx_untrained", rx, nrx_fn)
        rx.close()
    res["_sweep"] = {"snrs": list(sw.snrs), "blocks_per_point": int(batches[0].info.shape[0]),
                     "slots_per_point": sw.slots_per_point, "num_prb": sw.num_prb, "num_users": sw.num_users,
                     "bits": list(sw.mcs) if sw.mcs else sw.bits}
    if ldpc:
        b0 = ldpc_batches[0]
        res["_sweep"]["ldpc"] = {"transport_blocks_per_point": sum(len(u) for u in b0.users),
                                 "code_blocks_per_tb": int(b0.users[0][0].info.shape[0]),
                                 "Z": int(b0.users[0][0].Z), "E": int(b0.users[0][0].E), "rate": sw.ldpc_rate}
    return res
