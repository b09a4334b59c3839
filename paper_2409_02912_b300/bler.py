"""Block error rates of the receivers' LLRs (``include/nrx_eval.h``): with
the (133, 171) convolutional code (GPU Viterbi decoding) and with the
5G-structured LDPC code (transport blocks, GPU layered min-sum decoding);
coded slots from the transmitter in ``synth``; the SNR at a target BLER.

Decoding runs in ``libnrx.so`` (``nrx_conv_decode``, ``nrx_ldpc_decode``);
this module marshals arguments and counts errors.
"""
from __future__ import annotations

import ctypes
import dataclasses
from typing import Callable, List, Optional, Sequence

import numpy as np

from . import nrx, synth

EVAL_EXPORTED = ("nrx_conv_decode", "nrx_ldpc_decode")

_configured = False


def load():
    global _configured
    lib = nrx.load()
    if not _configured:
        P, I32 = ctypes.c_void_p, ctypes.c_int32
        lib.nrx_conv_decode.argtypes = [I32, I32, P, P, P, P, P]
        lib.nrx_conv_decode.restype = ctypes.c_int
        lib.nrx_ldpc_decode.argtypes = [I32, P, P, I32, I32, I32, I32, I32, P, P, P, I32, ctypes.c_float, I32, P, P,
                                        P]
        lib.nrx_ldpc_decode.restype = ctypes.c_int
        _configured = True
    return lib


def conv_decode(llr, block_offset, n_info: int, perm=None, out=None, stream=None):
    """Viterbi-decode blocks read from the device LLR vector ``llr`` (float32)
    at device int64 offsets ``block_offset`` through the optional device int32
    interleaver ``perm``; returns device uint8 [n_blocks, n_info]."""
    import torch
    nb = int(block_offset.numel())
    if out is None:
        out = torch.empty((nb, n_info), dtype=torch.uint8, device=llr.device)
    st = load().nrx_conv_decode(nb, n_info, llr.data_ptr(), block_offset.data_ptr(),
                                None if perm is None else perm.data_ptr(), out.data_ptr(), nrx._stream_ptr(stream))
    if st != nrx.NRX_OK:
        raise nrx.NrxError(st, "nrx_conv_decode")
    return out


def ldpc_decode(llr, block_offset, E: int, qm: int, Z: int, bg: synth.LdpcBaseGraph, iterations: int = 20,
                alpha: float = 0.75, stop_early: bool = True, stream=None):
    """Layered min-sum decoding (``nrx_ldpc_decode``) of the code blocks whose
    E received LLRs start at the device int64 offsets ``block_offset`` of the
    device float32 vector ``llr``; returns device uint8 [n_blocks, kb Z]."""
    import torch
    nb = int(block_offset.numel())
    row_ptr, col, shift = (np.ascontiguousarray(a, dtype=np.int32) for a in bg.edges())
    out = torch.empty((nb, bg.kb * Z), dtype=torch.uint8, device=llr.device)
    c2v = torch.empty(max(1, nb * int(row_ptr[-1]) * Z), dtype=torch.float32, device=llr.device)
    st = load().nrx_ldpc_decode(nb, llr.data_ptr(), block_offset.data_ptr(), E, qm, Z, bg.kb, bg.mb,
                                row_ptr.ctypes.data, col.ctypes.data, shift.ctypes.data, iterations, alpha,
                                int(bool(stop_early)), c2v.data_ptr(), out.data_ptr(), nrx._stream_ptr(stream))
    if st != nrx.NRX_OK:
        raise nrx.NrxError(st, "nrx_ldpc_decode")
    return out


@dataclasses.dataclass
class CodedBatch:
    """Same-geometry slots whose users carry interleaved code blocks, with
    each block's offset in the batch's packed LLR vector (slots back to back,
    users concatenated, user u holding n_data * m_u LLRs)."""

    slots: List[synth.Slot]
    info: np.ndarray          # uint8 [n_blocks, n_info]
    offsets: np.ndarray       # int64 [n_blocks]
    n_info: int
    perm: np.ndarray          # int32 [2 (n_info + 6)]

    @property
    def bits(self) -> List[List[int]]:
        return [list(s.cfg.bits_per_symbol) for s in self.slots]

    @property
    def noise_vars(self) -> List[float]:
        return [s.cfg.noise_var for s in self.slots]


def coded_batch(cfgs: Sequence[synth.SlotConfig], seeds: Sequence[int], n_info: int = 1024,
                perm_seed: int = 7) -> CodedBatch:
    perm = synth.interleaver(2 * (n_info + synth.CONV_TAIL), perm_seed)
    slots, infos, offs = [], [], []
    base = 0
    for cfg, seed in zip(cfgs, seeds):
        sl, users = synth.make_coded_slot(cfg, np.random.Generator(np.random.PCG64(seed)), n_info, perm)
        n_data = cfg.num_data_symbols * cfg.num_subcarriers
        ub = base
        for m, cu in zip(cfg.bits_per_symbol, users):
            infos.append(cu.info)
            offs.append(ub + cu.block_offset)
            ub += n_data * m
        base = ub
        slots.append(sl)
    return CodedBatch(slots=slots, info=np.concatenate(infos), offsets=np.concatenate(offs), n_info=n_info,
                      perm=perm)


def block_errors(llr, batch: CodedBatch) -> tuple:
    """(block errors, blocks, info-bit errors, info bits) of a packed device
    LLR vector of ``batch``."""
    import torch
    dev = llr.device
    dec = conv_decode(llr, torch.from_numpy(batch.offsets).to(dev), batch.n_info,
                      torch.from_numpy(batch.perm).to(dev)).cpu().numpy()
    err = dec != batch.info
    return int(err.any(axis=1).sum()), int(err.shape[0]), int(err.sum()), int(err.size)


@dataclasses.dataclass
class LdpcBatch:
    """Same-geometry slots whose users each carry one transport block of
    rate-matched LDPC code blocks (``synth.make_ldpc_slot``)."""

    slots: List[synth.Slot]
    bg: synth.LdpcBaseGraph
    users: List[List[synth.LdpcUser]]   # per slot, per user
    stream_offset: List[List[int]]       # per slot, per user: first LLR of the user in the packed vector

    @property
    def bits(self) -> List[List[int]]:
        return [list(s.cfg.bits_per_symbol) for s in self.slots]

    @property
    def noise_vars(self) -> List[float]:
        return [s.cfg.noise_var for s in self.slots]


def ldpc_batch(cfgs: Sequence[synth.SlotConfig], seeds: Sequence[int], bg: Optional[synth.LdpcBaseGraph] = None,
               rate: float = 0.5) -> LdpcBatch:
    bg = synth.ldpc_base_graph() if bg is None else bg
    slots, users, offs = [], [], []
    base = 0
    for cfg, seed in zip(cfgs, seeds):
        sl, us = synth.make_ldpc_slot(cfg, np.random.Generator(np.random.PCG64(seed)), bg, rate)
        n_data = cfg.num_data_symbols * cfg.num_subcarriers
        o = []
        for m in cfg.bits_per_symbol:
            o.append(base)
            base += n_data * m
        slots.append(sl)
        users.append(us)
        offs.append(o)
    return LdpcBatch(slots=slots, bg=bg, users=users, stream_offset=offs)


def tb_errors(llr, batch: LdpcBatch, iterations: int = 20) -> tuple:
    """(transport-block errors, transport blocks) of a packed device LLR
    vector of ``batch``: a user's block is in error when any of its code
    blocks decodes to a wrong information bit.  Code blocks with the same
    (Z, E, modulation order) are decoded in one call."""
    import torch
    groups = {}
    for si, (sl, us, offs) in enumerate(zip(batch.slots, batch.users, batch.stream_offset)):
        for ui, (cu, o, m) in enumerate(zip(us, offs, sl.cfg.bits_per_symbol)):
            for c in range(cu.info.shape[0]):
                groups.setdefault((cu.Z, cu.E, m), []).append((si, ui, o + c * cu.E, cu.info[c]))
    bad = set()
    for (Z, E, m), items in groups.items():
        offs = torch.tensor([it[2] for it in items], dtype=torch.int64, device=llr.device)
        dec = ldpc_decode(llr, offs, E, m, Z, batch.bg, iterations=iterations).cpu().numpy()
        for (si, ui, _, info), d in zip(items, dec):
            if not np.array_equal(d, info):
                bad.add((si, ui))
    n_tb = sum(len(us) for us in batch.users)
    return len(bad), n_tb


def snr_at_bler(snrs: Sequence[float], bler: Sequence[float], target: float = 0.1) -> Optional[float]:
    """SNR where the BLER curve crosses ``target`` (linear in SNR, log in
    BLER, between the first bracketing pair of grid points); None when the
    grid does not bracket it."""
    for i in range(len(snrs) - 1):
        a, b = bler[i], bler[i + 1]
        if a >= target > b:
            la = np.log10(max(a, 1e-9))
            lb = np.log10(max(b, 1e-9))
            f = (la - np.log10(target)) / (la - lb) if la != lb else 0.0
            return float(snrs[i] + f * (snrs[i + 1] - snrs[i]))
    return None


def bler_curve(detect: Callable, batches: Sequence[CodedBatch]) -> List[float]:
    """BLER of a receiver on each batch; ``detect(batch) -> packed device LLRs``."""
    out = []
    for b in batches:
        e, n, _, _ = block_errors(detect(b), b)
        out.append(e / max(n, 1))
    return out
