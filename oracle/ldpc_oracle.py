"""FP64 oracle of the quasi-cyclic LDPC decoding used for transport-block
error rates (the paper's receiver hands its LLRs to the 5G LDPC decoder,
Sec. II; TBLER in Fig. 3).

Test infrastructure: only the tests, the smoke check and the benchmark's CPU
leg use this module; the CUDA path never does.

The code is given by a base matrix V (int [mb, nb], -1 for an all-zero block,
else a circulant shift) and a lifting size Z: check r Z + i is connected to
variable c Z + ((i + V[r, c]) mod Z) for every nonzero block (r, c), so the
parity-check matrix is H = [P^(V[r,c] mod Z)] with (P^v x)[i] = x[(i+v) mod Z].
Receiver LLRs are ln P(b=1)/P(b=0) (Eq. 2); the decoders work on
L = ln P(b=0)/P(b=1) = -llr internally and return hard bits (1 where L < 0).

Functions:
  syndrome            H x over GF(2) (the definition of a codeword)
  rate_recover        inverse of the rate matching of TS 38.212 Sec. 5.4.2:
                      de-interleave and accumulate the E LLRs of a block into
                      the circular buffer, punctured and unsent positions 0
  sum_product         flooding belief propagation with the tanh rule
  layered_min_sum     row-layered normalised min-sum (the GPU decoder's
                      algorithm, in the same layer and edge order)
"""
from __future__ import annotations

import numpy as np


def _edges(V: np.ndarray, Z: int):
    """Lifted edges: (check index, variable index) arrays, grouped by base row
    then base column then i."""
    V = np.asarray(V)
    rows, cols = np.nonzero(V >= 0)
    i = np.arange(Z)
    chk = (rows[:, None] * Z + i[None, :]).reshape(-1)
    var = (cols[:, None] * Z + (i[None, :] + (V[rows, cols] % Z)[:, None]) % Z).reshape(-1)
    return chk, var


def syndrome(V: np.ndarray, Z: int, bits: np.ndarray) -> np.ndarray:
    """H x mod 2 for codeword candidates bits (uint8 [..., nb Z]) -> [..., mb Z]."""
    V = np.asarray(V)
    chk, var = _edges(V, Z)
    x = np.asarray(bits, dtype=np.int64)
    mbZ = V.shape[0] * Z
    out = np.zeros(x.shape[:-1] + (mbZ,), dtype=np.int64)
    np.add.at(out, (..., chk), x[..., var])
    return (out % 2).astype(np.uint8)


def rate_recover(llr_e: np.ndarray, Z: int, nb: int, qm: int) -> np.ndarray:
    """Codeword LLRs [nb Z] from the E received LLRs of one block: undo the
    qm-row bit interleaver (bit i of symbol j was e[i E/qm + j]), then add
    e[k] into circular-buffer position k mod (nb - 2) Z, which is codeword
    position 2 Z + that; the 2 Z punctured systematic bits stay 0."""
    f = np.asarray(llr_e, dtype=np.float64)
    E = f.shape[-1]
    e = f.reshape(E // qm, qm).T.reshape(-1)
    ncb = (nb - 2) * Z
    out = np.zeros(nb * Z)
    np.add.at(out, 2 * Z + np.arange(E) % ncb, e)
    return out


def sum_product(llr: np.ndarray, V: np.ndarray, Z: int, iterations: int = 30, stop_early: bool = True):
    """Flooding belief propagation.  llr: receiver LLRs [nb Z] (ln P1/P0).
    Each check-to-variable message is 2 atanh(prod over the check's other
    edges of tanh(v/2)), v the variable-to-check messages (posterior minus the
    check's own previous message).  Returns (hard bits uint8 [nb Z],
    posterior L = ln P0/P1 [nb Z], iterations run)."""
    V = np.asarray(V)
    chk, var = _edges(V, Z)
    order = np.argsort(chk, kind="stable")
    chk_s, var_s = chk[order], var[order]
    starts = np.r_[0, np.nonzero(np.diff(chk_s))[0] + 1]
    L0 = -np.asarray(llr, dtype=np.float64)
    post = L0.copy()
    c2v = np.zeros(chk_s.size)
    it = 0
    for it in range(1, iterations + 1):
        v2c = post[var_s] - c2v
        t = np.tanh(np.clip(v2c, -60.0, 60.0) / 2.0)
        sgn = np.where(t < 0, -1.0, 1.0)
        mag = np.maximum(np.abs(t), 1e-300)
        logm = np.log(mag)
        neg = (sgn < 0).astype(np.int64)
        sum_log = np.add.reduceat(logm, starts)
        cnt_neg = np.add.reduceat(neg, starts)
        deg = np.diff(np.r_[starts, chk_s.size])
        grp = np.repeat(np.arange(starts.size), deg)
        ext_mag = np.exp(sum_log[grp] - logm)              # product of the other |tanh|
        ext_sgn = np.where((cnt_neg[grp] - neg) % 2 == 1, -1.0, 1.0)
        c2v = 2.0 * np.arctanh(np.clip(ext_sgn * ext_mag, -1 + 1e-15, 1 - 1e-15))
        post = L0 + np.bincount(var_s, weights=c2v, minlength=L0.size)
        hard = (post < 0).astype(np.uint8)
        if stop_early and not syndrome(V, Z, hard).any():
            break
    return (post < 0).astype(np.uint8), post, it


def layered_min_sum(llr: np.ndarray, V: np.ndarray, Z: int, iterations: int = 20, alpha: float = 0.75,
                    stop_early: bool = False, dtype=np.float64):
    """Row-layered normalised min-sum: base rows in order; for row r and each
    of its Z checks, with t_e = post[v_e] - c2v_e over the row's edges e (in
    column order), the new message is alpha * (product of the other signs) *
    (the smallest other |t|), and post[v_e] = t_e + new message.  With
    stop_early, stops after an iteration whose hard decisions satisfy every
    check.  Returns (hard bits uint8 [nb Z], posterior L [nb Z], iterations run).

    ``dtype`` is the arithmetic of the messages and posteriors.  The hard
    decisions are integers decided by floating point, so a comparison with a
    decoder that runs in FP32 takes them in FP32 (``np.float32``): each
    message is then alpha * sign rounded once by the multiplication with the
    magnitude, and each posterior once by the addition."""
    V = np.asarray(V)
    L = -np.asarray(llr, dtype=np.float64).astype(dtype)
    alpha = dtype(alpha)
    post = L.copy()
    mb = V.shape[0]
    i = np.arange(Z)
    row_vars = []
    for r in range(mb):
        cols = np.nonzero(V[r] >= 0)[0]
        row_vars.append(np.stack([c * Z + (i + V[r, c] % Z) % Z for c in cols]))  # [d, Z]
    c2v = [np.zeros(rv.shape, dtype=dtype) for rv in row_vars]
    it = 0
    for it in range(1, iterations + 1):
        for r in range(mb):
            vs = row_vars[r]
            t = post[vs] - c2v[r]
            a = np.abs(t)
            sgn = np.where(t < 0, -1.0, 1.0).astype(dtype)
            tot = np.prod(sgn, axis=0)
            amin = np.argmin(a, axis=0)  # first minimum in edge order
            srt = np.sort(a, axis=0)
            m1, m2 = srt[0], srt[1] if a.shape[0] > 1 else srt[0]
            mag = np.where(np.arange(a.shape[0])[:, None] == amin[None, :], m2[None, :], m1[None, :])
            new = alpha * (tot[None, :] * sgn) * mag
            c2v[r] = new
            post[vs] = t + new
        if stop_early and not syndrome(V, Z, (post < 0).astype(np.uint8)).any():
            break
    return (post < 0).astype(np.uint8), post, it
