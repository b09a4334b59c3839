"""CPU oracle of the soft-input Viterbi decoder used for BLER evaluation.

TEST INFRASTRUCTURE ONLY (tests, smoke check and the benchmark's CPU leg).
It shares no code with the CUDA decoder.

The code is the textbook rate-1/2, constraint-length-7 convolutional code with
generators 133 and 171 (octal), zero-tail terminated; the receivers deliver
LLRs l = ln P(c=1)/P(c=0) (Eq. 2 sign), so the maximum-likelihood codeword
maximises sum_i c_i l_i.  The decoder is the Viterbi algorithm over the
64-state trellis, written from its definition:

* state = the six most recent inputs, newest in bit 5; input u moves state s
  to (u << 5) | (s >> 1), so the predecessors of s' are ((s' << 1) & 63) | b,
  b in {0, 1}, and the input is s' >> 5;
* the 7-bit register of a transition is (u << 6) | s, and output j is the
  parity of register & g_j;
* path metrics are float32 (the decoder's precision, so that both sides take
  the same integer decisions): candidate = (PM[s] + (c0 ? l0 : 0)) + (c1 ? l1 : 0);
  the b = 1 predecessor wins only when strictly larger; after each step the
  new metric of state 0 is subtracted from every state (renormalisation);
* start in state 0 (other states -inf), trace back from state 0 (zero tail).
"""
from __future__ import annotations

import numpy as np

G = (0o133, 0o171)
STATES = 64


def _parity(x: np.ndarray) -> np.ndarray:
    x = np.asarray(x, dtype=np.int64)
    p = np.zeros_like(x)
    for k in range(7):
        p ^= (x >> k) & 1
    return p


def transition_outputs():
    """For each new state s' and predecessor choice b: (c0, c1) of the
    transition from ((s' << 1) & 63) | b with input s' >> 5."""
    sp = np.arange(STATES)
    out = np.zeros((STATES, 2, 2), dtype=np.int64)
    for b in range(2):
        s = ((sp << 1) & 63) | b
        reg = ((sp >> 5) << 6) | s
        out[:, b, 0] = _parity(reg & G[0])
        out[:, b, 1] = _parity(reg & G[1])
    return out


def viterbi_decode(llr: np.ndarray, n_info: int) -> np.ndarray:
    """Decode one block: llr float [2 (n_info + 6)] in encoder output order
    -> info bits uint8 [n_info]."""
    l = np.asarray(llr, dtype=np.float32).reshape(-1, 2)
    T = l.shape[0]
    assert T == n_info + 6
    outs = transition_outputs()
    sp = np.arange(STATES)
    pred = np.stack([((sp << 1) & 63) | 0, ((sp << 1) & 63) | 1], axis=1)  # [64, 2]
    pm = np.full(STATES, -np.inf, dtype=np.float32)
    pm[0] = 0.0
    dec = np.zeros((T, STATES), dtype=np.uint8)
    zero = np.float32(0.0)
    for t in range(T):
        l0, l1 = l[t, 0], l[t, 1]
        cand = np.empty((STATES, 2), dtype=np.float32)
        for b in range(2):
            m0 = np.where(outs[:, b, 0] == 1, l0, zero).astype(np.float32)
            m1 = np.where(outs[:, b, 1] == 1, l1, zero).astype(np.float32)
            cand[:, b] = (pm[pred[:, b]] + m0) + m1
        take1 = cand[:, 1] > cand[:, 0]
        dec[t] = take1
        new = np.where(take1, cand[:, 1], cand[:, 0]).astype(np.float32)
        pm = (new - new[0]).astype(np.float32)
    s = 0
    bits = np.zeros(T, dtype=np.uint8)
    for t in range(T - 1, -1, -1):
        bits[t] = s >> 5
        s = ((s << 1) & 63) | int(dec[t, s])
    return bits[:n_info]
