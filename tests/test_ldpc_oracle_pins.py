"""Pins of the LDPC oracle (oracle/ldpc_oracle.py) and of the 5G-structured
code it decodes, against things other than themselves: the parity-check
definition (every encoded word has zero syndrome, and the encoder reaches
exactly the null space of H), exact bitwise MAP by enumeration on a tree code
(where belief propagation is exact), the closed form of a single check's
min-sum message, the inverse of the rate matching, and an AWGN waterfall.
CPU only."""
import itertools

import numpy as np
import pytest

from oracle import ldpc_oracle as LO
from paper_2409_02912_b300 import synth


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _gf2_rank(M: np.ndarray) -> int:
    M = (np.asarray(M) % 2).astype(np.uint8).copy()
    r = 0
    for c in range(M.shape[1]):
        piv = np.nonzero(M[r:, c])[0]
        if piv.size == 0:
            continue
        p = r + piv[0]
        M[[r, p]] = M[[p, r]]
        rows = np.nonzero(M[:, c])[0]
        rows = rows[rows != r]
        M[rows] ^= M[r]
        r += 1
        if r == M.shape[0]:
            break
    return r


def _dense_h(V, Z):
    chk, var = LO._edges(V, Z)
    H = np.zeros((V.shape[0] * Z, V.shape[1] * Z), dtype=np.uint8)
    H[chk, var] ^= 1
    return H


def test_lifting_sizes_are_the_38212_set():
    zs = synth.ldpc_lifting_sizes()
    assert len(zs) == 51 and zs[0] == 2 and zs[-1] == 384
    assert all(any(z == a << j for a in (2, 3, 5, 7, 9, 11, 13, 15) for j in range(8)) for z in zs)


@pytest.mark.parametrize("Z", [2, 7, 64, 320])
def test_encoded_words_have_zero_syndrome(Z):
    bg = synth.ldpc_base_graph()
    info = _rng(Z).integers(0, 2, size=(4, bg.kb * Z), dtype=np.uint8)
    cw = synth.ldpc_encode(bg, Z, info)
    assert np.array_equal(cw[:, :bg.kb * Z], info)  # systematic
    assert not LO.syndrome(bg.V, Z, cw).any()
    bad = cw.copy()
    bad[:, 5] ^= 1
    assert LO.syndrome(bg.V, Z, bad).any(axis=-1).all()


@pytest.mark.parametrize("kb,mb,Z", [(2, 4, 2), (3, 6, 3), (10, 42, 2)])
def test_encoder_spans_the_null_space_of_h(kb, mb, Z):
    """dim null(H) = nb Z - rank(H) equals kb Z and the encoder is injective:
    it reaches every codeword."""
    bg = synth.ldpc_base_graph(kb=kb, mb=mb, seed=3, check_z=())
    H = _dense_h(bg.V, Z)
    assert bg.nb * Z - _gf2_rank(H) == kb * Z
    K = kb * Z
    if K <= 12:
        infos = np.array(list(itertools.product([0, 1], repeat=K)), dtype=np.uint8)
        cws = synth.ldpc_encode(bg, Z, infos)
        assert len({c.tobytes() for c in cws}) == 2 ** K
        assert not LO.syndrome(bg.V, Z, cws).any()


def test_sum_product_is_exact_map_on_a_tree_code():
    """Two checks sharing one variable (x0+x1+x2 = 0, x2+x3+x4 = 0; Z = 1):
    the Tanner graph is a tree, so belief propagation returns the exact
    bitwise a-posteriori LLRs, computed here by enumerating the 8 codewords."""
    V = np.array([[0, 0, 0, -1, -1], [-1, -1, 0, 0, 0]])
    rng = _rng(5)
    words = [w for w in itertools.product([0, 1], repeat=5) if (w[0] ^ w[1] ^ w[2]) == 0 and (w[2] ^ w[3] ^ w[4]) == 0]
    words = np.array(words)
    for _ in range(5):
        llr = rng.normal(0.0, 2.0, size=5)  # ln P(1)/P(0) per bit
        logp = (words * llr).sum(axis=1)    # log-likelihood of each codeword (up to a constant)
        map_llr = np.array([np.logaddexp.reduce(logp[words[:, k] == 1]) - np.logaddexp.reduce(logp[words[:, k] == 0])
                            for k in range(5)])
        _, post, _ = LO.sum_product(llr, V, 1, iterations=4, stop_early=False)
        assert np.max(np.abs(-post - map_llr)) < 1e-9


def test_min_sum_single_check_closed_form():
    """One check of degree 5: each outgoing message is alpha times the product
    of the other inputs' signs times the smallest other magnitude."""
    V = np.array([[0, 0, 0, 0, 0]])
    llr = np.array([0.7, -2.0, 0.3, 1.5, -0.9])
    alpha = 0.75
    _, post, _ = LO.layered_min_sum(llr, V, 1, iterations=1, alpha=alpha)
    L = -llr
    for k in range(5):
        others = np.delete(L, k)
        want = L[k] + alpha * np.prod(np.sign(others)) * np.min(np.abs(others))
        assert abs(post[k] - want) < 1e-12


def test_min_sum_single_check_closed_form_fp32():
    """The same check in FP32: each message is alpha * sign times the smallest
    other magnitude, rounded once; each posterior is rounded once more."""
    V = np.array([[0, 0, 0, 0, 0]])
    llr = np.array([0.7, -2.0, 0.3, 1.5, -0.9], dtype=np.float32)
    _, post, _ = LO.layered_min_sum(llr, V, 1, iterations=1, alpha=0.75, dtype=np.float32)
    assert post.dtype == np.float32
    L = -llr
    for k in range(5):
        others = np.delete(L, k)
        msg = np.float32(0.75 * np.prod(np.sign(others))) * np.float32(np.min(np.abs(others)))
        assert post[k] == np.float32(L[k] + msg)


def test_min_sum_fp32_and_fp64_decode_the_same_block():
    """On a block that decodes, the FP32 and FP64 min-sum return the sent word."""
    bg = synth.ldpc_base_graph()
    Z = 32
    rng = _rng(5)
    info = rng.integers(0, 2, size=bg.kb * Z, dtype=np.uint8)
    cw = synth.ldpc_encode(bg, Z, info[None])[0]
    E = 2 * bg.kb * Z
    e = synth.ldpc_rate_match(bg, Z, cw[None], E, 1)[0]
    llr = -4.0 * (1.0 - 2.0 * e) + 1.5 * rng.standard_normal(E)  # ln P(1)/P(0)
    rec = LO.rate_recover(llr, Z, bg.nb, 1)
    for dt in (np.float64, np.float32):
        hard, _, _ = LO.layered_min_sum(rec, bg.V, Z, iterations=20, stop_early=True, dtype=dt)
        assert np.array_equal(hard, cw), dt


@pytest.mark.parametrize("E_mult", [0.4, 1.0, 1.7])
def test_rate_recover_inverts_rate_matching(E_mult):
    bg = synth.ldpc_base_graph()
    Z, qm = 16, 4
    ncb = (bg.nb - 2) * Z
    E = qm * int(E_mult * ncb / qm)
    pos = np.arange(bg.nb * Z, dtype=np.float64) + 1.0  # distinct values per codeword position
    # rate matching moves values: send the position values through it
    sent = synth.ldpc_rate_match(bg, Z, pos[None, :].astype(np.int64), E, qm)[0].astype(np.float64)
    got = LO.rate_recover(sent, Z, bg.nb, qm)
    want = np.zeros(bg.nb * Z)
    k = np.arange(E)
    np.add.at(want, 2 * Z + k % ncb, pos[2 * Z + k % ncb])
    assert np.array_equal(got, want)


def test_awgn_waterfall():
    """Rate 1/2 (K = 640, E = 1280, BPSK): sum-product block errors rare at
    Eb/N0 = 3 dB and nearly certain at -1 dB."""
    bg = synth.ldpc_base_graph()
    Z = 64
    K, E = bg.kb * Z, 2 * bg.kb * Z
    rng = _rng(11)

    def bler(ebn0_db, n):
        n0 = 1.0 / (2 * (K / E) * 10 ** (ebn0_db / 10))  # BPSK, Es = 1
        err = 0
        for _ in range(n):
            info = rng.integers(0, 2, size=K, dtype=np.uint8)
            e = synth.ldpc_rate_match(bg, Z, synth.ldpc_encode(bg, Z, info[None])[0][None], E, 1)[0]
            y = (1.0 - 2.0 * e) + np.sqrt(n0) * rng.standard_normal(E)
            llr = -2.0 * y / n0
            hard, _, _ = LO.sum_product(LO.rate_recover(llr, Z, bg.nb, 1), bg.V, Z, iterations=40)
            err += int(np.any(hard[:K] != info))
        return err / n

    assert bler(3.0, 40) <= 0.1
    assert bler(-1.0, 10) >= 0.9
