"""Pins of the TS 38.211 Sec. 5.2.1 pseudo-random sequence and the PUSCH DMRS
generator (transmitter side): the step-wise generator against jump-ahead by
GF(2) companion-matrix powers (an independent algorithm for the same linear
recurrences), and the DMRS mapping and c_init formula."""
import numpy as np

from paper_2409_02912_b300 import synth


def _companion(taps):
    """31x31 GF(2) matrix A with (x(n+1..n+31)) = A (x(n..n+30)), where
    x(n+31) = xor of x(n+t) over taps."""
    A = np.zeros((31, 31), dtype=np.int64)
    for i in range(30):
        A[i, i + 1] = 1
    for t in taps:
        A[30, t] = 1
    return A


def _matpow(A, e):
    R = np.eye(A.shape[0], dtype=np.int64)
    B = A.copy()
    while e:
        if e & 1:
            R = (R @ B) % 2
        B = (B @ B) % 2
        e >>= 1
    return R


def _jump(init, taps, n):
    """x(n) of the recurrence from the initial 31 values by A^n."""
    v = (_matpow(_companion(taps), n) @ np.asarray(init, dtype=np.int64)) % 2
    return int(v[0])


def test_gold_sequence_matches_jump_ahead():
    rng = np.random.Generator(np.random.PCG64(5))
    x1_0 = [1] + [0] * 30
    for c_init in (0, 1, 0x7FFFFFFF, int(rng.integers(0, 2 ** 31))):
        c = synth.gold_sequence(c_init, 300)
        x2_0 = [(c_init >> i) & 1 for i in range(31)]
        for n in (0, 1, 2, 27, 28, 29, 150, 299):
            ref = _jump(x1_0, (0, 3), 1600 + n) ^ _jump(x2_0, (0, 1, 2, 3), 1600 + n)
            assert c[n] == ref, (c_init, n)


def test_gold_sequence_is_balanced_and_c_init_sensitive():
    a = synth.gold_sequence(1234567, 20000)
    b = synth.gold_sequence(1234568, 20000)
    assert abs(a.mean() - 0.5) < 0.02 and abs((a ^ b).mean() - 0.5) < 0.02


def test_dmrs_c_init_and_mapping():
    assert synth.dmrs_c_init(0, 2, 0, 0) == 2 ** 17 * 3
    assert synth.dmrs_c_init(3, 11, 500, 1) == (2 ** 17 * (14 * 3 + 12) * 1001 + 1001) % 2 ** 31
    r = synth.dmrs_gold(2, (2, 11), 3, 77, 0)
    assert r.shape == (2, 12)
    assert np.allclose(np.abs(r), 1.0, atol=1e-6)
    c = synth.gold_sequence(synth.dmrs_c_init(3, 11, 77, 0), 24)
    assert np.allclose(r[1], ((1 - 2.0 * c[0::2]) + 1j * (1 - 2.0 * c[1::2])) / np.sqrt(2), atol=1e-7)


def test_gold_dmrs_slot_keeps_seeded_draws_otherwise():
    cfg = synth.SlotConfig(num_prb=2, num_users=1, num_rx_ant=1, dmrs_symbols=(2,), bits_per_symbol=(2,),
                           snr_db=10.0, num_taps=2, delay_spread_s=1e-7, doppler_hz=0.0, ula=False)
    a = synth.make_slot(cfg, np.random.Generator(np.random.PCG64(1)))
    g = synth.make_slot(synth.dataclasses.replace(cfg, n_id=10, slot_number=4),
                        np.random.Generator(np.random.PCG64(1)))
    assert np.allclose(g.dmrs, synth.dmrs_gold(2, (2,), 4, 10))
    assert not np.allclose(a.dmrs, g.dmrs)
