"""Pins of the counter-based link simulator's reference (the numpy twin of the
GPU training simulator): the Philox4x32-10 known-answer vectors, and
statistical and structural properties of the simulated link (Eq. 1)."""
import os

import numpy as np

from paper_2409_02912_b300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def test_philox_known_answers():
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = synth.philox4x32(np.array([v[:4]], dtype=np.uint64), np.array([v[4:6]], dtype=np.uint64))[0]
        assert [int(x) for x in out] == v[6:10]


def _params(n, U, ula=True, doppler=200.0, taps=8, bits=(2, 4, 6, 4), n0=0.05):
    return [synth.SimSlot(noise_var=n0, delay_spread_s=150e-9, doppler_hz=doppler if i % 2 == 0 else 0.0,
                          num_taps=taps, ula=ula, bits_per_symbol=tuple(bits[:U])) for i in range(n)]


def test_received_grid_is_channel_times_symbols_plus_noise_of_variance_n0():
    """y - sum_u H_u x_u, with x rebuilt from the returned bits and pilots by
    the transmitter, is white noise of variance N0 (Eq. 1)."""
    U, B = 3, 4
    sl = _params(4, U, ula=False, n0=0.05)
    tb = synth.simulate_philox(sl, U, B, 6, (2, 11), 6, seed=9, batch=1)
    S = 72
    res = []
    for i in range(4):
        cfg = synth.SlotConfig(num_prb=6, num_users=U, num_rx_ant=B, dmrs_symbols=(2, 11),
                               bits_per_symbol=sl[i].bits_per_symbol, snr_db=0.0, num_taps=8,
                               delay_spread_s=150e-9, doppler_hz=0.0, ula=False)
        bits = [tb.bits[i, u, :, :sl[i].bits_per_symbol[u]] for u in range(U)]
        x = synth.transmit_grid(cfg, tb.dmrs[i], bits)
        h = tb.h[i, ..., 0::2] + 1j * tb.h[i, ..., 1::2]  # [U, 14, S, B]
        y_clean = np.einsum("utsb,uts->bts", h, x)
        res.append(tb.y[i] - y_clean)
    r = np.concatenate([v.reshape(-1) for v in res])
    assert abs(np.var(r) / 0.05 - 1.0) < 0.05
    assert abs(np.mean(r.real * r.imag)) < 0.05 * 0.05


def test_channel_power_bits_and_pilots():
    sl = _params(48, 2, ula=True)
    tb = synth.simulate_philox(sl, 2, 4, 4, (2,), 6, seed=3, batch=7)
    p = np.mean(tb.h[..., 0::2] ** 2 + tb.h[..., 1::2] ** 2)
    assert 0.8 < p < 1.2  # unit average power per antenna
    assert np.allclose(np.abs(tb.dmrs), 1.0, atol=1e-6)
    m = tb.m_u
    assert m.tolist() == [[2, 4]] * 48
    assert abs(tb.bits[:, 0, :, :2].mean() - 0.5) < 0.01 and tb.bits[:, 0, :, 2:].max() == 0


def test_counters_make_batches_reproducible_and_distinct():
    sl = _params(2, 2)
    a = synth.simulate_philox(sl, 2, 2, 2, (2, 11), 4, seed=5, batch=3)
    b = synth.simulate_philox(sl, 2, 2, 2, (2, 11), 4, seed=5, batch=3)
    c = synth.simulate_philox(sl, 2, 2, 2, (2, 11), 4, seed=5, batch=4)
    assert np.array_equal(a.y, b.y) and np.array_equal(a.bits, b.bits)
    assert not np.array_equal(a.bits, c.bits) and not np.allclose(a.y, c.y)
