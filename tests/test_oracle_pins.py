"""Pins of the FP64 oracle against things other than itself: library routines
(scipy / torch convolutions and linear layers, numpy least squares), closed
forms (MRC, QPSK/16-QAM max-log, AWGN BER), exact cases (LS on noiseless
pilots, interpolation of affine channels), invariants (permutation
equivariance of message passing, masking of inactive users) and hand-worked
fixtures under tests/golden/.  CPU only."""
import os

import numpy as np
import pytest
import scipy.signal
import scipy.special
import torch

from oracle import nrx_oracle as O
from paper_2409_02912_b300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rng(seed=0):
    return np.random.Generator(np.random.PCG64(seed))


def _cfg(U=1, B=2, prb=2, dmrs=(2, 11), bits=None, snr=10.0):
    bits = bits or tuple([2] * U)
    return synth.SlotConfig(num_prb=prb, num_users=U, num_rx_ant=B, dmrs_symbols=dmrs,
                            bits_per_symbol=bits, snr_db=snr, num_taps=4,
                            delay_spread_s=100e-9, doppler_hz=0.0, ula=False)


def _noiseless_slot(cfg, h, rng):
    slot = synth.make_slot(cfg, rng, channel=h)
    y = np.einsum("ubts,uts->bts", h, slot.x)  # recompute without noise, in complex128
    return slot, y


# ----------------------------------------------------------------------------
# Constellation (Gray QAM, recursive labels: Sec. II, Sec. III)
# ----------------------------------------------------------------------------

def test_qam16_matches_ts38211_table():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "qam16_gray_ts38211.txt")) if not l.startswith("#")]
    labels, pts = O.constellation(4)
    table = {tuple(int(v) for v in r[:4]): complex(float(r[4]), float(r[5])) / np.sqrt(10) for r in rows}
    assert len(table) == 16
    for lab, p in zip(labels, pts):
        assert abs(table[tuple(int(b) for b in lab)] - p) < 1e-12


@pytest.mark.parametrize("m", [2, 4, 6])
def test_constellation_energy_gray_and_transmitter(m):
    labels, pts = O.constellation(m)
    assert abs(np.mean(np.abs(pts) ** 2) - 1.0) < 1e-12
    # Gray: nearest neighbours differ in exactly one bit
    dmin = np.min(np.abs(pts[:, None] - pts[None, :]) + 10 * np.eye(len(pts)))
    for i in range(len(pts)):
        for j in range(len(pts)):
            if i != j and abs(abs(pts[i] - pts[j]) - dmin) < 1e-9:
                assert int(np.sum(labels[i] != labels[j])) == 1
    # the transmitter's TS 38.211 formulas give the same points for the same labels
    assert np.allclose(synth.qam_modulate(labels, m), pts, atol=1e-12)


@pytest.mark.parametrize("m", [4, 6])
def test_recursive_labels_quadrant_is_qpsk(m):
    """Sec. III: points of a higher order within a quadrant carry the QPSK bits."""
    labels, pts = O.constellation(m)
    ql, qp = O.constellation(2)
    for lab, p in zip(labels, pts):
        k = int(np.argmin(np.abs(qp - (np.sign(p.real) + 1j * np.sign(p.imag)) / np.sqrt(2))))
        assert tuple(lab[:2]) == tuple(ql[k])


# ----------------------------------------------------------------------------
# Max-log demapper (Eq. 2 sign)
# ----------------------------------------------------------------------------

def test_maxlog_qpsk_closed_form():
    rng = _rng(1)
    x = rng.standard_normal(200) + 1j * rng.standard_normal(200)
    var = rng.uniform(0.05, 2.0, 200)
    l = O.maxlog_llr(x, var, 2)
    assert np.allclose(l[:, 0], -2 * np.sqrt(2) * x.real / var, atol=1e-12)
    assert np.allclose(l[:, 1], -2 * np.sqrt(2) * x.imag / var, atol=1e-12)


def test_maxlog_qpsk_equals_exact_app_for_flat_awgn():
    """QPSK on a flat channel: max-log equals the exact APP LLR of Eq. 2."""
    rng = _rng(2)
    y = rng.standard_normal(100) + 1j * rng.standard_normal(100)
    n0 = 0.3
    labels, pts = O.constellation(2)
    lik = np.exp(-np.abs(y[:, None] - pts[None, :]) ** 2 / n0)
    for i in range(2):
        exact = np.log(lik[:, labels[:, i] == 1].sum(1) / lik[:, labels[:, i] == 0].sum(1))
        assert np.allclose(O.maxlog_llr(y, np.full(100, n0), 2)[:, i], exact, atol=1e-9)


def test_maxlog_16qam_piecewise_linear():
    """Textbook per-dimension max-log expressions for Gray 16-QAM."""
    rng = _rng(3)
    x = 1.5 * (rng.standard_normal(500) + 1j * rng.standard_normal(500))
    var = np.full(500, 0.7)
    l = O.maxlog_llr(x, var, 4)
    for dim, comp in ((0, x.real), (1, x.imag)):
        a = np.sqrt(10) * comp
        sign_bit = np.where(np.abs(a) <= 2, -4 * a, -8 * a + 8 * np.sign(a)) / (10 * var)
        mag_bit = (4 * np.abs(a) - 8) / (10 * var)
        assert np.allclose(l[:, dim], sign_bit, atol=1e-9)
        assert np.allclose(l[:, 2 + dim], mag_bit, atol=1e-9)


@pytest.mark.parametrize("m", [4, 6])
def test_masked_demapper_sign_property(m):
    """Sec. III: a mismatched (masked) higher-order demapper gives the matched
    QPSK demapper's signs on the two sign bits."""
    rng = _rng(4)
    x = rng.standard_normal(1000) + 1j * rng.standard_normal(1000)
    var = np.full(1000, 0.5)
    hi = O.maxlog_llr(x, var, m)[:, :2]
    lo = O.maxlog_llr(x, var, 2)
    assert np.array_equal(np.sign(hi), np.sign(lo))


# ----------------------------------------------------------------------------
# LS estimation, interpolation, positional encoding
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("U", [1, 3])
def test_ls_exact_on_noiseless_pilots_single_port(U):
    """One port in the CDM group: per-pilot LS equals the channel exactly."""
    rng = _rng(5)
    cfg = _cfg(U=U, B=2, prb=2)
    S = cfg.num_subcarriers
    h = rng.standard_normal((U, 2, 14, S)) + 1j * rng.standard_normal((U, 2, 14, S))
    slot, y = _noiseless_slot(cfg, h, rng)
    u = U - 1 if U == 3 else 0  # the user alone in its group
    pos, est = O.ls_estimates(y, slot.dmrs, u, U, cfg.dmrs_symbols)
    g = u // 2
    for d, t in enumerate(cfg.dmrs_symbols):
        assert np.allclose(pos, np.arange(g, S, 2))
        assert np.max(np.abs(est[:, d] - h[u, :, t, g::2])) < 1e-12


def test_ls_exact_with_occ_when_flat_over_pilot_pair():
    """Two ports share a group: de-spread LS is exact when each user's channel
    is constant over every pilot pair."""
    rng = _rng(6)
    U, cfg = 4, _cfg(U=4, B=3, prb=3)
    S = cfg.num_subcarriers
    base = rng.standard_normal((U, 3, 14, S // 4)) + 1j * rng.standard_normal((U, 3, 14, S // 4))
    h = np.repeat(base, 4, axis=3)  # constant over 4-subcarrier blocks
    slot, y = _noiseless_slot(cfg, h, rng)
    for u in range(U):
        pos, est = O.ls_estimates(y, slot.dmrs, u, U, cfg.dmrs_symbols)
        assert np.allclose(pos, 4 * np.arange(S // 4) + 1 + u // 2)
        for d, t in enumerate(cfg.dmrs_symbols):
            assert np.max(np.abs(est[:, d] - h[u, :, t][:, pos.astype(int)])) < 1e-12


@pytest.mark.parametrize("U,dmrs", [(1, (2, 11)), (3, (2, 11)), (2, (3, 10)), (1, (2,))])
def test_interpolation_exact_on_affine_channel(U, dmrs):
    """Linear interpolation reproduces a channel affine in (s, t) inside the
    pilot hull and holds the edge values outside it.  For OCC groups the
    channel is affine in t and flat in s (otherwise the pair average is not
    the midpoint value)."""
    rng = _rng(7)
    cfg = _cfg(U=U, B=2, prb=2, dmrs=dmrs)
    S = cfg.num_subcarriers
    s = np.arange(S)[None, :]
    t = np.arange(14)[:, None]
    h = np.zeros((U, 2, 14, S), dtype=np.complex128)
    for u in range(U):
        for b in range(2):
            c = rng.standard_normal(3) + 1j * rng.standard_normal(3)
            slope_s = c[1] if not O.group_shared(u, U) else 0.0
            slope_t = c[2] if len(dmrs) == 2 else 0.0
            h[u, b] = c[0] + 0.05 * slope_s * s + 0.05 * slope_t * t
    slot, y = _noiseless_slot(cfg, h, rng)
    H = O.channel_estimate(y, slot.dmrs, U, dmrs)
    for u in range(U):
        pos, _ = O.ls_estimates(y, slot.dmrs, u, U, dmrs)
        lo, hi = int(pos[0]), int(pos[-1])
        tl, th = (dmrs[0], dmrs[-1])
        sc = np.clip(np.arange(S), lo, hi)
        tc = np.clip(np.arange(14), tl, th)
        want = h[u][:, tc][:, :, sc]
        assert np.max(np.abs(H[u] - want)) < 1e-12


def test_positional_encoding_hand_values():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "pe_dmrs2_11_s12.txt")) if not l.startswith("#")]
    for r in rows:
        if r[0] == "t":
            pe = O.positional_encoding(0, 12, (2, 11))
            assert abs(pe[int(r[1]), 0, 0] * 7 - float(r[2])) < 1e-12
        else:
            u = 2 * int(r[1])
            pe = O.positional_encoding(u, 12, (2, 11))
            assert abs(pe[0, int(r[2]), 1] * 2 - float(r[3])) < 1e-12


# ----------------------------------------------------------------------------
# Layers
# ----------------------------------------------------------------------------

def test_depthwise_matches_scipy_and_torch():
    rng = _rng(8)
    x = rng.standard_normal((14, 12, 4))
    k = rng.standard_normal((4, 3, 3))
    out = O.depthwise3x3(x, k)
    for c in range(4):
        ref = scipy.signal.correlate2d(x[:, :, c], k[c], mode="same", boundary="fill", fillvalue=0)
        assert np.max(np.abs(out[:, :, c] - ref)) < 1e-12
    tx = torch.from_numpy(x).permute(2, 0, 1)[None]
    tk = torch.from_numpy(k)[:, None]
    ref = torch.nn.functional.conv2d(tx, tk, padding=1, groups=4)[0].permute(1, 2, 0).numpy()
    assert np.max(np.abs(out - ref)) < 1e-12


def test_dense_matches_torch_linear():
    rng = _rng(9)
    x = rng.standard_normal((14, 12, 10))
    w = rng.standard_normal((6, 10))
    b = rng.standard_normal(6)
    ref = torch.nn.functional.linear(torch.from_numpy(x), torch.from_numpy(w), torch.from_numpy(b)).numpy()
    assert np.max(np.abs(O.dense(x, w, b) - ref)) < 1e-12


def _torch_nrx(y, dmrs, U, dmrs_syms, bits, W, net):
    """The NRX layer stack re-expressed with torch library layers (NCHW conv2d
    with groups=C for depthwise, 1x1 via linear), fed the oracle's features."""
    F = torch.nn.functional
    S = y.shape[2]
    H = O.channel_estimate(y, dmrs, U, dmrs_syms)
    pes = [O.positional_encoding(u, S, dmrs_syms) for u in range(U)]
    Wt = {k: torch.from_numpy(np.asarray(v, dtype=np.float64)) for k, v in W.items()}

    def dw(x, k):  # x [U, T, S, C]
        C = x.shape[-1]
        return F.conv2d(x.permute(0, 3, 1, 2), k[:, None], padding=1, groups=C).permute(0, 2, 3, 1)

    x = torch.stack([torch.from_numpy(O.input_features(y, H[u], pes[u])) for u in range(U)])
    pe = torch.stack([torch.from_numpy(p) for p in pes])
    st = F.relu(dw(F.linear(x, Wt["init.pw.w"], Wt["init.pw.b"]), Wt["init.dw"]))
    for k in range(net.iterations):
        p = f"it{k}."
        m = F.linear(F.relu(F.linear(st, Wt[p + "mp1.w"], Wt[p + "mp1.b"])), Wt[p + "mp2.w"], Wt[p + "mp2.b"])
        a = m.sum(0, keepdim=True) - m
        z = F.linear(torch.cat([st, a, pe], -1), Wt[p + "in.w"], Wt[p + "in.b"])
        for r in range(net.res_blocks):
            q = f"{p}blk{r}."
            hh = F.relu(F.linear(dw(z, Wt[q + "dw1"]), Wt[q + "pw1.w"], Wt[q + "pw1.b"]))
            z = z + F.linear(F.relu(dw(hh, Wt[q + "dw2"])), Wt[q + "pw2.w"], Wt[q + "pw2.b"])
        st = st + z
    l = F.linear(F.relu(F.linear(st, Wt["ro1.w"], Wt["ro1.b"])), Wt["ro2.w"], Wt["ro2.b"]).numpy()
    return O.pack_llrs(l, bits, dmrs_syms)


@pytest.mark.parametrize("U", [1, 2, 4])
def test_nrx_forward_matches_torch_layer_stack(U):
    net = synth.NetConfig(num_rx_ant=2, channels=8, res_blocks=2, iterations=2, m_max=6)
    W = synth.make_weights(net, seed=11)
    rng = _rng(10)
    bits = tuple([2, 4, 6, 4][:U])
    cfg = synth.SlotConfig(num_prb=2, num_users=U, num_rx_ant=2, dmrs_symbols=(2, 11),
                           bits_per_symbol=bits, snr_db=5.0, num_taps=4, delay_spread_s=200e-9,
                           doppler_hz=100.0, ula=False)
    sl = synth.make_slot(cfg, rng)
    ours = O.nrx_forward(sl.y, sl.dmrs, U, cfg.dmrs_symbols, bits, W, 2, 2)
    ref = _torch_nrx(sl.y, sl.dmrs, U, cfg.dmrs_symbols, bits, W, net)
    assert ours.shape == (12 * 24 * sum(bits),)
    assert np.max(np.abs(ours - ref)) < 1e-10 * max(1.0, np.max(np.abs(ref)))


def test_nrx_zero_branches_is_readout_of_stateinit():
    """Zeroed CNN-update input layers and residual outputs leave the state
    unchanged, so the NRX reduces to ReadoutLLRs(StateInit(x))."""
    net = synth.NetConfig(num_rx_ant=2, channels=8, res_blocks=2, iterations=2, m_max=2)
    W = synth.zero_like_residual(net, synth.make_weights(net, seed=12))
    rng = _rng(11)
    cfg = _cfg(U=2, B=2, prb=2)
    sl = synth.make_slot(cfg, rng)
    ours = O.nrx_forward(sl.y, sl.dmrs, 2, cfg.dmrs_symbols, (2, 2), W, 2, 2)
    H = O.channel_estimate(sl.y, sl.dmrs, 2, cfg.dmrs_symbols)
    l = [O.readout(O.state_init(O.input_features(sl.y, H[u], O.positional_encoding(u, 24, cfg.dmrs_symbols)), W), W)
         for u in range(2)]
    assert np.max(np.abs(ours - O.pack_llrs(l, (2, 2), cfg.dmrs_symbols))) < 1e-12


# ----------------------------------------------------------------------------
# Message passing invariants (Sec. II-A)
# ----------------------------------------------------------------------------

def _one_iteration(states, pes, W, active, res_blocks=1):
    msgs = np.stack([O.messages(states[u], W, 0) for u in range(len(states))])
    agg = O.aggregate(msgs, active)
    return np.stack([O.cnn_update(states[u], agg[u], pes[u], W, 0, res_blocks) for u in active]), agg


def test_message_passing_permutation_equivariance():
    net = synth.NetConfig(num_rx_ant=2, channels=6, res_blocks=1, iterations=1, m_max=2)
    W = synth.make_weights(net, seed=13)
    rng = _rng(12)
    U = 4
    states = rng.standard_normal((U, 14, 8, 6))
    pes = rng.standard_normal((U, 14, 8, 2))
    out, _ = _one_iteration(states, pes, W, list(range(U)))
    perm = [2, 0, 3, 1]
    out_p, _ = _one_iteration(states[perm], pes[perm], W, list(range(U)))
    assert np.max(np.abs(out_p - out[perm])) < 1e-12


def test_single_user_aggregate_is_zero_and_inactive_users_ignored():
    net = synth.NetConfig(num_rx_ant=2, channels=6, res_blocks=1, iterations=1, m_max=2)
    W = synth.make_weights(net, seed=14)
    rng = _rng(13)
    states = rng.standard_normal((3, 14, 8, 6))
    pes = rng.standard_normal((3, 14, 8, 2))
    _, agg = _one_iteration(states[:1], pes[:1], W, [0])
    assert np.all(agg[0] == 0.0)
    msgs = np.stack([O.messages(states[u], W, 0) for u in range(3)])
    assert np.allclose(O.aggregate(msgs, [0, 1, 2])[1], msgs.sum(0) - msgs[1], atol=1e-12)
    garbage = states.copy()
    garbage[2] = np.nan
    a, _ = _one_iteration(states, pes, W, [0, 1])
    b, _ = _one_iteration(garbage, pes, W, [0, 1])
    assert np.array_equal(a, b)


# ----------------------------------------------------------------------------
# LMMSE (the LS + LMMSE baseline)
# ----------------------------------------------------------------------------

def test_lmmse_zero_noise_is_zero_forcing_lstsq():
    rng = _rng(15)
    U, B, n = 3, 4, 50
    H = rng.standard_normal((U, B, n)) + 1j * rng.standard_normal((U, B, n))
    y = rng.standard_normal((B, n)) + 1j * rng.standard_normal((B, n))
    xhat, xt, _ = O.lmmse_equalize(y, H, 0.0)
    for i in range(n):
        ref = np.linalg.lstsq(H[:, :, i].T, y[:, i], rcond=None)[0]
        assert np.max(np.abs(xhat[:, i] - ref)) < 1e-10
        assert np.max(np.abs(xt[:, i] - ref)) < 1e-10


def test_lmmse_single_user_is_mrc():
    rng = _rng(16)
    B, n, n0 = 4, 80, 0.2
    h = rng.standard_normal((1, B, n)) + 1j * rng.standard_normal((1, B, n))
    y = rng.standard_normal((B, n)) + 1j * rng.standard_normal((B, n))
    xhat, xt, var = O.lmmse_equalize(y, h, n0)
    nh = np.sum(np.abs(h[0]) ** 2, axis=0)
    mrc = np.sum(np.conj(h[0]) * y, axis=0)
    d = nh / (nh + n0)
    assert np.max(np.abs(xhat[0] - mrc / (nh + n0))) < 1e-12
    assert np.max(np.abs(xt[0] - mrc / nh)) < 1e-12
    assert np.max(np.abs(var[0] - (1 / d - 1))) < 1e-12


def test_cholesky_solve_matches_numpy_solve():
    rng = _rng(17)
    A = rng.standard_normal((30, 4, 4)) + 1j * rng.standard_normal((30, 4, 4))
    G = np.conj(np.swapaxes(A, -1, -2)) @ A + 0.1 * np.eye(4)
    Bm = rng.standard_normal((30, 4, 3)) + 1j * rng.standard_normal((30, 4, 3))
    assert np.max(np.abs(O.cholesky_solve(G, Bm) - np.linalg.solve(G, Bm))) < 1e-10


@pytest.mark.parametrize("m,snr_db", [(2, 2.0), (4, 9.0)])
def test_awgn_ber_matches_closed_form(m, snr_db):
    """Flat known channel, B-antenna LMMSE (= scaled MRC for one user) and
    max-log hard decisions: Monte-Carlo BER inside a 99% binomial interval
    around the exact Gray QPSK / 16-QAM bit error rate."""
    rng = _rng(18 + m)
    B, n = 2, 60000
    n0 = 10 ** (-snr_db / 10)
    hv = np.array([0.8 + 0.3j, -0.4 + 0.5j])
    gamma = np.sum(np.abs(hv) ** 2) / n0
    bits = rng.integers(0, 2, size=(n, m))
    x = synth.qam_modulate(bits, m)
    y = hv[:, None] * x[None, :] + np.sqrt(n0 / 2) * (rng.standard_normal((B, n)) + 1j * rng.standard_normal((B, n)))
    H = np.repeat(hv[None, :, None], n, axis=2)
    _, xt, var = O.lmmse_equalize(y, H, n0)
    ber = np.mean((O.maxlog_llr(xt[0], var[0], m) > 0) != bits)
    Q = lambda v: 0.5 * scipy.special.erfc(v / np.sqrt(2))
    if m == 2:
        p = Q(np.sqrt(gamma))
    else:
        a = np.sqrt(gamma / 5)
        p = 0.25 * (3 * Q(a) + 2 * Q(3 * a) - Q(5 * a))
    nb = n * m
    half = 2.576 * np.sqrt(p * (1 - p) / nb)
    assert abs(ber - p) < half + 1e-4, (ber, p, half)


def test_pack_llrs_order_and_count():
    S, dm = 12, (2,)
    grids = [np.arange(14 * S * 6, dtype=float).reshape(14, S, 6) + 1e4 * u for u in range(2)]
    out = O.pack_llrs(grids, (2, 4), dm)
    assert out.size == O.llr_count(1, dm, (2, 4)) == 13 * 12 * 6
    # first user: data symbol 0 (t=0), s=0, bits 0,1; then s=1 ...
    assert out[0] == grids[0][0, 0, 0] and out[1] == grids[0][0, 0, 1] and out[2] == grids[0][0, 1, 0]
    # first RE of t=3 (the third data symbol after DMRS symbol 2) for user 0
    assert out[2 * 2 * S] == grids[0][3, 0, 0]
    off = 13 * 12 * 2
    assert out[off] == grids[1][0, 0, 0] and out[off + 3] == grids[1][0, 0, 3]


# ----------------------------------------------------------------------------
# Var-IO heads (Sec. III)
# ----------------------------------------------------------------------------

def _var_io_copy_of(net1, W1):
    """A Var-IO network whose every StateInit equals the single head and whose
    order-m ReadoutLLRs is the first m rows of the single ReadoutLLRs."""
    netv = synth.NetConfig(num_rx_ant=net1.num_rx_ant, channels=net1.channels, res_blocks=net1.res_blocks,
                           iterations=net1.iterations, m_max=net1.m_max, var_io=True)
    Wv = {}
    for name, _ in synth.weight_layout(netv):
        if name.startswith("init.m"):
            Wv[name] = W1["init." + name.split(".", 2)[2]]
        elif name.startswith("ro.m"):
            m = int(name.split(".")[1][1:])
            part = name.split(".", 2)[2]
            src = {"1.w": "ro1.w", "1.b": "ro1.b", "2.w": "ro2.w", "2.b": "ro2.b"}[part]
            Wv[name] = W1[src][:m] if part.startswith("2") else W1[src]
        else:
            Wv[name] = W1[name]
    return netv, Wv


def test_var_io_with_shared_heads_equals_masking():
    """Masking the shared head (Sec. III) and Var-IO heads that copy it give
    identical LLRs."""
    net1 = synth.NetConfig(num_rx_ant=2, channels=8, res_blocks=1, iterations=2, m_max=6)
    W1 = synth.make_weights(net1, seed=21)
    netv, Wv = _var_io_copy_of(net1, W1)
    assert netv.heads == (2, 4, 6)
    cfg = synth.SlotConfig(num_prb=2, num_users=3, num_rx_ant=2, dmrs_symbols=(2, 11), bits_per_symbol=(6, 2, 4),
                           snr_db=7.0, num_taps=4, delay_spread_s=1e-7, doppler_hz=50.0, ula=False)
    sl = synth.make_slot(cfg, _rng(31))
    a = O.nrx_forward(sl.y, sl.dmrs, 3, cfg.dmrs_symbols, cfg.bits_per_symbol, W1, 2, 1)
    b = O.nrx_forward(sl.y, sl.dmrs, 3, cfg.dmrs_symbols, cfg.bits_per_symbol, Wv, 2, 1)
    assert np.array_equal(a, b)


def test_var_io_heads_act_only_on_their_users():
    """Changing the 16-QAM heads changes the LLRs of the 16-QAM user (and,
    through message passing, the others'), while changing the unused 64-QAM
    head changes nothing."""
    netv = synth.NetConfig(num_rx_ant=2, channels=8, res_blocks=1, iterations=1, m_max=6, var_io=True)
    W = synth.make_weights(netv, seed=22)
    cfg = synth.SlotConfig(num_prb=2, num_users=2, num_rx_ant=2, dmrs_symbols=(2,), bits_per_symbol=(2, 4),
                           snr_db=7.0, num_taps=4, delay_spread_s=1e-7, doppler_hz=0.0, ula=False)
    sl = synth.make_slot(cfg, _rng(32))
    run = lambda Wx: O.nrx_forward(sl.y, sl.dmrs, 2, (2,), (2, 4), Wx, 1, 1)  # noqa: E731
    base = run(W)
    W6 = dict(W, **{"ro.m6.2.w": W["ro.m6.2.w"] + 1.0, "init.m6.pw.b": W["init.m6.pw.b"] + 1.0})
    assert np.array_equal(run(W6), base)
    n_data = 13 * 24
    W4 = dict(W, **{"ro.m4.2.b": W["ro.m4.2.b"] + 1.0})
    d = run(W4) - base
    assert np.all(d[:n_data * 2] == 0.0) and np.allclose(d[n_data * 2:], 1.0)


def test_var_io_blob_layout():
    netv = synth.NetConfig(num_rx_ant=4, channels=64, res_blocks=2, iterations=2, m_max=6, var_io=True)
    blob = synth.pack_weights(netv, synth.make_weights(netv))
    hdr = np.frombuffer(blob[:32], dtype="<i4")
    F, C = 18, 64
    per_it = 2 * (C * C + C) + C * (2 * C + 2) + C + 2 * 2 * (9 * C + C * C + C)
    heads = sum(C * F + C + 9 * C + C * C + C + m * C + m for m in (2, 4, 6))
    assert hdr[1] == 2 and hdr[7] == 2 * per_it + heads and len(blob) == 32 + 4 * hdr[7]
