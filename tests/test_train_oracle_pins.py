"""Pins of the FP64 training oracle (Sec. II-B) to facts other than itself:
closed forms of the BCE and MSE terms, the masking and multi-loss structure,
central finite differences of the numpy loss for the autograd gradient, the
numpy forward oracle for the torch loss, and closed forms of Adam."""
import numpy as np
import pytest

from oracle import nrx_oracle as O
from oracle import nrx_train_oracle as TO
from paper_2409_02912_b300 import synth

NET = synth.NetConfig(num_rx_ant=2, channels=4, res_blocks=1, iterations=2, m_max=4)


def _slots(U=2, bits=(2, 4), n=2, prb=1, dmrs=(2, 11), seed=5, snr=8.0):
    out = []
    for i in range(n):
        rng = np.random.Generator(np.random.PCG64(seed * 100 + i))
        cfg = synth.SlotConfig(num_prb=prb, num_users=U, num_rx_ant=NET.num_rx_ant, dmrs_symbols=dmrs,
                               bits_per_symbol=tuple(bits[:U]), snr_db=snr, num_taps=4, delay_spread_s=150e-9,
                               doppler_hz=80.0, ula=False)
        out.append(synth.make_slot(cfg, rng))
    return out


def _weights(seed=3):
    return synth.make_weights(NET, seed=seed), synth.make_chest_weights(NET, seed=seed + 1)


def test_softplus_closed_forms():
    x = np.array([-800.0, -3.0, 0.0, 2.5, 800.0])
    ref = np.array([0.0, np.log1p(np.exp(-3.0)), np.log(2.0), 2.5 + np.log1p(np.exp(-2.5)), 800.0])
    assert np.allclose(TO.softplus(x), ref, rtol=1e-15, atol=1e-300)


def test_zero_llrs_give_ln2_per_bit_in_every_iteration():
    """With ReadoutLLRs' last layer zeroed, every LLR is 0, P(b)=1/2 and each
    iteration's BCE mean is exactly ln 2, whatever the bits (Sec. II-B)."""
    W, Wc = _weights()
    W["ro2.w"][...] = 0.0
    W["ro2.b"][...] = 0.0
    total, bce, mse = TO.training_loss(_slots(), W, Wc, 2, 1, gamma=0.0)
    assert np.allclose(bce, [np.log(2.0)] * 2, rtol=1e-14)
    assert abs(total - 2 * np.log(2.0)) < 1e-13


def test_constant_llr_closed_form():
    """LLR = c on every output (ro2 zero, bias c): BCE mean = softplus(c) - c * (fraction of ones)."""
    W, Wc = _weights()
    c = float(np.float32(1.7))  # the weights are float32
    W["ro2.w"][...] = 0.0
    W["ro2.b"][...] = c
    sl = _slots()
    ones = sum(float(np.sum(s.bits[u])) for s in sl for u in range(2))
    count = sum(s.bits[u].size for s in sl for u in range(2))
    _, bce, _ = TO.training_loss(sl, W, Wc, 2, 1, gamma=0.0)
    ref = np.log1p(np.exp(c)) - c * ones / count
    assert np.allclose(bce, [ref, ref], rtol=1e-13)


def test_zero_chest_head_gives_channel_power():
    """h_hat = 0: the MSE is the mean channel power over (slot, user, antenna, RE)."""
    W, Wc = _weights()
    Wc["chest.2.w"][...] = 0.0
    Wc["chest.2.b"][...] = 0.0
    sl = _slots()
    power = np.mean([np.mean(np.abs(s.h) ** 2) for s in sl])
    total, bce, mse = TO.training_loss(sl, W, Wc, 2, 1, gamma=0.5)
    assert np.allclose(mse, [power, power], rtol=1e-12)
    assert abs(total - (sum(bce) + 0.5 * 2 * power)) < 1e-12


def test_masked_outputs_do_not_enter_the_loss():
    """Var-MCS masking (Sec. III): outputs j >= m_u of every user do not count;
    with m_u = 2 for all users the last two ReadoutLLRs rows are free."""
    W, Wc = _weights()
    sl = _slots(bits=(2, 2))
    a = TO.training_loss(sl, W, Wc, 2, 1, gamma=0.3)[0]
    W2 = {k: v.copy() for k, v in W.items()}
    W2["ro2.w"][2:] += 5.0
    W2["ro2.b"][2:] -= 3.0
    assert abs(TO.training_loss(sl, W2, Wc, 2, 1, gamma=0.3)[0] - a) < 1e-14
    W2["ro2.w"][1] += 0.5
    assert abs(TO.training_loss(sl, W2, Wc, 2, 1, gamma=0.3)[0] - a) > 1e-6


def test_multi_loss_sums_identical_iterations():
    """Zeroed CNN-update branches keep the state fixed, so both iterations'
    read-outs are equal and the multi-loss is twice the single loss."""
    W, Wc = _weights()
    W = synth.zero_like_residual(NET, W)
    total, bce, mse = TO.training_loss(_slots(), W, Wc, 2, 1, gamma=0.7)
    assert abs(bce[0] - bce[1]) < 1e-14 and abs(mse[0] - mse[1]) < 1e-14
    single, _, _ = TO.training_loss(_slots(), W, Wc, 1, 1, gamma=0.7)
    assert abs(total - 2 * single) < 1e-12


@pytest.mark.parametrize("U,dmrs", [(2, (2, 11)), (1, (2,)), (3, (3, 12))])
def test_torch_loss_matches_numpy_forward(U, dmrs):
    import torch
    W, Wc = _weights(seed=7)
    sl = _slots(U=U, bits=(4, 2, 4), dmrs=dmrs, seed=9)
    ref, _, _ = TO.training_loss(sl, W, Wc, 2, 1, gamma=0.4)
    Wt = {k: torch.from_numpy(np.asarray(v, dtype=np.float64)) for k, v in W.items()}
    Wct = {k: torch.from_numpy(np.asarray(v, dtype=np.float64)) for k, v in Wc.items()}
    got = float(TO._torch_loss(sl, Wt, Wct, 2, 1, 0.4))
    assert abs(got - ref) < 1e-12 * max(1.0, abs(ref))


def test_autograd_gradient_matches_finite_differences():
    """Central differences of the numpy loss (independent of autograd) on a
    few entries of every weight tensor, including the ReadoutChEst head."""
    W, Wc = _weights(seed=11)
    sl = _slots(U=2, bits=(2, 4), n=1, seed=13)
    gamma = 0.6
    _, g = TO.training_grads(sl, W, Wc, 2, 1, gamma)
    rng = np.random.Generator(np.random.PCG64(17))
    h = 1e-6
    checked = 0
    for name in list(W) + list(Wc):
        src = W if name in W else Wc
        flat_idx = rng.choice(src[name].size, size=min(3, src[name].size), replace=False)
        for fi in flat_idx:
            idx = np.unravel_index(fi, src[name].shape)
            base = {k: np.asarray(v, dtype=np.float64).copy() for k, v in W.items()}
            basec = {k: np.asarray(v, dtype=np.float64).copy() for k, v in Wc.items()}
            tgt = base if name in W else basec
            tgt[name][idx] += h
            lp = TO.training_loss(sl, base, basec, 2, 1, gamma)[0]
            tgt[name][idx] -= 2 * h
            lm = TO.training_loss(sl, base, basec, 2, 1, gamma)[0]
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[name][idx]) < 1e-6 * max(1.0, abs(fd)), (name, idx, fd, g[name][idx])
            checked += 1
    assert checked > 60


def test_gradient_of_masked_rows_and_unused_head_is_zero():
    W, Wc = _weights(seed=19)
    sl = _slots(bits=(2, 2), n=1)
    _, g = TO.training_grads(sl, W, Wc, 2, 1, gamma=0.0)
    assert np.all(g["ro2.w"][2:] == 0.0) and np.all(g["ro2.b"][2:] == 0.0)
    assert all(np.all(g[k] == 0.0) for k in Wc)
    assert np.any(g["ro2.w"][:2] != 0.0)


def test_adam_first_step_is_lr_times_sign():
    """Adam's first bias-corrected step moves each weight by lr sign(g) when
    |g| >> eps (Kingma and Ba, Sec. 2.1)."""
    rng = np.random.Generator(np.random.PCG64(23))
    w = rng.standard_normal(50)
    g = rng.standard_normal(50)
    w1, _, _ = TO.adam_step(w, g, np.zeros(50), np.zeros(50), 1, lr=1e-3, eps=1e-12)
    assert np.allclose(w - w1, 1e-3 * np.sign(g), rtol=1e-9, atol=0)


def test_adam_constant_gradient_moves_lr_per_step():
    """With a constant gradient the bias-corrected moments equal g and g^2, so
    every step moves by lr sign(g)."""
    w = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-2])
    m1 = np.zeros(3)
    m2 = np.zeros(3)
    for t in range(1, 8):
        w_new, m1, m2 = TO.adam_step(w, g, m1, m2, t, lr=0.01, eps=0.0)
        assert np.allclose(w - w_new, 0.01 * np.sign(g), rtol=1e-12)
        w = w_new


def test_snr_offset_orders_samples_by_mcs_and_users():
    assert synth.snr_offset_db((2,)) == 0.0
    assert synth.snr_offset_db((4, 4)) > synth.snr_offset_db((2, 4)) > synth.snr_offset_db((2, 2))
    assert synth.snr_offset_db((2, 2, 2)) > synth.snr_offset_db((2, 2))


def test_active_users_follow_the_triangular_distribution():
    """U_A per batch (Sec. II-B): P(U_A = k) = 2k / (U (U+1)) on 1..U (this
    build's reading of the triangular distribution), and the drawn number of
    users reaches the slots of a worker batch."""
    rng = np.random.Generator(np.random.PCG64(5))
    for U in (1, 2, 4):
        n = 40_000
        draws = np.array([synth.draw_active_users(U, rng) for _ in range(n)])
        assert draws.min() >= 1 and draws.max() <= U
        want = 2.0 * np.arange(1, U + 1) / (U * (U + 1))
        got = np.bincount(draws, minlength=U + 1)[1:] / n
        assert np.all(np.abs(got - want) <= 4.0 * np.sqrt(want * (1 - want) / n) + 1e-12), (U, got, want)
    from paper_2409_02912_b300 import train
    w = synth.Workload(name="active_check", seed_base=1, batch=3, num_prb=1, num_users=4, num_rx_ant=2,
                       dmrs_symbols=(2,), mcs_choices=(2, 4), snr_db_range=(0.0, 10.0), num_taps=2,
                       delay_spread_range_s=(1e-8, 5e-8), doppler_range_hz=(0.0, 10.0), ula=False,
                       net=synth.NetConfig(num_rx_ant=2, channels=8, res_blocks=1, iterations=1, m_max=4))
    users = {train._make_batch((w, seed, True)).m_u.shape[1] for seed in range(40)}
    assert users == {1, 2, 3, 4}
    assert {train._make_batch((w, seed, False)).m_u.shape[1] for seed in range(5)} == {4}


def test_training_batch_layout():
    sl = _slots(U=2, bits=(2, 4), n=2)
    tb = synth.training_batch(sl, m_max=6)
    assert tb.bits.shape == (2, 2, 12 * 12, 6) and tb.m_u.tolist() == [[2, 4], [2, 4]]
    assert np.array_equal(tb.bits[1, 1, :, :4], sl[1].bits[1]) and np.all(tb.bits[1, 0, :, 2:] == 0)
    assert np.allclose(tb.h[0, 1, 5, 7, 2] + 1j * tb.h[0, 1, 5, 7, 3], sl[0].h[1, 1, 5, 7], atol=1e-6)
    assert np.allclose(TO.channel_target(sl[0].h[1])[5, 7], tb.h[0, 1, 5, 7], atol=1e-6)


def test_var_io_training_loss_and_gradient():
    """Var-IO (Sec. III): the loss of a Var-IO network whose heads copy a
    single masked head equals the masked network's loss, the torch loss equals
    the numpy loss, and the autograd gradient of a head equals central finite
    differences; heads of orders no user carries get zero gradient."""
    import torch
    netv = synth.NetConfig(num_rx_ant=2, channels=4, res_blocks=1, iterations=2, m_max=6, var_io=True)
    Wv = synth.make_weights(netv, seed=27)
    Wc = synth.make_chest_weights(NET, seed=28)
    sl = _slots(U=2, bits=(2, 4), n=1, seed=31)
    a = TO.training_loss(sl, Wv, Wc, 2, 1, 0.3)[0]
    Wt = {k: torch.from_numpy(np.asarray(v, dtype=np.float64)) for k, v in Wv.items()}
    Wct = {k: torch.from_numpy(np.asarray(v, dtype=np.float64)) for k, v in Wc.items()}
    assert abs(float(TO._torch_loss(sl, Wt, Wct, 2, 1, 0.3)) - a) < 1e-12 * max(1.0, abs(a))
    _, g = TO.training_grads(sl, Wv, Wc, 2, 1, 0.3)
    assert all(np.all(g[k] == 0.0) for k in g if k.startswith("init.m6") or k.startswith("ro.m6"))
    h = 1e-6
    for name, idx in (("init.m4.pw.w", (1, 3)), ("ro.m2.2.w", (1, 2)), ("ro.m4.1.b", (3,)), ("init.m2.dw", (0, 1, 2))):
        base = {k: np.asarray(v, dtype=np.float64).copy() for k, v in Wv.items()}
        base[name][idx] += h
        lp = TO.training_loss(sl, base, Wc, 2, 1, 0.3)[0]
        base[name][idx] -= 2 * h
        lm = TO.training_loss(sl, base, Wc, 2, 1, 0.3)[0]
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[name][idx]) < 1e-6 * max(1.0, abs(fd)), (name, fd, g[name][idx])
