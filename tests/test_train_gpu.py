"""Training path on the GPU (Sec. II-B): the layer kernels against plain
definitions, the trainer's loss and gradient against the FP64 training oracle
(torch autograd, pinned by finite differences), Adam against its definition,
the exported blob against the inference path, and a short training run."""
import numpy as np
import pytest

from oracle import nrx_oracle as O
from oracle import nrx_train_oracle as TO
from paper_2409_02912_b300 import nrx, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2409_02912_b300 import train  # noqa: E402

# FP32 kernels with float-atomic reductions against FP64: the gradient of each
# tensor must match to 1e-4 of its norm (FP32 unit roundoff 6e-8 times the
# depth and reduction lengths of these small cases, with margin).
TOL_GRAD = 1e-4
TOL_LOSS = 1e-5


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _slots(net, U, bits, n, prb, dmrs, seed, snr=6.0):
    out = []
    for i in range(n):
        rng = np.random.Generator(np.random.PCG64(seed * 100 + i))
        cfg = synth.SlotConfig(num_prb=prb, num_users=U, num_rx_ant=net.num_rx_ant, dmrs_symbols=dmrs,
                               bits_per_symbol=tuple(bits[:U]), snr_db=snr, num_taps=6, delay_spread_s=200e-9,
                               doppler_hz=150.0, ula=True)
        out.append(synth.make_slot(cfg, rng))
    return out


# ----------------------------------------------------------------------------
# Layer kernels against their definitions
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (130, 70, 37), (64, 64, 64), (300, 9, 130)])
def test_gemm_strided_epilogues(M, N, K):
    rng = np.random.Generator(np.random.PCG64(M * 7 + N))
    ops = train._Ops(torch.cuda.current_stream().cuda_stream)
    A = rng.standard_normal((M, K + 3)).astype(np.float32)        # row stride K+3
    W = rng.standard_normal((N, K)).astype(np.float32)            # B(k,n) = W[n][k]
    bias = rng.standard_normal(N).astype(np.float32)
    Rm = rng.standard_normal((M, N)).astype(np.float32)
    dA, dW, db, dR = _t(A), _t(W), _t(bias), _t(Rm)
    out = torch.empty((M, N), device="cuda")
    ops.gemm(M, N, K, dA.data_ptr(), K + 3, 1, dW.data_ptr(), 1, K, out.data_ptr(), N, bias=db.data_ptr(),
             R=dR.data_ptr(), ldr=N, relu=True)
    ref = np.maximum(A[:, :K].astype(np.float64) @ W.T.astype(np.float64) + bias + Rm, 0.0)
    assert np.max(np.abs(out.cpu().numpy() - ref)) < 1e-5 * max(1.0, np.max(np.abs(ref)))
    # transposed operand (weight-gradient form), split K with atomics, into a strided slice
    G = rng.standard_normal((K, M)).astype(np.float32)            # A(m,k) = G[k][m]
    X = rng.standard_normal((K, N)).astype(np.float32)
    acc0 = rng.standard_normal((M, N + 5)).astype(np.float32)
    dG, dX, dacc = _t(G), _t(X), _t(acc0)
    ops.gemm(M, N, K, dG.data_ptr(), 1, M, dX.data_ptr(), N, 1, dacc.data_ptr(), N + 5, accumulate=True,
             split_k=3)
    ref2 = acc0.astype(np.float64)
    ref2[:, :N] += G.T.astype(np.float64) @ X.astype(np.float64)
    assert np.max(np.abs(dacc.cpu().numpy() - ref2)) < 1e-5 * max(1.0, np.max(np.abs(ref2)))


@pytest.mark.parametrize("planes,S,C", [(1, 12, 1), (3, 24, 5), (2, 36, 64)])
def test_depthwise_forward_adjoint_and_tap_gradient(planes, S, C):
    rng = np.random.Generator(np.random.PCG64(planes * 31 + S + C))
    ops = train._Ops(torch.cuda.current_stream().cuda_stream)
    X = rng.standard_normal((planes, 14, S, C)).astype(np.float32)
    G = rng.standard_normal((planes, 14, S, C)).astype(np.float32)
    k = rng.standard_normal((C, 3, 3)).astype(np.float32)
    dX, dG, dk = _t(X), _t(G), _t(k)
    Y = torch.empty_like(dX)
    ops.dw3(planes, S, C, dX.data_ptr(), dk.data_ptr(), Y.data_ptr())
    ref = np.stack([O.depthwise3x3(X[p].astype(np.float64), k) for p in range(planes)])
    assert np.max(np.abs(Y.cpu().numpy() - ref)) < 1e-5 * np.max(np.abs(ref))
    # adjoint: <DW(X), G> == <X, DW^T(G)>
    ops.dw3(planes, S, C, dG.data_ptr(), dk.data_ptr(), Y.data_ptr(), flip=True)
    lhs = np.sum(ref * G.astype(np.float64))
    rhs = np.sum(X.astype(np.float64) * Y.cpu().numpy().astype(np.float64))
    assert abs(lhs - rhs) < 1e-4 * max(1.0, abs(lhs))
    # tap gradient: d<DW(X), G>/dk[c,i,j] = sum G * shifted X (brute force)
    gk = torch.zeros((C, 3, 3), device="cuda")
    ops.dw3_wgrad(planes, S, C, dX.data_ptr(), dG.data_ptr(), gk.data_ptr())
    Xp = np.zeros((planes, 16, S + 2, C))
    Xp[:, 1:-1, 1:-1] = X
    refk = np.zeros((C, 3, 3))
    for i in range(3):
        for j in range(3):
            refk[:, i, j] = np.sum(G * Xp[:, i:i + 14, j:j + S], axis=(0, 1, 2))
    assert np.max(np.abs(gk.cpu().numpy() - refk)) < 1e-4 * max(1.0, np.max(np.abs(refk)))


@pytest.mark.parametrize("U", [1, 2, 3, 4])
def test_aggregate_is_sum_over_other_users(U):
    rng = np.random.Generator(np.random.PCG64(U))
    ops = train._Ops(torch.cuda.current_stream().cuda_stream)
    m = rng.standard_normal((2, U, 14, 12, 8)).astype(np.float32)
    dm = _t(m)
    a = torch.empty_like(dm)
    ops.aggregate(2, U, 14 * 12 * 8, dm.data_ptr(), a.data_ptr())
    ref = np.stack([O.aggregate(m[s].astype(np.float64), list(range(U))) for s in range(2)])
    assert np.max(np.abs(a.cpu().numpy() - ref)) < 1e-5


def test_adam_kernel_matches_definition():
    rng = np.random.Generator(np.random.PCG64(29))
    n = 10007
    w, g = rng.standard_normal(n), rng.standard_normal(n)
    m1, m2 = 0.1 * rng.standard_normal(n), np.abs(rng.standard_normal(n))
    t, lr = 7, 3e-3
    ref_w, ref_m1, ref_m2 = TO.adam_step(w, g, m1, m2, t, lr)
    dw, dg, dm1, dm2 = (_t(v.astype(np.float32)) for v in (w, g, m1, m2))
    lr_t = torch.tensor([lr * np.sqrt(1 - 0.999 ** t) / (1 - 0.9 ** t)], dtype=torch.float32).cuda()
    lib = train.load()
    st = lib.nrx_train_adam(n, dw.data_ptr(), dg.data_ptr(), dm1.data_ptr(), dm2.data_ptr(), lr_t.data_ptr(), 0.9,
                            0.999, 1e-8, torch.cuda.current_stream().cuda_stream)
    assert st == nrx.NRX_OK
    assert np.max(np.abs(dm1.cpu().numpy() - ref_m1)) < 1e-6
    assert np.max(np.abs(dm2.cpu().numpy() - ref_m2)) < 1e-5
    assert np.max(np.abs(dw.cpu().numpy() - ref_w)) < 1e-6


# ----------------------------------------------------------------------------
# Loss and gradient against the FP64 training oracle
# ----------------------------------------------------------------------------

GRAD_CASES = [
    # (B, C, R, N_it, m_max, U, bits, prb, dmrs, n_slots, gamma)
    (2, 8, 1, 2, 4, 2, (2, 4), 2, (2, 11), 2, 0.5),
    (2, 16, 2, 2, 6, 4, (2, 4, 6, 4), 1, (2, 11), 1, 1.0),
    (4, 8, 2, 1, 4, 1, (4,), 3, (2,), 2, 0.0),
    (1, 8, 1, 3, 2, 3, (2, 2, 2), 2, (3, 12), 1, 2.0),
]


@pytest.mark.parametrize("case", GRAD_CASES, ids=[f"B{c[0]}C{c[1]}U{c[5]}" for c in GRAD_CASES])
def test_trainer_loss_and_gradient_match_oracle(case):
    B, C, R, K, mm, U, bits, prb, dmrs, n, gamma = case
    net = synth.NetConfig(num_rx_ant=B, channels=C, res_blocks=R, iterations=K, m_max=mm)
    W = synth.make_weights(net, seed=5)
    Wc = synth.make_chest_weights(net, seed=6)
    sl = _slots(net, U, bits, n, prb, dmrs, seed=C + U)
    ref_loss, ref_g = TO.training_grads(sl, W, Wc, K, R, gamma)
    tr = train.Trainer(net, W, Wc, gamma=gamma)
    out = tr.loss_and_grad(train.DeviceBatch(synth.training_batch(sl, mm)))
    assert abs(out["loss"] - ref_loss) < TOL_LOSS * max(1.0, abs(ref_loss))
    ref_total, ref_bce, ref_mse = TO.training_loss(sl, W, Wc, K, R, gamma)
    assert np.allclose(out["bce"], ref_bce, rtol=TOL_LOSS)
    if gamma > 0:
        assert np.allclose(out["mse"], ref_mse, rtol=TOL_LOSS)
    g = tr.grads()
    for name, ref in ref_g.items():
        nrm = np.linalg.norm(ref)
        err = np.linalg.norm(g[name] - ref)
        if nrm == 0.0:
            assert err == 0.0, name
        else:
            assert err <= TOL_GRAD * nrm, (name, err / nrm)


def test_exported_blob_runs_the_same_network_in_the_inference_path():
    """The trainer's FP32 weights, exported as a blob, give inference LLRs whose
    masked BCE equals the trainer's last-iteration BCE."""
    net = synth.NetConfig(num_rx_ant=4, channels=64, res_blocks=2, iterations=2, m_max=6)
    W = synth.make_weights(net, seed=8)
    sl = _slots(net, 2, (2, 6), 3, 4, (2, 11), seed=4)
    tr = train.Trainer(net, W, gamma=0.0)
    out = tr.loss_and_grad(train.DeviceBatch(synth.training_batch(sl, 6)))
    rx = nrx.Receiver(tr.blob(), 4, 2, 4, max_slots=3, precision="fp32")
    y = _t(synth.stack_batch(sl))
    dm = _t(np.stack([s.dmrs for s in sl]))
    llr = rx.nrx_detect_batch(y, dm, (2, 11), [[2, 6]] * 3).cpu().numpy().astype(np.float64)
    bits = np.concatenate([np.concatenate([s.bits[0].reshape(-1), s.bits[1].reshape(-1)]) for s in sl])
    bce = float(np.mean(TO.softplus(llr) - bits * llr))
    assert abs(bce - out["bce"][-1]) < 1e-5 * bce


def test_training_reduces_the_loss():
    """A few hundred Adam steps on fresh random slots lower the BCE of a
    randomly initialised NRX (2 users, 4 Rx, QPSK/16-QAM mix)."""
    w = synth.Workload(name="train_mu2", seed_base=50, batch=8, num_prb=4, num_users=2, num_rx_ant=4,
                       dmrs_symbols=(2, 11), mcs_choices=(2, 4), snr_db_range=(5.0, 15.0), num_taps=8,
                       delay_spread_range_s=(30e-9, 200e-9), doppler_range_hz=(0.0, 200.0), ula=True,
                       net=synth.NetConfig(num_rx_ant=4, channels=32, res_blocks=1, iterations=2, m_max=4))
    tr = train.Trainer(w.net, synth.make_weights(w.net, seed=1), lr=2e-3, gamma=0.5)
    rng = np.random.Generator(np.random.PCG64(77))
    val = train.DeviceBatch(synth.training_batch([synth.training_slot(w, rng) for _ in range(8)], 4))
    before = tr.loss_and_grad(val)["bce"][-1]
    for _ in range(300):
        tr.step(train.DeviceBatch(synth.training_batch([synth.training_slot(w, rng) for _ in range(8)], 4)))
    after = tr.loss_and_grad(val)["bce"][-1]
    assert np.isfinite(after) and after < 0.75 * before, (before, after)


def test_graph_step_matches_eager_steps():
    """The captured training step (one graph replay per step, batches of
    different modulation orders uploaded into fixed buffers) follows the
    eager launch sequence step for step."""
    net = synth.NetConfig(num_rx_ant=2, channels=16, res_blocks=1, iterations=2, m_max=4)
    w = synth.Workload(name="graph_check", seed_base=51, batch=3, num_prb=2, num_users=2, num_rx_ant=2,
                       dmrs_symbols=(2, 11), mcs_choices=(2, 4), snr_db_range=(0.0, 10.0), num_taps=4,
                       delay_spread_range_s=(50e-9, 100e-9), doppler_range_hz=(0.0, 100.0), ula=False, net=net)
    rng = np.random.Generator(np.random.PCG64(3))
    batches = [synth.training_batch([synth.training_slot(w, rng) for _ in range(3)], 4) for _ in range(4)]
    assert len({tuple(b.m_u.reshape(-1)) for b in batches}) > 1
    W = synth.make_weights(net, seed=9)
    eager = train.Trainer(net, W, lr=1e-2, gamma=0.5)
    graph = train.Trainer(net, W, lr=1e-2, gamma=0.5)
    for tb in batches:
        a = eager.step(train.DeviceBatch(tb))
        b = graph.graph_step(tb)
        assert abs(a["loss"] - b["loss"]) < 1e-4 * abs(a["loss"]), (a, b)
    wa, wb = eager.w.cpu().numpy(), graph.w.cpu().numpy()
    assert np.max(np.abs(wa - wb)) < 1e-4 * np.max(np.abs(wa))
    assert graph.t == eager.t == 4


def test_recompute_gives_the_same_loss_and_gradient_with_less_memory():
    """Recomputing each residual block's conv activations in the reverse pass
    (instead of storing them for every block and iteration) leaves the loss
    and the gradient unchanged up to the rounding order of atomic reductions,
    in eager and graph-captured steps, and takes fewer activation bytes; the
    automatic mode switches to it when the stored activations exceed the
    memory fraction."""
    net = synth.NetConfig(num_rx_ant=4, channels=32, res_blocks=2, iterations=2, m_max=4)
    W, Wc = synth.make_weights(net, seed=21), synth.make_chest_weights(net, seed=22)
    sl = _slots(net, 2, (2, 4), 3, 6, (2, 11), seed=23)
    db = train.DeviceBatch(synth.training_batch(sl, 4))
    keep = train.Trainer(net, W, Wc, gamma=0.5, recompute=False)
    rec = train.Trainer(net, W, Wc, gamma=0.5, recompute=True)
    a, b = keep.loss_and_grad(db), rec.loss_and_grad(db)
    assert not keep.recomputing and rec.recomputing
    # the forward is the same launch sequence; only the FP64 atomic loss sums may round differently
    assert np.allclose([a["loss"]] + a["bce"] + a["mse"], [b["loss"]] + b["bce"] + b["mse"], rtol=1e-12, atol=0)
    ga, gb = keep.grads(), rec.grads()
    for name, ref in ga.items():
        assert np.linalg.norm(gb[name] - ref) <= 1e-5 * max(np.linalg.norm(ref), 1e-30), name
    n, U, S = 3, 2, 72
    full, small = keep.activation_bytes(n, U, S, False), keep.activation_bytes(n, U, S, True)
    assert small < full
    # the saving is exactly the 3 (K R - 1) conv activation tensors
    assert full - small == 4 * n * U * 14 * S * net.channels * 3 * (net.iterations * net.res_blocks - 1)
    auto = train.Trainer(net, W, Wc, gamma=0.5, memory_fraction=1e-12)
    assert abs(auto.loss_and_grad(db)["loss"] - a["loss"]) <= 1e-12 * a["loss"] and auto.recomputing
    # graph-captured steps with recompute follow the eager steps
    tb = synth.training_batch(sl, 4)
    e1 = train.Trainer(net, W, Wc, gamma=0.5, lr=1e-2, recompute=True)
    g1 = train.Trainer(net, W, Wc, gamma=0.5, lr=1e-2, recompute=True)
    for _ in range(3):
        x, y = e1.step(train.DeviceBatch(tb)), g1.graph_step(tb)
        assert abs(x["loss"] - y["loss"]) < 1e-5 * abs(x["loss"])


# ----------------------------------------------------------------------------
# BF16 tensor-core compute
# ----------------------------------------------------------------------------

def _bf16(x):
    """Round float32 to BF16 (round to nearest even), returned as float64."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return u.view(np.float32).astype(np.float64)


@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (130, 70, 37), (300, 9, 130), (64, 64, 1000)])
def test_gemm_bf16_equals_product_of_rounded_operands(M, N, K):
    """The tensor-core GEMM equals the FP64 product of the BF16-rounded
    operands up to FP32 accumulation order (products of BF16 are exact)."""
    rng = np.random.Generator(np.random.PCG64(M * 11 + N + K))
    ops = train._Ops(torch.cuda.current_stream().cuda_stream, "bf16")
    A = rng.standard_normal((M, K + 3)).astype(np.float32)
    W = rng.standard_normal((N, K)).astype(np.float32)
    bias = rng.standard_normal(N).astype(np.float32)
    Rm = rng.standard_normal((M, N)).astype(np.float32)
    out = torch.empty((M, N), device="cuda")
    dA, dW, db, dR = _t(A), _t(W), _t(bias), _t(Rm)
    ops.gemm(M, N, K, dA.data_ptr(), K + 3, 1, dW.data_ptr(), 1, K, out.data_ptr(), N, bias=db.data_ptr(),
             R=dR.data_ptr(), ldr=N, relu=True)
    prod = _bf16(A[:, :K]) @ _bf16(W).T
    ref = np.maximum(prod + bias + Rm, 0.0)
    scale = np.abs(_bf16(A[:, :K])) @ np.abs(_bf16(W)).T + 1.0
    assert np.all(np.abs(out.cpu().numpy() - ref) <= 1e-5 * scale)
    G = rng.standard_normal((K, M)).astype(np.float32)
    X = rng.standard_normal((K, N)).astype(np.float32)
    acc0 = rng.standard_normal((M, N + 5)).astype(np.float32)
    dG, dX, dacc = _t(G), _t(X), _t(acc0)
    ops.gemm(M, N, K, dG.data_ptr(), 1, M, dX.data_ptr(), N, 1, dacc.data_ptr(), N + 5, accumulate=True, split_k=3)
    ref2 = acc0.astype(np.float64)
    ref2[:, :N] += _bf16(G).T @ _bf16(X)
    scale2 = np.abs(acc0).astype(np.float64)
    scale2[:, :N] += np.abs(_bf16(G)).T @ np.abs(_bf16(X))
    assert np.all(np.abs(dacc.cpu().numpy() - ref2) <= 1e-5 * (scale2 + 1.0))


# BF16 operands carry a relative rounding error of 2^-9 at every dense layer of
# the forward and reverse passes (about 20 layers deep here).  A CPU emulation
# of this arithmetic on these cases gives 0.7-5.2% per-tensor error against the
# FP64 oracle (largest on small bias gradients); the test holds each tensor's
# gradient to 10% of its norm (a wrong gradient is off by order 100%).
TOL_GRAD_BF16 = 1e-1


@pytest.mark.parametrize("case", GRAD_CASES[:2], ids=[f"B{c[0]}C{c[1]}U{c[5]}" for c in GRAD_CASES[:2]])
def test_trainer_bf16_gradient_near_oracle(case):
    B, C, R, K, mm, U, bits, prb, dmrs, n, gamma = case
    net = synth.NetConfig(num_rx_ant=B, channels=C, res_blocks=R, iterations=K, m_max=mm)
    W = synth.make_weights(net, seed=5)
    Wc = synth.make_chest_weights(net, seed=6)
    sl = _slots(net, U, bits, n, prb, dmrs, seed=C + U)
    ref_loss, ref_g = TO.training_grads(sl, W, Wc, K, R, gamma)
    tr = train.Trainer(net, W, Wc, gamma=gamma, precision="bf16")
    out = tr.loss_and_grad(train.DeviceBatch(synth.training_batch(sl, mm)))
    assert abs(out["loss"] - ref_loss) < 1e-2 * abs(ref_loss)
    g = tr.grads()
    errs = {name: float(np.linalg.norm(g[name] - ref) / np.linalg.norm(ref))
            for name, ref in ref_g.items() if np.linalg.norm(ref) > 0}
    assert max(errs.values()) <= TOL_GRAD_BF16, sorted(errs.items(), key=lambda kv: -kv[1])[:5]


def test_bf16_training_reduces_the_loss():
    w = synth.Workload(name="train_mu2_bf16", seed_base=53, batch=8, num_prb=4, num_users=2, num_rx_ant=4,
                       dmrs_symbols=(2, 11), mcs_choices=(2, 4), snr_db_range=(5.0, 15.0), num_taps=8,
                       delay_spread_range_s=(30e-9, 200e-9), doppler_range_hz=(0.0, 200.0), ula=True,
                       net=synth.NetConfig(num_rx_ant=4, channels=32, res_blocks=1, iterations=2, m_max=4))
    tr = train.Trainer(w.net, synth.make_weights(w.net, seed=1), lr=2e-3, gamma=0.5, precision="bf16")
    rng = np.random.Generator(np.random.PCG64(78))
    val = train.DeviceBatch(synth.training_batch([synth.training_slot(w, rng) for _ in range(8)], 4))
    before = tr.loss_and_grad(val)["bce"][-1]
    for _ in range(300):
        tr.graph_step(synth.training_batch([synth.training_slot(w, rng) for _ in range(8)], 4))
    after = tr.loss_and_grad(val)["bce"][-1]
    assert np.isfinite(after) and after < 0.75 * before, (before, after)


# ----------------------------------------------------------------------------
# GPU link simulator
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("ula,dmrs,U", [(True, (2, 11), 3), (False, (3,), 2), (True, (2,), 4)])
def test_gpu_simulator_matches_counter_based_reference(ula, dmrs, U):
    """The device simulator reproduces the numpy restatement from the same
    Philox counters: bits, pilots and modulation orders exactly, the channel
    and the received grid to FP32 accuracy."""
    w = synth.Workload(name="simcheck", seed_base=0, batch=4, num_prb=5, num_users=U, num_rx_ant=4,
                       dmrs_symbols=dmrs, mcs_choices=(2, 4, 6), snr_db_range=(0.0, 20.0), num_taps=9,
                       delay_spread_range_s=(30e-9, 300e-9), doppler_range_hz=(0.0, 400.0), ula=ula,
                       net=synth.NetConfig(num_rx_ant=4, channels=8, res_blocks=1, iterations=1, m_max=6))
    sim = train.GpuSimulator(w, seed=1234567890123, param_seed=4)
    sim.draw()
    b = sim.draw()  # second batch: batch index 1
    params = list(sim.last_params)
    params[0] = synth.dataclasses.replace(params[0], doppler_hz=0.0)  # keep a static slot in the check
    sim.batch_index = 1
    import ctypes
    arr = (train.nrx_sim_slot * len(params))()
    for i, sp in enumerate(params):
        arr[i].noise_var, arr[i].delay_spread_s, arr[i].doppler_hz = sp.noise_var, sp.delay_spread_s, sp.doppler_hz
        arr[i].num_taps, arr[i].ula = sp.num_taps, int(sp.ula)
        for u, m in enumerate(sp.bits_per_symbol):
            arr[i].bits_per_symbol[u] = m
    ds = np.asarray(dmrs, dtype=np.int32)
    st = train.load().nrx_train_simulate(len(params), arr, U, 4, 5, len(dmrs), ds.ctypes.data, 6, sim.seed, 1,
                                         sim.scratch.data_ptr(), b.y.data_ptr(), b.dmrs.data_ptr(), b.bits.data_ptr(),
                                         b.m_u.data_ptr(), b.h.data_ptr(), None)
    assert st == nrx.NRX_OK
    torch.cuda.synchronize()
    ref = synth.simulate_philox(params, U, 4, 5, dmrs, 6, seed=sim.seed, batch=1)
    assert np.array_equal(b.bits.cpu().numpy(), ref.bits)
    assert np.array_equal(b.m_u.cpu().numpy(), ref.m_u)
    assert np.array_equal(b.dmrs.cpu().numpy(), ref.dmrs)
    h = b.h.cpu().numpy()
    assert np.max(np.abs(h - ref.h)) < 1e-4 * max(1.0, np.max(np.abs(ref.h)))
    y = b.y.cpu().numpy()
    assert np.max(np.abs(y - ref.y)) < 1e-4 * max(1.0, np.max(np.abs(ref.y)))


def test_active_user_batches_replay_per_shape_graphs():
    """Training with U_A drawn per batch (Sec. II-B): the GPU simulator fills
    one device batch per number of active users, each equal to the numpy
    Philox twin for its draw; the trainer keeps one captured graph per batch
    shape and its graph steps follow eager steps on the same batches."""
    net = synth.NetConfig(num_rx_ant=2, channels=16, res_blocks=1, iterations=2, m_max=4)
    w = synth.Workload(name="active_sim", seed_base=0, batch=3, num_prb=2, num_users=3, num_rx_ant=2,
                       dmrs_symbols=(2, 11), mcs_choices=(2, 4), snr_db_range=(0.0, 15.0), num_taps=4,
                       delay_spread_range_s=(30e-9, 200e-9), doppler_range_hz=(0.0, 200.0), ula=True, net=net)
    sim = train.GpuSimulator(w, seed=99, param_seed=3, active_users=True)
    W = synth.make_weights(net, seed=12)
    eager = train.Trainer(net, W, lr=1e-2, gamma=0.5)
    graph = train.Trainer(net, W, lr=1e-2, gamma=0.5)
    seen = set()
    for k in range(12):
        b = sim.draw()
        U = b.U
        seen.add(U)
        assert b is sim.batches[U] and 1 <= U <= 3
        ref = synth.simulate_philox(sim.last_params, U, 2, 2, (2, 11), 4, seed=sim.seed, batch=k)
        torch.cuda.synchronize()
        assert np.array_equal(b.bits.cpu().numpy(), ref.bits) and np.array_equal(b.m_u.cpu().numpy(), ref.m_u)
        e = eager.step(train.DeviceBatch(synth.TrainingBatch(
            y=b.y.cpu().numpy(), dmrs=b.dmrs.cpu().numpy(), bits=b.bits.cpu().numpy(), m_u=b.m_u.cpu().numpy(),
            h=b.h.cpu().numpy(), dmrs_symbols=(2, 11), noise_var=np.ones(3))))
        gr = graph.graph_step(b)
        assert abs(e["loss"] - gr["loss"]) < 1e-4 * abs(e["loss"]), (k, U, e, gr)
    assert len(seen) >= 2
    assert len(graph._graphs) == len(seen) and len(graph._bufs) == len(seen)
    wa, wb = eager.w.cpu().numpy(), graph.w.cpu().numpy()
    assert np.max(np.abs(wa - wb)) < 1e-4 * np.max(np.abs(wa))


def test_training_on_the_gpu_simulator_reduces_the_loss():
    w = synth.Workload(name="train_gpu_sim", seed_base=54, batch=8, num_prb=4, num_users=2, num_rx_ant=4,
                       dmrs_symbols=(2, 11), mcs_choices=(2, 4), snr_db_range=(5.0, 15.0), num_taps=8,
                       delay_spread_range_s=(30e-9, 200e-9), doppler_range_hz=(0.0, 200.0), ula=True,
                       net=synth.NetConfig(num_rx_ant=4, channels=32, res_blocks=1, iterations=2, m_max=4))
    tr = train.Trainer(w.net, synth.make_weights(w.net, seed=1), lr=2e-3, gamma=0.5)
    val_sim = train.GpuSimulator(w, seed=99, param_seed=98)
    val = val_sim.draw()
    before = tr.loss_and_grad(val)["bce"][-1]
    sim = train.GpuSimulator(w, seed=5, param_seed=6)
    for _ in range(300):
        tr.graph_step(sim.draw())
    after = tr.loss_and_grad(val)["bce"][-1]
    assert np.isfinite(after) and after < 0.75 * before, (before, after)


# ----------------------------------------------------------------------------
# Var-IO heads (Sec. III)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("U,bits,mm", [(2, (2, 4), 4), (4, (2, 4, 6, 4), 6)])
def test_var_io_trainer_gradient_matches_oracle(U, bits, mm):
    net = synth.NetConfig(num_rx_ant=2, channels=8, res_blocks=1, iterations=2, m_max=mm, var_io=True)
    W = synth.make_weights(net, seed=15)
    Wc = synth.make_chest_weights(net, seed=16)
    sl = _slots(net, U, bits, 2, 2, (2, 11), seed=40 + U)
    ref_loss, ref_g = TO.training_grads(sl, W, Wc, 2, 1, 0.5)
    tr = train.Trainer(net, W, Wc, gamma=0.5)
    out = tr.loss_and_grad(train.DeviceBatch(synth.training_batch(sl, mm)))
    assert abs(out["loss"] - ref_loss) < TOL_LOSS * max(1.0, abs(ref_loss))
    g = tr.grads()
    for name, ref in ref_g.items():
        nrm = np.linalg.norm(ref)
        err = np.linalg.norm(g[name] - ref)
        assert (err == 0.0) if nrm == 0.0 else (err <= TOL_GRAD * nrm), (name, err, nrm)


def test_var_io_blob_from_the_trainer_runs_in_the_inference_path():
    net = synth.NetConfig(num_rx_ant=4, channels=64, res_blocks=2, iterations=2, m_max=6, var_io=True)
    sl = _slots(net, 3, (6, 2, 4), 2, 4, (2, 11), seed=8)
    tr = train.Trainer(net, synth.make_weights(net, seed=9), gamma=0.0)
    out = tr.loss_and_grad(train.DeviceBatch(synth.training_batch(sl, 6)))
    rx = nrx.Receiver(tr.blob(), 4, 3, 4, max_slots=2, precision="fp32")
    y = _t(synth.stack_batch(sl))
    dm = _t(np.stack([s.dmrs for s in sl]))
    llr = rx.nrx_detect_batch(y, dm, (2, 11), [[6, 2, 4]] * 2).cpu().numpy().astype(np.float64)
    bits = np.concatenate([np.concatenate([s.bits[u].reshape(-1) for u in range(3)]) for s in sl])
    bce = float(np.mean(TO.softplus(llr) - bits * llr))
    assert abs(bce - out["bce"][-1]) < 1e-5 * bce


def test_autograd_function_drives_a_torch_optimiser():
    """The kernels behind torch.autograd: the loss is differentiable in the
    flat weight vector, its gradient is the reverse pass's, and a torch
    optimiser updating the shared parameter updates the trainer's weights."""
    net = synth.NetConfig(num_rx_ant=2, channels=8, res_blocks=1, iterations=2, m_max=4)
    W = synth.make_weights(net, seed=5)
    sl = _slots(net, 2, (2, 4), 2, 2, (2, 11), seed=60)
    tr = train.Trainer(net, W, gamma=0.5)
    batch = train.DeviceBatch(synth.training_batch(sl, 4))
    param = torch.nn.Parameter(tr.w)
    loss = train.nrx_training_loss(param, tr, batch)
    loss.backward()
    ref = tr.loss_and_grad(batch)
    assert abs(float(loss.detach()) - ref["loss"]) < 1e-5 * ref["loss"]
    assert torch.allclose(param.grad, tr.g, rtol=1e-4, atol=1e-6 * float(tr.g.abs().max()))
    w0 = tr.w.clone()
    opt = torch.optim.SGD([param], lr=1e-3)
    opt.step()
    assert torch.allclose(tr.w, w0 - 1e-3 * param.grad)
