"""Failure paths and linearity on the GPU, without faulting it.

* A bounded device wait that runs out (nothing arrives on its barrier) is
  reported by nrx_check as NRX_ETIMEDOUT, and the context stays usable.
* A NaN in one slot's received grid stays in that slot: the other slots of the
  batch get the LLRs they get without it, and the call succeeds.
* Latency grows linearly with the number of CGNN iterations run (early exit of
  an N_it = 8 network, Sec. IV-B)."""
import numpy as np
import pytest

from paper_2409_02912_b300 import build as nrx_build
from paper_2409_02912_b300 import nrx, synth
from tests import helpers as H

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a GPU", allow_module_level=True)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    nrx_build.build()
    nrx.load()


def _receiver(net, slots, prec):
    c = slots[0].cfg
    return nrx.Receiver(synth.pack_weights(net, synth.make_weights(net)), net.num_rx_ant, c.num_users,
                        c.num_prb, len(slots), prec)


@pytest.mark.parametrize("prec", ["bf16", "fp16", "fp8"])
def test_expired_wait_is_reported_and_the_context_recovers(prec):
    w, slots = H.slots_for("mu2_4rx_24prb", 2)
    rx = _receiver(w.net, slots, prec)
    y, dmrs, bits, _ = H.device_inputs(slots)
    before = rx.nrx_detect_batch(y, dmrs, w.dmrs_symbols, bits).cpu().numpy()
    rx.nrx_check()
    rx.nrx_expire_wait(2000)  # 2 ms
    with pytest.raises(nrx.NrxError) as e:
        rx.nrx_check()
    assert e.value.status == nrx.NRX_ETIMEDOUT
    rx.nrx_check()  # the status word was cleared
    after = rx.nrx_detect_batch(y, dmrs, w.dmrs_symbols, bits).cpu().numpy()
    rx.nrx_check()
    assert np.array_equal(before, after)
    for bad in (0, 1_000_001):
        with pytest.raises(nrx.NrxError) as e:
            rx.nrx_expire_wait(bad)
        assert e.value.status == nrx.NRX_EINVAL
    rx.close()


def test_expire_wait_needs_a_status_word():
    w, slots = H.slots_for("mu2_4rx_24prb", 1)
    rx = _receiver(w.net, slots, "fp32")
    with pytest.raises(nrx.NrxError) as e:
        rx.nrx_expire_wait(100)
    assert e.value.status == nrx.NRX_EUNSUPPORTED
    rx.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_nan_input_stays_in_its_slot(prec):
    w, slots = H.slots_for("mu2_4rx_24prb", 3)
    rx = _receiver(w.net, slots, prec)
    y, dmrs, bits, nv = H.device_inputs(slots)
    clean = rx.nrx_detect_batch(y, dmrs, w.dmrs_symbols, bits).cpu().numpy()
    clean_l = rx.lmmse_detect_batch(y, dmrs, w.dmrs_symbols, bits, nv).cpu().numpy()
    y_bad = y.clone()
    y_bad[1, 2, 5, 100] = complex(float("nan"), 0.0)  # slot 1, antenna 2, data symbol 5
    dirty = rx.nrx_detect_batch(y_bad, dmrs, w.dmrs_symbols, bits).cpu().numpy()
    dirty_l = rx.lmmse_detect_batch(y_bad, dmrs, w.dmrs_symbols, bits, nv).cpu().numpy()
    rx.nrx_check()
    for got, ref in ((dirty, clean), (dirty_l, clean_l)):
        g, _ = H.split(got, slots)
        r, _ = H.split(ref, slots)
        for i in (0, 2):  # the other slots are untouched, bit for bit
            for gu, ru in zip(g[i], r[i]):
                assert np.array_equal(gu, ru)
    rx.close()


def test_latency_is_linear_in_the_iterations():
    """Early exit after 1..8 iterations of an N_it = 8 network (the paper's
    large NRX depth): the batch time fits a + b N with R^2 > 0.99."""
    net = synth.NetConfig(num_rx_ant=4, channels=64, res_blocks=2, iterations=8, m_max=4)
    w = synth.WORKLOADS["mu2_4rx_24prb"]
    slots = synth.workload_slots(synth.dataclasses.replace(w, num_prb=106, net=net), 4)
    rx = _receiver(net, slots, "bf16")
    y, dmrs, bits, _ = H.device_inputs(slots)
    its = list(range(1, 9))

    def sweep():
        ts = []
        for n in its:
            for _ in range(3):
                rx.nrx_detect_batch(y, dmrs, w.dmrs_symbols, bits, iterations=n)
            samples = []
            for _ in range(7):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                rx.nrx_detect_batch(y, dmrs, w.dmrs_symbols, bits, iterations=n)
                b.record()
                torch.cuda.synchronize()
                samples.append(a.elapsed_time(b))
            ts.append(float(np.median(samples)))
        return ts

    # the lower of two sweeps' medians per depth: one sweep on a shared GPU machine was once
    # disturbed at a single depth (R^2 0.963)
    ts = [min(a, b) for a, b in zip(sweep(), sweep())]
    rx.nrx_check()
    A = np.stack([np.ones(len(its)), np.asarray(its, dtype=np.float64)], axis=1)
    coef, *_ = np.linalg.lstsq(A, np.asarray(ts), rcond=None)
    pred = A @ coef
    r2 = 1.0 - np.sum((np.asarray(ts) - pred) ** 2) / np.sum((np.asarray(ts) - np.mean(ts)) ** 2)
    assert coef[1] > 0 and r2 > 0.99, (ts, coef, r2)
    rx.close()
