"""The allocation-free entry point (for callers that cannot call cudaMalloc,
e.g. while a stream is being captured or under a fixed start-up memory budget)
gives the same LLRs as the context entry point, on two calls in a row that
reuse its static scratch, and rejects slots beyond its scratch limit.

Collected last on purpose: it runs after every other test in a full run."""
import numpy as np
import pytest

from paper_2409_02912_b300 import build as nrx_build
from paper_2409_02912_b300 import nrx, synth
from tests import helpers as H

pytestmark = pytest.mark.gpu
TOL_FP32 = 1e-4


def test_noalloc_matches_context_entry_point_twice():
    import torch
    nrx_build.build()
    w = synth.WORKLOADS["mu2_4rx_24prb"]
    blob = synth.pack_weights(w.net, synth.make_weights(w.net))
    wdev = torch.from_numpy(np.frombuffer(blob[32:], dtype=np.float32).copy()).cuda()
    slots = synth.workload_slots(w, 2, start=5)
    rx = nrx.Receiver(blob, w.net.num_rx_ant, w.num_users, w.num_prb, 1, "fp32")
    for s in slots:  # two calls in a row, different slots
        y, dmrs, bits, _ = H.device_inputs([s])
        ref = rx.nrx_detect_batch(y, dmrs, w.dmrs_symbols, bits).cpu().numpy()
        got = nrx.nrx_detect_noalloc(blob, wdev, y[0], dmrs[0], w.dmrs_symbols, bits[0]).cpu().numpy()
        torch.cuda.synchronize()
        err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
        assert err <= TOL_FP32, err
    rx.close()


def test_noalloc_rejects_slots_beyond_scratch():
    import torch
    nrx_build.build()
    w = synth.WORKLOADS["mu4_4rx_273prb"]
    blob = synth.pack_weights(w.net, synth.make_weights(w.net))
    wdev = torch.from_numpy(np.frombuffer(blob[32:], dtype=np.float32).copy()).cuda()
    s = synth.workload_slots(w, 1)[0]
    y, dmrs, bits, _ = H.device_inputs([s])
    with pytest.raises(nrx.NrxError) as e:
        nrx.nrx_detect_noalloc(blob, wdev, y[0], dmrs[0], w.dmrs_symbols, bits[0])
    assert e.value.status == nrx.NRX_EINVAL


def test_noalloc_net_near_the_weight_limit():
    """A net whose weights fill most of the 1 MiB weight region (C=64, R=1,
    N_it=9: 967 KB in kernel layout, 115 layer tensors) gives the context
    entry point's LLRs."""
    import torch
    nrx_build.build()
    net = synth.NetConfig(num_rx_ant=4, channels=64, res_blocks=1, iterations=9, m_max=6)
    blob = synth.pack_weights(net, synth.make_weights(net, seed=9))
    wdev = torch.from_numpy(np.frombuffer(blob[32:], dtype=np.float32).copy()).cuda()
    rng = np.random.Generator(np.random.PCG64(91))
    cfg = synth.SlotConfig(num_prb=4, num_users=2, num_rx_ant=4, dmrs_symbols=(2, 11), bits_per_symbol=(6, 2),
                           snr_db=12.0, num_taps=6, delay_spread_s=100e-9, doppler_hz=100.0, ula=True)
    s = synth.make_slot(cfg, rng)
    rx = nrx.Receiver(blob, 4, 2, 4, 1, "fp32")
    y, dmrs, bits, _ = H.device_inputs([s])
    ref = rx.nrx_detect_batch(y, dmrs, cfg.dmrs_symbols, bits).cpu().numpy()
    got = nrx.nrx_detect_noalloc(blob, wdev, y[0], dmrs[0], cfg.dmrs_symbols, bits[0]).cpu().numpy()
    err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    assert err <= TOL_FP32, err
    W64 = {k: v.astype(np.float64) for k, v in synth.make_weights(net, seed=9).items()}
    errs = H.rel_errors(got, H.oracle_nrx([s], W64, net), [s])
    assert max(errs) <= TOL_FP32, errs
    rx.close()
