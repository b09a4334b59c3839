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
