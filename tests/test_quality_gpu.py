"""Matched-BLER quality of the trained network (Sec. II-B training, Sec. IV
comparison at 10% BLER) on coded synthetic slots: the trained NRX against the
untrained one and LS+LMMSE on the same slots, and the reduced-precision modes
against FP32.  The paper's own curves are not reproducible (its data and
weights are absent), so the comparison is against this build's LMMSE."""
import pytest

from paper_2409_02912_b300 import evaluate, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a GPU", allow_module_level=True)


@pytest.fixture(scope="module")
def quality():
    net = synth.WORKLOADS["mu2_4rx_24prb"].net
    with open(evaluate.TRAINED_MU2, "rb") as f:
        blob = f.read()
    return evaluate.compare(blob, untrained_blob=synth.pack_weights(net, synth.make_weights(net)))


def test_trained_beats_untrained(quality):
    assert all(b == 1.0 for b in quality["nrx_untrained"]["bler"])
    assert quality["nrx_fp32"]["snr_at_10pct"] is not None
    assert quality["nrx_fp32"]["bler"][-1] < 0.02


def test_trained_beats_lmmse_on_the_same_slots(quality):
    """Fewer block errors than LS+LMMSE at 4-8 dB, and a lower SNR at the 10%
    BLER operating point."""
    snrs = quality["_sweep"]["snrs"]
    for i, snr in enumerate(snrs):
        if 4.0 <= snr <= 8.0:
            assert quality["nrx_fp32"]["bler"][i] < quality["lmmse"]["bler"][i], snr
    assert quality["nrx_fp32"]["snr_at_10pct"] < quality["lmmse"]["snr_at_10pct"]


def test_bf16_and_fp16_within_0p2_db_of_fp32(quality):
    ref = quality["nrx_fp32"]["snr_at_10pct"]
    for p in ("bf16", "fp16"):
        assert abs(quality[f"nrx_{p}"]["snr_at_10pct"] - ref) <= 0.2, p
    assert quality["nrx_fp8"]["snr_at_10pct"] is not None  # reported, not gated
