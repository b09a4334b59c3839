"""GPU Viterbi decoder against the FP32 Viterbi oracle (bit-exact decoded
bits: both take the same FP32 add-compare-select decisions), with offsets,
interleaver, ragged block lengths and the limits."""
import numpy as np
import pytest

from oracle import conv_oracle as CO
from paper_2409_02912_b300 import bler, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a GPU", allow_module_level=True)


@pytest.mark.parametrize("n_blocks,n_info,use_perm,sigma", [
    (37, 1024, True, 1.5), (5, 1, False, 1.0), (9, 100, True, 3.0), (3, 4096, False, 2.0), (1, 7, True, 0.0)])
def test_decoder_matches_oracle(n_blocks, n_info, use_perm, sigma):
    rng = np.random.Generator(np.random.PCG64(n_blocks * 1000 + n_info))
    n_coded = 2 * (n_info + 6)
    perm = synth.interleaver(n_coded, seed=n_info) if use_perm else None
    gap = 13
    offsets = np.arange(n_blocks, dtype=np.int64) * (n_coded + gap) + 5
    buf = rng.standard_normal(int(offsets[-1]) + n_coded + gap).astype(np.float32) * 50.0
    info = rng.integers(0, 2, (n_blocks, n_info), dtype=np.uint8)
    expect = []
    for b in range(n_blocks):
        c = synth.conv_encode(info[b])
        l = ((2.0 * c - 1.0) * 2.0 + sigma * rng.standard_normal(n_coded)).astype(np.float32)
        span = np.empty(n_coded, dtype=np.float32)
        if perm is None:
            span[:] = l
        else:
            span[perm] = l
        buf[offsets[b]:offsets[b] + n_coded] = span
        expect.append(CO.viterbi_decode(l, n_info))
    dev = torch.from_numpy(buf).cuda()
    out = bler.conv_decode(dev, torch.from_numpy(offsets).cuda(), n_info,
                           None if perm is None else torch.from_numpy(perm).cuda()).cpu().numpy()
    assert np.array_equal(out, np.stack(expect))
    if sigma == 0.0:
        assert np.array_equal(out, info)


def test_coded_batch_block_errors_of_perfect_llrs():
    cfgs = [synth.SlotConfig(num_prb=4, num_users=2, num_rx_ant=2, dmrs_symbols=(2, 11), bits_per_symbol=(2, 4),
                             snr_db=10.0, num_taps=4, delay_spread_s=1e-7, doppler_hz=0.0, ula=False)] * 2
    cb = bler.coded_batch(cfgs, [1, 2], n_info=200)
    llr = np.concatenate([np.concatenate([np.where(s.bits[u].reshape(-1) == 1, 8.0, -8.0) for u in range(2)])
                          for s in cb.slots]).astype(np.float32)
    e, n, be, nb = bler.block_errors(torch.from_numpy(llr).cuda(), cb)
    assert n == cb.info.shape[0] > 0 and e == 0 and be == 0
    assert bler.snr_at_bler([0, 2, 4], [0.5, 0.2, 0.05]) == pytest.approx(2 + 2 * np.log10(2) / np.log10(4))


@pytest.mark.parametrize("n_id,n_scid,prb,syms", [(0, 0, 1, (2,)), (77, 1, 24, (2, 11)), (65535, 0, 273, (3, 12))])
def test_dmrs_gold_matches_transmitter(n_id, n_scid, prb, syms):
    """Device DMRS sequences equal the transmitter's TS 38.211 generator bit
    for bit (+-1/sqrt(2) in float32)."""
    from paper_2409_02912_b300 import nrx
    slots = [0, 5, 159]
    out = nrx.nrx_dmrs_gold(slots, n_id, prb, syms, n_scid).cpu().numpy()
    ref = np.stack([synth.dmrs_gold(prb, syms, s, n_id, n_scid) for s in slots])
    assert out.shape == ref.shape and np.array_equal(out, ref)


def test_receivers_with_device_generated_gold_pilots():
    """A slot transmitted with TS 38.211 Gold-sequence DMRS, received with the
    pilots generated on the device by nrx_dmrs_gold: LS+LMMSE and the FP32 NRX
    match the FP64 oracle fed the transmitter's pilots."""
    from oracle import nrx_oracle as O
    from paper_2409_02912_b300 import nrx
    w = synth.WORKLOADS["mu2_4rx_24prb"]
    cfg = synth.dataclasses.replace(synth.draw_slot_config(w, np.random.Generator(np.random.PCG64(5))),
                                    n_id=321, slot_number=7)
    sl = synth.make_slot(cfg, np.random.Generator(np.random.PCG64(6)))
    W = synth.make_weights(w.net)
    rx = nrx.Receiver(synth.pack_weights(w.net, W), 4, 2, 24, max_slots=1, precision="fp32")
    dm = nrx.nrx_dmrs_gold([7], 321, 24, cfg.dmrs_symbols)
    y = torch.from_numpy(sl.y[None]).cuda()
    bits = [list(cfg.bits_per_symbol)]
    l = rx.lmmse_detect_batch(y, dm, cfg.dmrs_symbols, bits, [cfg.noise_var]).cpu().numpy()
    ref = O.lmmse_receiver(sl.y, sl.dmrs, 2, cfg.dmrs_symbols, cfg.bits_per_symbol, cfg.noise_var)
    assert np.max(np.abs(l - ref)) <= 1e-4 * np.max(np.abs(ref))
    l = rx.nrx_detect_batch(y, dm, cfg.dmrs_symbols, bits).cpu().numpy()
    W64 = {k: v.astype(np.float64) for k, v in W.items()}
    ref = O.nrx_forward(sl.y, sl.dmrs, 2, cfg.dmrs_symbols, cfg.bits_per_symbol, W64, 2, 2)
    assert np.max(np.abs(l - ref)) <= 1e-4 * np.max(np.abs(ref))
