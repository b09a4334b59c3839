"""The GPU LDPC decoder (nrx_ldpc_decode, through the C ABI) against the
oracle decoders on the same received LLRs: the same layered normalised
min-sum, run in FP32 like the decoder, gives the same hard decisions after
1, 3 and 10 passes, and on
encoded QAM blocks over AWGN the GPU decodes every block the oracle's
sum-product decodes, with the same rate recovery."""
import numpy as np
import pytest

from oracle import ldpc_oracle as LO
from paper_2409_02912_b300 import bler, nrx, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2409_02912_b300 import build as nrx_build
    nrx_build.build()
    nrx.load()


def _device(arr, dtype):
    import torch
    return torch.from_numpy(np.ascontiguousarray(arr, dtype=dtype)).cuda()


@pytest.mark.parametrize("iterations", [1, 3, 10])
@pytest.mark.parametrize("Z,qm,E_factor", [(64, 4, 2.0), (13, 2, 1.6), (352, 6, 2.2)])
def test_layered_min_sum_matches_oracle(iterations, Z, qm, E_factor):
    bg = synth.ldpc_base_graph()
    rng = np.random.Generator(np.random.PCG64(Z * 31 + iterations))
    E = qm * int(E_factor * bg.kb * Z / qm)
    n_blocks = 3
    llr = rng.normal(0.0, 3.0, size=(n_blocks, E)).astype(np.float32)  # noisy, mostly undecodable
    got = bler.ldpc_decode(_device(llr.reshape(-1), np.float32), _device(np.arange(n_blocks) * E, np.int64), E, qm,
                           Z, bg, iterations=iterations, alpha=0.75, stop_early=False).cpu().numpy()
    for b in range(n_blocks):
        # decisions in the decoder's precision (FP32); no position is repeated at these E, so the
        # recovered LLRs are the received ones exactly
        hard, _, _ = LO.layered_min_sum(LO.rate_recover(llr[b].astype(np.float64), Z, bg.nb, qm), bg.V, Z,
                                        iterations=iterations, alpha=0.75, dtype=np.float32)
        assert np.array_equal(got[b], hard[:bg.kb * Z]), (b, int(np.sum(got[b] != hard[:bg.kb * Z])))


@pytest.mark.parametrize("qm,snr_db", [(2, 3.0), (4, 9.0), (6, 14.0)])
def test_decodes_qam_blocks_over_awgn(qm, snr_db):
    """Rate-1/2 blocks (Z = 96, E = 2 kb Z) on Gray QAM over AWGN with exact
    max-log LLRs: the GPU decoder (20 passes, early stop) recovers every block
    that the oracle's sum-product recovers, and most blocks at these SNRs."""
    from oracle import nrx_oracle as O
    bg = synth.ldpc_base_graph()
    Z = 96
    E = 2 * bg.kb * Z
    rng = np.random.Generator(np.random.PCG64(qm))
    n_blocks = 8
    info = rng.integers(0, 2, size=(n_blocks, bg.kb * Z), dtype=np.uint8)
    e = synth.ldpc_rate_match(bg, Z, synth.ldpc_encode(bg, Z, info), E, qm)
    n0 = 10 ** (-snr_db / 10)
    llr = np.zeros((n_blocks, E), dtype=np.float32)
    for b in range(n_blocks):
        x = synth.qam_modulate(e[b].reshape(-1, qm), qm)
        y = x + np.sqrt(n0 / 2) * (rng.standard_normal(x.shape) + 1j * rng.standard_normal(x.shape))
        llr[b] = O.maxlog_llr(y, np.full(y.shape, n0), qm).reshape(-1)
    got = bler.ldpc_decode(_device(llr.reshape(-1), np.float32), _device(np.arange(n_blocks) * E, np.int64), E, qm,
                           Z, bg, iterations=20).cpu().numpy()
    gpu_ok = [np.array_equal(got[b], info[b]) for b in range(n_blocks)]
    ref_ok = []
    for b in range(n_blocks):
        hard, _, _ = LO.sum_product(LO.rate_recover(llr[b].astype(np.float64), Z, bg.nb, qm), bg.V, Z, iterations=40)
        ref_ok.append(np.array_equal(hard[:bg.kb * Z], info[b]))
    assert all(g for g, r in zip(gpu_ok, ref_ok) if r), (gpu_ok, ref_ok)
    assert sum(gpu_ok) >= n_blocks - 2, gpu_ok
