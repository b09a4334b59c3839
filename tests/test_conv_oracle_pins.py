"""Pins of the BLER-evaluation code and of the Viterbi oracle to facts other
than themselves: the generator polynomials' impulse response, linearity and
the free distance 10 of the (133, 171) code, brute-force maximum-likelihood
decoding of short blocks, and error correction within the free distance."""
import itertools

import numpy as np

from oracle import conv_oracle as CO
from paper_2409_02912_b300 import synth


def test_impulse_response_is_the_generator_polynomials():
    """A single 1 followed by zeros emits the generators' coefficients,
    current input first: 133 octal = 1011011, 171 octal = 1111001."""
    out = synth.conv_encode(np.array([1, 0, 0, 0, 0, 0, 0], dtype=np.uint8))
    assert out[0::2][:7].tolist() == [1, 0, 1, 1, 0, 1, 1]
    assert out[1::2][:7].tolist() == [1, 1, 1, 1, 0, 0, 1]
    assert out.size == 2 * (7 + 6) and not out[14:].any()


def test_encoder_is_linear_and_terminates():
    rng = np.random.Generator(np.random.PCG64(1))
    a = rng.integers(0, 2, 50, dtype=np.uint8)
    b = rng.integers(0, 2, 50, dtype=np.uint8)
    assert np.array_equal(synth.conv_encode(a ^ b), synth.conv_encode(a) ^ synth.conv_encode(b))


def test_free_distance_is_10():
    """The (133, 171) K=7 code has free distance 10 (minimum codeword weight
    over nonzero inputs; short inputs suffice to reach it)."""
    best = 99
    for n in range(1, 11):
        for v in range(1, 2 ** n):
            if not (v >> (n - 1)) & 1:
                continue
            u = np.array([(v >> k) & 1 for k in range(n)], dtype=np.uint8)
            best = min(best, int(synth.conv_encode(u).sum()))
    assert best == 10


def test_viterbi_is_maximum_likelihood_on_short_blocks():
    rng = np.random.Generator(np.random.PCG64(2))
    for n in (1, 4, 8):
        cws = np.array([synth.conv_encode(np.array(u, dtype=np.uint8))
                        for u in itertools.product([0, 1], repeat=n)])
        infos = np.array(list(itertools.product([0, 1], repeat=n)), dtype=np.uint8)
        done = 0
        for _ in range(60):
            l = rng.standard_normal(cws.shape[1]).astype(np.float32) * 2.0
            score = cws.astype(np.float64) @ l.astype(np.float64)
            order = np.sort(score)
            if order[-1] - order[-2] < 1e-3:
                continue  # near tie: ML not unique at float32 precision
            assert np.array_equal(CO.viterbi_decode(l, n), infos[np.argmax(score)])
            done += 1
        assert done > 40


def test_noiseless_round_trip_and_four_errors_corrected():
    rng = np.random.Generator(np.random.PCG64(3))
    info = rng.integers(0, 2, 1024, dtype=np.uint8)
    c = synth.conv_encode(info)
    l = np.where(c == 1, 4.0, -4.0).astype(np.float32)
    assert np.array_equal(CO.viterbi_decode(l, 1024), info)
    l[[100, 101, 102, 103]] *= -1.0   # four errors in a burst: within d_free = 10
    l[[900, 1500]] *= -1.0
    assert np.array_equal(CO.viterbi_decode(l, 1024), info)


def test_interleaved_blocks_in_the_bit_stream():
    rng = np.random.Generator(np.random.PCG64(4))
    n_info = 100
    perm = synth.interleaver(2 * (n_info + 6), seed=9)
    assert np.array_equal(np.sort(perm), np.arange(perm.size))
    stream, cu = synth.coded_bits(1000, n_info, perm, rng)
    assert cu.info.shape == (4, n_info) and cu.block_offset.tolist() == [0, 212, 424, 636]
    for b in range(4):
        blk = stream[cu.block_offset[b]:cu.block_offset[b] + 212]
        assert np.array_equal(blk[perm], synth.conv_encode(cu.info[b]))
