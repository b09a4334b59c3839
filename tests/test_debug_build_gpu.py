"""The bounds-checked build (libnrx_debug.so, compiled with NRX_DEBUG) on the
odd-size parity cases: every instrumented shared-memory and global index of
the kernels stays inside its array (zero recorded violations) and the results
still match the FP64 oracle.  This stands in for a memory checker: the checks
record and skip a bad access instead of faulting.

The debug library is loaded in a child process (one library per binding)."""
import os
import subprocess
import sys
import textwrap

import pytest

from paper_2409_02912_b300 import build as nrx_build

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent('''
    import numpy as np, torch
    from paper_2409_02912_b300 import bler, nrx, synth
    from oracle import ldpc_oracle as LO
    from tests import helpers as H
    assert nrx._LIB_PATH.endswith("libnrx_debug.so"), nrx._LIB_PATH
    nrx.debug_counters(reset=True)
    cases = [  # (U, B, num_prb, dmrs, R, N_it, bits): ragged user counts, 1 and 2 DMRS symbols, 1..8 antennas
        (1, 4, 1, (2,), 1, 1, (6,)),
        (3, 2, 5, (2, 11), 2, 2, (6, 2, 4)),
        (2, 8, 3, (3, 10), 2, 1, (4, 4)),
        (4, 4, 7, (5, 6), 1, 3, (2, 4, 6, 2)),
    ]
    worst = {}
    for U, B, prb, dmrs, R, N_it, bits in cases:
        net = synth.NetConfig(num_rx_ant=B, channels=64, res_blocks=R, iterations=N_it, m_max=6)
        rng = np.random.Generator(np.random.PCG64(91))
        slots = [synth.make_slot(synth.SlotConfig(num_prb=prb, num_users=U, num_rx_ant=B, dmrs_symbols=dmrs,
                                                  bits_per_symbol=bits, snr_db=float(rng.uniform(0, 15)),
                                                  num_taps=5, delay_spread_s=150e-9, doppler_hz=200.0,
                                                  ula=bool(i % 2)), rng) for i in range(3)]
        W = synth.make_weights(net)
        ref = H.oracle_nrx(slots, {k: v.astype(np.float64) for k, v in W.items()}, net)
        y, d, b, nv = H.device_inputs(slots)
        for prec in ("fp32", "bf16", "fp16", "fp8"):
            rx = nrx.Receiver(synth.pack_weights(net, W), B, U, prb, len(slots), prec)
            llr = rx.nrx_detect_batch(y, d, dmrs, b).cpu().numpy()
            rx.nrx_check()
            e = max(H.rel_errors(llr, ref, slots))
            worst[prec] = max(worst.get(prec, 0.0), e)
            if prec == "fp32" and B in (1, 2, 4, 8):
                l2 = rx.lmmse_detect_batch(y, d, dmrs, b, nv).cpu().numpy()
                worst["lmmse"] = max(worst.get("lmmse", 0.0), max(H.rel_errors(l2, H.oracle_lmmse(slots), slots)))
            rx.close()
    # LDPC decoder at a lifting size that is not a multiple of 32
    bg = synth.ldpc_base_graph()
    Z, qm = 13, 2
    E = qm * int(1.6 * bg.kb * Z / qm)
    llr = np.random.Generator(np.random.PCG64(3)).normal(0, 3, size=(2, E)).astype(np.float32)
    got = bler.ldpc_decode(torch.from_numpy(llr.reshape(-1)).cuda(), torch.tensor([0, E]).cuda(), E, qm, Z, bg,
                           iterations=3, stop_early=False).cpu().numpy()
    for k in range(2):
        hard, _, _ = LO.layered_min_sum(LO.rate_recover(llr[k].astype(np.float64), Z, bg.nb, qm), bg.V, Z, 3,
                                        dtype=np.float32)
        assert np.array_equal(got[k], hard[:bg.kb * Z])
    torch.cuda.synchronize()
    print("WORST", worst)
    print("DEBUG", nrx.debug_counters())
''')


def test_bounds_checked_build_on_odd_sizes():
    lib = nrx_build.build(debug=True)
    env = dict(os.environ, NRX_LIBRARY=lib, PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True, timeout=1500)
    print(r.stdout[-3000:], r.stderr[-3000:])
    assert r.returncode == 0
    dbg = eval(r.stdout.split("DEBUG", 1)[1].strip().splitlines()[0])
    worst = eval(r.stdout.split("WORST", 1)[1].strip().splitlines()[0])
    assert dbg["violations"] == 0, dbg
    assert worst["fp32"] <= 1e-4 and worst["lmmse"] <= 1e-4, worst
    assert worst["bf16"] <= 2e-2 and worst["fp16"] <= 2e-2, worst
