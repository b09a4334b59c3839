"""The C-ABI library loads, exports every symbol include/nrx.h declares, and
its host-side validation works without a GPU (no compute calls here)."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

from paper_2409_02912_b300 import build as nrx_build
from paper_2409_02912_b300 import bler, nrx, server, synth, train

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    nrx_build.build()
    return nrx.load()


def declared_functions():
    names = set()
    for h in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(
            r"^\s*(?:const\s+)?(?:nrx_status|void|size_t|int32_t|int64_t|char\s*\*|char)\s*\*?\s*(\w+)\s*\(",
            text, flags=re.M))
    return sorted(names)


def test_header_declares_the_binding_exports():
    assert sorted(nrx.EXPORTED + train.TRAIN_EXPORTED + bler.EVAL_EXPORTED + server.SERVER_EXPORTED) == \
        declared_functions()


def test_training_entry_points_validate_without_a_gpu(lib):
    """Host-side argument checks of the training ABI run before any launch."""
    tl = train.load()
    assert tl.nrx_train_gemm(0, 4, 4, 1, 4, 1, 1, 1, 4, None, None, 0, 1, 4, 0, 0, 1, None) == nrx.NRX_EINVAL
    # split K without accumulation, accumulation with an epilogue
    assert tl.nrx_train_gemm(4, 4, 4, 1, 4, 1, 1, 1, 4, None, None, 0, 1, 4, 0, 0, 2, None) == nrx.NRX_EINVAL
    assert tl.nrx_train_gemm(4, 4, 4, 1, 4, 1, 1, 1, 4, 1, None, 0, 1, 4, 0, 1, 1, None) == nrx.NRX_EINVAL
    assert tl.nrx_train_aggregate(1, 5, 16, 1, 2, None) == nrx.NRX_EINVAL
    assert tl.nrx_train_aggregate(1, 2, 16, 1, 1, None) == nrx.NRX_EINVAL
    assert tl.nrx_train_dw3(0, 12, 4, 1, 1, 0, 0, 2, None) == nrx.NRX_EINVAL
    assert tl.nrx_train_adam(0, 1, 1, 1, 1, 1, 0.9, 0.999, 1e-8, None) == nrx.NRX_EINVAL
    assert tl.nrx_train_adam(4, 1, 1, 1, 1, None, 0.9, 0.999, 1e-8, None) == nrx.NRX_EINVAL
    assert tl.nrx_train_zero(0, None, None) == nrx.NRX_OK
    assert tl.nrx_train_zero(-1, None, None) == nrx.NRX_EINVAL
    cfg = nrx.make_cfgs(1, 4, 2, (2, 11), [0], [1.0])
    assert tl.nrx_train_features(1, 2, 1, cfg, 1, None) == nrx.NRX_EINVAL   # null DMRS pointer
    assert tl.nrx_train_bce(1, cfg, 9, 1, 1, 1, 1.0, 1, 1, None) == nrx.NRX_EINVAL
    el = bler.load()
    assert el.nrx_conv_decode(1, 4097, 1, 1, None, 1, None) == nrx.NRX_EINVAL
    assert el.nrx_conv_decode(1, 0, 1, 1, None, 1, None) == nrx.NRX_EINVAL
    assert el.nrx_conv_decode(1, 64, None, 1, None, 1, None) == nrx.NRX_EINVAL
    assert el.nrx_conv_decode(0, 64, None, None, None, None, None) == nrx.NRX_OK
    sn = np.array([0, 160], dtype=np.int32)
    ds = np.array([2, 11], dtype=np.int32)
    assert lib.nrx_dmrs_gold(2, sn.ctypes.data, 1, 0, 4, 2, ds.ctypes.data, 1, None) == nrx.NRX_EINVAL
    assert lib.nrx_dmrs_gold(1, sn.ctypes.data, 65536, 0, 4, 2, ds.ctypes.data, 1, None) == nrx.NRX_EINVAL
    assert lib.nrx_dmrs_gold(1, sn.ctypes.data, 1, 2, 4, 2, ds.ctypes.data, 1, None) == nrx.NRX_EINVAL


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_struct_layout_matches_header():
    assert ctypes.sizeof(nrx.nrx_slot_cfg) == 40
    assert nrx.nrx_slot_cfg.dmrs_seq.offset == 32


def test_llr_count_and_status_strings(lib):
    cfg = nrx.make_cfgs(1, 273, 4, (2, 11), [0], [1.0])[0]
    bits = np.array([2, 4, 6, 6], dtype=np.int32)
    assert lib.nrx_llr_count(ctypes.byref(cfg), bits.ctypes.data) == 12 * 3276 * 18
    bad = np.array([2, 3, 6, 6], dtype=np.int32)
    assert lib.nrx_llr_count(ctypes.byref(cfg), bad.ctypes.data) == 0
    assert lib.nrx_status_string(nrx.NRX_EINVAL) == b"NRX_EINVAL"


def _create(lib, blob, B=2, users=1, prb=4, slots=1, prec=0):
    ctx = ctypes.c_void_p()
    buf = ctypes.create_string_buffer(blob, len(blob))
    st = lib.nrx_create(buf, len(blob), B, users, prb, slots, prec, ctypes.byref(ctx))
    if st == nrx.NRX_OK:
        lib.nrx_destroy(ctx)
    return st


def test_create_rejects_bad_blobs(lib):
    net = synth.WORKLOADS["su_2rx_4prb"].net
    blob = synth.pack_weights(net, synth.make_weights(net))
    assert _create(lib, blob[:-4]) == nrx.NRX_EINVAL            # truncated
    assert _create(lib, b"XXXX" + blob[4:]) == nrx.NRX_EINVAL    # magic
    assert _create(lib, blob, B=4) == nrx.NRX_EINVAL             # antenna mismatch
    assert _create(lib, blob, users=5) == nrx.NRX_EINVAL         # limits
    assert _create(lib, blob, prb=276) == nrx.NRX_EINVAL
    assert _create(lib, blob, slots=65) == nrx.NRX_EINVAL
    assert _create(lib, blob, prec=7) == nrx.NRX_EINVAL


def test_create_without_gpu_fails_loudly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    net = synth.WORKLOADS["su_2rx_4prb"].net
    blob = synth.pack_weights(net, synth.make_weights(net))
    assert _create(lib, blob) == nrx.NRX_ECUDA
    with pytest.raises(nrx.NrxError):
        nrx.Receiver(blob, 2, 1, 4)


def test_server_structs_and_validation(lib):
    """ctypes layouts of the serving ABI and its host-side config checks."""
    import ctypes
    assert ctypes.sizeof(server.nrx_request) == 72
    assert server.nrx_request.arrival_ns.offset == 56
    assert server.nrx_request.slot_number.offset == 68
    assert ctypes.sizeof(server.nrx_server_stats) == 120
    assert ctypes.sizeof(server.nrx_completion) == 40
    sl = server.load()
    net = synth.WORKLOADS["su_2rx_4prb"].net
    blob = synth.pack_weights(net, synth.make_weights(net))
    buf = ctypes.create_string_buffer(blob, len(blob))
    h = ctypes.c_void_p()
    for field, bad in (("num_buckets", 0), ("max_users", 5), ("max_batch", 65), ("queue_capacity", 0),
                       ("num_dmrs_symbols", 3), ("deadline_us", 0.0)):
        c = server.nrx_server_cfg(num_buckets=1, max_users=1, max_batch=1, queue_capacity=4, num_dmrs_symbols=1,
                                  precision=0, deadline_us=500.0, hbm_budget_bytes=1 << 30)
        c.bucket_prb[0] = 4
        c.dmrs_symbols[0] = 2
        setattr(c, field, bad)
        assert sl.nrx_server_create(buf, len(blob), 2, ctypes.byref(c), ctypes.byref(h)) == nrx.NRX_EINVAL, field
    assert sl.nrx_server_now_ns() > 0


def test_every_header_function_is_documented():
    """Each function the C headers declare is directly preceded by its own
    comment (arguments, layout, ownership, errors)."""
    import glob
    import re
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    missing = []
    for h in sorted(glob.glob(os.path.join(root, "include", "*.h"))):
        lines = open(h).read().splitlines()
        for i, line in enumerate(lines):
            m = re.match(r"^\s*(?:const\s+)?(?:nrx_status|void|size_t|int32_t|int64_t|char\s*\*|const char\s*\*)"
                         r"\s*\*?\s*(\w+)\s*\(", line)
            if not m:
                continue
            prev = next((lines[j].strip() for j in range(i - 1, -1, -1) if lines[j].strip()), "")
            if not (prev.endswith("*/") or prev.startswith("//")):
                missing.append(f"{os.path.basename(h)}:{m.group(1)}")
    assert not missing, missing


def _noalloc_header(B, C, R, N_it, m_max):
    F = 4 * B + 2
    n = (C * F + C + 9 * C + N_it * (2 * (C * C + C) + C * (2 * C + 2) + C + R * 2 * (9 * C + C * C + C))
         + C * C + C + m_max * C + m_max)
    return np.array([0x5758524E, 1, B, C, R, N_it, m_max, n], dtype=np.int32)


@pytest.mark.parametrize("B,C,R,N_it", [(4, 64, 4, 16), (4, 64, 4, 5), (4, 32, 2, 7), (4, 64, 1, 10)])
def test_noalloc_rejects_nets_beyond_its_tables_without_a_gpu(lib, B, C, R, N_it):
    """Nets whose copy plan (7 + N_it (6 + 6R) tensors > 128) or kernel-layout
    weights (> 1 MiB) exceed the allocation-free entry point's fixed tables
    are rejected from the header alone, before any CUDA call: the pointers
    below are aligned stand-ins that are never dereferenced."""
    hdr = _noalloc_header(B, C, R, N_it, 6)
    cfg = nrx.make_cfgs(1, 2, 2, (2, 11), [0x10000], [1.0])
    bits = np.array([2, 4], dtype=np.int32)
    st = lib.nrx_detect_noalloc(hdr.ctypes.data, 0x20000, 0x30000, cfg, bits.ctypes.data, 0x40000, None)
    assert st == nrx.NRX_EINVAL


def test_ldpc_decode_validates_without_a_gpu(lib):
    """Host-side checks of nrx_ldpc_decode run before any launch."""
    from paper_2409_02912_b300 import bler
    el = bler.load()
    bg = synth.ldpc_base_graph()
    rp, col, sh = (np.ascontiguousarray(a, dtype=np.int32) for a in bg.edges())
    args = lambda **k: dict(dict(n=1, E=64, qm=2, Z=16, kb=bg.kb, mb=bg.mb, rp=rp, col=col, sh=sh, it=10), **k)

    def call(a):
        return el.nrx_ldpc_decode(a["n"], None, None, a["E"], a["qm"], a["Z"], a["kb"], a["mb"], a["rp"].ctypes.data,
                                  a["col"].ctypes.data, a["sh"].ctypes.data, a["it"], 0.75, 1, None, None, None)
    assert call(args(n=0)) == nrx.NRX_OK                   # nothing to decode
    assert call(args()) == nrx.NRX_EINVAL                  # null device buffers
    assert call(args(n=0, Z=385)) == nrx.NRX_EINVAL        # lifting size
    assert call(args(n=0, E=63)) == nrx.NRX_EINVAL         # E not a multiple of qm
    assert call(args(n=0, it=0)) == nrx.NRX_EINVAL
    bad = col.copy()
    bad[0] = bg.nb
    assert call(args(n=0, col=bad)) == nrx.NRX_EINVAL      # column out of range
    dense = np.arange(bg.mb + 1, dtype=np.int32) * 17      # 17 edges per row
    assert call(args(n=0, rp=dense)) == nrx.NRX_EINVAL
