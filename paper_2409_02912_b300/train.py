"""NRX training on the GPU (Sec. II-B): forward pass with saved activations,
hand-written reverse pass and Adam, composed from the layer kernels of
``include/nrx_train.h``.

Loss: for every CGNN iteration k (multi-loss), the masked BCE of
ReadoutLLRs(S^(k)) against the bits (mean over the batch's counted bits) plus
gamma times the MSE of ReadoutChEst(S^(k)) against the true channel (mean over
slot, user, antenna and RE of |h_hat - h|^2), summed over k.

This module only marshals arguments and orders the launches: every arithmetic
step (features, dense and depthwise layers and their gradients, aggregation,
losses, Adam) runs in the CUDA kernels of ``libnrx.so``.  torch provides the
device memory and the stream.  The FP32 master weights live in one flat device
vector in the inference blob order followed by the ReadoutChEst head, so the
trained network exports directly as a weight blob for ``nrx_create``.
"""
from __future__ import annotations

import collections
import ctypes
import math
import struct
from typing import Dict, List, Optional

import numpy as np

from . import nrx, synth

TRAIN_EXPORTED = (
    "nrx_train_features", "nrx_train_gemm", "nrx_train_gemm_bf16", "nrx_train_check", "nrx_train_colsum", "nrx_train_dw3", "nrx_train_dw3_wgrad",
    "nrx_train_relu_mask", "nrx_train_aggregate", "nrx_train_axpy", "nrx_train_bce", "nrx_train_mse",
    "nrx_train_zero", "nrx_train_copy", "nrx_train_adam", "nrx_train_sim_scratch_bytes", "nrx_train_simulate",
    "nrx_train_plane_mask",
)


class nrx_sim_slot(ctypes.Structure):
    _fields_ = [("noise_var", ctypes.c_float), ("delay_spread_s", ctypes.c_float), ("doppler_hz", ctypes.c_float),
                ("num_taps", ctypes.c_int32), ("ula", ctypes.c_int32), ("bits_per_symbol", ctypes.c_int32 * 4)]

_configured = False


def load():
    """``libnrx.so`` with the training entry points' signatures set."""
    global _configured
    lib = nrx.load()
    if _configured:
        return lib
    P, I32, I64, F32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float
    CFG = ctypes.POINTER(nrx.nrx_slot_cfg)
    sig = {
        "nrx_train_features": [I32, I32, P, CFG, P, P],
        "nrx_train_gemm": [I32, I32, I32, P, I64, I64, P, I64, I64, P, P, I64, P, I64, I32, I32, I32, P],
        "nrx_train_gemm_bf16": [I32, I32, I32, P, I64, I64, P, I64, I64, P, P, I64, P, I64, I32, I32, I32, P],
        "nrx_train_check": [P],
        "nrx_train_colsum": [I32, I32, P, I64, P, P],
        "nrx_train_dw3": [I32, I32, I32, P, P, I32, I32, P, P],
        "nrx_train_dw3_wgrad": [I32, I32, I32, P, P, P, P],
        "nrx_train_relu_mask": [I64, P, P, P],
        "nrx_train_aggregate": [I32, I32, I64, P, P, P],
        "nrx_train_axpy": [I64, F32, P, P, P],
        "nrx_train_bce": [I32, CFG, I32, P, P, P, F32, P, P, P],
        "nrx_train_mse": [I64, P, P, F32, P, P, P],
        "nrx_train_zero": [I64, P, P],
        "nrx_train_copy": [I64, P, P, P],
        "nrx_train_adam": [I64, P, P, P, P, P, F32, F32, F32, P],
        "nrx_train_simulate": [I32, ctypes.POINTER(nrx_sim_slot), I32, I32, I32, I32, P, I32, ctypes.c_uint64,
                               ctypes.c_uint32, P, P, P, P, P, P, P],
        "nrx_train_plane_mask": [I64, I64, I32, I64, I64, P, I32, P, P, I32, P],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.nrx_train_sim_scratch_bytes.argtypes = [I32, I32, I32, I32]
    lib.nrx_train_sim_scratch_bytes.restype = ctypes.c_size_t
    _configured = True
    return lib


def _ptr(t) -> Optional[int]:
    return None if t is None else t.data_ptr()


class _Ops:
    """Thin wrappers: one C call each, raising on a non-OK status."""

    def __init__(self, stream_ptr, precision: str = "fp32"):
        self.lib = load()
        self.st = stream_ptr
        if precision not in ("fp32", "bf16"):
            raise ValueError(f"training precision {precision!r}: fp32 or bf16")
        self._gemm = self.lib.nrx_train_gemm_bf16 if precision == "bf16" else self.lib.nrx_train_gemm

    def _ok(self, st, what):
        if st != nrx.NRX_OK:
            raise nrx.NrxError(st, what)

    def gemm(self, M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, bias=None, R=None, ldr=0, relu=False,
             accumulate=False, split_k=1):
        self._ok(self._gemm(M, N, K, A, sam, sak, B, sbk, sbn, bias, R, ldr, C, ldc, int(relu), int(accumulate),
                            split_k, self.st), "nrx_train_gemm")

    def colsum(self, M, N, X, ldx, out):
        self._ok(self.lib.nrx_train_colsum(M, N, X, ldx, out, self.st), "nrx_train_colsum")

    def dw3(self, planes, S, C, X, k, Y, flip=False, relu=False):
        self._ok(self.lib.nrx_train_dw3(planes, S, C, X, k, int(flip), int(relu), Y, self.st), "nrx_train_dw3")

    def dw3_wgrad(self, planes, S, C, X, G, gk):
        self._ok(self.lib.nrx_train_dw3_wgrad(planes, S, C, X, G, gk, self.st), "nrx_train_dw3_wgrad")

    def relu_mask(self, n, G, Y):
        self._ok(self.lib.nrx_train_relu_mask(n, G, Y, self.st), "nrx_train_relu_mask")

    def aggregate(self, n_slots, U, per_user, m, a):
        self._ok(self.lib.nrx_train_aggregate(n_slots, U, per_user, m, a, self.st), "nrx_train_aggregate")

    def axpy(self, n, alpha, x, y):
        self._ok(self.lib.nrx_train_axpy(n, alpha, x, y, self.st), "nrx_train_axpy")

    def zero(self, nbytes, p):
        self._ok(self.lib.nrx_train_zero(nbytes, p, self.st), "nrx_train_zero")

    def copy(self, nbytes, dst, src):
        self._ok(self.lib.nrx_train_copy(nbytes, dst, src, self.st), "nrx_train_copy")

    def plane_mask(self, planes, rows, width, ld_src, ld_dst, m_u, m_head, src, dst, accumulate=False):
        self._ok(self.lib.nrx_train_plane_mask(planes, rows, width, ld_src, ld_dst, m_u, m_head, src, dst,
                                               int(accumulate), self.st), "nrx_train_plane_mask")


class Trainer:
    """Training state of one network (FP32 master weights, gradients, Adam
    moments) on the current CUDA device.  ``precision`` selects the GEMMs of
    the forward and reverse passes: "fp32" (CUDA cores) or "bf16" (tensor
    cores, BF16 operands, FP32 accumulation); everything else is FP32.

    ``loss_and_grad(batch)`` runs the forward and reverse passes and leaves the
    gradient in ``self.g``; ``step(batch)`` adds the Adam update.

    ``recompute``: keep only each residual block's input and rebuild its three
    conv activations (DW1, ReLU(PW1), ReLU(DW2)) from it in the reverse pass,
    one block at a time, instead of storing them for every block of every
    iteration.  ``None`` decides per batch shape: recompute when the stored
    activations would take more than ``memory_fraction`` of the free device
    memory.  The recomputed activations are bit-identical to the stored ones
    (the forward kernels are deterministic), so the gradient is the same.
    """

    def __init__(self, net: synth.NetConfig, weights: Dict[str, np.ndarray],
                 chest: Optional[Dict[str, np.ndarray]] = None, lr: float = 1e-3, gamma: float = 1.0,
                 beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8, precision: str = "fp32",
                 recompute: Optional[bool] = None, memory_fraction: float = 0.5):
        import torch
        self.torch = torch
        self.precision = precision
        self.recompute = recompute
        self.memory_fraction = memory_fraction
        self.recomputing = False  # mode of the current buffers
        _Ops(None, precision)  # validates the precision
        self.net = net
        self.lr, self.gamma, self.beta1, self.beta2, self.eps = lr, gamma, beta1, beta2, eps
        chest = synth.make_chest_weights(net) if chest is None else chest
        self.layout = synth.weight_layout(net) + synth.chest_layout(net)
        self.offset: Dict[str, int] = {}
        flat = []
        o = 0
        for name, shape in self.layout:
            src = weights[name] if name in weights else chest[name]
            a = np.ascontiguousarray(src, dtype=np.float32).reshape(-1)
            assert a.size == int(np.prod(shape)), name
            self.offset[name] = o
            flat.append(a)
            o += a.size
        self.n_blob = sum(int(np.prod(s)) for _, s in synth.weight_layout(net))
        self.n_total = o
        dev = torch.device("cuda")
        self.w = torch.from_numpy(np.concatenate(flat)).to(dev)
        self.g = torch.zeros_like(self.w)
        self.m1 = torch.zeros_like(self.w)
        self.m2 = torch.zeros_like(self.w)
        self.t = 0
        self._bufs: "collections.OrderedDict[tuple, dict]" = collections.OrderedDict()
        self.loss_dev = torch.zeros(2 * net.iterations, dtype=torch.float64, device=dev)
        self.lr_t_dev = torch.zeros(1, dtype=torch.float32, device=dev)
        self._lr_host = torch.zeros(1, dtype=torch.float32).pin_memory()
        # captured steps: key -> (graph, its device batch, key of the buffers it uses)
        self._graphs: Dict[tuple, tuple] = {}

    # -- weights ------------------------------------------------------------
    def _wp(self, name: str) -> int:
        return self.w.data_ptr() + 4 * self.offset[name]

    def _gp(self, name: str) -> int:
        return self.g.data_ptr() + 4 * self.offset[name]

    def weights(self) -> Dict[str, np.ndarray]:
        """Current master weights (float32 numpy, inference and head)."""
        host = self.w.cpu().numpy()
        return {n: host[self.offset[n]:self.offset[n] + int(np.prod(s))].reshape(s).copy() for n, s in self.layout}

    def grads(self) -> Dict[str, np.ndarray]:
        host = self.g.cpu().numpy()
        return {n: host[self.offset[n]:self.offset[n] + int(np.prod(s))].reshape(s).copy() for n, s in self.layout}

    def save(self, path: str):
        """Checkpoint (weights, Adam moments, step count, hyper-parameters) to
        an ``.npz`` file."""
        net = self.net
        np.savez(path, w=self.w.cpu().numpy(), m1=self.m1.cpu().numpy(), m2=self.m2.cpu().numpy(),
                 t=np.int64(self.t), net=np.array([net.num_rx_ant, net.channels, net.res_blocks, net.iterations,
                                                   net.m_max], dtype=np.int64))

    def restore(self, path: str):
        """Resume from a ``save`` checkpoint of the same network shape."""
        z = np.load(path)
        net = self.net
        want = [net.num_rx_ant, net.channels, net.res_blocks, net.iterations, net.m_max]
        if list(z["net"]) != want or z["w"].size != self.n_total:
            raise ValueError(f"checkpoint is for network {list(z['net'])}, not {want}")
        for dst, key in ((self.w, "w"), (self.m1, "m1"), (self.m2, "m2")):
            dst.copy_(self.torch.from_numpy(z[key]))
        self.t = int(z["t"])

    def blob(self) -> bytes:
        """Inference weight blob (nrx.h layout) of the current weights."""
        net = self.net
        hdr = struct.pack("<8i", synth.WEIGHT_MAGIC,
                          synth.WEIGHT_VERSION_VAR_IO if net.var_io else synth.WEIGHT_VERSION, net.num_rx_ant,
                          net.channels, net.res_blocks, net.iterations, net.m_max, self.n_blob)
        return hdr + self.w[:self.n_blob].cpu().numpy().tobytes()

    # -- buffers ------------------------------------------------------------
    def activation_bytes(self, n: int, U: int, S: int, recompute: bool) -> int:
        """Device bytes of the saved activations and reverse-pass scratch for
        a batch of n slots x U users x S subcarriers, in either mode."""
        net = self.net
        C, F, R, K, B, mm = net.channels, net.in_features, net.res_blocks, net.iterations, net.num_rx_ant, net.m_max
        conv = 3 if recompute else 3 * K * R
        cols = (F + C + (K + 1) * C + 3 * K * C + K * (R + 1) * C + conv * C + K * (C + mm + C + 2 * B)
                + 4 * C + mm + 2 * B)
        if net.var_io:
            H = net.heads
            cols += 2 * len(H) * C + K * (len(H) * C + sum(H)) + sum(H) + C
        return 4 * n * U * 14 * S * cols

    def _use_recompute(self, n, U, S) -> bool:
        if self.recompute is not None:
            return bool(self.recompute)
        free, _ = self.torch.cuda.mem_get_info()
        return self.activation_bytes(n, U, S, False) > self.memory_fraction * free

    MAX_SHAPES = 4  # batch shapes kept resident (e.g. one per number of active users)

    def _buffers(self, n, U, S):
        key = (n, U, S)
        if key in self._bufs:
            self._bufs.move_to_end(key)
            self.recomputing = self._bufs[key]["rc"]
            return self._bufs[key]
        torch = self.torch
        net = self.net
        C, F, R, K = net.channels, net.in_features, net.res_blocks, net.iterations
        M = n * U * 14 * S
        while len(self._bufs) >= self.MAX_SHAPES:  # drop the oldest shape and the graphs that use it
            old, _ = self._bufs.popitem(last=False)
            for gk in [gk for gk, ent in self._graphs.items() if ent[2] == old]:
                del self._graphs[gk]
        rc = self._use_recompute(n, U, S)
        self.recomputing = rc
        e = lambda w: torch.empty((M, w), dtype=torch.float32, device="cuda")  # noqa: E731
        def conv():  # conv activations of every (iteration, block), or one shared
            if rc:      # set that the reverse pass refills block by block
                t = e(C)
                return [[t] * R for _ in range(K)]
            return [[e(C) for _ in range(R)] for _ in range(K)]

        b = {"rc": rc, "x": e(F), "P0": e(C), "S": [e(C) for _ in range(K + 1)],
             "h1": [e(C) for _ in range(K)], "msg": [e(C) for _ in range(K)], "a": [e(C) for _ in range(K)],
             "z": [[e(C) for _ in range(R + 1)] for _ in range(K)],
             "d1": conv(), "p1": conv(), "d2": conv(),
             "r1": [e(C) for _ in range(K)], "l": [e(net.m_max) for _ in range(K)],
             "c1": [e(C) for _ in range(K)], "hh": [e(2 * net.num_rx_ant) for _ in range(K)],
             "gS": e(C), "gz": e(C), "t1": e(C), "t2": e(C), "gl": e(net.m_max),
             "ghh": e(2 * net.num_rx_ant)}
        if net.var_io:  # per-head StateInit and read-out activations (Sec. III)
            H = net.heads
            b.update({"P0h": [e(C) for _ in H], "S0h": [e(C) for _ in H],
                      "r1h": [[e(C) for _ in H] for _ in range(K)], "lh": [[e(m) for m in H] for _ in range(K)],
                      "glh": [e(m) for m in H], "gSh": e(C)})
        self._bufs[key] = b
        return b

    # -- forward / backward -------------------------------------------------
    def _enqueue(self, batch: "DeviceBatch", st, adam: bool):
        """Enqueue one step on stream `st` with no host synchronisation (so it
        can be captured into a CUDA graph): zero the gradient and the loss
        words, forward pass with saved activations, losses, reverse pass, and
        with `adam` the update (step size read from ``self.lr_t_dev``)."""
        net = self.net
        ops = _Ops(st, self.precision)
        lib = ops.lib
        n, U, S = batch.n, batch.U, batch.S
        C, F, R, K, B = net.channels, net.in_features, net.res_blocks, net.iterations, net.num_rx_ant
        mm = net.m_max
        M = n * U * 14 * S
        planes = n * U
        bf = self._buffers(n, U, S)
        p = lambda t: t.data_ptr()  # noqa: E731
        wp, gp = self._wp, self._gp
        split = max(1, min(1184, math.ceil(M / 128)))

        ops.zero(4 * self.n_total, self.g.data_ptr())
        ops.zero(8 * 2 * K, self.loss_dev.data_ptr())

        def dense(X, ldx, name, in_dim, out_dim, Y, relu=False, R_=None, bias=True):
            ops.gemm(M, out_dim, in_dim, X, ldx, 1, wp(name + ".w"), 1, in_dim, Y, out_dim,
                     bias=wp(name + ".b") if bias else None, R=R_, ldr=out_dim if R_ else 0, relu=relu)

        def dense_bwd(G, X, ldx, name, in_dim, out_dim, gX=None, accumulate_into_gX=False):
            """G [M][out] gradient of y = W x + b: dW += G^T X, db += colsum G,
            gX (=|+=) G W."""
            ops.gemm(out_dim, in_dim, M, G, 1, out_dim, X, ldx, 1, gp(name + ".w"), in_dim,
                     accumulate=True, split_k=split)
            ops.colsum(M, out_dim, G, out_dim, gp(name + ".b"))
            if gX is not None:
                ops.gemm(M, in_dim, out_dim, G, out_dim, 1, wp(name + ".w"), in_dim, 1, gX, in_dim,
                         R=gX if accumulate_into_gX else None, ldr=in_dim if accumulate_into_gX else 0)

        # ---- forward ----
        self._ok(lib.nrx_train_features(n, B, batch.y.data_ptr(), batch.cfgs, p(bf["x"]), st), "features")
        m_u = batch.m_u.data_ptr()
        rows = 14 * S
        if net.var_io:  # every head over all REs, then each user's plane from its own head
            for h, m in enumerate(net.heads):
                dense(p(bf["x"]), F, f"init.m{m}.pw", F, C, p(bf["P0h"][h]))
                ops.dw3(planes, S, C, p(bf["P0h"][h]), wp(f"init.m{m}.dw"), p(bf["S0h"][h]), relu=True)
                ops.plane_mask(planes, rows, C, C, C, m_u, m, p(bf["S0h"][h]), p(bf["S"][0]), accumulate=h > 0)
        else:
            dense(p(bf["x"]), F, "init.pw", F, C, p(bf["P0"]))
            ops.dw3(planes, S, C, p(bf["P0"]), wp("init.dw"), p(bf["S"][0]), relu=True)
        for k in range(K):
            q = f"it{k}."
            Sk = p(bf["S"][k])
            dense(Sk, C, q + "mp1", C, C, p(bf["h1"][k]), relu=True)
            dense(p(bf["h1"][k]), C, q + "mp2", C, C, p(bf["msg"][k]))
            ops.aggregate(n, U, 14 * S * C, p(bf["msg"][k]), p(bf["a"][k]))
            z0 = p(bf["z"][k][0])
            W_in, D_in = wp(q + "in.w"), 2 * C + 2
            ops.gemm(M, C, C, Sk, C, 1, W_in, 1, D_in, z0, C, bias=wp(q + "in.b"))
            ops.gemm(M, C, C, p(bf["a"][k]), C, 1, W_in + 4 * C, 1, D_in, z0, C, R=z0, ldr=C)
            ops.gemm(M, C, 2, p(bf["x"]) + 4 * 4 * B, F, 1, W_in + 4 * 2 * C, 1, D_in, z0, C, R=z0, ldr=C)
            for r in range(R):
                bq = f"{q}blk{r}."
                zr, zn = p(bf["z"][k][r]), p(bf["z"][k][r + 1])
                ops.dw3(planes, S, C, zr, wp(bq + "dw1"), p(bf["d1"][k][r]))
                dense(p(bf["d1"][k][r]), C, bq + "pw1", C, C, p(bf["p1"][k][r]), relu=True)
                ops.dw3(planes, S, C, p(bf["p1"][k][r]), wp(bq + "dw2"), p(bf["d2"][k][r]), relu=True)
                dense(p(bf["d2"][k][r]), C, bq + "pw2", C, C, zn, R_=zr)
            # S^(k+1) = S^(k) + z_R
            ops.copy(4 * M * C, p(bf["S"][k + 1]), Sk)
            ops.axpy(M * C, 1.0, p(bf["z"][k][R]), p(bf["S"][k + 1]))
            # read-outs after iteration k (multi-loss)
            Sn = p(bf["S"][k + 1])
            if net.var_io:  # LLRs of each plane from its own head, m outputs (the rest stay zero)
                ops.zero(4 * M * mm, p(bf["l"][k]))
                for h, m in enumerate(net.heads):
                    dense(Sn, C, f"ro.m{m}.1", C, C, p(bf["r1h"][k][h]), relu=True)
                    dense(p(bf["r1h"][k][h]), C, f"ro.m{m}.2", C, m, p(bf["lh"][k][h]))
                    ops.plane_mask(planes, rows, m, m, mm, m_u, m, p(bf["lh"][k][h]), p(bf["l"][k]),
                                   accumulate=True)
            else:
                dense(Sn, C, "ro1", C, C, p(bf["r1"][k]), relu=True)
                dense(p(bf["r1"][k]), C, "ro2", C, mm, p(bf["l"][k]))
            if self.gamma > 0:
                dense(Sn, C, "chest.1", C, C, p(bf["c1"][k]), relu=True)
                dense(p(bf["c1"][k]), C, "chest.2", C, 2 * B, p(bf["hh"][k]))

        # ---- reverse ----
        gS, gz, t1, t2 = p(bf["gS"]), p(bf["gz"]), p(bf["t1"]), p(bf["t2"])
        ops.zero(4 * M * C, gS)
        n_mse = float(n * U * 14 * S * B)
        for k in reversed(range(K)):
            q = f"it{k}."
            Sn = p(bf["S"][k + 1])
            # LLR read-out k
            gl = p(bf["gl"])
            self._ok(lib.nrx_train_bce(n, batch.cfgs, mm, p(bf["l"][k]), batch.bits.data_ptr(),
                                       batch.m_u.data_ptr(), 1.0, gl, self.loss_dev.data_ptr() + 8 * k, st), "bce")
            if net.var_io:  # route each plane's LLR gradient to its head
                for h, m in enumerate(net.heads):
                    glh = p(bf["glh"][h])
                    ops.plane_mask(planes, rows, m, mm, m, m_u, m, gl, glh)
                    dense_bwd(glh, p(bf["r1h"][k][h]), C, f"ro.m{m}.2", C, m, gX=t1)
                    ops.relu_mask(M * C, t1, p(bf["r1h"][k][h]))
                    dense_bwd(t1, Sn, C, f"ro.m{m}.1", C, C, gX=gS, accumulate_into_gX=True)
            else:
                dense_bwd(gl, p(bf["r1"][k]), C, "ro2", C, mm, gX=t1)
                ops.relu_mask(M * C, t1, p(bf["r1"][k]))
                dense_bwd(t1, Sn, C, "ro1", C, C, gX=gS, accumulate_into_gX=True)
            if self.gamma > 0:
                ghh = p(bf["ghh"])
                self._ok(lib.nrx_train_mse(M * 2 * B, p(bf["hh"][k]), batch.h.data_ptr(), self.gamma / n_mse, ghh,
                                           self.loss_dev.data_ptr() + 8 * (K + k), st), "mse")
                dense_bwd(ghh, p(bf["c1"][k]), C, "chest.2", C, 2 * B, gX=t1)
                ops.relu_mask(M * C, t1, p(bf["c1"][k]))
                dense_bwd(t1, Sn, C, "chest.1", C, C, gX=gS, accumulate_into_gX=True)
            # CNN update: S^(k+1) = S^(k) + z_R; gradient of z_R is gS
            ops.copy(4 * M * C, gz, gS)
            for r in reversed(range(R)):
                bq = f"{q}blk{r}."
                d1, p1, d2 = p(bf["d1"][k][r]), p(bf["p1"][k][r]), p(bf["d2"][k][r])
                if bf["rc"]:  # rebuild this block's conv activations from its input
                    zr = p(bf["z"][k][r])
                    ops.dw3(planes, S, C, zr, wp(bq + "dw1"), d1)
                    dense(d1, C, bq + "pw1", C, C, p1, relu=True)
                    ops.dw3(planes, S, C, p1, wp(bq + "dw2"), d2, relu=True)
                dense_bwd(gz, d2, C, bq + "pw2", C, C, gX=t1)
                ops.relu_mask(M * C, t1, d2)
                ops.dw3(planes, S, C, t1, wp(bq + "dw2"), t2, flip=True)
                ops.dw3_wgrad(planes, S, C, p1, t1, gp(bq + "dw2"))
                ops.relu_mask(M * C, t2, p1)
                dense_bwd(t2, d1, C, bq + "pw1", C, C, gX=t1)
                ops.dw3(planes, S, C, t1, wp(bq + "dw1"), t2, flip=True)
                ops.dw3_wgrad(planes, S, C, p(bf["z"][k][r]), t1, gp(bq + "dw1"))
                ops.axpy(M * C, 1.0, t2, gz)
            # z0 = in([S, a, PE])
            Sk, ak = p(bf["S"][k]), p(bf["a"][k])
            W_in, G_in, D_in = wp(q + "in.w"), gp(q + "in.w"), 2 * C + 2
            ops.gemm(M, C, C, gz, C, 1, W_in, D_in, 1, gS, C, R=gS, ldr=C)
            ops.gemm(M, C, C, gz, C, 1, W_in + 4 * C, D_in, 1, t1, C)  # gradient of a
            ops.gemm(C, C, M, gz, 1, C, Sk, C, 1, G_in, D_in, accumulate=True, split_k=split)
            ops.gemm(C, C, M, gz, 1, C, ak, C, 1, G_in + 4 * C, D_in, accumulate=True, split_k=split)
            ops.gemm(C, 2, M, gz, 1, C, p(bf["x"]) + 4 * 4 * B, F, 1, G_in + 4 * 2 * C, D_in, accumulate=True,
                     split_k=split)
            ops.colsum(M, C, gz, C, gp(q + "in.b"))
            # messages: a = sum over the other users (symmetric)
            ops.aggregate(n, U, 14 * S * C, t1, t2)
            dense_bwd(t2, p(bf["h1"][k]), C, q + "mp2", C, C, gX=t1)
            ops.relu_mask(M * C, t1, p(bf["h1"][k]))
            dense_bwd(t1, Sk, C, q + "mp1", C, C, gX=gS, accumulate_into_gX=True)
        # StateInit: S0 = ReLU(DW(P0)), P0 = PW(x)
        if net.var_io:  # each head receives the gradient of its planes only
            gSh = p(bf["gSh"])
            for h, m in enumerate(net.heads):
                ops.plane_mask(planes, rows, C, C, C, m_u, m, gS, gSh)
                ops.relu_mask(M * C, gSh, p(bf["S0h"][h]))
                ops.dw3(planes, S, C, gSh, wp(f"init.m{m}.dw"), t1, flip=True)
                ops.dw3_wgrad(planes, S, C, p(bf["P0h"][h]), gSh, gp(f"init.m{m}.dw"))
                dense_bwd(t1, p(bf["x"]), F, f"init.m{m}.pw", F, C)
        else:
            ops.relu_mask(M * C, gS, p(bf["S"][0]))
            ops.dw3(planes, S, C, gS, wp("init.dw"), t1, flip=True)
            ops.dw3_wgrad(planes, S, C, p(bf["P0"]), gS, gp("init.dw"))
            dense_bwd(t1, p(bf["x"]), F, "init.pw", F, C)
        if adam:
            ops.copy(4, self.lr_t_dev.data_ptr(), self._lr_host.data_ptr())
            self._ok(lib.nrx_train_adam(self.n_total, self.w.data_ptr(), self.g.data_ptr(), self.m1.data_ptr(),
                                        self.m2.data_ptr(), self.lr_t_dev.data_ptr(), self.beta1, self.beta2,
                                        self.eps, st), "adam")

    def _read_loss(self) -> Dict[str, List[float]]:
        K = self.net.iterations
        ld = self.loss_dev.cpu().numpy()
        self._ok(load().nrx_train_check(nrx._stream_ptr(None)), "nrx_train_check")
        bce = [float(v) for v in ld[:K]]
        mse = [float(v) / self.gamma for v in ld[K:]] if self.gamma > 0 else [0.0] * K
        return {"bce": bce, "mse": mse, "loss": float(sum(bce) + self.gamma * sum(mse))}

    def _advance(self):
        """Step counter and this step's bias-corrected Adam step size (written
        to pinned host memory; the enqueued copy moves it to the device)."""
        self.t += 1
        self._lr_host[0] = self.lr * math.sqrt(1.0 - self.beta2 ** self.t) / (1.0 - self.beta1 ** self.t)

    def loss_and_grad(self, batch: "DeviceBatch", stream=None) -> Dict[str, List[float]]:
        """Forward + reverse pass over one batch; gradient left in ``self.g``.
        Returns the per-iteration BCE and MSE means and the total loss."""
        self._enqueue(batch, nrx._stream_ptr(stream), adam=False)
        return self._read_loss()

    def step(self, batch: "DeviceBatch", stream=None) -> Dict[str, List[float]]:
        """One training step: loss, gradient, Adam update of the master weights."""
        self._advance()
        self._enqueue(batch, nrx._stream_ptr(stream), adam=True)
        return self._read_loss()

    def graph_step(self, tb) -> Dict[str, List[float]]:
        """``step`` through a CUDA graph of the whole launch sequence, captured
        on the first call per batch shape and replayed after, so the host
        issues one launch per step instead of a few hundred.  ``tb`` is a host
        ``synth.TrainingBatch`` (uploaded into fixed device buffers of its
        shape) or a ``DeviceBatch`` filled in place (e.g. by ``GpuSimulator``;
        one graph per such object).  Graphs of up to ``MAX_SHAPES`` batch
        shapes stay resident, so batches with different numbers of active
        users alternate without recapture."""
        if isinstance(tb, DeviceBatch):
            key = ("device", id(tb))
            ent = self._graphs.get(key)
            if ent is None or ent[1] is not tb:
                self.step(tb)  # eager step: the buffers exist before capture
                self._capture(key, tb)
                return self._read_loss()
        else:
            key = ("host", tb.y.shape, tb.m_u.shape, tb.bits.shape, tuple(tb.dmrs_symbols))
            ent = self._graphs.get(key)
            if ent is None:
                static = DeviceBatch(tb)
                self.step(static)
                self._capture(key, static)
                return self._read_loss()
            ent[1].load(tb)
        self._buffers(ent[1].n, ent[1].U, ent[1].S)  # mark the shape as recently used
        self._advance()
        ent[0].replay()
        return self._read_loss()

    def _capture(self, key, static: "DeviceBatch"):
        torch = self.torch
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            with torch.cuda.graph(g, stream=side):
                self._enqueue(static, side.cuda_stream, adam=True)
        torch.cuda.current_stream().wait_stream(side)
        self._graphs[key] = (g, static, (static.n, static.U, static.S))

    @staticmethod
    def _ok(st, what):
        if st != nrx.NRX_OK:
            raise nrx.NrxError(st, what)


def _autograd_function():
    import torch

    class NrxTrainingLoss(torch.autograd.Function):
        """torch.autograd interface to the training kernels.  forward(w,
        trainer, batch) returns the multi-loss of Sec. II-B for the trainer's
        flat FP32 weight vector ``w`` (a tensor sharing ``trainer.w``'s
        storage, e.g. a ``torch.nn.Parameter`` made from it); backward returns
        the gradient of the hand-written reverse pass, which runs in the same
        launch sequence as the forward (one fused, graph-capturable sequence),
        so a torch optimiser can drive the kernels."""

        @staticmethod
        def forward(ctx, w, trainer, batch):
            if w.data_ptr() != trainer.w.data_ptr():
                raise ValueError("w must share storage with trainer.w")
            out = trainer.loss_and_grad(batch)
            ctx.trainer = trainer
            return torch.tensor(out["loss"], dtype=torch.float32, device=w.device)

        @staticmethod
        def backward(ctx, grad):
            return ctx.trainer.g * grad, None, None

    return NrxTrainingLoss


def nrx_training_loss(w, trainer: "Trainer", batch: "DeviceBatch"):
    """``NrxTrainingLoss.apply(w, trainer, batch)``: the differentiable
    training loss (see ``_autograd_function``)."""
    global _NRX_FN
    if _NRX_FN is None:
        _NRX_FN = _autograd_function()
    return _NRX_FN.apply(w, trainer, batch)


_NRX_FN = None


class DeviceBatch:
    """A ``synth.TrainingBatch`` resident on the GPU, with its slot configs."""

    def __init__(self, tb: synth.TrainingBatch):
        import torch
        dev = torch.device("cuda")
        self.n, self.B = tb.y.shape[0], tb.y.shape[1]
        self.S = tb.y.shape[3]
        self.U = tb.m_u.shape[1]
        assert self.n <= 64, "at most 64 slots per batch"
        self.y = torch.from_numpy(np.ascontiguousarray(tb.y)).to(dev)
        self.dmrs = torch.from_numpy(np.ascontiguousarray(tb.dmrs)).to(dev)
        self.bits = torch.from_numpy(np.ascontiguousarray(tb.bits)).to(dev)
        self.m_u = torch.from_numpy(np.ascontiguousarray(tb.m_u)).to(dev)
        self.h = torch.from_numpy(np.ascontiguousarray(tb.h)).to(dev)
        self.dmrs_symbols = tb.dmrs_symbols
        self.n_data = (14 - len(tb.dmrs_symbols)) * self.S
        self.cfgs = nrx.make_cfgs(self.n, self.S // 12, self.U, tb.dmrs_symbols,
                                  [self.dmrs[i].data_ptr() for i in range(self.n)], tb.noise_var)
        self._pinned = None

    @classmethod
    def empty(cls, n: int, num_users: int, num_rx_ant: int, num_prb: int, m_max: int, dmrs_symbols) -> "DeviceBatch":
        """Device buffers of a batch shape, to be filled on the GPU."""
        S = 12 * num_prb
        nd = len(dmrs_symbols)
        n_data = (14 - nd) * S
        tb = synth.TrainingBatch(y=np.zeros((n, num_rx_ant, 14, S), np.complex64),
                                 dmrs=np.ones((n, nd, S // 2), np.complex64),
                                 bits=np.zeros((n, num_users, n_data, m_max), np.uint8),
                                 m_u=np.full((n, num_users), 2, np.int32),
                                 h=np.zeros((n, num_users, 14, S, 2 * num_rx_ant), np.float32),
                                 dmrs_symbols=tuple(dmrs_symbols), noise_var=np.ones(n))
        return cls(tb)

    def load(self, tb: synth.TrainingBatch, stream=None):
        """Upload a batch of the same shape into these buffers (through pinned
        staging, asynchronous on the stream; the staging is reused, so the
        caller synchronises before the next load, as ``graph_step`` does by
        reading the loss)."""
        import torch
        pairs = [(self.y, tb.y), (self.dmrs, tb.dmrs), (self.bits, tb.bits), (self.m_u, tb.m_u), (self.h, tb.h)]
        if self._pinned is None:
            self._pinned = [torch.empty(d.shape, dtype=d.dtype).pin_memory() for d, _ in pairs]
        lib = load()
        st = nrx._stream_ptr(stream)
        for (dev, src), pin in zip(pairs, self._pinned):
            assert tuple(src.shape) == tuple(dev.shape), "batch shape differs from the captured one"
            pin.numpy()[...] = src
            r = lib.nrx_train_copy(dev.numel() * dev.element_size(), dev.data_ptr(), pin.data_ptr(), st)
            if r != nrx.NRX_OK:
                raise nrx.NrxError(r, "nrx_train_copy")
        self.dmrs_symbols = tb.dmrs_symbols


class GpuSimulator:
    """Training batches drawn on the GPU (``nrx_train_simulate``) into one
    ``DeviceBatch``: per-slot parameters (random MCS association, SNR with
    offsets, delay spread, Doppler) from ``synth.sim_slot_params`` on the host,
    every per-RE draw from Philox on the device."""

    def __init__(self, workload: synth.Workload, seed: int = 7, param_seed: int = 11, active_users: bool = False):
        import torch
        w = workload
        self.w = w
        self.seed = seed
        self.batch_index = 0
        self.active_users = active_users  # draw U_A per batch (synth.draw_active_users)
        self.rng = np.random.Generator(np.random.PCG64(param_seed))
        self.batches: Dict[int, DeviceBatch] = {}  # one device batch per number of active users
        self.batch = self._batch(w.num_users)
        nbytes = load().nrx_train_sim_scratch_bytes(w.batch, w.num_users, w.num_rx_ant, synth.SIM_MAX_TAPS)
        self.scratch = torch.empty(max(int(nbytes), 16), dtype=torch.uint8, device="cuda")
        self._ds = np.ascontiguousarray(np.asarray(w.dmrs_symbols, dtype=np.int32))

    def _batch(self, U: int) -> DeviceBatch:
        w = self.w
        if U not in self.batches:
            self.batches[U] = DeviceBatch.empty(w.batch, U, w.num_rx_ant, w.num_prb, w.net.m_max, w.dmrs_symbols)
        return self.batches[U]

    def draw(self, stream=None) -> DeviceBatch:
        """Simulate the next batch (asynchronous) into the device batch of its
        number of active users, which is returned (and kept as ``self.batch``)."""
        w = self.w
        U = synth.draw_active_users(w.num_users, self.rng) if self.active_users else w.num_users
        params = [synth.sim_slot_params(w, self.rng, U) for _ in range(w.batch)]
        arr = (nrx_sim_slot * w.batch)()
        for i, sp in enumerate(params):
            arr[i].noise_var = sp.noise_var
            arr[i].delay_spread_s = sp.delay_spread_s
            arr[i].doppler_hz = sp.doppler_hz
            arr[i].num_taps = sp.num_taps
            arr[i].ula = int(sp.ula)
            for u, m in enumerate(sp.bits_per_symbol):
                arr[i].bits_per_symbol[u] = m
        b = self.batch = self._batch(U)
        st = load().nrx_train_simulate(w.batch, arr, U, w.num_rx_ant, w.num_prb, len(w.dmrs_symbols),
                                       self._ds.ctypes.data, w.net.m_max, self.seed, self.batch_index,
                                       self.scratch.data_ptr(), b.y.data_ptr(), b.dmrs.data_ptr(), b.bits.data_ptr(),
                                       b.m_u.data_ptr(), b.h.data_ptr(), nrx._stream_ptr(stream))
        if st != nrx.NRX_OK:
            raise nrx.NrxError(st, "nrx_train_simulate")
        self.batch_index += 1
        self.last_params = params
        return b


# ----------------------------------------------------------------------------
# Training loop
# ----------------------------------------------------------------------------


def _make_batch(args):
    """Worker: one seeded training batch (runs in a spawned process); with
    ``active`` its number of active users is drawn (synth.draw_active_users)."""
    wl, seed, active = args
    rng = np.random.Generator(np.random.PCG64(seed))
    U = synth.draw_active_users(wl.num_users, rng) if active else wl.num_users
    return synth.training_batch([synth.training_slot(wl, rng, U) for _ in range(wl.batch)], wl.net.m_max)


def fit(workload: synth.Workload, seconds: float, lr: float = 2e-3, lr_final: float = 5e-5, gamma: float = 1.0,
        seed: int = 1, resume: Optional[str] = None, workers: Optional[int] = None, log_every: int = 2000,
        trainer: Optional[Trainer] = None, precision: str = "fp32", simulator: str = "cpu",
        recompute: Optional[bool] = None, active_users: bool = True, init_blob: Optional[bytes] = None) -> Trainer:
    """Train for a wall-clock budget on fresh random batches of ``workload``
    (random MCS association and SNR offsets, Sec. IV-A; with ``active_users``
    the number of active users drawn per batch, Sec. II-B), with an exponential
    learning-rate decay from lr to lr_final over the budget.  Batches are
    generated by a pool of spawned CPU workers, at most 48 ahead of the GPU;
    each step is one CUDA-graph replay.  The read-out layers start at zero
    (LLRs and channel estimates 0, i.e. BCE ln 2) unless resuming; with
    ``init_blob`` the network starts from that inference blob instead (a
    narrower single-head read-out widened with zero rows)."""
    import multiprocessing as mp
    import os
    import time
    net = workload.net
    if trainer is None:
        W = synth.make_weights(net, seed=seed)
        Wc = synth.make_chest_weights(net, seed=seed + 1)
        for k in ("ro2.w", "ro2.b"):
            W[k][...] = 0.0
        Wc["chest.2.w"][...] = 0.0
        if init_blob is not None:
            net0, W0 = synth.unpack_weights(init_blob)
            if (net0.num_rx_ant, net0.channels, net0.res_blocks, net0.iterations, net0.var_io) != \
                    (net.num_rx_ant, net.channels, net.res_blocks, net.iterations, net.var_io):
                raise ValueError("the initial blob's network does not match the workload's")
            W = synth.widen_readout(net0, W0, net.m_max) if net0.m_max != net.m_max else W0
        trainer = Trainer(net, W, Wc, lr=lr, gamma=gamma, precision=precision, recompute=recompute)
    if resume:
        trainer.restore(resume)
    if simulator == "gpu":  # every batch drawn on the device, no host workers
        sim = GpuSimulator(workload, seed=seed * 1_000_003 + trainer.t, active_users=active_users)
        t0 = time.time()
        hist = []
        while time.time() - t0 < seconds:
            trainer.lr = lr * (lr_final / lr) ** min(1.0, (time.time() - t0) / seconds)
            hist.append(trainer.graph_step(sim.draw())["loss"])
            if log_every and len(hist) % log_every == 0:
                print(f"step {trainer.t} {time.time() - t0:.0f}s lr {trainer.lr:.2e} "
                      f"loss {np.mean(hist[-log_every:]):.4f}", flush=True)
        return trainer
    nw = workers or max(2, min(14, (os.cpu_count() or 4) - 2))
    pool = mp.get_context("spawn").Pool(nw)
    try:
        seed0 = 1_000_003 * (seed + 1) + trainer.t
        window = [pool.apply_async(_make_batch, ((workload, seed0 + i, active_users),)) for i in range(48)]
        nxt = seed0 + 48
        t0 = time.time()
        hist = []
        while time.time() - t0 < seconds:
            tb = window.pop(0).get(timeout=300)
            window.append(pool.apply_async(_make_batch, ((workload, nxt, active_users),)))
            nxt += 1
            frac = min(1.0, (time.time() - t0) / seconds)
            trainer.lr = lr * (lr_final / lr) ** frac
            hist.append(trainer.graph_step(tb)["loss"])
            if log_every and len(hist) % log_every == 0:
                print(f"step {trainer.t} {time.time() - t0:.0f}s lr {trainer.lr:.2e} "
                      f"loss {np.mean(hist[-log_every:]):.4f}", flush=True)
    finally:
        pool.terminate()
        pool.join()
    return trainer


def main(argv=None):
    import argparse
    ap = argparse.ArgumentParser(description="Train the NRX on synthetic slots (Sec. II-B)")
    ap.add_argument("--workload", default="mu2_4rx_24prb", choices=sorted(synth.WORKLOADS))
    ap.add_argument("--prb", type=int, default=8, help="PRBs of the training slots (the net is size-agnostic)")
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--mcs", default="2,4", help="modulation orders drawn per user")
    ap.add_argument("--snr", default=None, help="lo,hi: SNR range in dB before the offsets (default: workload's)")
    ap.add_argument("--seconds", type=float, default=600.0)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--lr-final", type=float, default=5e-5)
    ap.add_argument("--gamma", type=float, default=1.0)
    ap.add_argument("--resume", default=None)
    ap.add_argument("--init-blob", default=None,
                    help="start from this inference blob (its read-out widened to the workload's m_max)")
    ap.add_argument("--precision", default="fp32", choices=("fp32", "bf16"), help="GEMM compute of the passes")
    ap.add_argument("--simulator", default="cpu", choices=("cpu", "gpu"),
                    help="draw batches with CPU workers (synth) or on the GPU (nrx_train_simulate)")
    ap.add_argument("--recompute", default="auto", choices=("auto", "on", "off"),
                    help="rebuild the conv activations in the reverse pass (auto: when memory asks)")
    ap.add_argument("--all-users", action="store_true",
                    help="every batch with all users active (default: U_A drawn per batch, Sec. II-B)")
    ap.add_argument("--checkpoint", default=None, help="write an .npz checkpoint here")
    ap.add_argument("--out", required=True, help="write the inference weight blob here")
    a = ap.parse_args(argv)
    base = synth.WORKLOADS[a.workload]
    snr = tuple(float(v) for v in a.snr.split(",")) if a.snr else base.snr_db_range
    wl = dataclasses_replace(base, num_prb=a.prb, batch=a.batch, snr_db_range=snr,
                             mcs_choices=tuple(int(v) for v in a.mcs.split(",")))
    tr = fit(wl, a.seconds, lr=a.lr, lr_final=a.lr_final, gamma=a.gamma, resume=a.resume, precision=a.precision,
             simulator=a.simulator, recompute={"auto": None, "on": True, "off": False}[a.recompute],
             active_users=not a.all_users,
             init_blob=open(a.init_blob, "rb").read() if a.init_blob else None)
    if a.checkpoint:
        tr.save(a.checkpoint)
    with open(a.out, "wb") as f:
        f.write(tr.blob())
    print(f"trained {tr.t} steps -> {a.out}")


def dataclasses_replace(obj, **kw):
    import dataclasses
    return dataclasses.replace(obj, **kw)


if __name__ == "__main__":
    main()
