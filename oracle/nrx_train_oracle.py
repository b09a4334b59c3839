"""FP64 CPU oracle of the NRX training objective, its gradient and Adam.

TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
the benchmark's CPU-baseline leg may import this module; the library never
does.  It shares no code with the CUDA path: the forward pass reuses the
pinned FP64 forward oracle (``nrx_oracle``), and the gradient is torch
autograd (a library primitive) over a float64 torch expression of the same
layers, pinned by the tests against central finite differences of the numpy
loss and against the numpy forward.

What is computed, with the passage each part follows:

* Training loss (Sec. II-B): binary cross-entropy between the LLRs of
  ReadoutLLRs and the transmitted bits.  With the LLR sign of Eq. 2,
  P(b=1 | y) = sigmoid(l), so the per-bit loss is
  -[b ln sigmoid(l) + (1-b) ln sigmoid(-l)] = softplus(l) - b l.
  Masking (Sec. III): only each user's first m_u outputs on data REs count.
* Double read-out (Sec. II-B): a second head (ReadoutChEst) maps the state to
  the user's channel; its MSE against the true channel, weighted by gamma, is
  added to the loss.
* Multi-loss (Sec. II-B): both read-outs are applied after every CGNN
  iteration and the per-iteration losses are summed.
* Var-IO (Sec. III): in a network with modulation-specific input and output
  layers, each user runs the StateInit and ReadoutLLRs of its own order.
* Normalisation (this build's reading): each BCE term is the mean over the
  counted bits of the whole batch, each MSE term the mean over (slot, user,
  antenna, RE) of |h_hat - h|^2 (the sum of the real and imaginary squared
  errors).
* Adam (Kingma and Ba, Algorithm 1, with the step size folded into
  lr_t = lr sqrt(1 - b2^t) / (1 - b1^t) and eps added to sqrt(v)).
"""
from __future__ import annotations

from typing import Dict, List, Sequence, Tuple

import numpy as np

from . import nrx_oracle as O


# ----------------------------------------------------------------------------
# Loss terms
# ----------------------------------------------------------------------------


def softplus(x: np.ndarray) -> np.ndarray:
    """ln(1 + e^x), evaluated without overflow."""
    return np.maximum(x, 0.0) + np.log1p(np.exp(-np.abs(x)))


def bce_terms(llr_grid: np.ndarray, bits: np.ndarray, m: int, dmrs_symbols: Sequence[int]) -> Tuple[float, int]:
    """Summed BCE of one user's LLR grid [14, S, >= m] against its bits
    [n_data, m] (data REs symbol-major then subcarrier), and the bit count."""
    ds = O.data_symbols(dmrs_symbols)
    l = np.asarray(llr_grid, dtype=np.float64)[ds, :, :m].reshape(-1, m)
    b = np.asarray(bits, dtype=np.float64)[:, :m]
    return float(np.sum(softplus(l) - b * l)), b.size


def readout_chest(S_u: np.ndarray, Wc: Dict[str, np.ndarray]) -> np.ndarray:
    """ReadoutChEst (Sec. II-B): h_hat = W_c2 ReLU(W_c1 S + b_c1) + b_c2,
    [.., 2B] = [Re h_0, Im h_0, ...]."""
    return O.dense(O.relu(O.dense(S_u, Wc["chest.1.w"], Wc["chest.1.b"])), Wc["chest.2.w"], Wc["chest.2.b"])


def channel_target(h_u: np.ndarray) -> np.ndarray:
    """True channel of one user h[b, t, s] (complex) as reals [14, S, 2B]."""
    h_u = np.asarray(h_u, dtype=np.complex128)
    B = h_u.shape[0]
    out = np.zeros(h_u.shape[1:] + (2 * B,))
    for b in range(B):
        out[..., 2 * b] = h_u[b].real
        out[..., 2 * b + 1] = h_u[b].imag
    return out


def training_loss(slots, W: Dict[str, np.ndarray], Wc: Dict[str, np.ndarray], iterations: int, res_blocks: int,
                  gamma: float) -> Tuple[float, List[float], List[float]]:
    """Total multi-loss of a batch of slots (see module docstring) and its
    per-iteration BCE and MSE means.  Each slot provides y, dmrs, bits, h and
    cfg (num_users, dmrs_symbols, bits_per_symbol), as ``synth.Slot``."""
    n_it = iterations
    bce_sum = np.zeros(n_it)
    mse_sum = np.zeros(n_it)
    n_bits = 0
    n_mse = 0
    for sl in slots:
        U = sl.cfg.num_users
        ds = sl.cfg.dmrs_symbols
        states = O.nrx_states(sl.y, sl.dmrs, U, ds, W, n_it, res_blocks, sl.cfg.bits_per_symbol)
        for u in range(U):
            m = sl.cfg.bits_per_symbol[u]
            target = channel_target(sl.h[u])
            for k in range(n_it):
                S_u = states[k + 1][u]
                v, cnt = bce_terms(O.readout(S_u, O.head_weights(W, m)), sl.bits[u], m, ds)
                bce_sum[k] += v
                mse_sum[k] += float(np.sum((readout_chest(S_u, Wc) - target) ** 2))
            n_bits += cnt
            n_mse += target.size // 2
    bce = list(bce_sum / n_bits)
    mse = list(mse_sum / n_mse)
    return float(sum(bce) + gamma * sum(mse)), bce, mse


# ----------------------------------------------------------------------------
# Gradient: torch autograd over the same layers in float64
# ----------------------------------------------------------------------------


_HEAD_NAMES = {"init.pw.w": "init.m{m}.pw.w", "init.pw.b": "init.m{m}.pw.b", "init.dw": "init.m{m}.dw",
               "ro1.w": "ro.m{m}.1.w", "ro1.b": "ro.m{m}.1.b", "ro2.w": "ro.m{m}.2.w", "ro2.b": "ro.m{m}.2.b"}


def _torch_loss(slots, Wt, Wct, iterations: int, res_blocks: int, gamma: float):
    import torch
    F = torch.nn.functional

    def hw(name, m):  # Var-IO (Sec. III): the modulation-specific input / output layers of order m
        return Wt[_HEAD_NAMES[name].format(m=m)] if "init.pw.w" not in Wt else Wt[name]

    def dw(x, k):  # x [U, 14, S, C]; cross-correlation with zero padding
        C = x.shape[-1]
        return F.conv2d(x.permute(0, 3, 1, 2), k[:, None], padding=1, groups=C).permute(0, 2, 3, 1)

    total_bce = [0.0] * iterations
    total_mse = [0.0] * iterations
    n_bits = 0
    n_mse = 0
    for sl in slots:
        U = sl.cfg.num_users
        ds = list(sl.cfg.dmrs_symbols)
        S = sl.y.shape[2]
        H = O.channel_estimate(sl.y, sl.dmrs, U, ds)
        pes = [O.positional_encoding(u, S, ds) for u in range(U)]
        x = torch.stack([torch.from_numpy(O.input_features(sl.y, H[u], pes[u])) for u in range(U)])
        pe = torch.stack([torch.from_numpy(p) for p in pes])
        bits_u = sl.cfg.bits_per_symbol
        st = torch.cat([F.relu(dw(F.linear(x[u:u + 1], hw("init.pw.w", bits_u[u]), hw("init.pw.b", bits_u[u])),
                                  hw("init.dw", bits_u[u]))) for u in range(U)])
        data = [t for t in range(14) if t not in ds]
        for k in range(iterations):
            p = f"it{k}."
            msg = F.linear(F.relu(F.linear(st, Wt[p + "mp1.w"], Wt[p + "mp1.b"])), Wt[p + "mp2.w"], Wt[p + "mp2.b"])
            a = msg.sum(0, keepdim=True) - msg
            z = F.linear(torch.cat([st, a, pe], -1), Wt[p + "in.w"], Wt[p + "in.b"])
            for r in range(res_blocks):
                q = f"{p}blk{r}."
                hh = F.relu(F.linear(dw(z, Wt[q + "dw1"]), Wt[q + "pw1.w"], Wt[q + "pw1.b"]))
                z = z + F.linear(F.relu(dw(hh, Wt[q + "dw2"])), Wt[q + "pw2.w"], Wt[q + "pw2.b"])
            st = st + z
            ls = [F.linear(F.relu(F.linear(st[u], hw("ro1.w", bits_u[u]), hw("ro1.b", bits_u[u]))),
                           hw("ro2.w", bits_u[u]), hw("ro2.b", bits_u[u])) for u in range(U)]
            hh = F.linear(F.relu(F.linear(st, Wct["chest.1.w"], Wct["chest.1.b"])), Wct["chest.2.w"],
                          Wct["chest.2.b"])
            for u in range(U):
                m = sl.cfg.bits_per_symbol[u]
                lu = ls[u][data][:, :, :m].reshape(-1, m)
                bu = torch.from_numpy(np.asarray(sl.bits[u], dtype=np.float64)[:, :m])
                total_bce[k] = total_bce[k] + (F.softplus(lu) - bu * lu).sum()
                tgt = torch.from_numpy(channel_target(sl.h[u]))
                total_mse[k] = total_mse[k] + ((hh[u] - tgt) ** 2).sum()
        for u in range(U):
            n_bits += len(data) * S * sl.cfg.bits_per_symbol[u]
            n_mse += 14 * S * sl.h.shape[1]
    loss = sum(b / n_bits for b in total_bce) + gamma * sum(m / n_mse for m in total_mse)
    return loss


def training_grads(slots, W: Dict[str, np.ndarray], Wc: Dict[str, np.ndarray], iterations: int, res_blocks: int,
                   gamma: float) -> Tuple[float, Dict[str, np.ndarray]]:
    """Loss and its gradient with respect to every weight of W and Wc
    (float64), by torch autograd over the layer stack."""
    import torch
    Wt = {k: torch.tensor(np.asarray(v, dtype=np.float64), requires_grad=True) for k, v in W.items()}
    Wct = {k: torch.tensor(np.asarray(v, dtype=np.float64), requires_grad=True) for k, v in Wc.items()}
    loss = _torch_loss(slots, Wt, Wct, iterations, res_blocks, gamma)
    names = list(Wt) + list(Wct)
    tensors = [Wt[k] for k in Wt] + [Wct[k] for k in Wct]
    grads = torch.autograd.grad(loss, tensors, allow_unused=True)
    out = {}
    for n, t, g in zip(names, tensors, grads):
        out[n] = np.zeros(t.shape) if g is None else g.detach().numpy()
    return float(loss.detach()), out


# ----------------------------------------------------------------------------
# Adam
# ----------------------------------------------------------------------------


def adam_step(w: np.ndarray, g: np.ndarray, m1: np.ndarray, m2: np.ndarray, t: int, lr: float,
              beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """One Adam update at step t >= 1; returns (w, m1, m2), float64."""
    m1 = beta1 * m1 + (1.0 - beta1) * g
    m2 = beta2 * m2 + (1.0 - beta2) * g * g
    lr_t = lr * np.sqrt(1.0 - beta2 ** t) / (1.0 - beta1 ** t)
    return w - lr_t * m1 / (np.sqrt(m2) + eps), m1, m2
