"""FP64 CPU oracle of the NRX forward pass and of the LS + LMMSE + max-log receiver.

TEST INFRASTRUCTURE ONLY.  This module is the slow, plain definition that the
CUDA path is checked against.  Only the test suite, the package smoke check and
the benchmark's CPU-baseline leg may import it; the library itself never does.
It shares no code with the CUDA path (no kernels, headers, helpers, tables or
constants); the two meet only at the seeded inputs of the synthetic-slot
generator, which carries none of the receiver's arithmetic.

Everything is float64 / complex128, vectorised with numpy where the vectorised
form is the definition itself (a matmul is a dense layer; a 3x3 correlation is
nine shifted multiply-adds).  No blocking, fusion or reordering.

What is computed, with the passage each part follows:

* System model, Eq. 1 (Sec. II): y = sum_u H_u x_u + n.  The oracle reads y.
* DMRS least-squares estimate (Sec. II-A, the LS estimator that feeds the
  CGNN): h = y p* / |p|^2 per pilot RE, and with two ports sharing a CDM group
  the frequency-domain OCC is undone by averaging each pilot pair.
* Linear interpolation of the LS estimates to every RE, frequency first then
  time, holding the edge values (the "LS lin" baseline of Fig. 3 / Fig. 6).
* Positional encoding of the distance to the nearest pilot (Sec. II-A).
* StateInit, N_it CGNN iterations (message passing over the *other* users +
  CNN update) and ReadoutLLRs (Sec. II-A), in the depthwise-separable layout
  of this build (see the layer list in ``nrx_forward``).
* Var-MCS masking: user u keeps the first m_u of the m_max LLR outputs
  (Sec. III, masking of higher-order LLRs); or, for a Var-IO network (Sec.
  III), user u runs the StateInit and ReadoutLLRs of its own modulation order.
* LLR sign: ln P(b=1|y)/P(b=0|y), Eq. 2.
* LMMSE equalisation with unbiased scaling and max-log demapping over the
  user's matched Gray QAM constellation (the "LS + LMMSE" baseline, Fig. 3).

Readings where the paper is silent (listed in the design notes too): zero
"same" padding at every depthwise input; ReLU activations; bias-free
depthwise taps; no N0 input to the NRX; DMRS type-1 comb with users 0,1 in CDM
group 0 (even subcarriers) and users 2,3 in CDM group 1 (odd subcarriers), OCC
[+1,+1] / [+1,-1]; PE = ((t - t_dmrs)/7, (s - s_pilot)/2) with ties to the
lower index.
"""
from __future__ import annotations

from typing import Dict, List, Sequence, Tuple

import numpy as np

T_SYMBOLS = 14

# ----------------------------------------------------------------------------
# DMRS least squares, interpolation, positional encoding
# ----------------------------------------------------------------------------


def cdm_group(u: int) -> int:
    """CDM group of user u's DMRS port (ports 0,1 -> group 0; 2,3 -> group 1)."""
    return u // 2


def occ_sign(u: int, m: np.ndarray) -> np.ndarray:
    """Frequency OCC weight of user u's port on comb position m."""
    return np.ones(m.shape) if u % 2 == 0 else np.where(m % 2 == 0, 1.0, -1.0)


def group_shared(u: int, num_users: int) -> bool:
    """True when the other port of user u's CDM group is also active."""
    partner = u ^ 1
    return partner < num_users


def ls_estimates(y: np.ndarray, dmrs: np.ndarray, u: int, num_users: int,
                 dmrs_symbols: Sequence[int]) -> Tuple[np.ndarray, np.ndarray]:
    """LS channel estimates of user u on its DMRS (Sec. II-A).

    y: complex [B, 14, S]; dmrs: complex [n_dmrs, S/2] base sequence r(m).
    Returns (positions [n_est] as float subcarrier indices, h [B, n_dmrs, n_est]).

    Per pilot: h(m) = y(2m+g) * conj(p(m)) / |p(m)|^2 with p(m) = w_u(m) r(m).
    If the partner port of the group is active, the OCC is undone by averaging
    pilot pairs (2n, 2n+1); the estimate sits midway, at subcarrier 4n+1+g.
    """
    y = np.asarray(y, dtype=np.complex128)
    g = cdm_group(u)
    S = y.shape[2]
    M = S // 2
    m = np.arange(M)
    est = []
    for d, t in enumerate(dmrs_symbols):
        p = np.asarray(dmrs[d], dtype=np.complex128) * occ_sign(u, m)
        z = y[:, t, 2 * m + g] * np.conj(p)[None, :] / (np.abs(p) ** 2)[None, :]
        if group_shared(u, num_users):
            z = 0.5 * (z[:, 0::2] + z[:, 1::2])
        est.append(z)
    h = np.stack(est, axis=1)  # [B, n_dmrs, n_est]
    if group_shared(u, num_users):
        pos = 4.0 * np.arange(M // 2) + 1.0 + g
    else:
        pos = 2.0 * m + g
    return pos, h


def interpolate(pos: np.ndarray, h: np.ndarray, S: int, dmrs_symbols: Sequence[int]) -> np.ndarray:
    """Linear interpolation of LS estimates to the full grid, holding the
    nearest estimate outside the first/last pilot.  Frequency first (on each
    DMRS symbol), then time between the DMRS symbols.

    h: [B, n_dmrs, n_est] -> returns [B, 14, S]."""
    B, n_dmrs, _ = h.shape
    s = np.arange(S, dtype=np.float64)
    hf = np.zeros((B, n_dmrs, S), dtype=np.complex128)
    for b in range(B):
        for d in range(n_dmrs):
            hf[b, d] = np.interp(s, pos, h[b, d].real) + 1j * np.interp(s, pos, h[b, d].imag)
    out = np.zeros((B, T_SYMBOLS, S), dtype=np.complex128)
    if n_dmrs == 1:
        out[:] = hf[:, 0:1, :]
        return out
    t0, t1 = dmrs_symbols[0], dmrs_symbols[1]
    for t in range(T_SYMBOLS):
        if t <= t0:
            out[:, t] = hf[:, 0]
        elif t >= t1:
            out[:, t] = hf[:, 1]
        else:
            a = (t - t0) / (t1 - t0)
            out[:, t] = hf[:, 0] + a * (hf[:, 1] - hf[:, 0])
    return out


def channel_estimate(y: np.ndarray, dmrs: np.ndarray, num_users: int,
                     dmrs_symbols: Sequence[int]) -> np.ndarray:
    """Interpolated LS estimate of every user on every RE: [U, B, 14, S]."""
    S = y.shape[2]
    out = []
    for u in range(num_users):
        pos, h = ls_estimates(y, dmrs, u, num_users, dmrs_symbols)
        out.append(interpolate(pos, h, S, dmrs_symbols))
    return np.stack(out)


def positional_encoding(u: int, S: int, dmrs_symbols: Sequence[int]) -> np.ndarray:
    """Distances to the nearest pilot (Sec. II-A): [14, S, 2] with channel 0 =
    (t - nearest DMRS symbol)/7 and channel 1 = (s - nearest pilot subcarrier
    of the user's CDM group)/2; ties go to the lower index."""
    tds = np.asarray(sorted(dmrs_symbols), dtype=np.float64)
    t = np.arange(T_SYMBOLS, dtype=np.float64)
    nearest_t = tds[np.argmin(np.abs(t[:, None] - tds[None, :]), axis=1)]
    pilots = np.arange(cdm_group(u), S, 2, dtype=np.float64)
    s = np.arange(S, dtype=np.float64)
    nearest_s = pilots[np.argmin(np.abs(s[:, None] - pilots[None, :]), axis=1)]
    pe = np.zeros((T_SYMBOLS, S, 2))
    pe[:, :, 0] = ((t - nearest_t) / 7.0)[:, None]
    pe[:, :, 1] = ((s - nearest_s) / 2.0)[None, :]
    return pe


def input_features(y: np.ndarray, h_u: np.ndarray, pe_u: np.ndarray) -> np.ndarray:
    """CGNN input of one user (Sec. II-A): per RE the received vector, the
    user's interpolated LS estimate and the PE, as reals:
    [Re y0, Im y0, ..., Re y_{B-1}, Im y_{B-1}, Re h0, Im h0, ..., dt, df]."""
    y = np.asarray(y, dtype=np.complex128)
    B = y.shape[0]
    feats = []
    for b in range(B):
        feats += [y[b].real, y[b].imag]
    for b in range(B):
        feats += [h_u[b].real, h_u[b].imag]
    x = np.stack(feats, axis=-1)  # [14, S, 4B]
    return np.concatenate([x, pe_u], axis=-1)


# ----------------------------------------------------------------------------
# Network layers
# ----------------------------------------------------------------------------


def relu(x: np.ndarray) -> np.ndarray:
    return np.maximum(x, 0.0)


def dense(x: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Pointwise (1x1) layer / MLP layer: x [..., in] -> x W^T + b."""
    return x @ np.asarray(w, dtype=np.float64).T + np.asarray(b, dtype=np.float64)


def depthwise3x3(x: np.ndarray, k: np.ndarray) -> np.ndarray:
    """Bias-free depthwise 3x3 cross-correlation over (symbol, subcarrier) with
    zero padding: out[t,s,c] = sum_{i,j} k[c,i,j] x[t+i-1, s+j-1, c]."""
    k = np.asarray(k, dtype=np.float64)
    T, S, C = x.shape
    xp = np.zeros((T + 2, S + 2, C))
    xp[1:-1, 1:-1] = x
    out = np.zeros_like(x)
    for i in range(3):
        for j in range(3):
            out += k[:, i, j] * xp[i:i + T, j:j + S]
    return out


def state_init(x_u: np.ndarray, W: Dict[str, np.ndarray]) -> np.ndarray:
    """StateInit (Sec. II-A): S^(0) = ReLU(DW(PW(x)))."""
    return relu(depthwise3x3(dense(x_u, W["init.pw.w"], W["init.pw.b"]), W["init.dw"]))


def messages(S_u: np.ndarray, W: Dict[str, np.ndarray], k: int) -> np.ndarray:
    """Per-user message MLP of CGNN iteration k: m = W2 ReLU(W1 S + b1) + b2."""
    p = f"it{k}."
    return dense(relu(dense(S_u, W[p + "mp1.w"], W[p + "mp1.b"])), W[p + "mp2.w"], W[p + "mp2.b"])


def aggregate(msgs: np.ndarray, active: Sequence[int]) -> np.ndarray:
    """For each user, the sum of the messages of all *other* active users
    (Sec. II-A).  msgs: [U, ...]; inactive users' entries are never read and
    their aggregate is returned as zero."""
    out = np.zeros_like(msgs)
    for u in active:
        for v in active:
            if v != u:
                out[u] += msgs[v]
    return out


def residual_block(z: np.ndarray, W: Dict[str, np.ndarray], k: int, r: int) -> np.ndarray:
    """z + PW2(ReLU(DW2(ReLU(PW1(DW1(z))))))."""
    q = f"it{k}.blk{r}."
    h = relu(dense(depthwise3x3(z, W[q + "dw1"]), W[q + "pw1.w"], W[q + "pw1.b"]))
    h = relu(depthwise3x3(h, W[q + "dw2"]))
    return z + dense(h, W[q + "pw2.w"], W[q + "pw2.b"])


def cnn_update(S_u: np.ndarray, a_u: np.ndarray, pe_u: np.ndarray, W: Dict[str, np.ndarray],
               k: int, res_blocks: int) -> np.ndarray:
    """CNN part of CGNN iteration k (Sec. II-A): from the previous state, the
    aggregated messages and the PE, z = PW_in([S, a, PE]) refined by the
    residual blocks; returns the new state S + z."""
    p = f"it{k}."
    z = dense(np.concatenate([S_u, a_u, pe_u], axis=-1), W[p + "in.w"], W[p + "in.b"])
    for r in range(res_blocks):
        z = residual_block(z, W, k, r)
    return S_u + z


def head_weights(W: Dict[str, np.ndarray], m: int) -> Dict[str, np.ndarray]:
    """Var-IO (Sec. III): a network with modulation-specific input and output
    layers keeps, for order m, StateInit under "init.m{m}.*" and ReadoutLLRs
    (m outputs) under "ro.m{m}.*"; this returns W with that pair under the
    single-head names.  A single-head network is returned unchanged."""
    if "init.pw.w" in W:
        return W
    out = dict(W)
    out["init.pw.w"] = W[f"init.m{m}.pw.w"]
    out["init.pw.b"] = W[f"init.m{m}.pw.b"]
    out["init.dw"] = W[f"init.m{m}.dw"]
    out["ro1.w"] = W[f"ro.m{m}.1.w"]
    out["ro1.b"] = W[f"ro.m{m}.1.b"]
    out["ro2.w"] = W[f"ro.m{m}.2.w"]
    out["ro2.b"] = W[f"ro.m{m}.2.b"]
    return out


def readout(S_u: np.ndarray, W: Dict[str, np.ndarray]) -> np.ndarray:
    """ReadoutLLRs (Sec. II-A): l = W_o2 ReLU(W_o1 S + b_o1) + b_o2, [.., m_max]."""
    return dense(relu(dense(S_u, W["ro1.w"], W["ro1.b"])), W["ro2.w"], W["ro2.b"])


# ----------------------------------------------------------------------------
# Full NRX forward
# ----------------------------------------------------------------------------


def nrx_states(y: np.ndarray, dmrs: np.ndarray, num_users: int, dmrs_symbols: Sequence[int],
               W: Dict[str, np.ndarray], iterations: int, res_blocks: int,
               bits_per_symbol: Sequence[int] | None = None) -> List[np.ndarray]:
    """States after StateInit and after each CGNN iteration: list of
    [U, 14, S, C] arrays (entry k = S^(k)).  A Var-IO network needs the users'
    modulation orders to pick each user's StateInit."""
    S = y.shape[2]
    H = channel_estimate(y, dmrs, num_users, dmrs_symbols)
    pes = [positional_encoding(u, S, dmrs_symbols) for u in range(num_users)]
    Wu = [W if bits_per_symbol is None else head_weights(W, bits_per_symbol[u]) for u in range(num_users)]
    state = np.stack([state_init(input_features(y, H[u], pes[u]), Wu[u]) for u in range(num_users)])
    out = [state]
    active = list(range(num_users))
    for k in range(iterations):
        msgs = np.stack([messages(state[u], W, k) for u in range(num_users)])
        agg = aggregate(msgs, active)
        state = np.stack([cnn_update(state[u], agg[u], pes[u], W, k, res_blocks)
                          for u in range(num_users)])
        out.append(state)
    return out


def data_symbols(dmrs_symbols: Sequence[int]) -> List[int]:
    return [t for t in range(T_SYMBOLS) if t not in dmrs_symbols]


def pack_llrs(llr_grid: Sequence[np.ndarray], bits_per_symbol: Sequence[int],
              dmrs_symbols: Sequence[int]) -> np.ndarray:
    """Masking (Sec. III) and output packing: user u's first m_u LLRs on the
    data REs, RE order symbol-major then subcarrier, users concatenated.
    llr_grid: per user [14, S, >= m_u]."""
    ds = data_symbols(dmrs_symbols)
    parts = []
    for u, m in enumerate(bits_per_symbol):
        g = np.asarray(llr_grid[u])
        parts.append(g[ds, :, :m].reshape(-1))
    return np.concatenate(parts)


def nrx_forward(y: np.ndarray, dmrs: np.ndarray, num_users: int, dmrs_symbols: Sequence[int],
                bits_per_symbol: Sequence[int], W: Dict[str, np.ndarray], iterations: int,
                res_blocks: int) -> np.ndarray:
    """The NRX over one slot: packed LLRs (float64), see ``pack_llrs``.

    Layers: StateInit; N_it x [messages, aggregate over other users, CNN
    update]; ReadoutLLRs; masking to each user's modulation order."""
    states = nrx_states(y, dmrs, num_users, dmrs_symbols, W, iterations, res_blocks, bits_per_symbol)
    llr = [readout(states[-1][u], head_weights(W, bits_per_symbol[u])) for u in range(num_users)]
    return pack_llrs(llr, bits_per_symbol, dmrs_symbols)


# ----------------------------------------------------------------------------
# LMMSE + max-log receiver
# ----------------------------------------------------------------------------


def pam_levels(k: int) -> Tuple[np.ndarray, np.ndarray]:
    """Gray PAM for one of I/Q with k label bits (c0 = sign bit), recursively:
    level = (1-2 c0) * mag_k(c1..), mag_1 = 1,
    mag_k(c1, c2, ..) = 2^(k-1) - (1-2 c1) mag_{k-1}(c2, ..).
    Returns (labels [2^k, k] uint8, unnormalised levels [2^k])."""
    labels = np.array([[(i >> (k - 1 - j)) & 1 for j in range(k)] for i in range(2 ** k)], dtype=np.uint8)

    def mag(c):
        if len(c) == 0:
            return 1.0
        return 2.0 ** len(c) - (1.0 - 2.0 * c[0]) * mag(c[1:])

    lv = np.array([(1.0 - 2.0 * c[0]) * mag(list(c[1:])) for c in labels])
    return labels, lv


def constellation(m: int) -> Tuple[np.ndarray, np.ndarray]:
    """Unit-energy Gray QAM with 2^m points: bits (b0, b1, b2, ...) where even
    bits label I and odd bits label Q.  Returns (labels [2^m, m], points)."""
    k = m // 2
    lab1, lv = pam_levels(k)
    n = 2 ** k
    labels = np.zeros((n * n, m), dtype=np.uint8)
    pts = np.zeros(n * n, dtype=np.complex128)
    for i in range(n):
        for q in range(n):
            idx = i * n + q
            labels[idx, 0::2] = lab1[i]
            labels[idx, 1::2] = lab1[q]
            pts[idx] = lv[i] + 1j * lv[q]
    pts /= np.sqrt(np.mean(np.abs(pts) ** 2))
    return labels, pts


def maxlog_llr(xt: np.ndarray, var: np.ndarray, m: int) -> np.ndarray:
    """Max-log LLRs (Eq. 2 sign) of equalised symbols xt with effective noise
    variance var: l_i = (min_{c: b_i=0} |x-c|^2 - min_{c: b_i=1} |x-c|^2) / var.
    xt, var: [...]; returns [..., m]."""
    labels, pts = constellation(m)
    d = np.abs(xt[..., None] - pts) ** 2 / np.asarray(var)[..., None]  # [..., 2^m]
    out = np.zeros(xt.shape + (m,))
    for i in range(m):
        d0 = np.min(d[..., labels[:, i] == 0], axis=-1)
        d1 = np.min(d[..., labels[:, i] == 1], axis=-1)
        out[..., i] = d0 - d1
    return out


def cholesky_solve(G: np.ndarray, Bm: np.ndarray) -> np.ndarray:
    """Solve G X = Bm for Hermitian positive definite G [.., U, U] through the
    Cholesky factor G = L L^H, by forward then back substitution."""
    L = np.linalg.cholesky(G)
    U = G.shape[-1]
    v = np.zeros(Bm.shape, dtype=np.complex128)
    for i in range(U):
        acc = Bm[..., i, :].copy()
        for j in range(i):
            acc -= L[..., i, j, None] * v[..., j, :]
        v[..., i, :] = acc / L[..., i, i, None]
    x = np.zeros(Bm.shape, dtype=np.complex128)
    for i in reversed(range(U)):
        acc = v[..., i, :].copy()
        for j in range(i + 1, U):
            acc -= np.conj(L[..., j, i])[..., None] * x[..., j, :]
        x[..., i, :] = acc / np.conj(L[..., i, i])[..., None]
    return x


def lmmse_equalize(y: np.ndarray, H: np.ndarray, noise_var: float) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Per-RE LMMSE with unbiased scaling.

    y: [B, ...REs]; H: [U, B, ...REs] channel estimates.  Per RE:
    G = H^H H + N0 I, xhat = G^-1 H^H y, d_u = [G^-1 H^H H]_uu,
    xt_u = xhat_u / d_u, var_u = 1/d_u - 1.
    Returns (xhat, xt, var), each [U, ...REs]."""
    y = np.asarray(y, dtype=np.complex128)
    H = np.asarray(H, dtype=np.complex128)
    U = H.shape[0]
    Hm = np.moveaxis(H, (0, 1), (-1, -2))        # [..., B, U]
    yv = np.moveaxis(y, 0, -1)[..., None]         # [..., B, 1]
    Hh = np.conj(np.swapaxes(Hm, -1, -2))         # [..., U, B]
    A = Hh @ Hm                                   # H^H H
    G = A + noise_var * np.eye(U)
    xhat = cholesky_solve(G, Hh @ yv)[..., 0]     # [..., U]
    d = np.real(np.diagonal(cholesky_solve(G, A), axis1=-2, axis2=-1))
    xt = xhat / d
    var = 1.0 / d - 1.0
    mv = lambda a: np.moveaxis(a, -1, 0)
    return mv(xhat), mv(xt), mv(var)


def lmmse_receiver(y: np.ndarray, dmrs: np.ndarray, num_users: int, dmrs_symbols: Sequence[int],
                   bits_per_symbol: Sequence[int], noise_var: float) -> np.ndarray:
    """LS + linear interpolation + LMMSE + max-log, packed like ``nrx_forward``."""
    H = channel_estimate(y, dmrs, num_users, dmrs_symbols)
    _, xt, var = lmmse_equalize(y, H, noise_var)  # [U, 14, S]
    llr = [maxlog_llr(xt[u], var[u], m) for u, m in enumerate(bits_per_symbol)]
    return pack_llrs(llr, bits_per_symbol, dmrs_symbols)


def llr_count(num_prb: int, dmrs_symbols: Sequence[int], bits_per_symbol: Sequence[int]) -> int:
    return (T_SYMBOLS - len(dmrs_symbols)) * 12 * num_prb * int(sum(bits_per_symbol))
