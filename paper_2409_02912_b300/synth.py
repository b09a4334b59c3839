"""Seeded synthetic PUSCH slots and seeded NRX weights.

This module is the transmitter and channel side of the link: random bits,
Gray QAM (3GPP TS 38.211 Sec. 5.1 mapping formulas), DMRS insertion with the
type-1 comb and frequency-domain OCC, a tapped-delay-line channel with an
exponential power-delay profile and Doppler, and AWGN, producing the received
resource grid of the system model (Eq. 1).  It also draws the seeded network
weights and serialises them into the flat weight blob that ``nrx_create``
consumes (format documented in ``include/nrx.h``).

It holds none of the receiver's arithmetic (no LS estimation, interpolation,
network layers, equalisation or demapping): both the CUDA path and the CPU
oracle consume what it produces, and nothing here depends on either of them.

Randomness: every draw comes from ``numpy.random.Generator(PCG64(seed))``.
Slot ``i`` of a workload uses seed ``1000 * workload.seed_base + i``; weights
use seed 42.
"""
from __future__ import annotations

import dataclasses
import struct
from typing import Dict, List, Optional, Sequence

import numpy as np

SUBCARRIER_SPACING_HZ = 30e3
NUM_SYMBOLS = 14
SLOT_DURATION_S = 0.5e-3

# ----------------------------------------------------------------------------
# Configuration records
# ----------------------------------------------------------------------------


@dataclasses.dataclass(frozen=True)
class NetConfig:
    """Hyper-parameters of the network: Rx antennas B, state depth C (d_S in
    Sec. II-A), residual conv blocks R per CGNN iteration, iterations N_it,
    and LLR head width m_max (bits of the highest supported modulation)."""

    num_rx_ant: int
    channels: int
    res_blocks: int
    iterations: int
    m_max: int = 6
    var_io: bool = False  # modulation-specific StateInit / ReadoutLLRs heads (Sec. III)

    @property
    def in_features(self) -> int:
        # [Re/Im y per antenna, Re/Im LS estimate per antenna, 2 PE channels]
        return 4 * self.num_rx_ant + 2

    @property
    def heads(self) -> tuple:
        """Modulation orders with their own input / output layers (Var-IO), or
        (m_max,) for the single masked head."""
        return tuple(m for m in (2, 4, 6) if m <= self.m_max) if self.var_io else (self.m_max,)


@dataclasses.dataclass(frozen=True)
class SlotConfig:
    """One slot's transmission: geometry, DMRS positions, modulation orders
    (bits per symbol per user) and channel/SNR draws."""

    num_prb: int
    num_users: int
    num_rx_ant: int
    dmrs_symbols: tuple
    bits_per_symbol: tuple  # one entry per user, each 2, 4 or 6
    snr_db: float
    num_taps: int
    delay_spread_s: float
    doppler_hz: float
    ula: bool
    n_id: int = -1          # DMRS scrambling identity; -1: seeded random QPSK pilots
    slot_number: int = 0    # slot index within the frame (Gold-sequence DMRS only)
    n_scid: int = 0

    @property
    def num_subcarriers(self) -> int:
        return 12 * self.num_prb

    @property
    def num_data_symbols(self) -> int:
        return NUM_SYMBOLS - len(self.dmrs_symbols)

    @property
    def noise_var(self) -> float:
        return float(10.0 ** (-self.snr_db / 10.0))


@dataclasses.dataclass(frozen=True)
class Workload:
    """A named family of slots (shape + the distributions of the random draws)
    and the network it is run with."""

    name: str
    seed_base: int
    batch: int
    num_prb: int
    num_users: int
    num_rx_ant: int
    dmrs_symbols: tuple
    mcs_choices: tuple  # modulation orders drawn per user (uniformly)
    snr_db_range: tuple  # (lo, hi); lo == hi means fixed
    num_taps: int
    delay_spread_range_s: tuple
    doppler_range_hz: tuple
    ula: bool
    net: NetConfig


# The three workloads.  Shapes follow the paper's evaluation setting (Sec. III-B:
# 2 users x 4 Rx antennas, 30 kHz SCS, DMRS type A with one additional position)
# scaled to a tiny single-user case, a 24-PRB two-user case and the full
# 273-PRB four-user slot.
WORKLOADS: Dict[str, Workload] = {
    "su_2rx_4prb": Workload(
        name="su_2rx_4prb", seed_base=1, batch=1, num_prb=4, num_users=1,
        num_rx_ant=2, dmrs_symbols=(2,), mcs_choices=(2,), snr_db_range=(10.0, 10.0),
        num_taps=6, delay_spread_range_s=(100e-9, 100e-9), doppler_range_hz=(0.0, 0.0),
        ula=False, net=NetConfig(num_rx_ant=2, channels=32, res_blocks=2, iterations=1, m_max=2)),
    "mu2_4rx_24prb": Workload(
        name="mu2_4rx_24prb", seed_base=2, batch=16, num_prb=24, num_users=2,
        num_rx_ant=4, dmrs_symbols=(2, 11), mcs_choices=(4,), snr_db_range=(-2.0, 20.0),
        num_taps=12, delay_spread_range_s=(10e-9, 300e-9), doppler_range_hz=(0.0, 400.0),
        ula=True, net=NetConfig(num_rx_ant=4, channels=64, res_blocks=2, iterations=2, m_max=4)),
    "mu4_4rx_273prb": Workload(
        name="mu4_4rx_273prb", seed_base=3, batch=8, num_prb=273, num_users=4,
        num_rx_ant=4, dmrs_symbols=(2, 11), mcs_choices=(2, 4, 6), snr_db_range=(-2.0, 20.0),
        num_taps=12, delay_spread_range_s=(10e-9, 300e-9), doppler_range_hz=(0.0, 400.0),
        ula=True, net=NetConfig(num_rx_ant=4, channels=64, res_blocks=2, iterations=2, m_max=6)),
}


def draw_slot_config(w: Workload, rng: np.random.Generator, num_users: Optional[int] = None) -> SlotConfig:
    """Draw one slot's per-slot parameters from the workload's distributions
    (``num_users`` active users, default all of the workload's)."""
    U = w.num_users if num_users is None else num_users
    bits = tuple(int(rng.choice(w.mcs_choices)) for _ in range(U))
    snr = float(rng.uniform(*w.snr_db_range)) if w.snr_db_range[0] != w.snr_db_range[1] \
        else float(w.snr_db_range[0])
    ds = float(rng.uniform(*w.delay_spread_range_s))
    fd = float(rng.uniform(*w.doppler_range_hz))
    return SlotConfig(num_prb=w.num_prb, num_users=U, num_rx_ant=w.num_rx_ant,
                      dmrs_symbols=tuple(w.dmrs_symbols), bits_per_symbol=bits, snr_db=snr,
                      num_taps=w.num_taps, delay_spread_s=ds, doppler_hz=fd, ula=w.ula)


# ----------------------------------------------------------------------------
# Transmitter
# ----------------------------------------------------------------------------


def qam_modulate(bits: np.ndarray, m: int) -> np.ndarray:
    """Map bit vectors [..., m] to unit-energy Gray QAM symbols with the
    TS 38.211 Sec. 5.1.3-5.1.5 formulas (b0/b1 are the I/Q sign bits)."""
    b = 1.0 - 2.0 * bits.astype(np.float64)
    if m == 2:
        return (b[..., 0] + 1j * b[..., 1]) / np.sqrt(2.0)
    if m == 4:
        re = b[..., 0] * (2.0 - b[..., 2])
        im = b[..., 1] * (2.0 - b[..., 3])
        return (re + 1j * im) / np.sqrt(10.0)
    if m == 6:
        re = b[..., 0] * (4.0 - b[..., 2] * (2.0 - b[..., 4]))
        im = b[..., 1] * (4.0 - b[..., 3] * (2.0 - b[..., 5]))
        return (re + 1j * im) / np.sqrt(42.0)
    raise ValueError(f"unsupported bits per symbol {m}")


def dmrs_port_values(base: np.ndarray, port: int) -> np.ndarray:
    """Values a DMRS port transmits on its comb: port p in {0,1,2,3} uses CDM
    group p//2 and frequency OCC [+1,+1] (even p) or [+1,-1] (odd p) over each
    pair of consecutive comb positions.  ``base`` is the base sequence r(m) of
    one DMRS symbol, m = 0..S/2-1, placed on subcarrier 2m + p//2."""
    m = np.arange(base.shape[-1])
    occ = np.ones_like(m, dtype=np.float64) if port % 2 == 0 else (-1.0) ** m
    return base * occ


def transmit_grid(cfg: SlotConfig, dmrs: np.ndarray, bits: List[np.ndarray]) -> np.ndarray:
    """Resource grids x_u[t, s] of all users (complex128 [U, 14, S]).  DMRS
    symbols carry only pilots (both CDM groups reserved, no data)."""
    S = cfg.num_subcarriers
    x = np.zeros((cfg.num_users, NUM_SYMBOLS, S), dtype=np.complex128)
    data_syms = [t for t in range(NUM_SYMBOLS) if t not in cfg.dmrs_symbols]
    for u in range(cfg.num_users):
        sym = qam_modulate(bits[u], cfg.bits_per_symbol[u]).reshape(len(data_syms), S)
        for i, t in enumerate(data_syms):
            x[u, t, :] = sym[i]
        for d, t in enumerate(cfg.dmrs_symbols):
            x[u, t, (u // 2)::2] = dmrs_port_values(dmrs[d].astype(np.complex128), u)
    return x


# ----------------------------------------------------------------------------
# Channel
# ----------------------------------------------------------------------------


def tdl_channel(cfg: SlotConfig, rng: np.random.Generator) -> np.ndarray:
    """Frequency response h[u, b, t, s] (complex128) of an exponential-PDP
    tapped delay line per user.

    Taps: tau_l = l * 4 * DS / (L-1), power ~ exp(-tau_l / DS), normalised to 1.
    Time variation: a sum of M = 16 complex sinusoids per tap with equally
    spaced, randomly rotated arrival angles (Clarke's model), unit power; a
    static channel (zero Doppler) draws CN(0, 1) gains instead.  Antennas: a
    half-wavelength ULA (one arrival angle in [-60, 60] degrees per tap) or
    independent gains per antenna.
    """
    U, B, S, L = cfg.num_users, cfg.num_rx_ant, cfg.num_subcarriers, cfg.num_taps
    tau = np.arange(L) * (4.0 * cfg.delay_spread_s / max(L - 1, 1))
    pdp = np.exp(-tau / cfg.delay_spread_s)
    pdp /= pdp.sum()
    t_n = np.arange(NUM_SYMBOLS) * (SLOT_DURATION_S / NUM_SYMBOLS)
    f_s = (np.arange(S) - S / 2) * SUBCARRIER_SPACING_HZ
    n_ant_draws = 1 if cfg.ula else B
    M = 16
    h = np.zeros((U, B, NUM_SYMBOLS, S), dtype=np.complex128)
    for u in range(U):
        # gains a[l, b', t]
        if cfg.doppler_hz == 0.0:
            g = (rng.standard_normal((L, n_ant_draws)) + 1j * rng.standard_normal((L, n_ant_draws))) / np.sqrt(2.0)
            a = np.repeat(g[:, :, None], NUM_SYMBOLS, axis=2)
        else:
            theta = rng.uniform(-np.pi, np.pi, size=(L, n_ant_draws, 1))
            phi = rng.uniform(0.0, 2.0 * np.pi, size=(L, n_ant_draws, M))
            alpha = (2.0 * np.pi * np.arange(1, M + 1) - np.pi + theta) / M  # [L, b', M]
            ph = 2.0 * np.pi * cfg.doppler_hz * np.cos(alpha)[..., None] * t_n + phi[..., None]
            a = np.exp(1j * ph).sum(axis=2) / np.sqrt(M)  # [L, b', T]
        a = a * np.sqrt(pdp)[:, None, None]
        if cfg.ula:
            aoa = rng.uniform(-np.pi / 3.0, np.pi / 3.0, size=L)
            steer = np.exp(1j * np.pi * np.arange(B)[None, :] * np.sin(aoa)[:, None])  # [L, B]
            a = a[:, 0:1, :] * steer[:, :, None]  # [L, B, T]
        phase = np.exp(-2j * np.pi * f_s[None, :] * tau[:, None])  # [L, S]
        h[u] = np.einsum("lbt,ls->bts", a, phase)
    return h


# ----------------------------------------------------------------------------
# Slots
# ----------------------------------------------------------------------------


@dataclasses.dataclass
class Slot:
    cfg: SlotConfig
    y: np.ndarray          # complex64 [B, 14, S]: the received grid
    dmrs: np.ndarray       # complex64 [n_dmrs, S/2]: DMRS base sequence per DMRS symbol
    bits: List[np.ndarray]  # per user uint8 [n_data_RE, m_u], RE order t-major then s
    h: np.ndarray          # complex128 [U, B, 14, S]: true channel
    x: np.ndarray          # complex128 [U, 14, S]: transmitted grid


def slot_dmrs(cfg: SlotConfig, rng: np.random.Generator) -> np.ndarray:
    """DMRS base sequence r(m) of each DMRS symbol (complex64 [n_dmrs, S/2]):
    TS 38.211 Gold-sequence pilots when ``cfg.n_id >= 0``, else seeded random
    unit-modulus QPSK."""
    S = cfg.num_subcarriers
    if cfg.n_id >= 0:
        return dmrs_gold(cfg.num_prb, cfg.dmrs_symbols, cfg.slot_number, cfg.n_id, cfg.n_scid)
    qpsk = (1.0 - 2.0 * rng.integers(0, 2, size=(len(cfg.dmrs_symbols), S // 2, 2))) / np.sqrt(2.0)
    return (qpsk[..., 0] + 1j * qpsk[..., 1]).astype(np.complex64)


def make_slot(cfg: SlotConfig, rng: np.random.Generator, channel: np.ndarray | None = None) -> Slot:
    """Generate one received slot (Eq. 1).  ``channel`` overrides the TDL draw
    (shape [U, B, 14, S]); used by tests that need e.g. a flat channel."""
    S = cfg.num_subcarriers
    dmrs = slot_dmrs(cfg, rng)
    n_data = cfg.num_data_symbols * S
    bits = [rng.integers(0, 2, size=(n_data, m), dtype=np.uint8) for m in cfg.bits_per_symbol]
    x = transmit_grid(cfg, dmrs, bits)
    h = tdl_channel(cfg, rng) if channel is None else np.asarray(channel, dtype=np.complex128)
    n0 = cfg.noise_var
    noise = np.sqrt(n0 / 2.0) * (rng.standard_normal((cfg.num_rx_ant, NUM_SYMBOLS, S))
                                + 1j * rng.standard_normal((cfg.num_rx_ant, NUM_SYMBOLS, S)))
    y = np.einsum("ubts,uts->bts", h, x) + noise
    return Slot(cfg=cfg, y=y.astype(np.complex64), dmrs=dmrs, bits=bits, h=h, x=x)


def workload_slots(w: Workload, n: int | None = None, start: int = 0) -> List[Slot]:
    """Slots ``start .. start+n-1`` of a workload (seed 1000*seed_base + i)."""
    n = w.batch if n is None else n
    out = []
    for i in range(start, start + n):
        rng = np.random.Generator(np.random.PCG64(1000 * w.seed_base + i))
        out.append(make_slot(draw_slot_config(w, rng), rng))
    return out


# ----------------------------------------------------------------------------
# Weights
# ----------------------------------------------------------------------------

WEIGHT_MAGIC = 0x5758524E  # "NRXW" little-endian
WEIGHT_VERSION = 1
WEIGHT_VERSION_VAR_IO = 2


def weight_layout(net: NetConfig) -> List[tuple]:
    """(name, shape) of every tensor in blob order.  Dense weights are
    [out, in] row-major (y = W x + b); depthwise kernels are [C, 3, 3] indexed
    [channel, symbol offset + 1, subcarrier offset + 1].  A Var-IO network
    (Sec. III) has one StateInit per modulation order m first ("init.m{m}.*")
    and one ReadoutLLRs per order last ("ro.m{m}.*", m outputs)."""
    C, F, m = net.channels, net.in_features, net.m_max
    if net.var_io:
        lay = []
        for mh in net.heads:
            lay += [(f"init.m{mh}.pw.w", (C, F)), (f"init.m{mh}.pw.b", (C,)), (f"init.m{mh}.dw", (C, 3, 3))]
    else:
        lay = [("init.pw.w", (C, F)), ("init.pw.b", (C,)), ("init.dw", (C, 3, 3))]
    for k in range(net.iterations):
        p = f"it{k}."
        lay += [(p + "mp1.w", (C, C)), (p + "mp1.b", (C,)),
                (p + "mp2.w", (C, C)), (p + "mp2.b", (C,)),
                (p + "in.w", (C, 2 * C + 2)), (p + "in.b", (C,))]
        for r in range(net.res_blocks):
            q = f"{p}blk{r}."
            lay += [(q + "dw1", (C, 3, 3)), (q + "pw1.w", (C, C)), (q + "pw1.b", (C,)),
                    (q + "dw2", (C, 3, 3)), (q + "pw2.w", (C, C)), (q + "pw2.b", (C,))]
    if net.var_io:
        for mh in net.heads:
            lay += [(f"ro.m{mh}.1.w", (C, C)), (f"ro.m{mh}.1.b", (C,)), (f"ro.m{mh}.2.w", (mh, C)),
                    (f"ro.m{mh}.2.b", (mh,))]
    else:
        lay += [("ro1.w", (C, C)), ("ro1.b", (C,)), ("ro2.w", (m, C)), ("ro2.b", (m,))]
    return lay


def make_weights(net: NetConfig, seed: int = 42) -> Dict[str, np.ndarray]:
    """Seeded Gaussian initialisation (float32): He-normal N(0, 2/fan_in) for
    dense layers, N(0, 2/9) for depthwise taps, N(0, 0.01^2) biases; the last
    dense layer of each residual branch is scaled by 1/sqrt(R * N_it)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    scale_last = 1.0 / np.sqrt(net.res_blocks * net.iterations)
    out = {}
    for name, shape in weight_layout(net):
        if name.endswith(".b"):
            v = 0.01 * rng.standard_normal(shape)
        elif name.endswith("dw") or name.endswith("dw1") or name.endswith("dw2"):
            v = np.sqrt(2.0 / 9.0) * rng.standard_normal(shape)
        else:
            v = np.sqrt(2.0 / shape[1]) * rng.standard_normal(shape)
            if name.endswith("pw2.w"):
                v = v * scale_last
        out[name] = v.astype(np.float32)
    return out


def pack_weights(net: NetConfig, weights: Dict[str, np.ndarray]) -> bytes:
    """Serialise to the flat blob: a 32-byte header of eight little-endian
    int32 (magic, version, B, C, R, N_it, m_max, total float count) followed by
    the float32 tensors in ``weight_layout`` order."""
    arrs = [np.ascontiguousarray(weights[n], dtype=np.float32).reshape(-1) for n, _ in weight_layout(net)]
    total = int(sum(a.size for a in arrs))
    hdr = struct.pack("<8i", WEIGHT_MAGIC, WEIGHT_VERSION_VAR_IO if net.var_io else WEIGHT_VERSION,
                      net.num_rx_ant, net.channels, net.res_blocks, net.iterations, net.m_max, total)
    return hdr + b"".join(a.tobytes() for a in arrs)


def unpack_weights(blob: bytes) -> tuple:
    """Inverse of ``pack_weights``: (NetConfig, weights) of a blob."""
    hdr = struct.unpack("<8i", blob[:32])
    if hdr[0] != WEIGHT_MAGIC or hdr[1] not in (WEIGHT_VERSION, WEIGHT_VERSION_VAR_IO):
        raise ValueError("not an NRX weight blob")
    net = NetConfig(num_rx_ant=hdr[2], channels=hdr[3], res_blocks=hdr[4], iterations=hdr[5], m_max=hdr[6],
                    var_io=hdr[1] == WEIGHT_VERSION_VAR_IO)
    flat = np.frombuffer(blob[32:], dtype=np.float32)
    if flat.size != hdr[7]:
        raise ValueError("blob size does not match its header")
    out, o = {}, 0
    for name, shape in weight_layout(net):
        n = int(np.prod(shape))
        out[name] = flat[o:o + n].reshape(shape).copy()
        o += n
    if o != flat.size:
        raise ValueError("blob size does not match the layout")
    return net, out


def widen_readout(net: NetConfig, weights: Dict[str, np.ndarray], m_max: int) -> Dict[str, np.ndarray]:
    """Weights of a single-head network with its ReadoutLLRs widened to m_max
    outputs: the first rows keep the trained bit outputs, the added rows
    (higher-order bits) start at zero."""
    if net.var_io or m_max < net.m_max:
        raise ValueError("only a single-head read-out can be widened")
    out = {k: v.copy() for k, v in weights.items()}
    w2 = np.zeros((m_max, net.channels), np.float32)
    b2 = np.zeros((m_max,), np.float32)
    w2[:net.m_max] = weights["ro2.w"]
    b2[:net.m_max] = weights["ro2.b"]
    out["ro2.w"], out["ro2.b"] = w2, b2
    return out


def zero_like_residual(net: NetConfig, weights: Dict[str, np.ndarray]) -> Dict[str, np.ndarray]:
    """Copy of ``weights`` with every message-MLP output layer, CNN-update input
    layer and residual branch output layer zeroed (used by composition tests)."""
    w = {k: v.copy() for k, v in weights.items()}
    for k in w:
        if any(k.endswith(s) for s in ("mp2.w", "mp2.b", "in.w", "in.b", "pw2.w", "pw2.b")):
            w[k][...] = 0.0
    return w


def stack_batch(slots: Sequence[Slot]) -> np.ndarray:
    """Contiguous complex64 [n_slots, B, 14, S] grid of same-shaped slots."""
    return np.stack([s.y for s in slots]).astype(np.complex64)


# ----------------------------------------------------------------------------
# Training data (Sec. II-B, Sec. IV-A)
# ----------------------------------------------------------------------------


def chest_layout(net: NetConfig) -> List[tuple]:
    """(name, shape) of the training-only channel-estimate read-out
    (ReadoutChEst, Sec. II-B): a two-layer MLP from the state to the 2B reals
    [Re h_0, Im h_0, ..., Re h_{B-1}, Im h_{B-1}] of the user's channel."""
    C, B2 = net.channels, 2 * net.num_rx_ant
    return [("chest.1.w", (C, C)), ("chest.1.b", (C,)), ("chest.2.w", (B2, C)), ("chest.2.b", (B2,))]


def make_chest_weights(net: NetConfig, seed: int = 43) -> Dict[str, np.ndarray]:
    """Seeded He-normal initialisation of the ReadoutChEst head (float32)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = {}
    for name, shape in chest_layout(net):
        v = 0.01 * rng.standard_normal(shape) if name.endswith(".b") else \
            np.sqrt(2.0 / shape[1]) * rng.standard_normal(shape)
        out[name] = v.astype(np.float32)
    return out


def snr_offset_db(bits_per_symbol: Sequence[int]) -> float:
    """SNR offset of a training sample (Sec. IV-A: samples with higher MCS and
    more active users are drawn at higher SNR so they do not dominate the
    batch loss).  The paper gives no values; this build uses +3 dB per two bits
    of the users' mean modulation order above QPSK and +1 dB per additional
    active user."""
    m = float(np.mean(bits_per_symbol))
    return 3.0 * (m - 2.0) / 2.0 + 1.0 * (len(bits_per_symbol) - 1)


def draw_active_users(num_users: int, rng: np.random.Generator) -> int:
    """Number of active users of one training batch, 1 <= U_A <= U, from a
    triangular distribution (Sec. II-B).  The paper does not give its shape;
    this build's reading is the discrete distribution rising to U,
    P(U_A = k) = 2 k / (U (U + 1))."""
    k = np.arange(1, num_users + 1, dtype=np.float64)
    return int(rng.choice(np.arange(1, num_users + 1), p=k / k.sum()))


def training_slot(w: Workload, rng: np.random.Generator, num_users: Optional[int] = None) -> Slot:
    """One training sample: an i.i.d. uniform modulation order per user from
    ``w.mcs_choices`` (random MCS-to-user association, Sec. IV-A), SNR uniform
    in ``w.snr_db_range`` plus ``snr_offset_db``, channel draws as
    ``draw_slot_config``; ``num_users`` active users (default all)."""
    c = draw_slot_config(w, rng, num_users)
    c = dataclasses.replace(c, snr_db=c.snr_db + snr_offset_db(c.bits_per_symbol))
    return make_slot(c, rng)


@dataclasses.dataclass
class TrainingBatch:
    """Same-geometry slots with their labels in the layouts the trainer reads."""

    y: np.ndarray        # complex64 [n, B, 14, S]
    dmrs: np.ndarray     # complex64 [n, n_dmrs, S/2]
    bits: np.ndarray     # uint8 [n, U, n_data, m_max] (zero beyond m_u)
    m_u: np.ndarray      # int32 [n, U]
    h: np.ndarray        # float32 [n, U, 14, S, 2B]: true channel, Re/Im per antenna
    dmrs_symbols: tuple
    noise_var: np.ndarray  # float64 [n]


def training_batch(slots: Sequence[Slot], m_max: int) -> TrainingBatch:
    """Stack same-geometry slots into a ``TrainingBatch``."""
    s0 = slots[0].cfg
    n, U, S, B = len(slots), s0.num_users, s0.num_subcarriers, s0.num_rx_ant
    n_data = s0.num_data_symbols * S
    bits = np.zeros((n, U, n_data, m_max), dtype=np.uint8)
    m_u = np.zeros((n, U), dtype=np.int32)
    h = np.zeros((n, U, NUM_SYMBOLS, S, 2 * B), dtype=np.float32)
    for i, sl in enumerate(slots):
        assert sl.cfg.num_subcarriers == S and sl.cfg.num_users == U and sl.cfg.dmrs_symbols == s0.dmrs_symbols
        for u in range(U):
            m = sl.cfg.bits_per_symbol[u]
            m_u[i, u] = m
            bits[i, u, :, :m] = sl.bits[u]
            hu = np.transpose(sl.h[u], (1, 2, 0))  # [14, S, B]
            h[i, u, :, :, 0::2] = hu.real
            h[i, u, :, :, 1::2] = hu.imag
    return TrainingBatch(y=stack_batch(slots), dmrs=np.stack([s.dmrs for s in slots]), bits=bits, m_u=m_u, h=h,
                         dmrs_symbols=tuple(s0.dmrs_symbols),
                         noise_var=np.array([s.cfg.noise_var for s in slots]))


# ----------------------------------------------------------------------------
# 5G-structured quasi-cyclic LDPC code (transport-block decoding, Sec. II)
# ----------------------------------------------------------------------------
# TS 38.212 Sec. 5.3.2 structure: a base graph of mb rows and nb = kb + mb
# columns whose nonzero entries are circulant shifts V; lifting by Z from the
# set a 2^j (a in {2, 3, 5, 7, 9, 11, 13, 15}, Z <= 384) with shift V mod Z;
# kb systematic columns, a 4 x 4 core parity block (first column of weight 3
# with shifts 1, 0, 1 and a dual diagonal of identities, so the core parities
# follow from the row sums in linear time) and one degree-1 parity column per
# extension row; the first 2 Z systematic bits are punctured.  The standard's
# shift tables are not reproduced here: this build's base graph draws the
# systematic / extension connections and their shifts from a seeded rule
# (BG2-like degrees, 4-cycles rejected at the lifting sizes used).

LDPC_A = (2, 3, 5, 7, 9, 11, 13, 15)
LDPC_ZMAX = 384


def ldpc_lifting_sizes() -> List[int]:
    """The lifting sizes a 2^j <= 384 of TS 38.212 Sec. 5.3.2, ascending."""
    return sorted({a << j for a in LDPC_A for j in range(8) if (a << j) <= LDPC_ZMAX})


@dataclasses.dataclass(frozen=True)
class LdpcBaseGraph:
    kb: int             # systematic columns
    mb: int             # rows (4 core + extension)
    V: np.ndarray       # int32 [mb, kb + mb]: shift in [0, 384), -1 where the block is zero

    @property
    def nb(self) -> int:
        return self.kb + self.mb

    def edges(self):
        """Row-major edge list: (row_ptr int32 [mb+1], col int32 [nnz], shift int32 [nnz])."""
        rows, cols = np.nonzero(self.V >= 0)
        row_ptr = np.zeros(self.mb + 1, dtype=np.int32)
        np.add.at(row_ptr, rows + 1, 1)
        return np.cumsum(row_ptr).astype(np.int32), cols.astype(np.int32), self.V[rows, cols].astype(np.int32)


def _four_cycles(V: np.ndarray, Z: int) -> int:
    """Number of length-4 cycles of the lifted graph's base pattern at size Z
    (row pairs x column pairs with V11 - V12 + V22 - V21 = 0 mod Z)."""
    n = 0
    nz = V >= 0
    for r1 in range(V.shape[0]):
        for r2 in range(r1 + 1, V.shape[0]):
            cs = np.nonzero(nz[r1] & nz[r2])[0]
            for a in range(len(cs)):
                for b in range(a + 1, len(cs)):
                    c1, c2 = cs[a], cs[b]
                    if (V[r1, c1] - V[r1, c2] + V[r2, c2] - V[r2, c1]) % Z == 0:
                        n += 1
    return n


def ldpc_base_graph(kb: int = 10, mb: int = 42, seed: int = 17, check_z=(96, 192, 384)) -> LdpcBaseGraph:
    """BG2-like base graph (kb = 10, mb = 42 by default): core rows 0..3 on
    every-few systematic columns plus the core parity block; extension row r
    on 2..4 of the first kb + 4 columns plus its own parity column kb + r.
    Shifts are redrawn (up to a bound) where they close a 4-cycle at the
    lifting sizes ``check_z``."""
    if kb < 2 or mb < 4:
        raise ValueError("need kb >= 2 and the 4 core rows")
    rng = np.random.Generator(np.random.PCG64(seed))
    nb = kb + mb
    V = -np.ones((mb, nb), dtype=np.int64)
    # core rows: systematic connections (each column in at least two core rows)
    deg = [max(2, kb - 3), max(2, kb - 4), max(2, kb - 3), max(2, kb - 4)]
    for r in range(4):
        V[r, rng.choice(kb, size=min(deg[r], kb), replace=False)] = 0
    for c in range(kb):
        while np.count_nonzero(V[:4, c] >= 0) < 2:
            V[rng.integers(0, 4), c] = 0
    # extension rows: a few of the systematic and core parity columns
    for r in range(4, mb):
        d = 4 if r < 12 else (3 if r < 28 else 2)
        V[r, rng.choice(kb + 4, size=min(d, kb + 4), replace=False)] = 0
    free = V >= 0  # entries whose shift is drawn
    V[free] = rng.integers(0, LDPC_ZMAX, size=int(free.sum()))
    # core parity block (fixed shifts) and the extension parities (identities)
    core = {(0, kb): 1, (1, kb): 0, (3, kb): 1, (0, kb + 1): 0, (1, kb + 1): 0, (1, kb + 2): 0, (2, kb + 2): 0,
            (2, kb + 3): 0, (3, kb + 3): 0}
    for (r, c), v in core.items():
        V[r, c] = v
    for r in range(4, mb):
        V[r, kb + r] = 0
    fixed = np.zeros_like(free)
    for (r, c) in core:
        fixed[r, c] = True
    for r in range(4, mb):
        fixed[r, kb + r] = True
    drawn = free & ~fixed
    for _ in range(200):  # redraw shifts that close 4-cycles at the checked sizes
        bad = [z for z in check_z if _four_cycles(V, z)]
        if not bad:
            break
        z = bad[0]
        for r1 in range(mb):
            for r2 in range(r1 + 1, mb):
                cs = np.nonzero((V[r1] >= 0) & (V[r2] >= 0))[0]
                for a in range(len(cs)):
                    for b in range(a + 1, len(cs)):
                        c1, c2 = cs[a], cs[b]
                        if (V[r1, c1] - V[r1, c2] + V[r2, c2] - V[r2, c1]) % z == 0:
                            for (rr, cc) in ((r2, c2), (r2, c1), (r1, c2), (r1, c1)):
                                if drawn[rr, cc]:
                                    V[rr, cc] = rng.integers(0, LDPC_ZMAX)
                                    break
    return LdpcBaseGraph(kb=kb, mb=mb, V=V.astype(np.int32))


def _circ(x: np.ndarray, v: int) -> np.ndarray:
    """Circulant P^v applied to a length-Z block: (P^v x)[i] = x[(i + v) mod Z]."""
    return np.roll(x, -v, axis=-1)


def ldpc_encode(bg: LdpcBaseGraph, Z: int, info: np.ndarray) -> np.ndarray:
    """Systematic encoding of info bits (uint8 [..., kb Z]) into the full
    codeword (uint8 [..., nb Z]): core parities from the core row sums (the
    weight-3 first parity column sums to the identity), then the dual
    diagonal, then each extension parity from its row."""
    info = np.asarray(info, dtype=np.uint8)
    kb, mb, nb = bg.kb, bg.mb, bg.nb
    lead = info.shape[:-1]
    x = np.zeros(lead + (nb, Z), dtype=np.uint8)
    x[..., :kb, :] = info.reshape(lead + (kb, Z))
    V = bg.V % Z

    def row_sum(r, cols):
        acc = np.zeros(lead + (Z,), dtype=np.uint8)
        for c in cols:
            if bg.V[r, c] >= 0:
                acc ^= _circ(x[..., c, :], int(V[r, c]))
        return acc
    sysc = range(kb)
    s = [row_sum(r, sysc) for r in range(4)]
    p0 = s[0] ^ s[1] ^ s[2] ^ s[3]
    x[..., kb, :] = p0
    x[..., kb + 1, :] = s[0] ^ _circ(p0, int(V[0, kb]))
    x[..., kb + 2, :] = s[1] ^ p0 ^ x[..., kb + 1, :]
    x[..., kb + 3, :] = s[2] ^ x[..., kb + 2, :]
    for r in range(4, mb):
        x[..., kb + r, :] = row_sum(r, range(kb + 4))
    return x.reshape(lead + (nb * Z,))


def ldpc_rate_match(bg: LdpcBaseGraph, Z: int, cw: np.ndarray, E: int, qm: int) -> np.ndarray:
    """TS 38.212 Sec. 5.4.2 bit selection and interleaving (redundancy version
    0, no filler bits): the circular buffer is the codeword without its first
    2 Z bits; E bits are read from its start (wrapping), then written row-wise
    into qm rows and read column-wise (bit i of modulation symbol j is
    e[i E/qm + j])."""
    if E % qm:
        raise ValueError("E must be a multiple of the modulation order")
    w = np.asarray(cw)[..., 2 * Z:]
    e = w[..., np.arange(E) % w.shape[-1]]
    return e.reshape(e.shape[:-1] + (qm, E // qm)).swapaxes(-1, -2).reshape(e.shape)


def ldpc_params(n_bits: int, qm: int, rate: float = 0.5, kb: int = 10) -> tuple:
    """Code blocks for a user stream of n_bits coded bits at modulation order
    qm: (number of blocks C, lifting size Z, E bits per block), with C the
    fewest blocks of at most kb * 384 information bits at the target rate and Z
    the largest lifting size with kb Z <= rate * E."""
    C = max(1, int(np.ceil(rate * n_bits / (kb * LDPC_ZMAX))))
    E = qm * (n_bits // (C * qm))
    zs = [z for z in ldpc_lifting_sizes() if kb * z <= rate * E]
    if not zs:
        raise ValueError("stream too short for a code block")
    return C, zs[-1], E


@dataclasses.dataclass
class LdpcUser:
    info: np.ndarray        # uint8 [C, kb Z]
    Z: int
    E: int


def ldpc_coded_bits(bg: LdpcBaseGraph, n_bits: int, qm: int, rng: np.random.Generator, rate: float = 0.5):
    """A user's bit stream of n_bits (the receivers' LLR order) filled with C
    rate-matched code blocks back to back, random filler after them.  Returns
    (bits uint8 [n_bits], LdpcUser)."""
    C, Z, E = ldpc_params(n_bits, qm, rate, bg.kb)
    info = rng.integers(0, 2, size=(C, bg.kb * Z), dtype=np.uint8)
    stream = rng.integers(0, 2, size=n_bits, dtype=np.uint8)
    stream[:C * E] = ldpc_rate_match(bg, Z, ldpc_encode(bg, Z, info), E, qm).reshape(-1)
    return stream, LdpcUser(info=info, Z=Z, E=E)


def make_ldpc_slot(cfg: SlotConfig, rng: np.random.Generator, bg: LdpcBaseGraph, rate: float = 0.5):
    """A slot whose users carry LDPC code blocks (one transport block per user
    and slot).  Returns (Slot, [LdpcUser per user])."""
    S = cfg.num_subcarriers
    n_data = cfg.num_data_symbols * S
    users, bits = [], []
    for m in cfg.bits_per_symbol:
        stream, cu = ldpc_coded_bits(bg, n_data * m, m, rng, rate)
        bits.append(stream.reshape(n_data, m))
        users.append(cu)
    dmrs = slot_dmrs(cfg, rng)
    x = transmit_grid(cfg, dmrs, bits)
    h = tdl_channel(cfg, rng)
    n0 = cfg.noise_var
    noise = np.sqrt(n0 / 2.0) * (rng.standard_normal((cfg.num_rx_ant, NUM_SYMBOLS, S))
                                + 1j * rng.standard_normal((cfg.num_rx_ant, NUM_SYMBOLS, S)))
    y = np.einsum("ubts,uts->bts", h, x) + noise
    return Slot(cfg=cfg, y=y.astype(np.complex64), dmrs=dmrs, bits=bits, h=h, x=x), users


# ----------------------------------------------------------------------------
# Channel code for BLER evaluation
# ----------------------------------------------------------------------------
# The paper reports LDPC TBLER; this build measures BLER with the textbook
# rate-1/2, constraint-length-7 convolutional code (generators 133 and 171
# octal), zero-tail terminated, and a seeded random interleaver per block.

CONV_K = 7
CONV_G = (0o133, 0o171)
CONV_TAIL = CONV_K - 1


def conv_encode(info: np.ndarray) -> np.ndarray:
    """Encode info bits (uint8 [..., n]) with 6 zero tail bits: output uint8
    [..., 2 (n + 6)], the two generator outputs of each step interleaved
    (c0(t), c1(t)).  Generator bit 6 (the MSB of the octal value) multiplies
    the current input, bit 0 the input six steps back."""
    info = np.asarray(info, dtype=np.uint8)
    n = info.shape[-1]
    u = np.concatenate([info, np.zeros(info.shape[:-1] + (CONV_TAIL,), dtype=np.uint8)], axis=-1)
    pad = np.concatenate([np.zeros(info.shape[:-1] + (CONV_TAIL,), dtype=np.uint8), u], axis=-1)
    out = np.zeros(info.shape[:-1] + (2 * (n + CONV_TAIL),), dtype=np.uint8)
    for j, g in enumerate(CONV_G):
        acc = np.zeros(u.shape, dtype=np.uint8)
        for d in range(CONV_K):  # tap on u[t - d] when bit (6 - d) of g is set
            if (g >> (CONV_K - 1 - d)) & 1:
                acc ^= pad[..., CONV_TAIL - d:CONV_TAIL - d + u.shape[-1]]
        out[..., j::2] = acc
    return out


def interleaver(n_coded: int, seed: int = 7) -> np.ndarray:
    """Seeded random interleaver: coded bit i of a block is sent at position
    perm[i] of the block's span (int32 [n_coded])."""
    return np.random.Generator(np.random.PCG64(seed)).permutation(n_coded).astype(np.int32)


@dataclasses.dataclass
class CodedUser:
    info: np.ndarray        # uint8 [n_blocks, n_info]
    block_offset: np.ndarray  # int64 [n_blocks]: first bit of each block in the user's bit stream


def coded_bits(n_bits: int, n_info: int, perm: np.ndarray, rng: np.random.Generator):
    """Fill a user's bit stream of n_bits (RE-major, then bit index: the LLR
    order of the receivers) with as many interleaved code blocks as fit, then
    random filler bits.  Returns (bits uint8 [n_bits], CodedUser)."""
    n_coded = 2 * (n_info + CONV_TAIL)
    nb = n_bits // n_coded
    info = rng.integers(0, 2, size=(nb, n_info), dtype=np.uint8)
    stream = rng.integers(0, 2, size=n_bits, dtype=np.uint8)
    if nb:
        cw = conv_encode(info)
        blocks = np.zeros_like(cw)
        blocks[:, perm] = cw
        stream[:nb * n_coded] = blocks.reshape(-1)
    return stream, CodedUser(info=info, block_offset=np.arange(nb, dtype=np.int64) * n_coded)


def make_coded_slot(cfg: SlotConfig, rng: np.random.Generator, n_info: int, perm: np.ndarray):
    """A slot whose users carry interleaved convolutional code blocks (see
    ``coded_bits``).  Returns (Slot, [CodedUser per user])."""
    S = cfg.num_subcarriers
    n_data = cfg.num_data_symbols * S
    dmrs = slot_dmrs(cfg, rng)
    bits, users = [], []
    for m in cfg.bits_per_symbol:
        stream, cu = coded_bits(n_data * m, n_info, perm, rng)
        bits.append(stream.reshape(n_data, m))
        users.append(cu)
    x = transmit_grid(cfg, dmrs, bits)
    h = tdl_channel(cfg, rng)
    n0 = cfg.noise_var
    noise = np.sqrt(n0 / 2.0) * (rng.standard_normal((cfg.num_rx_ant, NUM_SYMBOLS, S))
                                + 1j * rng.standard_normal((cfg.num_rx_ant, NUM_SYMBOLS, S)))
    y = np.einsum("ubts,uts->bts", h, x) + noise
    return Slot(cfg=cfg, y=y.astype(np.complex64), dmrs=dmrs, bits=bits, h=h, x=x), users


# ----------------------------------------------------------------------------
# TS 38.211 pseudo-random sequence and PUSCH DMRS
# ----------------------------------------------------------------------------

GOLD_NC = 1600


def gold_sequence(c_init: int, length: int) -> np.ndarray:
    """Pseudo-random sequence c(n), n < length, of TS 38.211 Sec. 5.2.1:
    c(n) = x1(n + Nc) xor x2(n + Nc), Nc = 1600, with
    x1(n+31) = x1(n+3) xor x1(n), x1(0) = 1, x1(1..30) = 0, and
    x2(n+31) = x2(n+3) xor x2(n+2) xor x2(n+1) xor x2(n), x2(i) = bit i of c_init.
    Computed 28 entries at a time (each new entry depends on entries at least
    28 positions back)."""
    total = GOLD_NC + length
    x1 = np.zeros(total + 31, dtype=np.uint8)
    x2 = np.zeros(total + 31, dtype=np.uint8)
    x1[0] = 1
    x2[:31] = [(c_init >> i) & 1 for i in range(31)]
    n = 0
    while n < total:
        k = min(28, total - n)
        x1[n + 31:n + 31 + k] = x1[n + 3:n + 3 + k] ^ x1[n:n + k]
        x2[n + 31:n + 31 + k] = x2[n + 3:n + 3 + k] ^ x2[n + 2:n + 2 + k] ^ x2[n + 1:n + 1 + k] ^ x2[n:n + k]
        n += k
    return (x1[GOLD_NC:total] ^ x2[GOLD_NC:total]).astype(np.uint8)


def dmrs_c_init(slot_number: int, symbol: int, n_id: int, n_scid: int = 0) -> int:
    """c_init of the PUSCH DMRS sequence (TS 38.211 Sec. 6.4.1.1.1.1, transform
    precoding disabled, CDM groups 0 and 1): (2^17 (14 n_s + l + 1)(2 N_ID + 1)
    + 2 N_ID + n_SCID) mod 2^31."""
    return (2 ** 17 * (14 * slot_number + symbol + 1) * (2 * n_id + 1) + 2 * n_id + n_scid) % (2 ** 31)


def dmrs_gold(num_prb: int, dmrs_symbols: Sequence[int], slot_number: int, n_id: int, n_scid: int = 0) -> np.ndarray:
    """r(m) = ((1 - 2c(2m)) + j (1 - 2c(2m+1))) / sqrt(2), m < 6 num_prb, per DMRS
    symbol (complex64 [n_dmrs, 6 num_prb]); the allocation starts at common
    resource block 0, so comb position m carries r(m)."""
    M = 6 * num_prb
    out = np.zeros((len(dmrs_symbols), M), dtype=np.complex64)
    for d, l in enumerate(dmrs_symbols):
        c = gold_sequence(dmrs_c_init(slot_number, l, n_id, n_scid), 2 * M).astype(np.float64)
        out[d] = ((1.0 - 2.0 * c[0::2]) + 1j * (1.0 - 2.0 * c[1::2])) / np.sqrt(2.0)
    return out


# ----------------------------------------------------------------------------
# Counter-based link simulator (the reference of the GPU simulator)
# ----------------------------------------------------------------------------
# The GPU training simulator draws every random number from the Philox4x32-10
# counter-based generator (Salmon et al., SC'11), so that this numpy
# restatement of the same link, from the same counters, reproduces its batches:
# key = (seed low word, seed high word), counter = (index low word, index high
# word, batch, stream).  Streams and indices:
#   1 bits     index ((slot U + u) n_data + re): bit j of word 0 is bit j of the RE
#   2 DMRS     index ((slot n_dmrs + d) S/2 + m): bits 0 / 1 of word 0 are the
#              QPSK signs of Re / Im
#   3 noise    index ((slot B + b) 14 + t) S + s: Box-Muller of words 0 and 1
#   4..8       channel gains, index ((slot U + u) L + l) Bd + bd (Bd = 1 for a
#              ULA, else B): stream 4 word 0 = arrival rotation theta (or, for
#              a static channel, words 0/1 = a Box-Muller CN(0,1) gain),
#              streams 5..8 words 0..3 = the 16 sinusoid phases
#   9 AoA      index ((slot U + u) L + l): word 0
# Uniform u(x) = (x >> 8) 2^-24; Box-Muller uses u1 = ((x0 >> 8) + 1) 2^-24 and
# u2 = u(x1): (re, im) = sqrt(-2 ln u1) (cos 2 pi u2, sin 2 pi u2).

PHILOX_M = (0xD2511F53, 0xCD9E8D57)
PHILOX_W = (0x9E3779B9, 0xBB67AE85)
SIM_STREAM_BITS, SIM_STREAM_DMRS, SIM_STREAM_NOISE, SIM_STREAM_GAIN, SIM_STREAM_AOA = 1, 2, 3, 4, 9
SIM_SINUSOIDS = 16
SIM_MAX_TAPS = 32


def philox4x32(ctr, key, rounds: int = 10) -> np.ndarray:
    """Philox4x32-R: ctr uint [..., 4], key uint [..., 2] -> uint32 [..., 4]."""
    c = [np.asarray(ctr[..., i], dtype=np.uint64) & 0xFFFFFFFF for i in range(4)]
    k0 = np.asarray(key[..., 0], dtype=np.uint64) & 0xFFFFFFFF
    k1 = np.asarray(key[..., 1], dtype=np.uint64) & 0xFFFFFFFF
    for r in range(rounds):
        if r > 0:
            k0 = (k0 + PHILOX_W[0]) & 0xFFFFFFFF
            k1 = (k1 + PHILOX_W[1]) & 0xFFFFFFFF
        p0 = np.uint64(PHILOX_M[0]) * c[0]
        p1 = np.uint64(PHILOX_M[1]) * c[2]
        c = [(p1 >> np.uint64(32)) ^ c[1] ^ k0, p1 & 0xFFFFFFFF, (p0 >> np.uint64(32)) ^ c[3] ^ k1,
             p0 & 0xFFFFFFFF]
    return np.stack(c, axis=-1).astype(np.uint32)


def _philox_draw(index, seed: int, batch: int, stream: int) -> np.ndarray:
    index = np.asarray(index, dtype=np.uint64)
    ctr = np.stack([index & 0xFFFFFFFF, index >> np.uint64(32), np.full_like(index, batch),
                    np.full_like(index, stream)], axis=-1)
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint64)
    return philox4x32(ctr, np.broadcast_to(key, ctr.shape[:-1] + (2,)))


def _uniform(x) -> np.ndarray:
    return (np.asarray(x, dtype=np.uint64) >> np.uint64(8)).astype(np.float64) * 2.0 ** -24


def _box_muller(x0, x1):
    u1 = ((np.asarray(x0, dtype=np.uint64) >> np.uint64(8)).astype(np.float64) + 1.0) * 2.0 ** -24
    r = np.sqrt(-2.0 * np.log(u1))
    a = 2.0 * np.pi * _uniform(x1)
    return r * np.cos(a), r * np.sin(a)


@dataclasses.dataclass(frozen=True)
class SimSlot:
    """Per-slot parameters of the counter-based simulator."""

    noise_var: float
    delay_spread_s: float
    doppler_hz: float
    num_taps: int
    ula: bool
    bits_per_symbol: tuple


def sim_slot_params(w: Workload, rng: np.random.Generator, num_users: Optional[int] = None) -> SimSlot:
    """Training-sample parameters as ``training_slot`` draws them (random MCS
    association, SNR with the offsets of Sec. IV-A, delay spread, Doppler)."""
    c = draw_slot_config(w, rng, num_users)
    snr = c.snr_db + snr_offset_db(c.bits_per_symbol)
    return SimSlot(noise_var=float(np.float32(10.0 ** (-snr / 10.0))), delay_spread_s=float(np.float32(c.delay_spread_s)),
                   doppler_hz=float(np.float32(c.doppler_hz)), num_taps=w.num_taps, ula=w.ula,
                   bits_per_symbol=c.bits_per_symbol)


def simulate_philox(slots: Sequence[SimSlot], num_users: int, num_rx_ant: int, num_prb: int,
                    dmrs_symbols: Sequence[int], m_max: int, seed: int, batch: int) -> TrainingBatch:
    """The link of ``make_slot`` (Eq. 1) with every draw from Philox (see
    above): bits -> Gray QAM, QPSK DMRS on the type-1 comb with OCC, TDL
    channel with the Clarke sum of sinusoids (or CN(0,1) static gains), ULA
    steering, AWGN.  float64 arithmetic; returns a ``TrainingBatch``."""
    n, U, B, S = len(slots), num_users, num_rx_ant, 12 * num_prb
    ds = tuple(dmrs_symbols)
    nd = len(ds)
    data = [t for t in range(NUM_SYMBOLS) if t not in ds]
    n_data = len(data) * S
    # DMRS
    idx = np.arange(n * nd * (S // 2))
    w = _philox_draw(idx, seed, batch, SIM_STREAM_DMRS)[:, 0].astype(np.int64)
    dm = (((1 - 2 * (w & 1)) + 1j * (1 - 2 * ((w >> 1) & 1))) / np.sqrt(2.0)).reshape(n, nd, S // 2)
    # bits
    bits = np.zeros((n, U, n_data, m_max), dtype=np.uint8)
    m_u = np.array([[s.bits_per_symbol[u] for u in range(U)] for s in slots], dtype=np.int32)
    wb = _philox_draw(np.arange(n * U * n_data), seed, batch, SIM_STREAM_BITS)[:, 0].reshape(n, U, n_data)
    for j in range(m_max):
        bits[..., j] = (wb >> j) & 1
    for i in range(n):
        for u in range(U):
            bits[i, u, :, m_u[i, u]:] = 0
    # transmitted grids
    x = np.zeros((n, U, NUM_SYMBOLS, S), dtype=np.complex128)
    for i in range(n):
        for u in range(U):
            m = int(m_u[i, u])
            sym = qam_modulate(bits[i, u, :, :m], m).reshape(len(data), S)
            for k, t in enumerate(data):
                x[i, u, t] = sym[k]
            for d, t in enumerate(ds):
                x[i, u, t, (u // 2)::2] = dmrs_port_values(dm[i, d], u)
    # channel
    t_n = np.arange(NUM_SYMBOLS) * (SLOT_DURATION_S / NUM_SYMBOLS)
    f_s = (np.arange(S) - S / 2) * SUBCARRIER_SPACING_HZ
    h = np.zeros((n, U, B, NUM_SYMBOLS, S), dtype=np.complex128)
    for i, sp in enumerate(slots):
        L = sp.num_taps
        DS = sp.delay_spread_s
        tau = np.arange(L) * (4.0 * DS / max(L - 1, 1))
        pdp = np.exp(-tau / DS)
        pdp /= pdp.sum()
        Bd = 1 if sp.ula else B
        for u in range(U):
            gidx = ((i * U + u) * L + np.arange(L))[:, None] * Bd + np.arange(Bd)[None, :]  # [L, Bd]
            w4 = _philox_draw(gidx, seed, batch, SIM_STREAM_GAIN)
            if sp.doppler_hz == 0.0:
                gr, gi = _box_muller(w4[..., 0], w4[..., 1])
                a = np.repeat(((gr + 1j * gi) / np.sqrt(2.0))[:, :, None], NUM_SYMBOLS, axis=2)
            else:
                theta = (2.0 * _uniform(w4[..., 0]) - 1.0) * np.pi  # [L, Bd]
                phi = np.concatenate([2.0 * np.pi * _uniform(_philox_draw(gidx, seed, batch, SIM_STREAM_GAIN + 1 + k))
                                      for k in range(4)], axis=-1)  # [L, Bd, 16]
                mm = np.arange(1, SIM_SINUSOIDS + 1)
                alpha = (2.0 * np.pi * mm - np.pi + theta[..., None]) / SIM_SINUSOIDS
                ph = 2.0 * np.pi * sp.doppler_hz * np.cos(alpha)[..., None] * t_n + phi[..., None]
                a = np.exp(1j * ph).sum(axis=2) / np.sqrt(SIM_SINUSOIDS)  # [L, Bd, T]
            a = a * np.sqrt(pdp)[:, None, None]
            if sp.ula:
                wa = _philox_draw((i * U + u) * L + np.arange(L), seed, batch, SIM_STREAM_AOA)[:, 0]
                aoa = (2.0 * _uniform(wa) - 1.0) * (np.pi / 3.0)
                steer = np.exp(1j * np.pi * np.arange(B)[None, :] * np.sin(aoa)[:, None])  # [L, B]
                a = a[:, 0:1, :] * steer[:, :, None]
            phase = np.exp(-2j * np.pi * f_s[None, :] * tau[:, None])  # [L, S]
            h[i, u] = np.einsum("lbt,ls->bts", a, phase)
    # received grid
    nidx = np.arange(n * B * NUM_SYMBOLS * S)
    wn = _philox_draw(nidx, seed, batch, SIM_STREAM_NOISE)
    nr, ni = _box_muller(wn[:, 0], wn[:, 1])
    noise = (nr + 1j * ni).reshape(n, B, NUM_SYMBOLS, S)
    n0 = np.array([s.noise_var for s in slots])
    y = np.einsum("nubts,nuts->nbts", h, x) + np.sqrt(n0 / 2.0)[:, None, None, None] * noise
    hr = np.zeros((n, U, NUM_SYMBOLS, S, 2 * B), dtype=np.float32)
    hr[..., 0::2] = np.transpose(h, (0, 1, 3, 4, 2)).real
    hr[..., 1::2] = np.transpose(h, (0, 1, 3, 4, 2)).imag
    return TrainingBatch(y=y.astype(np.complex64), dmrs=dm.astype(np.complex64), bits=bits, m_u=m_u, h=hr,
                         dmrs_symbols=ds, noise_var=n0)
