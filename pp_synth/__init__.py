"""Seeded synthetic inputs for the LiDAR pillar front end and its serving workloads.

This module is shared by the CUDA path's tests/bench and by the oracle's tests. It holds
configuration constants and random draws only -- none of the pillar method's arithmetic
(no cell indexing, no grouping, no features, no convolution, no urgency).

The paper evaluates on bus recordings from RS-Helios LiDARs (Section 6, ~22k-25k points per
frame for the 3D detection task, Table 4). Those recordings are not available, so seeded
synthetic clouds stand in for them:

* uniform clouds: x ~ U[0, 69.12), y ~ U[-39.68, 39.68), z ~ U[-3, 1), r ~ U[0, 1), float32;
* clustered clouds: 70 % of the points in 40 Gaussian blobs (sigma 0.5 m in x, y, z; centres
  uniform in x/y range, centre z ~ U[-2, 0]) and 30 % uniform as above.  Points a blob throws
  outside the range are kept in the cloud; the range filter drops them.

Every frame draws from ``numpy.random.default_rng(1000 + config * 100 + frame)``.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence, Tuple

import numpy as np

__all__ = [
    "Geometry", "Backbone", "GEOM_SMALL", "GEOM_FULL", "BACKBONE_SMALL", "BACKBONE_FULL",
    "frame_seed", "uniform_cloud", "clustered_cloud", "config_points", "batched_counts",
    "pillar_weights", "ChainSpec", "tight_chains", "serving_chains", "arrival_times", "splitmix64",
    "noise_factors",
]


@dataclasses.dataclass(frozen=True)
class Geometry:
    """Pillar grid. Ranges are half-open [min, max); nx*vx spans x, ny*vy spans y."""
    xmin: float
    xmax: float
    ymin: float
    ymax: float
    zmin: float
    zmax: float
    vx: float
    vy: float
    nx: int
    ny: int
    max_pillars: int
    max_pts: int = 32
    channels: int = 64

    @property
    def cells(self) -> int:
        return self.nx * self.ny


@dataclasses.dataclass(frozen=True)
class Backbone:
    """Conv3x3 backbone: block b has ``convs[b]`` layers of ``chans[b]`` channels; the first
    layer of the block has stride ``strides[b]``, the others stride 1."""
    convs: Tuple[int, ...]
    chans: Tuple[int, ...]
    strides: Tuple[int, ...]

    def layers(self, cin: int = 64) -> List[Tuple[int, int, int]]:
        """(cin, cout, stride) per conv layer, in order."""
        out = []
        for n, c, s in zip(self.convs, self.chans, self.strides):
            for i in range(n):
                out.append((cin, c, s if i == 0 else 1))
                cin = c
        return out


# 0.32 m grid, 216 x 248 cells, 4000 pillars; one block of three 64-channel convs (first s2).
GEOM_SMALL = Geometry(0.0, 69.12, -39.68, 39.68, -3.0, 1.0, 0.32, 0.32, 216, 248, 4000)
BACKBONE_SMALL = Backbone((3,), (64,), (2,))
# 0.16 m grid, 432 x 496 cells, 12000 pillars; blocks 64/128/256 ch x 4/6/6 convs, strides 2/2/2.
GEOM_FULL = Geometry(0.0, 69.12, -39.68, 39.68, -3.0, 1.0, 0.16, 0.16, 432, 496, 12000)
BACKBONE_FULL = Backbone((4, 6, 6), (64, 128, 256), (2, 2, 2))


def frame_seed(config: int, frame: int) -> int:
    return 1000 + config * 100 + frame


def _uniform(rng: np.random.Generator, n: int, g: Geometry) -> np.ndarray:
    pts = np.empty((n, 4), dtype=np.float32)
    pts[:, 0] = rng.uniform(g.xmin, g.xmax, n)
    pts[:, 1] = rng.uniform(g.ymin, g.ymax, n)
    pts[:, 2] = rng.uniform(g.zmin, g.zmax, n)
    pts[:, 3] = rng.uniform(0.0, 1.0, n)
    return pts


def uniform_cloud(n: int, seed: int, g: Geometry = GEOM_SMALL) -> np.ndarray:
    """``n`` points (x, y, z, r) float32, uniform over the grid's range."""
    return _uniform(np.random.default_rng(seed), n, g)


def clustered_cloud(n: int, seed: int, g: Geometry = GEOM_FULL, blobs: int = 40,
                    sigma: float = 0.5, frac: float = 0.7) -> np.ndarray:
    """70 % of the points in ``blobs`` Gaussian blobs, the rest uniform; rows shuffled."""
    rng = np.random.default_rng(seed)
    n_blob = int(round(n * frac))
    cx = rng.uniform(g.xmin, g.xmax, blobs)
    cy = rng.uniform(g.ymin, g.ymax, blobs)
    cz = rng.uniform(-2.0, 0.0, blobs)
    which = rng.integers(0, blobs, n_blob)
    pts = np.empty((n, 4), dtype=np.float32)
    pts[:n_blob, 0] = cx[which] + rng.normal(0.0, sigma, n_blob)
    pts[:n_blob, 1] = cy[which] + rng.normal(0.0, sigma, n_blob)
    pts[:n_blob, 2] = cz[which] + rng.normal(0.0, sigma, n_blob)
    pts[:n_blob, 3] = rng.uniform(0.0, 1.0, n_blob)
    pts[n_blob:] = _uniform(rng, n - n_blob, g)
    return pts[rng.permutation(n)]


def batched_counts(config: int, frames: int = 8, lo: int = 30000, hi: int = 150000) -> List[int]:
    """Point counts N_i ~ U{lo..hi} for a batch of frames (inclusive bounds)."""
    rng = np.random.default_rng(frame_seed(config, 99))
    return [int(v) for v in rng.integers(lo, hi + 1, frames)]


def config_points(config: int, frame: int = 0, n: int | None = None) -> np.ndarray:
    """The cloud of ``frame`` in workload ``config``:
    1 = 20k uniform points (0.32 m grid), 2 = 120k clustered points (0.16 m grid),
    3/4/5 = uniform clouds of 30k-150k points on the 0.32 m grid."""
    seed = frame_seed(config, frame)
    if config == 1:
        return uniform_cloud(20000 if n is None else n, seed, GEOM_SMALL)
    if config == 2:
        return clustered_cloud(120000 if n is None else n, seed, GEOM_FULL)
    if n is None:
        n = int(np.random.default_rng(seed).integers(30000, 150001))
    return uniform_cloud(n, seed + 7, GEOM_SMALL)


def pillar_weights(backbone: Backbone, seed: int = 7, cin: int = 64):
    """Random-init weights for the PointNet and the conv backbone.

    Returns ``(pfn_w [64,9], pfn_bn [4,64], conv_w list of [cout,cin,3,3], conv_bn list of
    [4,cout])``, all float32.  BN rows are (gamma, beta, mean, var).  Linear/conv weights are
    He-normal; gamma ~ U[0.5, 1.5], beta ~ U[-0.1, 0.1]; mean 0.  The PointNet BN variance is
    400 (the features carry coordinates of tens of metres), the conv BN variance is 1.
    """
    rng = np.random.default_rng(seed)
    pfn_w = rng.normal(0.0, np.sqrt(2.0 / 9.0), (64, 9)).astype(np.float32)
    pfn_bn = np.stack([rng.uniform(0.5, 1.5, 64), rng.uniform(-0.1, 0.1, 64),
                       np.zeros(64), np.full(64, 400.0)]).astype(np.float32)
    conv_w, conv_bn = [], []
    for ci, co, _s in backbone.layers(cin):
        conv_w.append(rng.normal(0.0, np.sqrt(2.0 / (9 * ci)), (co, ci, 3, 3)).astype(np.float32))
        conv_bn.append(np.stack([rng.uniform(0.5, 1.5, co), rng.uniform(-0.1, 0.1, co),
                                 np.zeros(co), np.ones(co)]).astype(np.float32))
    return pfn_w, pfn_bn, conv_w, conv_bn


NECK_CHANNELS = 128      # per upsampled block
HEAD_OUTPUTS = 72        # 6 anchors per location x (3 class scores + 7 box parameters + 2 direction scores)


def head_weights(backbone: Backbone, seed: int = 17, up_channels: int = NECK_CHANNELS,
                 head_outputs: int = HEAD_OUTPUTS):
    """Random-init weights for the neck and the detection head.

    Returns ``(up_w list of [cin, up_channels, s, s], up_bn list of [4, up_channels], head_w
    [head_outputs, n_blocks * up_channels], head_b [head_outputs])``, float32; block b's
    upsampling stride s is the product of the strides of blocks 1..b (its map's reduction
    relative to the first block's).
    Weights He-normal over the fan-in (cin for the transposed convs), BN as in the backbone
    (gamma ~ U[0.5, 1.5], beta ~ U[-0.1, 0.1], mean 0, var 1), bias ~ U[-0.1, 0.1].
    """
    rng = np.random.default_rng(seed)
    up_w, up_bn = [], []
    s = 1
    for b, ch in enumerate(backbone.chans):
        if b:
            s *= backbone.strides[b]
        up_w.append(rng.normal(0.0, np.sqrt(2.0 / ch), (ch, up_channels, s, s)).astype(np.float32))
        up_bn.append(np.stack([rng.uniform(0.5, 1.5, up_channels), rng.uniform(-0.1, 0.1, up_channels),
                               np.zeros(up_channels), np.ones(up_channels)]).astype(np.float32))
    cin = up_channels * len(backbone.chans)
    head_w = rng.normal(0.0, np.sqrt(1.0 / cin), (head_outputs, cin)).astype(np.float32)
    head_b = rng.uniform(-0.1, 0.1, head_outputs).astype(np.float32)
    return up_w, up_bn, head_w, head_b


@dataclasses.dataclass(frozen=True)
class ChainSpec:
    chain_id: int
    period_ms: float
    deadline_ms: float
    precision: int  # 0 = FP32, 1 = BF16


def tight_chains(n_chains: int, tight: float, seed: int = 1500) -> List[int]:
    """The chains whose deadlines are halved for a tight-deadline share ``tight`` (the paper's
    f_tight, Section 6.2): floor(tight * n_chains + 1/2) of them, the first ones of a seeded
    permutation of the chain ids (so a larger share keeps the chains of a smaller one)."""
    if not 0.0 <= tight <= 1.0:
        raise ValueError("tight must be in [0, 1]")
    k = int(math.floor(tight * n_chains + 0.5))
    return sorted(int(c) for c in np.random.default_rng(seed).permutation(n_chains)[:k])


def serving_chains(n_chains: int = 11, mixed: bool = False,
                   periods: Sequence[float] = (50.0, 100.0, 200.0), tight: float = 0.0,
                   tight_seed: int = 1500) -> List[ChainSpec]:
    """Periodic chains: period = periods[i mod 3], deadline = period, halved for the chains
    ``tight_chains(n_chains, tight, tight_seed)`` picks.
    ``mixed``: odd chains BF16, even chains FP32; otherwise all BF16."""
    halved = set(tight_chains(n_chains, tight, tight_seed))
    out = []
    for i in range(n_chains):
        p = float(periods[i % len(periods)])
        out.append(ChainSpec(i, p, p / 2.0 if i in halved else p, (i % 2) if mixed else 1))
    return out


def arrival_times(chains: Sequence[ChainSpec], duration_ms: float, rate: float = 1.0,
                  jitter_ms: float = 5.0, seed: int = 1400) -> List[Tuple[float, int, int]]:
    """Frame releases ``(t_ms, chain_id, n_points)`` sorted by time.  Chain i releases every
    ``period/rate`` ms with a phase ~ U[0, period/rate) and jitter ~ U[-jitter, +jitter];
    each frame's point count ~ U{30000..150000}."""
    rng = np.random.default_rng(seed)
    ev = []
    for c in chains:
        per = c.period_ms / rate
        t = rng.uniform(0.0, per)
        while t < duration_ms:
            tj = max(0.0, t + rng.uniform(-jitter_ms, jitter_ms))
            ev.append((float(tj), c.chain_id, int(rng.integers(30000, 150001))))
            t += per
    ev.sort()
    return ev


_MASK = (1 << 64) - 1


def splitmix64(seed: int, k: int) -> int:
    """The k-th output (k >= 1) of a SplitMix64 generator seeded with ``seed`` (Steele, Lea and
    Flood, OOPSLA 2014): the state advances by 0x9E3779B97F4A7C15 per output and each output is
    the state after two xor-shift-multiply rounds and a final xor-shift."""
    z = (seed + k * 0x9E3779B97F4A7C15) & _MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
    return z ^ (z >> 31)


def noise_factors(seed: int, ids: Sequence[int], eps: float) -> np.ndarray:
    """Estimate-noise factors 1 + eps (2u - 1), u = the top 53 bits of splitmix64(seed, id)
    scaled to [0, 1): one per frame id (the estimate-error experiment's per-instance draw)."""
    u = np.array([(splitmix64(seed, int(i)) >> 11) * 2.0 ** -53 for i in ids])
    return 1.0 + eps * (2.0 * u - 1.0)
