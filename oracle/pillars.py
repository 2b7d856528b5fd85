"""FP64 oracle of the pillar front end -- TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper's 3D-perception chains C0/C1 run PointPillars (Section 6, Table 4: 22k-25k points,
41 kernels) as a closed-source engine; the paper itself does not describe the network.  This
module restates its front end step by step as this library specifies it:

1. voxelise: cell index per point, range filter, pillars = occupied cells in ascending cell
   order, at most ``max_pillars``; each pillar keeps its first ``max_pts`` points by input index;
2. PointNet: 9 features per point, Linear (no bias), inference BN, ReLU, max over the pillar's
   valid points;
3. BEV scatter: each pillar's feature vector lands at its cell of a [ny][nx][C] canvas, zeros
   elsewhere;
4. backbone: conv3x3 (zero pad 1) + BN + ReLU layers;
5. neck and detection head (the rest of PointPillars' GPU segment): each block's output is
   upsampled to the first block's resolution by a transposed convolution whose kernel equals its
   stride (no overlap), followed by BN + ReLU; the upsampled maps are concatenated along
   channels in block order; a 1x1 convolution with bias produces the per-anchor class, box and
   direction outputs.

Readings where the specification is silent:
* ranges are half-open [min, max) in x, y and z;
* cell index contract: ix = floor(fl32(fl32(x - xmin) / vx)) with IEEE binary32 round-to-nearest
  subtraction and division on binary32 operands; a point is kept iff it is inside all three
  ranges and 0 <= ix < nx, 0 <= iy < ny; cell = iy * nx + ix;
* the 9 features are (x, y, z, r, x - mean_x, y - mean_y, z - mean_z, x - x_c, y - y_c): the
  means are over the pillar's kept points, (x_c, y_c) is the pillar's cell centre
  xmin + (ix + 0.5) vx, ymin + (iy + 0.5) vy with the binary32 geometry constants;
* BN is y = gamma (h - mean) / sqrt(var + 1e-3) + beta;
* the max runs over the pillar's valid points only (padding slots excluded);
* neck: block b is upsampled by s_b = (first block's height) / (block b's height) with a
  transposed convolution of kernel s_b and stride s_b (PyTorch ConvTranspose2d weight layout
  [cin][cout][s][s], no bias): out[s*y + dy, s*x + dx, co] = sum_ci in[y, x, ci] w[ci, co, dy, dx];
* head: one 1x1 convolution (weight [cout][cin], bias [cout]) over the concatenated map; its
  outputs are the anchors' class scores, box parameters and direction scores side by side.
"""
from __future__ import annotations

from typing import Dict, List, Sequence

import numpy as np

BN_EPS = 1e-3


def cell_indices(points: np.ndarray, g) -> tuple:
    """(ix, iy, keep) per point under the binary32 rounding contract described above."""
    p = np.ascontiguousarray(points, dtype=np.float32).reshape(-1, 4)
    x, y, z = p[:, 0], p[:, 1], p[:, 2]
    xmin, xmax = np.float32(g.xmin), np.float32(g.xmax)
    ymin, ymax = np.float32(g.ymin), np.float32(g.ymax)
    zmin, zmax = np.float32(g.zmin), np.float32(g.zmax)
    with np.errstate(invalid="ignore", over="ignore"):
        qx = np.floor((x - xmin) / np.float32(g.vx))  # each op rounded to binary32
        qy = np.floor((y - ymin) / np.float32(g.vy))
        keep = ((x >= xmin) & (x < xmax) & (y >= ymin) & (y < ymax) & (z >= zmin) & (z < zmax)
                & (qx >= 0) & (qx < g.nx) & (qy >= 0) & (qy < g.ny))
    ix = np.where(keep, qx, 0).astype(np.int64)
    iy = np.where(keep, qy, 0).astype(np.int64)
    return ix, iy, keep


def voxelise(points: np.ndarray, g) -> Dict[str, np.ndarray]:
    """Point -> pillar assignment.

    Returns ``cell`` int32[N] (-1 = dropped), ``cnt`` int64[G] points per cell,
    ``pillar_of_cell`` int32[G] (-1 = not a kept pillar), ``coord`` int32[P'] (cell of pillar p,
    strictly increasing), ``npts`` int32[P'] = min(count, max_pts), ``pt_idx`` int64[P', max_pts]
    (input index of each kept point, ascending, -1 padding), ``pts`` float32[P', max_pts, 4]
    (zero padding) and ``num_pillars`` = P'.
    """
    p = np.ascontiguousarray(points, dtype=np.float32).reshape(-1, 4)
    n = p.shape[0]
    G, T = g.nx * g.ny, g.max_pts
    ix, iy, keep = cell_indices(p, g)
    cell = np.full(n, -1, dtype=np.int64)
    cell[keep] = iy[keep] * g.nx + ix[keep]
    cnt = np.bincount(cell[keep], minlength=G).astype(np.int64)
    occupied = np.nonzero(cnt)[0]                 # ascending cell order
    kept = occupied[: g.max_pillars]
    num = len(kept)
    pillar_of_cell = np.full(G, -1, dtype=np.int32)
    pillar_of_cell[kept] = np.arange(num, dtype=np.int32)
    # points grouped by cell, input order preserved inside each group (stable sort)
    idx = np.nonzero(keep)[0]
    order = idx[np.argsort(cell[idx], kind="stable")]
    sorted_cells = cell[order]
    start = np.searchsorted(sorted_cells, kept, side="left")
    npts = np.minimum(cnt[kept], T).astype(np.int32)
    pt_idx = np.full((num, T), -1, dtype=np.int64)
    pts = np.zeros((num, T, 4), dtype=np.float32)
    for j in range(T):
        has = npts > j
        pt_idx[has, j] = order[start[has] + j]
        pts[has, j] = p[pt_idx[has, j]]
    return {
        "cell": cell.astype(np.int32), "cnt": cnt, "pillar_of_cell": pillar_of_cell,
        "coord": kept.astype(np.int32), "npts": npts, "pt_idx": pt_idx, "pts": pts,
        "num_pillars": num,
    }


def pointnet(pts: np.ndarray, npts: np.ndarray, coord: np.ndarray, pfn_w: np.ndarray,
             pfn_bn: np.ndarray, g) -> np.ndarray:
    """Per-pillar feature vector float64[P', C]: 9 features -> Linear (no bias) -> BN -> ReLU
    -> max over the valid points."""
    P, T = int(len(npts)), g.max_pts
    C = pfn_w.shape[0]
    if P == 0:
        return np.zeros((0, C))
    q = pts.astype(np.float64)[:, :T, :]
    npts = np.asarray(npts, dtype=np.int64)
    valid = np.arange(T)[None, :] < npts[:, None]
    mean = (q[:, :, :3] * valid[:, :, None]).sum(axis=1) / npts[:, None]
    ix = coord.astype(np.int64) % g.nx
    iy = coord.astype(np.int64) // g.nx
    xc = float(np.float32(g.xmin)) + (ix + 0.5) * float(np.float32(g.vx))
    yc = float(np.float32(g.ymin)) + (iy + 0.5) * float(np.float32(g.vy))
    f = np.empty((P, T, 9))
    f[:, :, 0:4] = q[:, :, 0:4]
    f[:, :, 4:7] = q[:, :, 0:3] - mean[:, None, :]
    f[:, :, 7] = q[:, :, 0] - xc[:, None]
    f[:, :, 8] = q[:, :, 1] - yc[:, None]
    h = f @ pfn_w.astype(np.float64).T                        # [P, T, C]
    gamma, beta, mu, var = (pfn_bn[i].astype(np.float64) for i in range(4))
    a = np.maximum(gamma * (h - mu) / np.sqrt(var + BN_EPS) + beta, 0.0)
    a = np.where(valid[:, :, None], a, -np.inf)
    return a.max(axis=1)


def scatter(feat: np.ndarray, coord: np.ndarray, g) -> np.ndarray:
    """BEV pseudo-image [ny, nx, C]: canvas[iy, ix] = feat[p] for pillar p at cell iy*nx+ix."""
    C = feat.shape[1] if feat.ndim == 2 and feat.shape[0] else g.channels
    canvas = np.zeros((g.ny, g.nx, C))
    c = coord.astype(np.int64)
    canvas[c // g.nx, c % g.nx] = feat
    return canvas


def conv3x3_bn_relu(x: np.ndarray, w: np.ndarray, bn: np.ndarray, stride: int) -> np.ndarray:
    """One backbone layer on an HWC map: out[oy, ox, co] = ReLU(BN(sum over ky, kx, ci of
    w[co, ci, ky, kx] * xpad[oy*s + ky, ox*s + kx, ci])) with a one-pixel zero border xpad.
    Output size floor((H + 2 - 3) / s) + 1.  Each tap's channel contraction is a matmul."""
    H, W, Cin = x.shape
    Cout = w.shape[0]
    Ho, Wo = (H - 1) // stride + 1, (W - 1) // stride + 1
    xp = np.zeros((H + 2, W + 2, Cin))
    xp[1:-1, 1:-1] = x
    w = w.astype(np.float64)
    acc = np.zeros((Ho, Wo, Cout))
    for ky in range(3):
        for kx in range(3):
            win = xp[ky: ky + stride * (Ho - 1) + 1: stride, kx: kx + stride * (Wo - 1) + 1: stride]
            acc += win @ w[:, :, ky, kx].T
    gamma, beta, mu, var = (bn[i].astype(np.float64) for i in range(4))
    return np.maximum(gamma * (acc - mu) / np.sqrt(var + BN_EPS) + beta, 0.0)


def backbone(canvas: np.ndarray, conv_w: Sequence[np.ndarray], conv_bn: Sequence[np.ndarray],
             layers: Sequence[tuple], convs: Sequence[int]) -> List[np.ndarray]:
    """Runs every layer; returns the output of the last layer of each block (HWC, float64)."""
    outs, x, li = [], canvas, 0
    for nb in convs:
        for _ in range(nb):
            x = conv3x3_bn_relu(x, conv_w[li], conv_bn[li], layers[li][2])
            li += 1
        outs.append(x)
    return outs


def deconv_bn_relu(x: np.ndarray, w: np.ndarray, bn: np.ndarray, s: int) -> np.ndarray:
    """Transposed convolution with kernel = stride = s (each input pixel writes its own s x s
    output block), then BN and ReLU.  x [H, W, cin], w [cin, cout, s, s] -> [s H, s W, cout]."""
    H, W, _ = x.shape
    cout = w.shape[1]
    out = np.zeros((s * H, s * W, cout))
    w = w.astype(np.float64)
    for dy in range(s):
        for dx in range(s):
            out[dy::s, dx::s] = x @ w[:, :, dy, dx]
    gamma, beta, mu, var = (bn[i].astype(np.float64) for i in range(4))
    return np.maximum(gamma * (out - mu) / np.sqrt(var + BN_EPS) + beta, 0.0)


def neck(blocks: Sequence[np.ndarray], up_w: Sequence[np.ndarray], up_bn: Sequence[np.ndarray]) -> np.ndarray:
    """Upsample every block output to the first block's resolution and concatenate channels."""
    H0 = blocks[0].shape[0]
    ups = []
    for x, w, bn in zip(blocks, up_w, up_bn):
        s = H0 // x.shape[0]
        ups.append(deconv_bn_relu(x, w, bn, s))
    return np.concatenate(ups, axis=2)


def head(x: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """1x1 convolution with bias: [H, W, cin] x w [cout, cin] + b [cout] -> [H, W, cout]."""
    return x @ w.astype(np.float64).T + b.astype(np.float64)


def frame(points: np.ndarray, g, bb, weights) -> Dict[str, object]:
    """Whole front end for one frame: voxelise -> PointNet -> scatter -> backbone."""
    pfn_w, pfn_bn, conv_w, conv_bn = weights
    v = voxelise(points, g)
    feat = pointnet(v["pts"], v["npts"], v["coord"], pfn_w, pfn_bn, g)
    canvas = scatter(feat, v["coord"], g)
    blocks = backbone(canvas, conv_w, conv_bn, bb.layers(g.channels), bb.convs)
    return {"vox": v, "feat": feat, "canvas": canvas, "blocks": blocks}
