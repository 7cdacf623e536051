"""Candidate centres for sampled voxels of images too large for the whole-
image oracle: every seed whose window can cover the voxel.  Seeds sit on the
lattice o_d + j S_d (reading R1) moved by at most one voxel per axis by the
perturbation (R3), and a window covers x when x - S < c <= x + S (R5), so
lattice index j can cover x only if o + j S lies in [x - S - 1, x + S + 1]."""
import numpy as np


def lattice(size, grid):
    n = [-(-N // S) for N, S in zip(size, grid)]
    o = [(N - 1 - (nn - 1) * S) // 2 for N, S, nn in zip(size, grid, n)]
    return n, o


def seed_candidates(size, grid, q):
    """CSR lists (start, idx) of the seeds that can cover raster voxels q."""
    size = tuple(int(v) for v in size)
    grid = tuple(int(v) for v in grid)
    nd = len(size)
    n, o = lattice(size, grid)
    q = np.asarray(q, np.int64)
    x, rem = [], q.copy()
    for d in range(nd):
        x.append(rem % size[d])
        rem //= size[d]
    per_axis = []
    for d in range(nd):
        lo = np.maximum(0, -((o[d] + grid[d] + 1 - x[d]) // grid[d]))    # ceil((x - S - 1 - o) / S)
        hi = np.minimum(n[d] - 1, (x[d] + grid[d] + 1 - o[d]) // grid[d])
        per_axis.append((lo, hi))
    span = max(int((h - l).max()) + 1 for l, h in per_axis)
    offs = np.arange(span)
    idx = np.zeros((q.shape[0],) + (span,) * nd, np.int64)
    ok = np.ones_like(idx, dtype=bool)
    stride = 1
    for d in range(nd):
        lo, hi = per_axis[d]
        j = lo[:, None] + offs[None, :]
        shape = [q.shape[0]] + [1] * nd
        shape[1 + d] = span
        idx += (j * stride).reshape(shape)
        ok &= (j <= hi[:, None]).reshape(shape)
        stride *= n[d]
    idx = idx.reshape(q.shape[0], -1)
    ok = ok.reshape(q.shape[0], -1)
    counts = ok.sum(1)
    start = np.zeros(q.shape[0] + 1, np.int64)
    np.cumsum(counts, out=start[1:])
    return start, idx[ok]
