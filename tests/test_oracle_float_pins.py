"""Pins of the oracle's float-image paths against independent numpy restatements.

The oracle (oracle/sslic_oracle.c) is the reference of every float-tolerance
claim: its FP64 mode defines the "FP64 oracle" that float images (the
CIE-Lab volume, the 64-band image) are compared with, and its FP32 mode on a
float image is the canonical single-precision evaluation.  Each pin below
restates one step of the method in numpy, in the same arithmetic and the same
order of operations, and asks for bit-for-bit equality:

  * assignment (Sec. 2.2, "for each cluster centre C_k ... if D < d(x)"): an
    exhaustive voxel x centre argmin of D^2 = d_c^2 + sum_d w_d (x_d - c_d)^2
    (Sec. 2.1; anisotropic w_d = m^2/S_d^2, Sec. 3.3) over the centres whose
    2S window covers the voxel, ties to the lowest index;
  * update (Sec. 2.2 "Update clusters", Sec. 3.1 map-reduce): centres are the
    member means, accumulated in double in raster order (numpy's bincount
    adds in index order, as the oracle's map loop does);
  * residual (Sec. 2.2 "Terminate iterations if", reading R10);
  * gradient (footnote of Sec. 2.2, reading R2) and the perturbation of the
    seeds to the lowest gradient in their 3^n box (reading R3).

The last test plants known mistakes in a copy of the oracle source (a float
accumulator, a dropped weight, ...) and checks that a pin fails for each.
"""
import numpy as np
import pytest

import oracle as O


def _coords(size):
    n = len(size)
    grids = np.meshgrid(*[np.arange(s) for s in reversed(size)], indexing="ij")
    return [grids[n - 1 - d].reshape(-1) for d in range(n)]  # x_d per voxel


def brute_assign_fp64(img, centres, grid, m):
    """Every voxel against every centre in double precision, in the order of
    reading R6: dc = ((e_0^2 + e_1^2) + ...), ds = ((t_0 + t_1) + ...),
    t_d = w_d (x_d - c_d)^2 with w_d = m^2 / S_d^2; window (x - S) < c <= (x + S)."""
    n = img.ndim - 1
    size = tuple(reversed(img.shape[:-1]))
    C = img.shape[-1]
    X = _coords(size)
    feat = img.reshape(-1, C).astype(np.float64)
    w = [np.float64(m) * np.float64(m) / (np.float64(S) * np.float64(S)) for S in grid]
    K = centres.shape[0]
    D = np.full((K, feat.shape[0]), np.inf, np.float64)
    for k in range(K):
        c = centres[k]
        e = feat - c[:C]
        dc = e[:, 0] * e[:, 0]
        for ch in range(1, C):
            dc = dc + e[:, ch] * e[:, ch]
        ds = None
        inwin = np.ones(feat.shape[0], bool)
        for d in range(n):
            delta = X[d].astype(np.float64) - c[C + d]
            t = w[d] * (delta * delta)
            ds = t if ds is None else ds + t
            inwin &= ((X[d] - grid[d]).astype(np.float64) < c[C + d]) & (c[C + d] <= (X[d] + grid[d]).astype(np.float64))
        D[k] = np.where(inwin, dc + ds, np.inf)
    lab = np.argmin(D, axis=0).astype(np.int32)   # first minimum: the lowest index wins ties
    lab[np.all(np.isinf(D), axis=0)] = -1
    return lab.reshape(img.shape[:-1])


FLOAT_CASES = [((41,), (5,), 1), ((37,), (4,), 3), ((23,), (6,), 64),
               ((13, 11), (3, 4), 1), ((14, 12), (4, 4), 3), ((12, 10), (4, 3), 64),
               ((9, 7, 5), (3, 3, 2), 3), ((8, 6, 5), (3, 2, 2), 64),
               ((5, 4, 4, 3), (2, 2, 2, 2), 1), ((6, 4, 3, 4), (3, 2, 2, 2), 3)]


def _float_img(size, C, seed):
    rng = np.random.default_rng(seed)
    shape = tuple(reversed(size)) + (C,)
    return rng.uniform(-2.0, 3.0, size=shape).astype(np.float32)


@pytest.mark.parametrize("size,grid,C", FLOAT_CASES)
def test_fp64_assign_brute_force_float_image(size, grid, C):
    img = _float_img(size, C, hash((size, C)) % 2 ** 32)
    rng = np.random.default_rng(5)
    n = len(size)
    p = O.params_for(img, grid, m=float(rng.uniform(0.2, 3.0)), max_iter=1, mode=O.FP64)
    K = O.num_clusters(p)
    for trial in range(3):
        cent = np.zeros((K, C + n))
        cent[:, :C] = rng.uniform(-2.0, 3.0, size=(K, C))
        for d in range(n):
            if trial == 0:   # integer positions and equal features: ties decided by the index
                cent[:, C + d] = rng.integers(0, size[d], size=K)
            else:
                cent[:, C + d] = rng.uniform(-0.5, size[d] - 0.5, size=K)
        if trial == 0:
            cent[:, :C] = cent[0, :C]
        got = O.assign(p, img, cent)
        np.testing.assert_array_equal(got, brute_assign_fp64(img, cent, grid, p.m))


@pytest.mark.parametrize("n,C", [(1, 1), (2, 3), (3, 3), (3, 64), (4, 2)])
def test_fp64_distance_in_the_order_of_r6(n, C):
    """The FP64 D^2 of one voxel and one centre, restated in double in the
    order of reading R6, bit for bit (random features, sub-voxel centres)."""
    rng = np.random.default_rng(n * 100 + C)
    grid = tuple(int(v) for v in rng.integers(2, 9, size=n))
    p = O.Params(size=(40,) * n, grid=grid, channels=C, dtype=O.F32, m=float(rng.uniform(0.1, 20)),
                 max_iter=1, mode=O.FP64)
    w = [np.float64(p.m) * np.float64(p.m) / (np.float64(S) * np.float64(S)) for S in grid]
    for _ in range(50):
        f = rng.uniform(-100, 100, size=C)
        x = rng.integers(0, 40, size=n)
        c = np.concatenate([rng.uniform(-100, 100, size=C), rng.uniform(0, 40, size=n)])
        e = f - c[:C]
        dc = e[0] * e[0]
        for ch in range(1, C):
            dc = dc + e[ch] * e[ch]
        ds = None
        for d in range(n):
            delta = np.float64(x[d]) - c[C + d]
            t = w[d] * (delta * delta)
            ds = t if ds is None else ds + t
        assert O.distance(p, f, x, c) == dc + ds


def _member_mean(img, lab, prev, fp64):
    """Member means accumulated in double in raster order; the FP32 mode
    stores each mean rounded to float; empty clusters keep their centre."""
    n = img.ndim - 1
    size = tuple(reversed(img.shape[:-1]))
    C = img.shape[-1]
    K = prev.shape[0]
    fl = lab.reshape(-1)
    m = fl >= 0
    cnt = np.bincount(fl[m], minlength=K)
    cols = [img[..., c].reshape(-1).astype(np.float64) for c in range(C)] + \
           [x.astype(np.float64) for x in _coords(size)]
    out = prev.copy()
    for j, vals in enumerate(cols):
        s = np.bincount(fl[m], weights=vals[m], minlength=K)
        mean = s / np.maximum(cnt, 1)
        if not fp64:
            mean = mean.astype(np.float32).astype(np.float64)
        out[:, j] = np.where(cnt > 0, mean, prev[:, j])
    return out, cnt


def _residual(prev, new, cnt, C, grid, m):
    """Reading R10: mean over non-empty clusters of sqrt(D^2(C_prev, C_new))
    in double, features first, then positions weighted by m^2 / S_d^2."""
    w = [np.float64(m) * np.float64(m) / (np.float64(S) * np.float64(S)) for S in grid]
    total, nonempty = 0.0, 0
    for k in range(prev.shape[0]):
        if cnt[k] == 0:
            continue
        D2 = 0.0
        for j in range(prev.shape[1]):
            diff = new[k, j] - prev[k, j]
            D2 += diff * diff if j < C else w[j - C] * (diff * diff)
        total += np.sqrt(D2)
        nonempty += 1
    return total / nonempty if nonempty else 0.0


@pytest.mark.parametrize("mode", [O.FP32, O.FP64])
@pytest.mark.parametrize("size,grid,C", [((37,), (4,), 3), ((15, 21), (5, 4), 2), ((9, 8, 7), (3, 3, 2), 5),
                                         ((12, 10), (4, 3), 64)])
def test_update_float_image_is_member_mean(mode, size, grid, C):
    """Float images: features summed in double (reading R9), positions as
    exact integers, one division per component; empty clusters keep their
    previous centre; and the residual of R10 in double."""
    img = _float_img(size, C, 31)
    p = O.params_for(img, grid, m=1.7, max_iter=1, mode=mode)
    K = O.num_clusters(p)
    rng = np.random.default_rng(12)
    lab = rng.integers(-1, K, size=img.shape[:-1]).astype(np.int32)
    lab[lab == 1] = 0                       # cluster 1 empty
    prev = rng.uniform(-2, 3, size=(K, C + len(size)))
    if mode == O.FP32:
        prev = prev.astype(np.float32).astype(np.float64)
    new, counts, res = O.update(p, img, lab, prev)
    expect, cnt = _member_mean(img, lab, prev, mode == O.FP64)
    np.testing.assert_array_equal(counts, cnt)
    np.testing.assert_array_equal(new, expect)
    np.testing.assert_array_equal(new[1], prev[1])
    assert res == _residual(prev, expect, cnt, C, grid, p.m)


def _gradient_field(img, fp64):
    """Reading R2 restated: edge-clamped central differences, summed over
    channels (outer) and axes (inner), left to right; FP32 canonical for the
    FP32 mode (difference and square rounded to float), double otherwise."""
    n = img.ndim - 1
    C = img.shape[-1]
    dt = np.float64 if fp64 else np.float32
    pad = np.pad(img.astype(dt), [(1, 1)] * n + [(0, 0)], mode="edge")
    acc = None
    for c in range(C):
        for d in range(n):
            ax = n - 1 - d
            hi = [slice(1, -1)] * n
            lo = [slice(1, -1)] * n
            hi[ax] = slice(2, None)
            lo[ax] = slice(0, -2)
            diff = pad[tuple(hi) + (c,)] - pad[tuple(lo) + (c,)]
            sq = diff * diff
            if acc is None:
                acc = sq if not fp64 else np.float64(0.0) + sq
            else:
                acc = acc + sq
    return acc.astype(np.float64)


@pytest.mark.parametrize("mode", [O.FP32, O.FP64])
@pytest.mark.parametrize("size,C", [((29,), 3), ((11, 9), 1), ((11, 9), 4), ((7, 6, 5), 3), ((5, 4, 3, 4), 2)])
def test_gradient_float_image(mode, size, C):
    img = _float_img(size, C, 17)
    p = O.params_for(img, (2,) * len(size), max_iter=1, mode=mode)
    field = _gradient_field(img, mode == O.FP64).reshape(-1)
    got = np.array([O.gradient(p, img, q) for q in range(field.size)])
    np.testing.assert_array_equal(got, field)


def _perturbed_seeds(img, grid, fp64):
    n = img.ndim - 1
    size = tuple(reversed(img.shape[:-1]))
    g = _gradient_field(img, fp64)
    ns = [-(-size[d] // grid[d]) for d in range(n)]
    off = [(size[d] - 1 - (ns[d] - 1) * grid[d]) // 2 for d in range(n)]
    rows = []
    for k in range(int(np.prod(ns))):
        j, r = [], k
        for d in range(n):
            j.append(r % ns[d])
            r //= ns[d]
        s = [off[d] + j[d] * grid[d] for d in range(n)]
        best, bg = list(s), g[tuple(reversed(s))]
        for o in np.ndindex(*([3] * n)):
            o = list(reversed([v - 1 for v in o]))  # dimension 0 fastest
            y = [s[d] + o[d] for d in range(n)]
            if any(y[d] < 0 or y[d] >= size[d] for d in range(n)):
                continue
            if g[tuple(reversed(y))] < bg:
                bg, best = g[tuple(reversed(y))], y
        rows.append(list(img[tuple(reversed(best))].astype(np.float64)) + [float(v) for v in best])
    return np.array(rows)


@pytest.mark.parametrize("mode", [O.FP32, O.FP64])
@pytest.mark.parametrize("size,grid,C", [((37,), (4,), 3), ((17, 12), (4, 3), 2), ((9, 8, 7), (3, 3, 2), 3),
                                         ((6, 5, 4, 5), (3, 2, 2, 3), 1)])
def test_perturbation_float_image(mode, size, grid, C):
    img = _float_img(size, C, 23)
    p = O.params_for(img, grid, perturb=True, max_iter=1, mode=mode)
    np.testing.assert_array_equal(O.seed(p, img), _perturbed_seeds(img, grid, mode == O.FP64))


# --------------------------------------------------------------------------
# planted mistakes: each must fail one of the pins above
# --------------------------------------------------------------------------

MUTATIONS = {
    # feature sums of float images kept in float instead of double (R9)
    "float_feature_sum": ("fsum[k * g->C + c] += pix(g, image, q, c);",
                          "fsum[k * g->C + c] = (float)(fsum[k * g->C + c] + pix(g, image, q, c));"),
    # a channel-offset slip in the feature sums
    "feature_sum_channel": ("fsum[k * g->C + c] += pix(g, image, q, c);",
                            "fsum[k * g->C + (c + 1) % g->C] += pix(g, image, q, c);"),
    # FP64 gradient accumulated in float (R2)
    "float_gradient_acc": ("    double acc = 0.0;\n    for (int c = 0; c < g->C; ++c) {",
                           "    float acc = 0.0f;\n    for (int c = 0; c < g->C; ++c) {"),
    # FP64 distance: the feature term squared in float (R6)
    "float_dist64_feature": ("dc = (c == 0) ? e * e : dc + e * e;",
                             "dc = (c == 0) ? (float)(e * e) : dc + (float)(e * e);"),
    # FP64 distance: the spatial weight dropped (Sec. 2.1)
    "dist64_no_weight": ("double t = g->w64[d] * (delta * delta);", "double t = (delta * delta);"),
    # residual: positions not weighted by m^2/S^2 (R10)
    "residual_weight": ("D2 += (j < g->C) ? diff * diff : g->w64[j - g->C] * (diff * diff);",
                        "D2 += diff * diff;"),
}

PIN_OF = {
    "float_feature_sum": lambda: test_update_float_image_is_member_mean(O.FP64, (9, 8, 7), (3, 3, 2), 5),
    "feature_sum_channel": lambda: test_update_float_image_is_member_mean(O.FP32, (15, 21), (5, 4), 2),
    "float_gradient_acc": lambda: test_gradient_float_image(O.FP64, (11, 9), 4),
    "float_dist64_feature": lambda: test_fp64_distance_in_the_order_of_r6(3, 64),
    "dist64_no_weight": lambda: test_fp64_assign_brute_force_float_image((13, 11), (3, 4), 1),
    "residual_weight": lambda: test_update_float_image_is_member_mean(O.FP64, (15, 21), (5, 4), 2),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistakes(name, tmp_path):
    src = O.source_text()
    old, new = MUTATIONS[name]
    assert src.count(old) == 1, f"mutation site of {name} not found exactly once"
    path = O.build_variant(src.replace(old, new), str(tmp_path / name))
    PIN_OF[name]()                       # the real oracle passes the pin
    with O.use_library(path):
        with pytest.raises(AssertionError):
            PIN_OF[name]()
