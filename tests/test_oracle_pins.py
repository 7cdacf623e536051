"""Pins of the CPU oracle against facts fixed by the paper and by mathematics
(arXiv 1806.08741): hand-derived worked cases, closed forms, brute force on
tiny inputs, exact rational arithmetic and invariants.  CPU only."""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _img1d(vals, channels):
    a = np.asarray(vals, dtype=np.uint8)
    return a.reshape(len(vals), channels)


# --------------------------------------------------------------------------
# hand-derived worked cases (tests/golden)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("case", _load("slic_1d_hand.json")["cases"], ids=lambda c: c["name"])
@pytest.mark.parametrize("mode", [O.FP32, O.FP64])
def test_hand_1d(case, mode):
    img = _img1d(case["image"], case["channels"])
    p = O.params_for(img, (case["grid"],), m=case["m"], max_iter=case["max_iter"],
                     perturb=case["perturb"], mode=mode)
    np.testing.assert_array_equal(O.seed(p, img), np.asarray(case["seeds"], float))
    r = O.slic(p, img)
    np.testing.assert_array_equal(r["labels"], case["labels"])
    if mode == O.FP32:
        np.testing.assert_array_equal(r["centres"], np.asarray(case["centres"], float))
    else:
        np.testing.assert_allclose(r["centres"], np.asarray(case["centres"], float), rtol=1e-7)
    if "residual" in case:
        assert r["residual"] == pytest.approx(case["residual"], abs=1e-12)
    else:
        assert r["residual"] == pytest.approx(case["residual_approx"], rel=1e-6)


@pytest.mark.parametrize("case", _load("perturb_1d_hand.json")["cases"], ids=lambda c: c["name"])
def test_hand_perturbation(case):
    img = _img1d(case["image"], 1)
    p = O.params_for(img, (case["grid"],), perturb=True, max_iter=1)
    for q, g in case["gradients"].items():
        assert O.gradient(p, img, int(q)) == g
    np.testing.assert_array_equal(O.seed(p, img), np.asarray(case["seeds"], float))


@pytest.mark.parametrize("case", _load("connectivity_2d_hand.json")["cases"],
                         ids=lambda c: c["name"])
def test_hand_connectivity(case):
    lab = np.asarray(case["labels"], np.int32)
    H, W = lab.shape
    p = O.Params(size=(W, H), grid=tuple(case["grid"]), channels=1, dtype=O.U8)
    centres = np.array([[0.0, x, y] for x, y in case["centres_xy"]])
    out, n = O.connectivity(p, centres, lab)
    np.testing.assert_array_equal(out, np.asarray(case["expected"], np.int32))
    assert n == case["num_labels"]


# --------------------------------------------------------------------------
# distance: exact rational arithmetic of Sec. 2.1 / Sec. 3.3
# --------------------------------------------------------------------------

def test_distance_against_exact_rationals():
    rng = np.random.default_rng(5)
    for n in (1, 2, 3):
        for C in (1, 3, 5):
            size = (40, 30, 20)[:n]
            grid = tuple(int(s) for s in rng.integers(1, 20, size=n))
            m = float(np.float32(rng.uniform(0.5, 40)))
            p = O.Params(size=size, grid=grid, channels=C, dtype=O.U16, m=m)
            for _ in range(20):
                f = rng.integers(0, 65536, size=C).astype(float)
                x = np.array([rng.integers(0, s) for s in size])
                c = np.concatenate([np.float32(rng.uniform(0, 65535, size=C)),
                                    np.float32(rng.uniform(0, 40, size=n))]).astype(float)
                exact = sum((Fraction(fi) - Fraction(ci)) ** 2 for fi, ci in zip(f, c[:C]))
                exact += sum((Fraction(int(xi)) - Fraction(ci)) ** 2 * Fraction(m) ** 2
                             / Fraction(g) ** 2 for xi, ci, g in zip(x, c[C:], grid))
                p.mode = O.FP64
                d64 = O.distance(p, f, x, c)
                assert abs(Fraction(d64) - exact) <= abs(exact) * Fraction(1, 10 ** 12)
                p.mode = O.FP32
                d32 = O.distance(p, f, x, c)
                # (C + 2n + ...) single-precision roundings
                assert abs(Fraction(d32) - exact) <= abs(exact) * Fraction(4 * (C + 3 * n), 2 ** 24) + Fraction(1, 10 ** 30)


def test_distance_weight_anisotropic():
    """Sec. 3.3: each axis is divided by its own S_i."""
    p = O.Params(size=(10, 10, 10), grid=(2, 4, 8), channels=1, dtype=O.U8, m=8.0, mode=O.FP64)
    # unit offset along each axis contributes m^2/S_i^2
    for d, S in enumerate((2, 4, 8)):
        x = np.zeros(3, np.int64)
        x[d] = 1
        assert O.distance(p, [0.0], x, [0.0, 0.0, 0.0, 0.0]) == pytest.approx(64.0 / S ** 2)
    assert O.distance(p, [3.0], [0, 0, 0], [7.0, 0, 0, 0]) == 16.0


# --------------------------------------------------------------------------
# brute force: every voxel against every centre, masked by the window
# --------------------------------------------------------------------------

def _coords(size):
    n = len(size)
    grids = np.meshgrid(*[np.arange(s) for s in reversed(size)], indexing="ij")
    return [grids[n - 1 - d].reshape(-1) for d in range(n)]  # x_d per voxel


def brute_assign_fp32(img, centres, grid, m):
    """Exhaustive voxel-centric argmin in float32 (one rounding per op),
    masked by c - S <= x < c + S; ties to the lowest index (np.argmin)."""
    n = img.ndim - 1
    size = tuple(reversed(img.shape[:-1]))
    C = img.shape[-1]
    X = _coords(size)
    feat = img.reshape(-1, C).astype(np.float32)
    w = [np.float32(np.float64(m) * np.float64(m) / (np.float64(S) * np.float64(S))) for S in grid]
    K = centres.shape[0]
    D = np.full((K, feat.shape[0]), np.inf, np.float32)
    for k in range(K):
        cf = centres[k].astype(np.float32)
        e = feat - cf[:C]
        sq = e * e
        dc = sq[:, 0]
        for c in range(1, C):
            dc = dc + sq[:, c]
        ds = None
        inwin = np.ones(feat.shape[0], bool)
        for d in range(n):
            xd = X[d].astype(np.float32)
            delta = xd - cf[C + d]
            t = w[d] * (delta * delta)
            ds = t if ds is None else ds + t
            inwin &= ((X[d] - grid[d]).astype(np.float32) < cf[C + d]) & \
                     (cf[C + d] <= (X[d] + grid[d]).astype(np.float32))
        D[k] = np.where(inwin, dc + ds, np.inf)
    lab = np.argmin(D, axis=0).astype(np.int32)
    lab[np.all(np.isinf(D), axis=0)] = -1
    return lab.reshape(img.shape[:-1])


CASES = [((37,), (5,), 1), ((37,), (4,), 3), ((13, 11), (3, 4), 1), ((13, 11), (4, 4), 3),
         ((9, 7, 5), (3, 3, 2), 1), ((9, 7, 5), (2, 3, 4), 3),
         ((5, 4, 4, 3), (2, 2, 2, 2), 1), ((6, 4, 3, 4), (3, 2, 2, 2), 3)]


@pytest.mark.parametrize("size,grid,C", CASES)
@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_assign_brute_force(size, grid, C, dtype):
    rng = np.random.default_rng(hash((size, grid, C)) % 2 ** 32)
    shape = tuple(reversed(size)) + (C,)
    hi = 256 if dtype == np.uint8 else 65536
    img = rng.integers(0, hi, size=shape).astype(dtype)
    p = O.params_for(img, grid, m=float(np.float32(rng.uniform(1, 40))), max_iter=1)
    K = O.num_clusters(p)
    n = len(size)
    for trial in range(3):
        cent = np.zeros((K, C + n))
        cent[:, :C] = np.float32(rng.uniform(0, hi, size=(K, C)))
        for d in range(n):
            if trial == 0:   # integer positions: many exact ties
                cent[:, C + d] = rng.integers(0, size[d], size=K)
            else:
                cent[:, C + d] = np.float32(rng.uniform(-0.5, size[d] - 0.5, size=K))
        if trial == 0:       # equal features too: ties decided by index only
            cent[:, :C] = cent[0, :C]
        got = O.assign(p, img, cent)
        np.testing.assert_array_equal(got, brute_assign_fp32(img, cent, grid, p.m))


def test_window_is_exactly_2S():
    """Sec. 2.2: a centre reaches 2S voxels per axis whatever its sub-voxel
    position; other centres far away leave those voxels to it."""
    img = np.zeros((1, 64, 1), np.uint8)[0]
    p = O.params_for(img, (5,), m=1.0, max_iter=1)
    K = O.num_clusters(p)
    for c in (20.0, 20.25, 20.5, 20.999, 21.0):
        cent = np.full((K, 2), 0.0)
        cent[:, 1] = 1000.0          # unreachable
        cent[0, 1] = c
        lab = O.assign(p, img, cent)
        covered = np.flatnonzero(lab == 0)
        assert len(covered) == 10
        assert covered[0] == int(np.ceil(c - 5)) and covered[-1] == int(np.ceil(c + 5)) - 1


# --------------------------------------------------------------------------
# gradient and perturbation
# --------------------------------------------------------------------------

def test_gradient_linear_ramp_closed_form():
    """I = a x + b y (+ c z): interior gradient^2 = sum_d (2 a_d)^2; at a
    clamped border the difference spans one voxel: a_d^2."""
    a = (3, 5, 7)
    for n in (1, 2, 3):
        size = (6, 5, 4)[:n]
        X = _coords(size)
        val = sum(a[d] * X[d] for d in range(n)).astype(np.uint16)
        img = val.reshape(tuple(reversed(size)) + (1,))
        p = O.params_for(img, (2,), max_iter=1)
        for q in range(int(np.prod(size))):
            x = [X[d][q] for d in range(n)]
            expect = sum((2 * a[d]) ** 2 if 0 < x[d] < size[d] - 1 else a[d] ** 2 for d in range(n))
            assert O.gradient(p, img, q) == expect


def test_gradient_frobenius_over_channels():
    """Footnote of Sec. 2.2: multi-channel uses the Frobenius norm of the
    Jacobian, i.e. the per-channel squared gradients add."""
    rng = np.random.default_rng(1)
    img = rng.integers(0, 256, size=(6, 7, 3)).astype(np.uint8)
    p = O.params_for(img, (3,), max_iter=1)
    for q in range(42):
        tot = sum(O.gradient(O.params_for(img[..., c:c + 1].copy(), (3,), max_iter=1),
                             img[..., c:c + 1].copy(), q) for c in range(3))
        assert O.gradient(p, img, q) == tot


def brute_perturbed_seeds(img, grid):
    """Independent restatement: numpy edge-padded central differences and a
    3^n argmin with the seed as first candidate."""
    n = img.ndim - 1
    size = tuple(reversed(img.shape[:-1]))
    pad = np.pad(img.astype(np.int64), [(1, 1)] * n + [(0, 0)], mode="edge")
    g = np.zeros(img.shape[:-1], np.int64)
    for d in range(n):
        ax = n - 1 - d
        sl_hi = [slice(1, -1)] * n
        sl_lo = [slice(1, -1)] * n
        sl_hi[ax] = slice(2, None)
        sl_lo[ax] = slice(0, -2)
        diff = pad[tuple(sl_hi)] - pad[tuple(sl_lo)]
        g += (diff * diff).sum(axis=-1)
    ns = [-(-size[d] // grid[d]) for d in range(n)]
    off = [(size[d] - 1 - (ns[d] - 1) * grid[d]) // 2 for d in range(n)]
    seeds = []
    for k in range(int(np.prod(ns))):
        j = []
        r = k
        for d in range(n):
            j.append(r % ns[d])
            r //= ns[d]
        s = [off[d] + j[d] * grid[d] for d in range(n)]
        best = list(s)
        bg = g[tuple(reversed(best))]
        for o in np.ndindex(*([3] * n)):
            o = list(reversed([v - 1 for v in o]))  # dimension 0 fastest
            y = [s[d] + o[d] for d in range(n)]
            if any(y[d] < 0 or y[d] >= size[d] for d in range(n)):
                continue
            gy = g[tuple(reversed(y))]
            if gy < bg:
                bg, best = gy, y
        seeds.append(list(img[tuple(reversed(best))].astype(float)) + [float(v) for v in best])
    return np.array(seeds)


@pytest.mark.parametrize("size,grid", [((37,), (4,)), ((17, 12), (4, 3)), ((9, 8, 7), (3, 3, 2)),
                                       ((6, 5, 4, 5), (3, 2, 2, 3))])
def test_perturbation_brute_force(size, grid):
    rng = np.random.default_rng(7)
    img = rng.integers(0, 256, size=tuple(reversed(size)) + (3,)).astype(np.uint8)
    p = O.params_for(img, grid, perturb=True, max_iter=1)
    np.testing.assert_array_equal(O.seed(p, img), brute_perturbed_seeds(img, grid))


def test_seed_lattice_counts():
    """K = prod ceil(N_d/S_d); the 3-D cryosection-volume workload gives the
    ~1.14M supervoxels of its recipe."""
    p = O.Params(size=(2048, 1216, 1871), grid=(16, 16, 16))
    assert O.num_clusters(p) == 128 * 76 * 117 == 1138176
    assert O.num_clusters(O.Params(size=(2048, 1216), grid=(16, 16))) == 9728
    assert O.num_clusters(O.Params(size=(256, 256), grid=(16, 16))) == 256


# --------------------------------------------------------------------------
# closed form: constant image
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 3, 4])
@pytest.mark.parametrize("S", [1, 2, 3, 16])
@pytest.mark.parametrize("C", [1, 3])
def test_constant_image_fixed_point(n, S, C):
    cells = {1: (5,), 2: (4, 3), 3: (3, 2, 2), 4: (2, 2, 1, 2)}[n]
    if S == 16 and n == 3:
        cells = (2, 2, 1)
    if S == 16 and n == 4:
        cells = (1, 2, 1, 1)
    size = tuple(c * S for c in cells)
    img = np.full(tuple(reversed(size)) + (C,), 77, np.uint8)
    p = O.params_for(img, (S,), m=10.0, max_iter=3, perturb=True, enforce_connectivity=True)
    K = O.num_clusters(p)
    assert K == int(np.prod(cells))
    seeds = O.seed(p, img)
    o = (S - 1) // 2
    r = O.slic(p, img)
    X = _coords(size)
    # first assignment = grid cells (ties on a cell's upper edge go to the lower k)
    cell_of = np.zeros(int(np.prod(size)), np.int64)
    mul = 1
    for d in range(n):
        cell_of += (X[d] // S) * mul
        mul *= cells[d]
    np.testing.assert_array_equal(r["labels"].reshape(-1), cell_of)
    for k in range(K):
        j = []
        rr = k
        for d in range(n):
            j.append(rr % cells[d])
            rr //= cells[d]
        assert list(seeds[k, C:]) == [o + j[d] * S for d in range(n)]
        assert list(r["centres"][k, :C]) == [77.0] * C
        assert list(r["centres"][k, C:]) == [(j[d] + 0.5) * S - 0.5 for d in range(n)]
    assert r["num_labels"] == K
    # fixed point: one more run from the result gives identical output, residual 0
    p2 = O.params_for(img, (S,), m=10.0, max_iter=2, perturb=True)
    r2 = O.slic(p2, img, init_centres=r["centres"])
    np.testing.assert_array_equal(r2["labels"], r["labels"])
    np.testing.assert_array_equal(r2["centres"], r["centres"])
    assert r2["residual"] == 0.0


def test_single_cluster():
    """K = 1: label 0 wherever the window covers, -1 elsewhere."""
    img = np.zeros((1, 30, 1), np.uint8)[0]
    p = O.params_for(img, (40,), m=5.0, max_iter=1, perturb=False)
    assert O.num_clusters(p) == 1
    cent = np.array([[0.0, 3.0]])
    lab = O.assign(p, img, cent)
    expect = np.where(np.arange(30) < 3 + 40, 0, -1)
    np.testing.assert_array_equal(lab, expect)
    cent = np.array([[0.0, 29.0]])
    p = O.params_for(img, (10,), m=5.0, max_iter=1, perturb=False)
    K = O.num_clusters(p)
    cent = np.tile(np.array([[0.0, 1000.0]]), (K, 1))
    cent[0, 1] = 5.0
    lab = O.assign(p, img, cent)
    np.testing.assert_array_equal(lab, np.where(np.arange(30) < 15, 0, -1))


def test_large_grid_one_seed_per_axis():
    img = np.random.default_rng(0).integers(0, 256, size=(7, 9, 2)).astype(np.uint8)
    p = O.params_for(img, (50,), max_iter=2, perturb=False)
    assert O.num_clusters(p) == 1
    r = O.slic(p, img)
    assert (r["labels"] == 0).all()
    np.testing.assert_array_equal(r["centres"][0, :2], img.reshape(-1, 2).mean(0).astype(np.float32))
    assert list(r["centres"][0, 2:]) == [4.0, 3.0]


def test_constant_image_is_windowed_voronoi():
    """d_c = 0 on a constant image, so the labels are the nearest centre in the
    weighted index metric among the covering windows (integer positions make
    the comparison exact)."""
    rng = np.random.default_rng(3)
    size = (23, 19)
    img = np.full((19, 23, 3), 9, np.uint8)
    grid = (5, 4)
    p = O.params_for(img, grid, m=7.0, max_iter=1)
    K = O.num_clusters(p)
    cent = np.zeros((K, 5))
    cent[:, :3] = 9.0
    cent[:, 3] = rng.integers(0, size[0], size=K)
    cent[:, 4] = rng.integers(0, size[1], size=K)
    lab = O.assign(p, img, cent).reshape(-1)
    X = _coords(size)
    w = [Fraction(49, g * g) for g in grid]
    for q in range(len(lab)):
        best, bk = None, -1
        for k in range(K):
            if all(cent[k, 3 + d] - grid[d] <= X[d][q] < cent[k, 3 + d] + grid[d] for d in range(2)):
                dd = sum(w[d] * int(X[d][q] - cent[k, 3 + d]) ** 2 for d in range(2))
                if best is None or dd < best:
                    best, bk = dd, k
        assert lab[q] == bk


# --------------------------------------------------------------------------
# update and whole-run invariants
# --------------------------------------------------------------------------

def test_update_is_member_mean():
    rng = np.random.default_rng(11)
    img = rng.integers(0, 65536, size=(15, 21, 2)).astype(np.uint16)
    p = O.params_for(img, (5,), max_iter=1)
    K = O.num_clusters(p)
    lab = rng.integers(-1, K, size=img.shape[:-1]).astype(np.int32)
    lab[lab == 3] = 4                       # cluster 3 empty: keeps its centre
    prev = rng.uniform(0, 100, size=(K, 4)).astype(np.float32).astype(float)
    new, counts, _ = O.update(p, img, lab, prev)
    X = _coords((21, 15))
    fl = lab.reshape(-1)
    m = fl >= 0
    cnt = np.bincount(fl[m], minlength=K)
    np.testing.assert_array_equal(counts, cnt)
    for j, vals in enumerate([img[..., 0].reshape(-1), img[..., 1].reshape(-1), X[0], X[1]]):
        s = np.bincount(fl[m], weights=vals[m].astype(np.float64), minlength=K)
        expect = np.where(cnt > 0, (s / np.maximum(cnt, 1)).astype(np.float32), prev[:, j])
        np.testing.assert_array_equal(new[:, j], expect)


def _run_invariants(img, grid, m, iters, mode=O.FP32):
    p = O.params_for(img, grid, m=m, max_iter=iters, mode=mode)
    r_prev = O.slic(O.params_for(img, grid, m=m, max_iter=iters - 1, mode=mode), img) if iters > 1 else None
    r = O.slic(p, img)
    C = img.shape[-1]
    n = img.ndim - 1
    size = tuple(reversed(img.shape[:-1]))
    lab = r["labels"].reshape(-1)
    K = O.num_clusters(p)
    # I1: output centres are the member means of the output labels
    X = _coords(size)
    cnt = np.bincount(lab[lab >= 0], minlength=K)
    for j in range(C + n):
        vals = img.reshape(-1, C)[:, j] if j < C else X[j - C]
        s = np.bincount(lab[lab >= 0], weights=vals[lab >= 0].astype(np.float64), minlength=K)
        nz = cnt > 0
        np.testing.assert_array_equal(r["centres"][nz, j], (s[nz] / cnt[nz]).astype(np.float32))
    # I2-I4 against the centres used by the last assignment
    cprev = r_prev["centres"]
    np.testing.assert_array_equal(r["labels"], brute_assign_fp32(img, cprev, grid, m))
    assert (lab >= 0).all()
    return r


def test_invariants_small_2d():
    rng = np.random.default_rng(21)
    img = rng.integers(0, 256, size=(40, 48, 3)).astype(np.uint8)
    _run_invariants(img, (8, 8), 10.0, 4)


def test_invariants_small_3d():
    rng = np.random.default_rng(22)
    img = rng.integers(0, 256, size=(10, 12, 14, 3)).astype(np.uint8)
    _run_invariants(img, (4, 4, 4), 10.0, 3)


def test_resume_equals_uninterrupted():
    """State after t iterations is the centre table: 5 + 5 == 10."""
    rng = np.random.default_rng(4)
    img = rng.integers(0, 256, size=(48, 64, 3)).astype(np.uint8)
    full = O.slic(O.params_for(img, (8,), max_iter=10), img)
    half = O.slic(O.params_for(img, (8,), max_iter=5), img)
    rest = O.slic(O.params_for(img, (8,), max_iter=5), img, init_centres=half["centres"])
    np.testing.assert_array_equal(rest["labels"], full["labels"])
    np.testing.assert_array_equal(rest["centres"], full["centres"])


def test_threshold_stops_early():
    img = np.full((32, 32, 1), 50, np.uint8)
    r = O.slic(O.params_for(img, (8,), max_iter=10, conv_threshold=1e-9), img)
    assert r["iterations"] == 2 and r["residual"] == 0.0
    r = O.slic(O.params_for(img, (8,), max_iter=10, conv_threshold=0.0), img)
    assert r["iterations"] == 10


def test_fp32_and_fp64_modes_agree_on_float_image():
    rng = np.random.default_rng(8)
    img = rng.uniform(0, 1, size=(40, 40, 4)).astype(np.float32)
    a = O.slic(O.params_for(img, (8,), m=0.5, max_iter=3, mode=O.FP32), img)
    b = O.slic(O.params_for(img, (8,), m=0.5, max_iter=3, mode=O.FP64), img)
    assert (a["labels"] == b["labels"]).mean() > 0.99
    np.testing.assert_allclose(a["centres"], b["centres"], rtol=1e-3, atol=1e-3)


def test_bad_params_rejected():
    img = np.zeros((4, 4, 1), np.uint8)
    with pytest.raises(RuntimeError):
        O.slic(O.params_for(img, (0,)), img)
    with pytest.raises(RuntimeError):
        O.slic(O.params_for(img, (2,), m=0.0), img)
    with pytest.raises(RuntimeError):
        O.slic(O.params_for(img, (2,), max_iter=0), img)


# --------------------------------------------------------------------------
# connectivity invariants (independent CCL from scipy)
# --------------------------------------------------------------------------

def _ccl(labels):
    from scipy import ndimage
    n = labels.ndim
    struct = ndimage.generate_binary_structure(n, 1)
    comp = np.zeros(labels.shape, np.int64)
    total = 0
    for v in np.unique(labels):
        c, k = ndimage.label(labels == v, structure=struct)
        comp[c > 0] = c[c > 0] + total
        total += k
    return comp, total


@pytest.mark.parametrize("seed", range(6))
def test_connectivity_invariants(seed):
    rng = np.random.default_rng(100 + seed)
    n = (2, 3, 4)[seed % 3]
    size = {2: (30, 26), 3: (14, 12, 10), 4: (9, 8, 7, 6)}[n]
    grid = {2: (6, 6), 3: (4, 4, 3), 4: (3, 3, 3, 2)}[n]
    img = rng.integers(0, 256, size=tuple(reversed(size)) + (3,)).astype(np.uint8)
    p = O.params_for(img, grid, m=2.0, max_iter=3, enforce_connectivity=False)
    r = O.slic(p, img)
    out, nlab = O.connectivity(p, r["centres"], r["labels"])
    K = O.num_clusters(p)
    sprod = int(np.prod(grid))
    assert out.min() >= 0 and out.max() < nlab
    # every output label is one face-connected region
    comp, ncomp = _ccl(out)
    assert ncomp == len(np.unique(out))
    # every region is larger than prod(S)/4 unless it holds the origin
    flat = out.reshape(-1)
    for v in np.unique(flat):
        size_v = int((flat == v).sum())
        assert 4 * size_v > sprod or flat[0] == v
    # new labels are K, K+1, ... with none skipped
    newl = sorted(set(np.unique(flat)) - set(range(K)))
    assert newl == list(range(K, nlab))
    # the pre-relabel components that survive keep their label
    incomp, _ = _ccl(r["labels"])
    for c in np.unique(incomp):
        msk = incomp == c
        vals = np.unique(out[msk])
        assert len(vals) == 1       # components are relabelled as a whole


# --------------------------------------------------------------------------
# CIE-Lab conversion (reading R16)
# --------------------------------------------------------------------------

def _cube():
    v = np.arange(256)
    return np.stack(np.meshgrid(v, v, v, indexing="ij"), -1).reshape(-1, 3).astype(np.uint8)


def test_lab_ranges_are_the_papers():
    # The extremes over every 8-bit colour are the ranges Sec. 2.1 prints (to
    # its three decimals: the last digit may be cut rather than rounded).
    ref = _load("lab_ranges_paper.json")
    lab = O.srgb_to_lab(_cube())
    lo, hi = lab.min(0), lab.max(0)
    for j, ch in enumerate("Lab"):
        assert abs(lo[j] - ref[ch][0]) <= 1e-3, (ch, lo[j])
        assert abs(hi[j] - ref[ch][1]) <= 1e-3, (ch, hi[j])
    # black and white are the ends of the L axis exactly (the Y row of the
    # sRGB matrix sums to 1)
    bw = O.srgb_to_lab(np.array([[0, 0, 0], [255, 255, 255]], np.uint8))
    assert bw[0].tolist() == [0.0, 0.0, 0.0]
    assert abs(bw[1, 0] - 100.0) < 1e-12


def test_lab_round_trip_through_the_textbook_inverse():
    # Invert Lab -> XYZ -> linear RGB -> sRGB code with the inverse
    # definitions (written here independently of the oracle's forward code);
    # every code must come back to within rounding.
    rng = np.random.default_rng(7)
    rgb = rng.integers(0, 256, size=(20000, 3), dtype=np.uint8)
    lab = O.srgb_to_lab(rgb)
    d = 6.0 / 29.0
    fy = (lab[:, 0] + 16.0) / 116.0
    fx = fy + lab[:, 1] / 500.0
    fz = fy - lab[:, 2] / 200.0

    def finv(f):
        return np.where(f > d, f ** 3, 3.0 * d * d * (f - 4.0 / 29.0))

    xyz = np.stack([finv(fx) * 0.95047, finv(fy), finv(fz) * 1.08883], -1)
    m = np.array([[0.4124, 0.3576, 0.1805], [0.2126, 0.7152, 0.0722], [0.0193, 0.1192, 0.9505]])
    lin = np.linalg.solve(m, xyz.T).T
    enc = np.where(lin <= 0.0031308, 12.92 * lin, 1.055 * np.abs(lin) ** (1 / 2.4) - 0.055)
    np.testing.assert_allclose(enc * 255.0, rgb.astype(np.float64), atol=1e-6)


def test_lab_grey_axis():
    # Greys lie on the L axis (a, b within the 4e-5 gap between the D65 white
    # and the matrix's row sums) and L rises with the code value.
    v = np.arange(256, dtype=np.uint8)
    lab = O.srgb_to_lab(np.stack([v, v, v], -1))
    assert np.all(np.diff(lab[:, 0]) > 0)
    assert np.abs(lab[:, 1:]).max() < 0.02


# --------------------------------------------------------------------------
# assignment at chosen voxels (for sampling images too large to assign whole)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("size,grid,C,mode", [((61,), (4,), 2, O.FP32), ((40, 33), (6, 5), 3, O.FP32),
                                              ((20, 17, 13), (4, 5, 3), 1, O.FP64),
                                              ((24, 18, 16), (8, 8, 8), 3, O.FP32),
                                              ((9, 8, 7, 6), (3, 3, 2, 3), 2, O.FP32)])
def test_assign_voxels_equals_assign(size, grid, C, mode):
    import _lattice
    rng = np.random.default_rng(sum(size))
    img = rng.integers(0, 256, size=tuple(reversed(size)) + (C,), dtype=np.uint8)
    p = O.params_for(img, grid, m=7.0, max_iter=2, mode=mode)
    seeds = O.seed(p, img)
    K = seeds.shape[0]
    V = int(np.prod(size))
    want = O.assign(p, img, seeds).reshape(-1)
    q = np.arange(V, dtype=np.int64)
    # every centre as a candidate, listed in a shuffled order
    start = np.arange(V + 1, dtype=np.int64) * K
    cand = np.concatenate([rng.permutation(K) for _ in range(V)])
    np.testing.assert_array_equal(O.assign_voxels(p, img, seeds, q, start, cand), want)
    # the lattice superset of the seeds that can cover each voxel
    start, cand = _lattice.seed_candidates(size, grid, q)
    np.testing.assert_array_equal(O.assign_voxels(p, img, seeds, q, start, cand), want)
    # and after an update (centres anywhere): with every centre listed
    cen, _, _ = O.update(p, img, want.reshape(img.shape[:-1]), seeds)
    start = np.arange(V + 1, dtype=np.int64) * K
    cand = np.tile(np.arange(K), V)
    np.testing.assert_array_equal(O.assign_voxels(p, img, cen, q, start, cand),
                                  O.assign(p, img, cen).reshape(-1))
