"""Parity of the CUDA path (through the C ABI) with the CPU oracle, step by
step and end to end.  Integer images: labels and centres bit-exact.  Float
images: labels equal to the FP32-canonical oracle for one iteration from the
same centres; against the FP64 oracle over a whole run, label agreement
>= 99.99 % and centre relative error <= 1e-5."""
import numpy as np
import pytest

import oracle as O
from paper_1806_08741_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch


def _S():
    from paper_1806_08741_gb300 import sslic as S
    return S


def _dev(a):
    torch = _torch()
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _gpu_seed(img, grid, **kw):
    torch, S = _torch(), _S()
    p = S.params_for(img, grid, **kw)
    with S.Context(p) as ctx:
        out = torch.empty((ctx.K, ctx.centre_width), dtype=torch.float32, device="cuda")
        ctx.seed(_dev(img), out)
        torch.cuda.synchronize()
        return out.cpu().numpy().astype(np.float64)


def _gpu_iterate(img, grid, centres, m=10.0):
    torch, S = _torch(), _S()
    p = S.params_for(img, grid, m=m, max_iter=1)
    with S.Context(p) as ctx:
        cin = _dev(centres.astype(np.float32))
        lab = torch.empty(img.shape[:-1], dtype=torch.int32, device="cuda")
        cout = torch.empty_like(cin)
        res = ctx.iterate(_dev(img), cin, lab, cout, residual=True)
        return lab.cpu().numpy(), cout.cpu().numpy().astype(np.float64), res


def _gpu_run(img, grid, **kw):
    torch, S = _torch(), _S()
    p = S.params_for(img, grid, **kw)
    with S.Context(p) as ctx:
        lab = torch.empty(img.shape[:-1], dtype=torch.int32, device="cuda")
        cen = torch.empty((ctx.K, ctx.centre_width), dtype=torch.float32, device="cuda")
        info = ctx.run(_dev(img), lab, cen)
        return lab.cpu().numpy(), cen.cpu().numpy().astype(np.float64), info


def _rand_img(shape, dtype, seed):
    rng = np.random.default_rng(seed)
    if dtype == np.float32:
        return rng.uniform(0, 1, size=shape).astype(np.float32)
    hi = 256 if dtype == np.uint8 else 65536
    return rng.integers(0, hi, size=shape).astype(dtype)


def _synth(size, C=3, dtype="u8", regions=None, sigma=6, seed=5, ramp=0):
    V = int(np.prod(size))
    regions = regions or max(2, V // 4000)
    return I.make_image(I.ImageSpec(tuple(size), C, dtype, seed, regions, sigma, ramp))


# ---------------------------------------------------------------------------
# a1 / a2: seeding and perturbation
# ---------------------------------------------------------------------------
SEED_CASES = [
    ("2d_rgb", lambda: _synth((256, 256)), (16, 16)),
    ("2d_ragged", lambda: _synth((203, 150)), (16, 16)),
    ("3d_rgb", lambda: _synth((70, 50, 37)), (8, 8, 8)),
    ("3d_aniso_u16", lambda: _synth((64, 40, 30), 1, "u16", sigma=300), (16, 8, 4)),
    ("1d", lambda: _synth((1000,), 3), (7,)),
    ("2d_f32_c4", lambda: _rand_img((60, 70, 4), np.float32, 3), (6, 6)),
    ("2d_u8_c2", lambda: _rand_img((40, 50, 2), np.uint8, 4), (5, 5)),
]


@pytest.mark.parametrize("name,mk,grid", SEED_CASES, ids=[c[0] for c in SEED_CASES])
@pytest.mark.parametrize("perturb", [True, False])
def test_seed_parity(name, mk, grid, perturb):
    img = mk()
    ref = O.seed(O.params_for(img, grid, perturb=perturb, max_iter=1), img)
    got = _gpu_seed(img, grid, perturb=perturb)
    np.testing.assert_array_equal(got, ref)


# ---------------------------------------------------------------------------
# a3 / a4: one assignment + update from the same centres
# ---------------------------------------------------------------------------
ITER_CASES = [
    ("2d_256", lambda: _synth((256, 256), regions=32, sigma=8), (16, 16), 10.0),
    ("2d_ragged", lambda: _synth((203, 150)), (16, 16), 10.0),
    ("2d_S8", lambda: _synth((190, 130)), (8, 8), 10.0),
    ("2d_S32", lambda: _synth((300, 260)), (32, 32), 20.0),
    ("3d_S16", lambda: _synth((96, 80, 48)), (16, 16, 16), 10.0),
    ("3d_ragged_S8", lambda: _synth((70, 50, 37)), (8, 8, 8), 10.0),
    ("3d_small_S_overflow", lambda: _synth((40, 30, 20)), (3, 3, 3), 5.0),
    ("3d_aniso", lambda: _synth((80, 48, 30)), (16, 8, 4), 10.0),
    # rows a multiple of 16 bytes (TMA-staged tiles), ragged along y and z
    ("3d_tma_ragged", lambda: _synth((45, 37, 64)), (16, 16, 16), 10.0),
    ("2d_tma_ragged", lambda: _synth((150, 208)), (16, 16), 10.0),
    ("3d_u16_tma", lambda: _synth((40, 24, 32), 1, "u16", sigma=300), (8, 8, 8), 10.0),
    ("3d_u16", lambda: _synth((64, 40, 30), 1, "u16", sigma=300), (8, 8, 8), 10.0),
    ("2d_gray_u8", lambda: _synth((150, 100), 1), (10, 10), 5.0),
    ("1d", lambda: _synth((1000,), 3), (7,), 10.0),
    ("2d_u8_c2_generic", lambda: _rand_img((40, 50, 2), np.uint8, 4), (5, 5), 10.0),
    ("2d_f32_c4", lambda: _rand_img((60, 70, 4), np.float32, 3), (6, 6), 0.5),
    ("2d_f32_c32_tile", lambda: _rand_img((70, 53, 32), np.float32, 5), (8, 8), 0.5),
    ("3d_f32_c16_tile", lambda: _rand_img((20, 19, 11, 16), np.float32, 6), (5, 5, 5), 0.5),
]


@pytest.mark.parametrize("name,mk,grid,m", ITER_CASES, ids=[c[0] for c in ITER_CASES])
@pytest.mark.parametrize("after", [0, 3])
def test_iterate_parity(name, mk, grid, m, after):
    img = mk()
    p = O.params_for(img, grid, m=m, max_iter=max(after, 1), perturb=True)
    cen = O.seed(p, img) if after == 0 else O.slic(p, img)["centres"]
    ref_lab = O.assign(p, img, cen)
    ref_cen, _, ref_res = O.update(p, img, ref_lab, cen)
    lab, got_cen, res = _gpu_iterate(img, grid, cen, m=m)
    np.testing.assert_array_equal(lab, ref_lab)
    if img.dtype == np.float32:
        # float sums are FP32 block partials added in FP64 (reading R9): the
        # centres, and the residual computed from them, carry that rounding
        np.testing.assert_allclose(got_cen, ref_cen, rtol=1e-6, atol=1e-6)
        assert res == pytest.approx(ref_res, rel=1e-6, abs=1e-9)
    else:
        np.testing.assert_array_equal(got_cen, ref_cen)
        assert res == pytest.approx(ref_res, rel=1e-9, abs=1e-12)


def _gpu_iterate_shape(img, grid, centres, m, shape):
    torch, S = _torch(), _S()
    p = S.params_for(img, grid, m=m, max_iter=1)
    with S.Context(p) as ctx:
        ctx.tile_shape = shape
        assert ctx.tile_shape == shape
        cin = _dev(centres.astype(np.float32))
        lab = torch.empty(img.shape[:-1], dtype=torch.int32, device="cuda")
        cout = torch.empty_like(cin)
        ctx.iterate(_dev(img), cin, lab, cout)
        return lab.cpu().numpy(), cout.cpu().numpy().astype(np.float64)


SHAPE_CASES = [c for c in ITER_CASES if c[0] in
               ("2d_256", "2d_ragged", "2d_S8", "3d_S16", "3d_ragged_S8", "3d_small_S_overflow", "3d_aniso",
                "3d_u16", "2d_gray_u8", "3d_tma_ragged", "2d_tma_ragged", "3d_u16_tma")]


@pytest.mark.parametrize("name,mk,grid,m", SHAPE_CASES, ids=[c[0] for c in SHAPE_CASES])
def test_every_tile_shape_is_exact(name, mk, grid, m):
    """Every tile extent and voxels-per-lane choice gives the oracle's labels
    and centres (the launch configuration never changes a result)."""
    S = _S()
    img = mk()
    p = O.params_for(img, grid, m=m, max_iter=2, perturb=True)
    cen = O.slic(p, img)["centres"]
    ref_lab = O.assign(p, img, cen)
    ref_cen, _, _ = O.update(p, img, ref_lab, cen)
    for shape in range(S.num_tile_shapes(img.ndim - 1)):
        lab, got = _gpu_iterate_shape(img, grid, cen, m, shape)
        np.testing.assert_array_equal(lab, ref_lab, err_msg=f"shape {shape}")
        np.testing.assert_array_equal(got, ref_cen, err_msg=f"shape {shape}")


def test_autotune_picks_a_measured_shape_and_keeps_results():
    torch, S = _torch(), _S()
    S.tune_forget()
    img = _synth((96, 80, 48))
    p = S.params_for(img, (16, 16, 16), max_iter=4)
    ref = O.slic(O.params_for(img, (16, 16, 16), max_iter=4), img)
    with S.Context(p) as ctx:
        dimg = _dev(img)
        lab = torch.empty(img.shape[:-1], dtype=torch.int32, device="cuda")
        t = ctx.autotune(dimg, lab, reps=2)
        assert 0 <= t["best"] < S.num_tile_shapes(3)
        assert len(t["ms"]) == S.num_tile_shapes(3) and all(v > 0 for v in t["ms"])
        assert t["ms"][t["best"]] == min(t["ms"])
        assert ctx.tile_shape == t["best"]
        cen = torch.empty((ctx.K, ctx.centre_width), dtype=torch.float32, device="cuda")
        ctx.run(dimg, lab, cen)
        np.testing.assert_array_equal(lab.cpu().numpy(), ref["labels"])
        np.testing.assert_array_equal(cen.cpu().numpy().astype(np.float64), ref["centres"])
    # a new context of the same type and grid starts from the measured shape
    with S.Context(p) as ctx2:
        assert ctx2.tile_shape == t["best"]
    S.tune_forget()
    # image types without a tile kernel refuse
    fimg = _rand_img((30, 40, 4), np.float32, 1)
    with S.Context(S.params_for(fimg, (6, 6))) as ctx3:
        assert ctx3.tile_shape == -1
        with pytest.raises(S.SSLICError):
            ctx3.autotune(_dev(fimg), torch.empty((30, 40), dtype=torch.int32, device="cuda"))


def test_iterate_random_centres_ties():
    """Integer centre positions and equal features: every tie is decided by
    the cluster index alone."""
    img = np.full((37, 45, 3), 100, np.uint8)
    p = O.params_for(img, (5, 5), m=3.0, max_iter=1)
    K = O.num_clusters(p)
    rng = np.random.default_rng(9)
    cen = np.zeros((K, 5))
    cen[:, :3] = 100.0
    cen[:, 3] = rng.integers(0, 45, size=K)
    cen[:, 4] = rng.integers(0, 37, size=K)
    ref_lab = O.assign(p, img, cen)
    lab, _, _ = _gpu_iterate(img, (5, 5), cen, m=3.0)
    np.testing.assert_array_equal(lab, ref_lab)


# ---------------------------------------------------------------------------
# a6: connectivity enforcement alone
# ---------------------------------------------------------------------------
def _gpu_conn(img_shape, grid, centres, labels, C=3):
    torch, S = _torch(), _S()
    size = tuple(reversed(img_shape))
    p = S.Params(size=size, grid=grid, channels=C, dtype=S.U8, enforce_connectivity=True)
    with S.Context(p) as ctx:
        lin = _dev(labels.astype(np.int32))
        lout = torch.empty_like(lin)
        n = ctx.connectivity(_dev(centres.astype(np.float32)), lin, lout)
        return lout.cpu().numpy(), n


@pytest.mark.parametrize("shape,grid,m", [((150, 203), (16, 16), 2.0), ((37, 50, 70), (8, 8, 8), 1.0),
                                          ((30, 40, 20), (4, 4, 4), 0.5), ((2000,), (9,), 1.0)])
def test_connectivity_parity(shape, grid, m):
    img = _rand_img(tuple(shape) + (3,), np.uint8, 12)
    p = O.params_for(img, grid, m=m, max_iter=3)
    r = O.slic(p, img)
    ref, nref = O.connectivity(p, r["centres"], r["labels"])
    got, n = _gpu_conn(shape, grid, r["centres"], r["labels"])
    np.testing.assert_array_equal(got, ref)
    assert n == nref


def test_connectivity_uncovered_and_blocky():
    """Labels with -1 holes, tiny islands and components spanning many tiles."""
    rng = np.random.default_rng(2)
    shape = (70, 130)
    grid = (10, 10)
    K = 7 * 13
    blocks = rng.integers(-1, K, size=(14, 26))
    lab = np.kron(blocks, np.ones((5, 5), np.int64))[:70, :130].astype(np.int32)
    noise = rng.random(shape) < 0.05
    lab[noise] = rng.integers(-1, K, size=noise.sum())
    cen = np.zeros((K, 5))
    cen[:, 3] = rng.uniform(0, 129, size=K)
    cen[:, 4] = rng.uniform(0, 69, size=K)
    p = O.Params(size=(130, 70), grid=grid, channels=3)
    ref, nref = O.connectivity(p, cen, lab)
    got, n = _gpu_conn(shape, grid, cen, lab)
    np.testing.assert_array_equal(got, ref)
    assert n == nref


def _spiral(h, w):
    """1 on a one-pixel-wide square spiral (one long winding component that
    crosses every row and tile boundary many times), 0 elsewhere."""
    a = np.zeros((h, w), np.int32)
    y, x, dy, dx = 0, 0, 0, 1
    a[0, 0] = 1
    turns = 0
    while turns < 2:
        ny, nx = y + dy, x + dx
        fy, fx = y + 2 * dy, x + 2 * dx   # keep one free pixel to the next arm
        ok = 0 <= ny < h and 0 <= nx < w and not a[ny, nx] and not (0 <= fy < h and 0 <= fx < w and a[fy, fx])
        if ok:
            y, x = ny, nx
            a[y, x] = 1
            turns = 0
        else:
            dy, dx = dx, -dy
            turns += 1
    return a


@pytest.mark.parametrize("case", ["checker2d", "checker3d", "spiral2d", "spiral3d", "stripes1d"])
def test_connectivity_adversarial_patterns(case):
    """Every voxel its own component (the most local components a tile can
    hold), and thin winding components that cross tiles and rows many times."""
    if case == "checker2d":
        y, x = np.mgrid[0:97, 0:131]
        lab = ((x + y) % 2).astype(np.int32)
        grid = (16, 16)
    elif case == "checker3d":
        z, y, x = np.mgrid[0:21, 0:19, 0:70]
        lab = ((x + y + z) % 2).astype(np.int32)
        grid = (8, 8, 8)
    elif case == "spiral2d":
        lab = _spiral(150, 203)
        grid = (32, 32)
    elif case == "spiral3d":
        sp = _spiral(40, 70)
        lab = np.stack([sp if z % 2 == 0 else 1 - sp for z in range(12)]).astype(np.int32)
        grid = (16, 16, 4)
    else:
        lab = (np.arange(5000) // 3 % 2).astype(np.int32)
        grid = (50,)
    shape = lab.shape
    n = len(shape)
    size = tuple(reversed(shape))
    nb = [-(-size[d] // grid[d]) for d in range(n)]
    K = int(np.prod(nb))
    cen = np.zeros((K, 3 + n))
    for k in range(K):
        j = np.unravel_index(k, tuple(reversed(nb)))[::-1]   # x fastest
        for d in range(n):
            cen[k, 3 + d] = min(size[d] - 1, j[d] * grid[d] + grid[d] / 2)
    p = O.Params(size=tuple(reversed(shape)), grid=grid, channels=3)
    ref, nref = O.connectivity(p, cen, lab)
    got, nn = _gpu_conn(shape, grid, cen, lab)
    assert nn == nref
    np.testing.assert_array_equal(got, ref)


def test_connectivity_many_components_and_capacity_growth():
    """~10^6 components on 8M voxels: many concurrent union-find walks, and a
    component count far above the initial record capacity (grown on demand)."""
    rng = np.random.default_rng(31)
    shape = (160, 224, 224)
    grid = (56, 56, 40)
    K = 4 * 4 * 4
    blocks = rng.integers(-1, K, size=(80, 112, 112))
    lab = np.kron(blocks, np.ones((2, 2, 2), np.int64)).astype(np.int32)
    flip = rng.random(shape) < 0.02
    lab[flip] = rng.integers(-1, K, size=int(flip.sum()))
    cen = np.zeros((K, 6))
    cen[:, 3] = rng.uniform(0, 223, size=K)
    cen[:, 4] = rng.uniform(0, 223, size=K)
    cen[:, 5] = rng.uniform(0, 159, size=K)
    p = O.Params(size=(224, 224, 160), grid=grid, channels=3)
    ref, nref = O.connectivity(p, cen, lab)
    got, n = _gpu_conn(shape, grid, cen, lab)
    assert n == nref
    np.testing.assert_array_equal(got, ref)


# ---------------------------------------------------------------------------
# end to end
# ---------------------------------------------------------------------------
def _cfg_image(name):
    w = I.WORKLOADS[name]
    return w, I.make_image(w.image)


@pytest.mark.parametrize("name", ["rgb2d_256", "rgb2d_2048x1216"])
def test_full_run_2d_workloads(name):
    w, img = _cfg_image(name)
    kw = dict(m=w.m, max_iter=w.max_iter, perturb=w.perturb, enforce_connectivity=w.connectivity)
    ref = O.slic(O.params_for(img, w.grid, **kw), img)
    lab, cen, info = _gpu_run(img, w.grid, **kw)
    np.testing.assert_array_equal(lab, ref["labels"])
    np.testing.assert_array_equal(cen, ref["centres"])
    assert info["num_labels"] == ref["num_labels"]
    assert info["iterations"] == ref["iterations"] == w.max_iter
    assert info["residual"] == pytest.approx(ref["residual"], rel=1e-9)


@pytest.mark.parametrize("size,grid,conn", [((128, 96, 64), (16, 16, 16), True),
                                            ((77, 61, 45), (8, 8, 8), True),
                                            ((100, 60, 40), (16, 8, 4), False)])
def test_full_run_3d(size, grid, conn):
    img = _synth(size, regions=int(np.prod(size)) // 20000 + 2)
    kw = dict(m=10.0, max_iter=5, perturb=True, enforce_connectivity=conn)
    ref = O.slic(O.params_for(img, grid, **kw), img)
    lab, cen, info = _gpu_run(img, grid, **kw)
    np.testing.assert_array_equal(lab, ref["labels"])
    np.testing.assert_array_equal(cen, ref["centres"])
    assert info["num_labels"] == ref["num_labels"]


def test_full_run_u16_blocks():
    img = _synth((96, 96, 96), 1, "u16", regions=60, sigma=300)
    kw = dict(m=10.0, max_iter=10, perturb=True, enforce_connectivity=True)
    ref = O.slic(O.params_for(img, (16, 16, 16), **kw), img)
    lab, cen, info = _gpu_run(img, (16, 16, 16), **kw)
    np.testing.assert_array_equal(lab, ref["labels"])
    np.testing.assert_array_equal(cen, ref["centres"])


def test_float_hyperspectral_vs_fp64_oracle():
    """Float tolerance: label agreement >= 99.99 %; the centre table's
    relative error ||C - C_ref||_F / ||C_ref||_F <= 1e-5; and every centre
    whose member set is the same on both sides within 1e-5 relative."""
    w = I.WORKLOADS["hyper64_1024"]
    img = I.make_hyperspectral()
    kw = dict(m=w.m, max_iter=w.max_iter, perturb=True)
    ref = O.slic(O.params_for(img, w.grid, mode=O.FP64, **kw), img)
    lab, cen, _ = _gpu_run(img, w.grid, **kw)
    agree = (lab == ref["labels"]).mean()
    assert agree >= 0.9999, agree
    table = np.linalg.norm(cen - ref["centres"]) / np.linalg.norm(ref["centres"])
    assert table <= 1e-5, table
    differ = np.unique(np.concatenate([lab[lab != ref["labels"]], ref["labels"][lab != ref["labels"]]]))
    same = np.setdiff1d(np.arange(cen.shape[0]), differ)
    rel = np.abs(cen[same] - ref["centres"][same]) / np.maximum(np.abs(ref["centres"][same]), 1e-3)
    assert rel.max() <= 1e-5, rel.max()


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("shape,grid", [((1, 1), (1, 1)), ((1, 1, 1), (4, 4, 4)), ((5, 7), (16, 16)),
                                        ((3, 200), (2, 2)), ((33, 17, 5), (40, 40, 40))])
def test_degenerate_shapes(shape, grid):
    img = _rand_img(tuple(shape) + (3,), np.uint8, 1)
    kw = dict(m=10.0, max_iter=3, perturb=True, enforce_connectivity=True)
    ref = O.slic(O.params_for(img, grid, **kw), img)
    lab, cen, info = _gpu_run(img, grid, **kw)
    np.testing.assert_array_equal(lab, ref["labels"])
    np.testing.assert_array_equal(cen, ref["centres"])
    assert info["num_labels"] == ref["num_labels"]


def test_threshold_iterations_match():
    img = _synth((160, 120))
    for thr in (1e-9, 0.5, 5.0):
        kw = dict(m=10.0, max_iter=10, conv_threshold=thr)
        ref = O.slic(O.params_for(img, (16, 16), **kw), img)
        lab, cen, info = _gpu_run(img, (16, 16), **kw)
        assert info["iterations"] == ref["iterations"]
        np.testing.assert_array_equal(lab, ref["labels"])


def test_resume_and_host_entry():
    torch, S = _torch(), _S()
    img = _synth((120, 90))
    p5 = S.params_for(img, (8, 8), max_iter=5)
    p10 = S.params_for(img, (8, 8), max_iter=10)
    l10, c10, _ = _gpu_run(img, (8, 8), max_iter=10)
    with S.Context(p5) as ctx:
        d = _dev(img)
        lab = torch.empty(img.shape[:-1], dtype=torch.int32, device="cuda")
        c5 = torch.empty((ctx.K, ctx.centre_width), dtype=torch.float32, device="cuda")
        ctx.run(d, lab, c5)
        c_res = torch.empty_like(c5)
        ctx.run_from(d, c5, lab, c_res)
        np.testing.assert_array_equal(lab.cpu().numpy(), l10)
        np.testing.assert_array_equal(c_res.cpu().numpy().astype(np.float64), c10)
    with S.Context(p10) as ctx:
        h_img = torch.from_numpy(img).pin_memory()
        h_lab = torch.empty(img.shape[:-1], dtype=torch.int32).pin_memory()
        h_cen = torch.empty((ctx.K, ctx.centre_width), dtype=torch.float32).pin_memory()
        ctx.run_host(h_img, h_lab, h_cen)
        np.testing.assert_array_equal(h_lab.numpy(), l10)
        np.testing.assert_array_equal(h_cen.numpy().astype(np.float64), c10)


def test_invalid_calls_raise():
    torch, S = _torch(), _S()
    with pytest.raises(S.SSLICError):
        S.Context(S.Params(size=(10, 10), grid=(0, 2)))
    img = _synth((40, 30))
    with S.Context(S.params_for(img, (8, 8))) as ctx:
        with pytest.raises(ValueError):
            ctx.run(_dev(img), torch.empty(5, dtype=torch.int32, device="cuda"))
        assert ctx.lib.sslic_run(ctx._c, None, None, None, None, None) == -1


# ---------------------------------------------------------------------------
# 4-D images (the paper's filter is n-dimensional, Sec. 3): per-voxel kernel,
# 4-D bins, 3^4 perturbation, 4-D connectivity
# ---------------------------------------------------------------------------
def _blocky4d(size, C, dtype, seed):
    """Piecewise-constant blocks (a few voxels per axis) plus noise."""
    rng = np.random.default_rng(seed)
    shape = tuple(reversed(size))
    hi = 256 if dtype == np.uint8 else (65536 if dtype == np.uint16 else 1.0)
    blocks = [max(1, s // 5) for s in shape]
    base = rng.uniform(0, hi, size=tuple(blocks) + (C,))
    idx = np.ix_(*[np.minimum(np.arange(s) * b // s, b - 1) for s, b in zip(shape, blocks)])
    img = base[idx] + rng.normal(0, 0.04 * hi, size=shape + (C,))
    if dtype == np.float32:
        return img.astype(np.float32)
    return np.clip(np.rint(img), 0, hi - 1).astype(dtype)


CASES_4D = [("u8_rgb", (20, 18, 14, 12), (6, 6, 5, 4), 3, np.uint8),
            ("u16_ragged_aniso", (17, 13, 11, 9), (5, 4, 3, 4), 1, np.uint16),
            ("u8_small_grid", (12, 10, 9, 8), (2, 3, 2, 2), 2, np.uint8)]


@pytest.mark.parametrize("name,size,grid,C,dtype", CASES_4D, ids=[c[0] for c in CASES_4D])
def test_4d_parity(name, size, grid, C, dtype):
    img = _blocky4d(size, C, dtype, sum(size))
    # seeds (3^4 perturbation)
    np.testing.assert_array_equal(_gpu_seed(img, grid, perturb=True), O.seed(O.params_for(img, grid), img))
    # one iteration from the oracle's centres after two iterations
    p = O.params_for(img, grid, m=10.0, max_iter=2)
    cen = O.slic(p, img)["centres"]
    lab, cout, _ = _gpu_iterate(img, grid, cen)
    np.testing.assert_array_equal(lab, O.assign(p, img, cen))
    ref_c, _, _ = O.update(p, img, lab, cen)
    np.testing.assert_array_equal(cout, ref_c)
    # whole runs, with and without connectivity
    for conn in (False, True):
        kw = dict(m=10.0, max_iter=5, perturb=True, enforce_connectivity=conn)
        ref = O.slic(O.params_for(img, grid, **kw), img)
        lab, cen, info = _gpu_run(img, grid, **kw)
        np.testing.assert_array_equal(lab, ref["labels"])
        np.testing.assert_array_equal(cen, ref["centres"])
        assert info["num_labels"] == ref["num_labels"]


def test_4d_float_assignment_is_fp32_canonical():
    img = _blocky4d((16, 14, 12, 10), 2, np.float32, 4)
    grid = (5, 5, 4, 4)
    p = O.params_for(img, grid, m=0.5, max_iter=2)
    cen = O.slic(p, img)["centres"]
    lab, _, _ = _gpu_iterate(img, grid, cen, m=0.5)
    np.testing.assert_array_equal(lab, O.assign(p, img, cen))
