"""Precision form (precision = 1): the feature term from BF16 tensor-core dot
products with an exact FP32 recheck of every voxel the error bound does not
decide.  Pinned three ways: the MMA's raw output against BF16 products
computed here; labels against the exact form and the FP32-canonical oracle
(bit for bit, from the same centres); whole runs against the FP64 oracle
within the float tolerance."""
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
    return _torch().from_numpy(np.ascontiguousarray(a)).cuda()


def _bf16(a):
    """Round float32 values to bfloat16 (nearest, ties to even), as float32."""
    b = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def _split(a):
    """Two-part BF16 split of float32 values: hi = bf16(a), lo = bf16(a - hi)
    (a - hi is exact in float32), both returned as float64."""
    a = np.ascontiguousarray(a, np.float32)
    hi = _bf16(a)
    lo = _bf16(a - hi)
    return hi.astype(np.float64), lo.astype(np.float64)


def test_bf16_rounding_helper():
    # bfloat16 keeps 8 significant bits: the spacing above 1.0 is 2^-7
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -9, 1.0 + 2 ** -8 + 2 ** -20, -2.5],
                 np.float32)
    np.testing.assert_array_equal(_bf16(x), [1.0, 1.0, 1.0 + 2 ** -6, 1.0, 1.0 + 2 ** -7, -2.5])


def _hyper(size, bands, regions=40, seed=7):
    if len(size) == 2:
        return I.make_hyperspectral(size=size, bands=bands, regions=regions, seed=seed)
    # 3-D: stack 2-D mixtures with a slow drift along z
    sl = [I.make_hyperspectral(size=size[:2], bands=bands, regions=regions, seed=seed + z) for z in range(size[2])]
    return np.ascontiguousarray(np.stack(sl, axis=0))


TILE = {2: (16, 8, 1), 3: (8, 4, 4)}


def _reaching(cen, C, grid, T0, E, n):
    ks = []
    for k in range(cen.shape[0]):
        ok = True
        for d in range(n):
            lo = int(np.ceil(np.float32(cen[k, C + d]))) - grid[d]
            ok = ok and lo <= T0[d] + E[d] - 1 and lo + 2 * grid[d] - 1 >= T0[d]
        if ok:
            ks.append(k)
    return ks


@pytest.mark.parametrize("size,bands,grid", [((96, 80), 64, (16, 16)), ((70, 45), 48, (12, 12)),
                                             ((20, 18, 10), 32, (8, 8, 8))])
def test_probe_dots_are_bf16_products(size, bands, grid):
    """The tensor core's x~.c~ for every voxel and candidate slot of a tile
    equals hi.hi + hi.lo + lo.hi of the two-part BF16 splits (within FP32
    accumulation),
    the slots hold the reaching centres in ascending order, and mu is their
    mean feature."""
    torch, S = _torch(), _S()
    img = _hyper(size, bands)
    n = len(size)
    p = S.params_for(img, grid, m=0.1, max_iter=1, precision=1)
    cen = O.seed(O.params_for(img, grid, m=0.1, max_iter=1), img).astype(np.float32)
    C = bands
    N = tuple(reversed(img.shape[:-1]))  # x first
    TX, TY, TZ = TILE[n]
    ntx, nty = -(-N[0] // TX), -(-N[1] // TY)
    ntz = -(-N[2] // TZ) if n == 3 else 1
    with S.Context(p) as ctx:
        dimg, dcen = _dev(img), _dev(cen)
        for tile in sorted({0, (ntx * nty * ntz) // 2, ntx * nty * ntz - 1}):
            r = ctx.precision_probe(dimg, dcen, tile)
            T0 = [(tile % ntx) * TX, ((tile // ntx) % nty) * TY, (tile // (ntx * nty)) * TZ]
            E = [min(TX, N[0] - T0[0]), min(TY, N[1] - T0[1]), min(TZ, N[2] - T0[2]) if n == 3 else 1]
            ks = _reaching(cen, C, grid, T0, E, n)
            assert len(ks) <= 32
            np.testing.assert_array_equal(r["cand"][:len(ks)], ks)
            assert (r["cand"][len(ks):] == -1).all()
            mu_ref = cen[ks, :C].astype(np.float64).mean(axis=0)
            np.testing.assert_allclose(r["mu"], mu_ref, rtol=1e-5, atol=1e-6)
            mu = r["mu"].astype(np.float32)
            ch, cl = np.zeros((32, C), np.float64), np.zeros((32, C), np.float64)
            ch[:len(ks)], cl[:len(ks)] = _split(cen[ks, :C] - mu)
            for v in range(128):
                xl, yl, zl = v % TX, (v // TX) % TY, v // (TX * TY)
                X = (T0[0] + xl, T0[1] + yl, T0[2] + zl)
                inside = X[0] < N[0] and X[1] < N[1] and (n == 2 or X[2] < N[2])
                if n == 2:
                    x = img[X[1], X[0]] if inside else np.zeros(C, np.float32)
                else:
                    x = img[X[2], X[1], X[0]] if inside else np.zeros(C, np.float32)
                xh, xl_ = _split(x - mu)
                terms = xh[None, :] * ch + xh[None, :] * cl + xl_[None, :] * ch
                want = terms.sum(axis=1)
                tol = (3 * C + 2) * 2.0 ** -22 * (np.abs(xh[None, :] * ch) + np.abs(xh[None, :] * cl) +
                                                  np.abs(xl_[None, :] * ch)).sum(axis=1) + 1e-30
                got = r["dots"][v].astype(np.float64)
                assert (np.abs(got - want) <= tol).all(), (tile, v, np.abs(got - want).max())


def _iterate(img, grid, cen, m, precision, ndim):
    torch, S = _torch(), _S()
    p = S.params_for(img, grid, m=m, max_iter=1, precision=precision)
    with S.Context(p) as ctx:
        cin = _dev(cen.astype(np.float32))
        lab = torch.empty(img.shape[:-1], dtype=torch.int32, device="cuda")
        cout = torch.empty_like(cin)
        ctx.profile_enable(True)
        ctx.iterate(_dev(img), cin, lab, cout)
        prof = ctx.profile_read()
        return lab.cpu().numpy(), cout.cpu().numpy().astype(np.float64), prof


@pytest.mark.parametrize("size,bands,grid,m", [((256, 192), 64, (16, 16), 0.1), ((90, 70), 32, (7, 9), 0.05),
                                               ((40, 36, 24), 48, (8, 8, 8), 0.1), ((64, 48), 128, (16, 16), 0.2),
                                               ((50, 40), 64, (2, 2), 0.1)])
def test_precision_labels_equal_exact_form(size, bands, grid, m):
    """One iteration from the same centres: the tensor-core form's labels are
    the exact form's and the FP32-canonical oracle's, bit for bit; rechecks
    are the minority (the bound is tight enough to decide most voxels)."""
    img = _hyper(size, bands)
    po = O.params_for(img, grid, m=m, max_iter=2)
    cen = O.slic(po, img)["centres"]
    ref_lab = O.assign(po, img, cen)
    ref_cen, _, _ = O.update(po, img, ref_lab, cen)
    lab1, cen1, prof1 = _iterate(img, grid, cen, m, 1, len(size))
    lab0, cen0, prof0 = _iterate(img, grid, cen, m, 0, len(size))
    np.testing.assert_array_equal(lab0, ref_lab)
    np.testing.assert_array_equal(lab1, ref_lab)
    np.testing.assert_allclose(cen1, ref_cen, rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(cen0, ref_cen, rtol=1e-6, atol=1e-6)
    assert prof0["rechecks"] == 0
    if grid[0] > 2:   # with S = 2 every tile is crowded and runs the per-voxel kernel
        assert prof1["rechecks"] < 0.5 * img.shape[0] * img.shape[1] * (img.shape[2] if len(size) == 3 else 1)


def test_precision_full_run_vs_fp64_oracle():
    """The hyperspectral workload (1024x1024, 64 bands, S = 16, m = 0.1, 10
    iterations) in the tensor-core form: label agreement >= 99.99 %, the
    centre table's relative error <= 1e-5 against the FP64 oracle, and every
    centre whose member set is the same on both sides within 1e-5 relative
    (the per-cluster half of the float tolerance)."""
    torch, S = _torch(), _S()
    w = I.WORKLOADS["hyper64_1024"]
    img = I.make_hyperspectral()
    kw = dict(m=w.m, max_iter=w.max_iter, perturb=True)
    ref = O.slic(O.params_for(img, w.grid, mode=O.FP64, **kw), img)
    p = S.params_for(img, w.grid, precision=1, **kw)
    with S.Context(p) as ctx:
        lab = torch.empty(img.shape[:-1], dtype=torch.int32, device="cuda")
        cen = torch.empty((ctx.K, ctx.centre_width), dtype=torch.float32, device="cuda")
        ctx.profile_enable(True)
        ctx.run(_dev(img), lab, cen)
        prof = ctx.profile_read()
        lab, cen = lab.cpu().numpy(), cen.cpu().numpy().astype(np.float64)
    agree = (lab == ref["labels"]).mean()
    assert agree >= 0.9999, agree
    table = np.linalg.norm(cen - ref["centres"]) / np.linalg.norm(ref["centres"])
    assert table <= 1e-5, table
    differ = np.unique(np.concatenate([lab[lab != ref["labels"]], ref["labels"][lab != ref["labels"]]]))
    same = np.setdiff1d(np.arange(cen.shape[0]), differ)
    assert same.size >= 0.99 * cen.shape[0], same.size
    rel = np.abs(cen[same] - ref["centres"][same]) / np.maximum(np.abs(ref["centres"][same]), 1e-3)
    assert rel.max() <= 1e-5, rel.max()
    assert prof["rechecks"] < 0.25 * lab.size * w.max_iter, prof["rechecks"]
