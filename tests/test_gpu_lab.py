"""Colour input (CIE-Lab, reading R16): the device sRGB -> Lab conversion
against the FP64 oracle, and SLIC on the converted float image against the
oracle.  Conversion tolerance: 1e-3 in every component.  The single-
precision evaluation errs by at most about 2e-4: a few ulp on f <= 1.1,
times the factor of 500 in a = 500 (f_x - f_y).  Segmentation tolerances
are those of every float image: label agreement >= 99.99 % and centre
relative error <= 1e-5 against FP64."""
import numpy as np
import pytest

import oracle as O
from paper_1806_08741_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-3


def _torch():
    import torch
    return torch


def _S():
    from paper_1806_08741_gb300 import sslic as S
    return S


def _cube():
    v = np.arange(256)
    return np.stack(np.meshgrid(v, v, v, indexing="ij"), -1).reshape(-1, 3).astype(np.uint8)


def _gpu_lab(rgb):
    torch, S = _torch(), _S()
    out = S.srgb_to_lab(torch.from_numpy(np.ascontiguousarray(rgb)).cuda())
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_every_8bit_colour_matches_the_oracle():
    cube = _cube()
    got = _gpu_lab(cube).astype(np.float64)
    ref = O.srgb_to_lab(cube)
    err = np.abs(got - ref).max(0)
    assert err.max() <= TOL, err


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7, 1027, 100003])
@pytest.mark.parametrize("offset", [(0, 0), (1, 0), (0, 1), (3, 2)])
def test_ragged_lengths_and_unaligned_buffers(n, offset):
    # offsets in voxels into larger buffers: (1, 0) leaves rgb 4-byte
    # misaligned, (0, 1) leaves lab off its 16-byte boundary
    torch, S = _torch(), _S()
    rng = np.random.default_rng(n)
    ro, lo = offset
    rgb_all = torch.from_numpy(rng.integers(0, 256, size=(n + ro) * 3, dtype=np.uint8)).cuda()
    lab_all = torch.full(((n + lo + 1) * 3,), -7.0, dtype=torch.float32, device="cuda")
    rgb = rgb_all[3 * ro:]
    lab = lab_all[3 * lo:3 * (lo + n)]
    L = S.load()
    rc = L.sslic_srgb_to_lab(S._ptr(rgb), S._ptr(lab), n, S._stream(None))
    assert rc == 0
    torch.cuda.synchronize()
    got = lab.cpu().numpy().reshape(n, 3).astype(np.float64)
    ref = O.srgb_to_lab(rgb.cpu().numpy().reshape(n, 3))
    assert np.abs(got - ref).max() <= TOL
    tail = lab_all.cpu().numpy()
    assert np.all(tail[:3 * lo] == -7.0) and np.all(tail[3 * (lo + n):] == -7.0)  # nothing outside written


def test_zero_voxels_is_a_no_op():
    S = _S()
    assert S.load().sslic_srgb_to_lab(None, None, 0, None) == 0


def _lab_image(size, seed=5, regions=None, sigma=6):
    rgb = I.make_image(I.ImageSpec(tuple(size), 3, "u8", seed, regions or max(2, int(np.prod(size)) // 4000), sigma, 0))
    return _gpu_lab(rgb)


def _gpu_run(img, grid, **kw):
    torch, S = _torch(), _S()
    p = S.params_for(img, grid, **kw)
    with S.Context(p) as ctx:
        lab = torch.empty(img.shape[:-1], dtype=torch.int32, device="cuda")
        cen = torch.empty((ctx.K, ctx.centre_width), dtype=torch.float32, device="cuda")
        info = ctx.run(torch.from_numpy(np.ascontiguousarray(img)).cuda(), lab, cen)
        return lab.cpu().numpy(), cen.cpu().numpy().astype(np.float64), info


def _gpu_iterate(img, grid, centres, m):
    torch, S = _torch(), _S()
    p = S.params_for(img, grid, m=m, max_iter=1)
    with S.Context(p) as ctx:
        cin = torch.from_numpy(centres.astype(np.float32)).cuda()
        lab = torch.empty(img.shape[:-1], dtype=torch.int32, device="cuda")
        cout = torch.empty_like(cin)
        ctx.iterate(torch.from_numpy(np.ascontiguousarray(img)).cuda(), cin, lab, cout)
        return lab.cpu().numpy()


LAB_CASES = [
    ("2d_512x384", (512, 384), (16, 16), False),
    ("2d_ragged_203x150", (203, 150), (16, 16), True),
    ("3d_96x80x40", (96, 80, 40), (16, 16, 16), True),
    ("3d_ragged_70x45x33", (70, 45, 33), (8, 8, 8), False),
]


@pytest.mark.parametrize("name,size,grid,conn", LAB_CASES, ids=[c[0] for c in LAB_CASES])
def test_lab_assignment_is_the_fp32_canonical_one(name, size, grid, conn):
    # one assignment from the same centres: labels identical to the oracle's
    # FP32-canonical assignment
    img = _lab_image(size)
    p = O.params_for(img, grid, m=10.0, max_iter=3)
    cen = O.slic(p, img)["centres"]
    got = _gpu_iterate(img, grid, cen, 10.0)
    np.testing.assert_array_equal(got, O.assign(p, img, cen))


@pytest.mark.parametrize("name,size,grid,conn", LAB_CASES, ids=[c[0] for c in LAB_CASES])
def test_lab_segmentation_vs_fp64_oracle(name, size, grid, conn):
    img = _lab_image(size)
    kw = dict(m=10.0, max_iter=10, perturb=True, enforce_connectivity=conn)
    ref = O.slic(O.params_for(img, grid, mode=O.FP64, **kw), img)
    lab, cen, info = _gpu_run(img, grid, **kw)
    agree = (lab == ref["labels"]).mean()
    assert agree >= 0.9999, agree
    table = np.linalg.norm(cen - ref["centres"]) / np.linalg.norm(ref["centres"])
    assert table <= 1e-5, table


def _gpu_iterate_shape(img, grid, centres, m, shape):
    torch, S = _torch(), _S()
    p = S.params_for(img, grid, m=m, max_iter=1)
    with S.Context(p) as ctx:
        ctx.tile_shape = shape
        cin = torch.from_numpy(centres.astype(np.float32)).cuda()
        lab = torch.empty(img.shape[:-1], dtype=torch.int32, device="cuda")
        cout = torch.empty_like(cin)
        ctx.iterate(torch.from_numpy(np.ascontiguousarray(img)).cuda(), cin, lab, cout)
        return lab.cpu().numpy(), cout.cpu().numpy().astype(np.float64)


SHAPE_CASES = [("3d", (75, 53, 27), (16, 16, 16), 12), ("3d_small_grid", (40, 36, 20), (5, 5, 5), 12),
               ("2d", (203, 150), (16, 16), 6), ("2d_small_grid", (130, 70), (3, 3), 6)]


@pytest.mark.parametrize("name,size,grid,nshapes", SHAPE_CASES, ids=[c[0] for c in SHAPE_CASES])
def test_every_float_tile_shape(name, size, grid, nshapes):
    # every tile shape (ragged tails; the small grids crowd tiles past the
    # candidate capacity, which go to the per-voxel kernel): labels identical
    # to the FP32-canonical assignment; the update's centres within FP32
    # summation error of the FP64 update of the same labels
    img = _lab_image(size)
    p32 = O.params_for(img, grid, m=10.0, max_iter=2)
    cen = O.slic(p32, img)["centres"]
    want = O.assign(p32, img, cen)
    ref, _, _ = O.update(O.params_for(img, grid, m=10.0, max_iter=1, mode=O.FP64), img, want, cen)
    for shape in range(nshapes):
        lab, cout = _gpu_iterate_shape(img, grid, cen, 10.0, shape)
        np.testing.assert_array_equal(lab, want, err_msg=f"shape {shape}")
        np.testing.assert_allclose(cout, ref, rtol=1e-5, atol=1e-4, err_msg=f"shape {shape}")
