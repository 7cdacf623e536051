"""sslic_run_host with host buffers: the image goes up in pieces (the planes
seeding reads first, then slabs of 64 planes along the last axis, each
slab's first assignment launched behind its upload).  Integer images: labels,
centres and result fields equal the oracle's whole run (Sec. 3.1) and the
device-resident sslic_run bit for bit, whether the upload is split or not;
float images: within the float tolerances of the device run."""
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


def _synth(size, C=3, dtype="u8", seed=7, sigma=6):
    V = int(np.prod(size))
    return I.make_image(I.ImageSpec(tuple(size), C, dtype, seed, max(2, V // 4000), sigma, 0))


def _host_run(img, p, exact=True):
    torch, S = _torch(), _S()
    with S.Context(p) as ctx:
        h_img = torch.from_numpy(np.ascontiguousarray(img)).pin_memory()
        h_lab = torch.empty(img.shape[:-1], dtype=torch.int32).pin_memory()
        h_cen = torch.empty((ctx.K, ctx.centre_width), dtype=torch.float32).pin_memory()
        info = ctx.run_host(h_img, h_lab, h_cen)
        # a second call on the same context (buffers and graph reused)
        h_lab2 = torch.empty_like(h_lab).pin_memory()
        info2 = ctx.run_host(h_img, h_lab2, None)
        if exact:
            assert info2 == info
            assert np.array_equal(h_lab2.numpy(), h_lab.numpy())
        else:  # float sums: FP64 atomics in no fixed order
            assert info2["residual"] == pytest.approx(info["residual"], rel=1e-6)
            assert (h_lab2.numpy() == h_lab.numpy()).mean() >= 0.9999
        return h_lab.numpy().copy(), h_cen.numpy().copy(), info


def _dev_run(img, p):
    torch, S = _torch(), _S()
    with S.Context(p) as ctx:
        d = torch.from_numpy(np.ascontiguousarray(img)).cuda()
        lab = torch.empty(img.shape[:-1], dtype=torch.int32, device="cuda")
        cen = torch.empty((ctx.K, ctx.centre_width), dtype=torch.float32, device="cuda")
        info = ctx.run(d, lab, cen)
        return lab.cpu().numpy(), cen.cpu().numpy(), info


# (name, image, grid, extra params): the last axis has >= 128 planes and a
# grid of >= 8 along it, so the upload is split; the last two fall back to one copy
CASES = [
    ("3d_rgb_conn", lambda: _synth((48, 40, 200)), (8, 8, 8), {"enforce_connectivity": True}),
    ("3d_rgb_ragged", lambda: _synth((37, 29, 131)), (8, 8, 9), {}),
    ("3d_u16_noperturb", lambda: _synth((40, 40, 160), C=1, dtype="u16", sigma=300), (10, 10, 10),
     {"perturb": False}),
    ("2d_rgb_conn", lambda: _synth((150, 300)), (16, 16), {"enforce_connectivity": True}),
    ("2d_grey_threshold", lambda: _synth((203, 333), C=1), (16, 16), {"conv_threshold": 0.05, "max_iter": 30}),
    ("2d_rgb_one_iteration", lambda: _synth((100, 256)), (16, 16), {"max_iter": 1}),
    ("3d_rgb_fine_grid", lambda: _synth((32, 32, 160)), (6, 6, 6), {}),
    ("2d_rgb_short", lambda: _synth((300, 100)), (16, 16), {}),
]


@pytest.mark.parametrize("name,make,grid,kw", CASES, ids=[c[0] for c in CASES])
def test_run_host_equals_oracle_and_device_run(name, make, grid, kw):
    S = _S()
    img = make()
    kw = dict(kw)
    kw.setdefault("max_iter", 5)
    p = S.params_for(img, grid, **kw)
    lh, ch, ih = _host_run(img, p)
    ld, cd, idv = _dev_run(img, p)
    assert np.array_equal(lh, ld)
    assert np.array_equal(ch.view(np.uint32), cd.view(np.uint32))
    assert ih == idv
    ref = O.slic(O.params_for(img, grid, **kw), img)
    assert np.array_equal(lh, ref["labels"])
    np.testing.assert_array_equal(ch.astype(np.float64), ref["centres"])
    assert ih["iterations"] == ref["iterations"]
    assert ih["num_labels"] == ref["num_labels"]


def test_run_host_float_lab_within_tolerance():
    """Float images: the split upload assigns slab by slab, so the FP64 sums
    of the first iteration are added in another order than in one launch."""
    S = _S()
    rng = np.random.default_rng(4)
    img = rng.uniform(0, 100, size=(160, 36, 40, 3)).astype(np.float32)
    p = S.params_for(img, (8, 8, 8), m=10.0, max_iter=4)
    lh, ch, ih = _host_run(img, p, exact=False)
    ld, cd, _ = _dev_run(img, p)
    assert (lh == ld).mean() >= 0.9999
    np.testing.assert_allclose(ch, cd, rtol=1e-5, atol=1e-4)
    assert ih["iterations"] == 4
