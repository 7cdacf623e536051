"""Streamed form (sslic_run_streamed): the image stays in host memory and
every iteration streams it through the GPU in slabs along its last axis.
Integer images: labels and centres bit-identical to sslic_run on the device
and to the oracle; float images: within the float tolerance of sslic_run."""
import numpy as np
import pytest

import oracle as O
from paper_1806_08741_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _run(img, grid, **kw):
    import torch
    from paper_1806_08741_gb300 import sslic as S
    p = S.params_for(img, grid, **kw)
    with S.Context(p) as ctx:
        lab = torch.empty(img.shape[:-1], dtype=torch.int32, device="cuda")
        cen = torch.empty((ctx.K, ctx.centre_width), dtype=torch.float32, device="cuda")
        info = ctx.run(torch.from_numpy(np.ascontiguousarray(img)).cuda(), lab, cen)
        return lab.cpu().numpy(), cen.cpu().numpy(), info


def _streamed(img, grid, slab, **kw):
    import torch
    from paper_1806_08741_gb300 import sslic as S
    p = S.params_for(img, grid, **kw)
    h_img = torch.from_numpy(np.ascontiguousarray(img)).pin_memory()
    with S.Context(p) as ctx:
        lab = torch.empty(img.shape[:-1], dtype=torch.int32).pin_memory()
        cen = np.empty((ctx.K, ctx.centre_width), np.float32)
        info = ctx.run_streamed(h_img, lab, cen, slab_planes=slab)
        return lab.numpy(), cen, info


def _synth(size, C=3, dtype="u8", sigma=6, seed=5):
    V = int(np.prod(size))
    return I.make_image(I.ImageSpec(tuple(size), C, dtype, seed, max(2, V // 4000), sigma))


INT_CASES = [("3d_rgb_ragged", lambda: _synth((70, 52, 150)), (16, 16, 16), 32),
             ("3d_rgb_one_slab", lambda: _synth((64, 48, 40)), (8, 8, 8), 64),
             ("3d_u16", lambda: _synth((48, 40, 100), 1, "u16", sigma=300), (8, 8, 8), 32),
             ("2d_rgb_rows", lambda: _synth((300, 230)), (16, 16), 64),
             ("3d_two_channel_voxel_kernel", lambda: _synth((40, 36, 70), 2), (8, 8, 8), 32)]


@pytest.mark.parametrize("name,mk,grid,slab", INT_CASES, ids=[c[0] for c in INT_CASES])
def test_streamed_equals_resident_and_oracle(name, mk, grid, slab):
    img = mk()
    kw = dict(m=10.0, max_iter=5, perturb=True)
    lab, cen, info = _streamed(img, grid, slab, **kw)
    ref_l, ref_c, ref_i = _run(img, grid, **kw)
    np.testing.assert_array_equal(lab, ref_l)
    np.testing.assert_array_equal(cen, ref_c)
    assert info["iterations"] == ref_i["iterations"] == 5
    assert info["residual"] == ref_i["residual"]
    o = O.slic(O.params_for(img, grid, **kw), img)
    np.testing.assert_array_equal(lab, o["labels"])
    np.testing.assert_array_equal(cen.astype(np.float64), o["centres"])


def test_streamed_threshold_stops_where_the_resident_run_stops():
    img = _synth((64, 48, 96))
    # a threshold just above the residual of the third iteration: the run
    # stops there (or earlier), well before the cap
    r3 = _run(img, (8, 8, 8), m=10.0, max_iter=3, perturb=True)[2]["residual"]
    kw = dict(m=10.0, max_iter=10, perturb=True, conv_threshold=r3 * 1.0001)
    lab, cen, info = _streamed(img, (8, 8, 8), 32, **kw)
    ref_l, ref_c, ref_i = _run(img, (8, 8, 8), **kw)
    assert info["iterations"] == ref_i["iterations"] < 10
    np.testing.assert_array_equal(lab, ref_l)
    np.testing.assert_array_equal(cen, ref_c)


@pytest.mark.parametrize("C", [3, 32])
def test_streamed_float_within_tolerance(C):
    rng = np.random.default_rng(C)
    rgb = _synth((60, 44, 96))
    if C == 3:
        img = O.srgb_to_lab(rgb).astype(np.float32)
    else:
        img = (rng.uniform(0, 1, size=rgb.shape[:-1] + (C,)) * 0.05 +
               np.repeat(rgb[..., :1].astype(np.float32) / 255.0, C, axis=-1)).astype(np.float32)
    kw = dict(m=10.0 if C == 3 else 0.5, max_iter=4, perturb=True)
    lab, cen, _ = _streamed(img, (8, 8, 8), 32, **kw)
    ref_l, ref_c, _ = _run(img, (8, 8, 8), **kw)
    assert (lab == ref_l).mean() >= 0.9999
    flip = lab != ref_l
    differ = np.unique(np.concatenate([lab[flip], ref_l[flip]]))
    same = np.setdiff1d(np.arange(cen.shape[0]), differ)
    rel = np.abs(cen[same] - ref_c[same]) / np.maximum(np.abs(ref_c[same]), 1e-3)
    assert rel.max() <= 1e-5


CONN_CASES = [("3d_rgb_ragged", lambda: _synth((70, 52, 150)), (16, 16, 16), 32),
              ("3d_rgb_s8", lambda: _synth((64, 48, 100)), (8, 8, 8), 32),
              ("3d_u16", lambda: _synth((48, 40, 100), 1, "u16", sigma=300), (8, 8, 8), 64),
              ("2d_rgb_rows", lambda: _synth((300, 230)), (16, 16), 64),
              ("2d_rgb_one_slab", lambda: _synth((130, 60)), (16, 16), 64)]


@pytest.mark.parametrize("name,mk,grid,slab", CONN_CASES, ids=[c[0] for c in CONN_CASES])
def test_streamed_connectivity_equals_resident_and_oracle(name, mk, grid, slab):
    """With connectivity enforcement (Sec. 3.1 stage 3) the labels pass
    through the device slab by slab: the result is sslic_run's and the
    oracle's, bit for bit, label count included."""
    img = mk()
    kw = dict(m=10.0, max_iter=4, perturb=True, enforce_connectivity=True)
    lab, cen, info = _streamed(img, grid, slab, **kw)
    ref_l, ref_c, ref_i = _run(img, grid, **kw)
    np.testing.assert_array_equal(lab, ref_l)
    np.testing.assert_array_equal(cen, ref_c)
    assert info["num_labels"] == ref_i["num_labels"]
    o = O.slic(O.params_for(img, grid, **kw), img)
    np.testing.assert_array_equal(lab, o["labels"])
    assert info["num_labels"] == o["num_labels"]


def test_streamed_rejects():
    import torch
    from paper_1806_08741_gb300 import sslic as S
    img = _synth((64, 48, 40))
    h = torch.from_numpy(img).pin_memory()
    lab = torch.empty(img.shape[:-1], dtype=torch.int32)
    with S.Context(S.params_for(img, (40, 40, 40), enforce_connectivity=True)) as ctx:
        with pytest.raises(S.SSLICError) as e:   # slabs thinner than S along the last axis
            ctx.run_streamed(h, lab, None, slab_planes=32)
        assert e.value.code == -1
    img2 = _synth((64, 96))
    with S.Context(S.params_for(img2, (8, 8), enforce_connectivity=True)) as ctx:
        with pytest.raises(S.SSLICError) as e:   # 2-D connectivity wants slabs of 64 rows
            ctx.run_streamed(torch.from_numpy(img2).pin_memory(), torch.empty((96, 64), dtype=torch.int32),
                             None, slab_planes=32)
        assert e.value.code == -1
    with S.Context(S.params_for(img, (8, 8, 8))) as ctx:
        for bad in (0, 31, 48):
            with pytest.raises(S.SSLICError) as e:
                ctx.run_streamed(h, lab, None, slab_planes=bad)
            assert e.value.code == -1
