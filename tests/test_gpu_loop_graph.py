"""The iterated loop of a run (Sec. 3.1, steps 2-3) replayed from a CUDA graph
gives the eagerly launched loop's labels, centres and result fields bit for
bit, for every assignment kernel family (tile kernels of each integer type,
the 3-channel float tile kernel, the per-voxel kernel in 1-D and 4-D, the
high-channel exact and tensor-core forms), with and without connectivity,
when the cached graph is updated for other buffers or re-instantiated for
another tile shape, and on a non-default stream.  It launches the same
kernels the eager loop does."""
import numpy as np
import pytest

from paper_1806_08741_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch


def _S():
    from paper_1806_08741_gb300 import sslic as S
    return S


def _synth(size, C=3, dtype="u8", seed=5, sigma=6):
    V = int(np.prod(size))
    return I.make_image(I.ImageSpec(tuple(size), C, dtype, seed, max(2, V // 4000), sigma, 0))


def _rand(shape, dtype, seed):
    rng = np.random.default_rng(seed)
    if dtype == np.float32:
        return rng.uniform(0, 1, size=shape).astype(np.float32)
    return rng.integers(0, 256 if dtype == np.uint8 else 65536, size=shape).astype(dtype)


CASES = [
    ("2d_rgb_u8", lambda: _synth((256, 256)), (16, 16), {}),
    ("2d_ragged_rgb_conn", lambda: _synth((203, 150)), (16, 16), {"enforce_connectivity": True}),
    ("3d_rgb_u8", lambda: _synth((64, 48, 40)), (8, 8, 8), {}),
    ("3d_rgb_u8_conn", lambda: _synth((70, 45, 33)), (8, 8, 8), {"enforce_connectivity": True}),
    ("3d_u16_grey", lambda: _synth((64, 64, 32), C=1, dtype="u16"), (8, 8, 8), {}),
    ("2d_u8_grey", lambda: _synth((300, 200), C=1), (16, 16), {}),
    ("2d_f32_lab_tile", lambda: _rand((90, 110, 3), np.float32, 2), (10, 10), {"m": 0.5}),
    ("1d_voxel", lambda: _synth((1000,)), (7,), {}),
    ("4d_voxel", lambda: _rand((8, 10, 12, 12, 1), np.uint8, 3), (4, 4, 4, 4), {}),
    ("2d_f32_c32_exact", lambda: _rand((70, 53, 32), np.float32, 5), (8, 8), {"m": 0.5}),
    ("2d_f32_c32_tensor", lambda: _rand((70, 53, 32), np.float32, 5), (8, 8), {"m": 0.5, "precision": 1}),
]


def _run(img_dev, p, graph, stream=None, shape=None):
    torch, S = _torch(), _S()
    with S.Context(p) as ctx:
        ctx.set_loop_graph(graph)
        if shape is not None:
            ctx.tile_shape = shape
        ctx.profile_enable(False)  # resets the launch counter; timing stays off
        lab = torch.empty(img_dev.shape[:-1], dtype=torch.int32, device="cuda")
        cen = torch.empty((ctx.K, ctx.centre_width), dtype=torch.float32, device="cuda")
        info = ctx.run(img_dev, lab, cen, stream=stream)
        launches = ctx.profile_read()["kernel_launches"]
        torch.cuda.synchronize()
        return lab.cpu().numpy(), cen.cpu().numpy(), info, launches


@pytest.mark.parametrize("name,make,grid,kw", CASES, ids=[c[0] for c in CASES])
def test_graph_loop_equals_eager_loop(name, make, grid, kw):
    torch, S = _torch(), _S()
    img = make()
    d = torch.from_numpy(np.ascontiguousarray(img)).cuda()
    p = S.params_for(img, grid, max_iter=6, **kw)
    lg, cg, ig, ng = _run(d, p, True)
    le, ce, ie, ne = _run(d, p, False)
    assert np.array_equal(lg, le)
    assert np.array_equal(cg.view(np.uint32), ce.view(np.uint32))
    assert ig == ie
    assert ig["iterations"] == 6
    assert ng == ne  # the replayed graph holds the eager iteration's kernels


def test_graph_updated_for_new_buffers_and_reinstantiated_for_new_shape():
    torch, S = _torch(), _S()
    a = _synth((128, 96, 40), seed=11)
    b = _synth((128, 96, 40), seed=12)
    p = S.params_for(a, (8, 8, 8), max_iter=5)
    da = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    db = torch.from_numpy(np.ascontiguousarray(b)).cuda()
    expect = {}
    for key, d, sh in (("a", da, None), ("b", db, None), ("b1", db, 1), ("a0", da, 0)):
        expect[key] = _run(d, p, False, shape=sh)[:2]
    with S.Context(p) as ctx:
        ctx.set_loop_graph(True)
        for key, d, sh in (("a", da, None), ("b", db, None), ("b1", db, 1), ("a0", da, 0)):
            if sh is not None:
                ctx.tile_shape = sh
            lab = torch.empty(d.shape[:-1], dtype=torch.int32, device="cuda")
            cen = torch.empty((ctx.K, ctx.centre_width), dtype=torch.float32, device="cuda")
            ctx.run(d, lab, cen)
            torch.cuda.synchronize()
            le, ce = expect[key]
            assert np.array_equal(lab.cpu().numpy(), le), key
            assert np.array_equal(cen.cpu().numpy().view(np.uint32), ce.view(np.uint32)), key


def test_graph_loop_on_a_side_stream():
    torch, S = _torch(), _S()
    img = _synth((512, 384), seed=21)
    d = torch.from_numpy(np.ascontiguousarray(img)).cuda()
    p = S.params_for(img, (16, 16), max_iter=10)
    le, ce, _, _ = _run(d, p, False)
    s = torch.cuda.Stream()
    with S.Context(p) as ctx:
        lab = torch.empty(d.shape[:-1], dtype=torch.int32, device="cuda")
        cen = torch.empty((ctx.K, ctx.centre_width), dtype=torch.float32, device="cuda")
        s.wait_stream(torch.cuda.current_stream())
        for _ in range(3):
            ctx.run_async(d, lab, cen, stream=s)
        s.synchronize()
        assert np.array_equal(lab.cpu().numpy(), le)
        assert np.array_equal(cen.cpu().numpy().view(np.uint32), ce.view(np.uint32))


def test_threshold_runs_stay_eager_and_equal():
    torch, S = _torch(), _S()
    img = _synth((256, 256), seed=31)
    d = torch.from_numpy(np.ascontiguousarray(img)).cuda()
    p = S.params_for(img, (16, 16), max_iter=20, conv_threshold=1e-3)
    lg, cg, ig, _ = _run(d, p, True)
    le, ce, ie, _ = _run(d, p, False)
    assert np.array_equal(lg, le) and np.array_equal(cg.view(np.uint32), ce.view(np.uint32))
    assert ig == ie
