"""sslic_iterate_static -- the iteration entry point that allocates nothing,
for callers that cannot call cudaMalloc (an allocator or pool that must not
grow, a pre-budgeted plug-in, a latency-critical path).  Its output must equal
the context-based sslic_iterate on the same inputs, on two calls in a row
(the second call reuses the fixed device array the first one left behind).
Kept in a file collected last."""
import numpy as np
import pytest

from paper_1806_08741_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _cases():
    rng = np.random.default_rng(77)
    return [
        ("rgb2d_u8", I.make_image(I.ImageSpec((300, 200), 3, "u8", 41, 40, 6)), (16, 16), 10.0),
        ("gray3d_u16", I.make_image(I.ImageSpec((64, 48, 40), 1, "u16", 42, 20, 300)), (8, 8, 8), 10.0),
        ("f32_c4", rng.uniform(0, 1, size=(60, 70, 4)).astype(np.float32), (6, 6), 0.5),
        # the 3-D 8-bit colour volume's kernel (ragged tiles on every axis)
        ("rgb3d_u8", I.make_image(I.ImageSpec((72, 56, 44), 3, "u8", 43, 30, 6)), (8, 8, 8), 10.0),
        # three float channels: the float tile kernel
        ("lab3d_f32", rng.uniform(0, 100, size=(36, 40, 48, 3)).astype(np.float32), (8, 8, 8), 10.0),
    ]


def _compare(p, img):
    import torch
    from paper_1806_08741_gb300 import sslic as S

    dimg = torch.from_numpy(img).cuda()
    with S.Context(p) as ctx:
        cin = torch.empty((ctx.K, ctx.centre_width), dtype=torch.float32, device="cuda")
        ctx.seed(dimg, cin)
        for call in range(2):
            lab_ref = torch.empty(img.shape[:-1], dtype=torch.int32, device="cuda")
            cen_ref = torch.empty_like(cin)
            ctx.iterate(dimg, cin, lab_ref, cen_ref)
            lab = torch.full(img.shape[:-1], -7, dtype=torch.int32, device="cuda")
            cen = torch.full_like(cin, -7.0)
            S.iterate_static(p, dimg, cin, lab, cen)
            torch.cuda.synchronize()
            assert torch.equal(lab, lab_ref), f"labels differ on call {call}"
            if img.dtype == np.float32:
                torch.testing.assert_close(cen, cen_ref, rtol=1e-6, atol=1e-6)
            else:
                assert torch.equal(cen, cen_ref), f"centres differ on call {call}"
            cin = cen_ref


@pytest.mark.parametrize("name,img,grid,m", _cases(), ids=[c[0] for c in _cases()])
def test_static_iterate_matches_context_iterate(name, img, grid, m):
    from paper_1806_08741_gb300 import sslic as S

    _compare(S.params_for(img, grid, m=m, max_iter=1), img)


def test_static_iterate_after_a_tma_shape_was_recorded():
    """A tile shape recorded for this image type may be a TMA-staged one,
    which needs a status word the fixed array does not hold: the call must
    then run the same tile with plain-load staging, with the same result."""
    from paper_1806_08741_gb300 import sslic as S

    img = I.make_image(I.ImageSpec((64, 48, 40), 3, "u8", 44, 24, 6))  # rows of 192 bytes: TMA applies
    p = S.params_for(img, (8, 8, 8), m=10.0, max_iter=1)
    base = S.num_tile_shapes(3) // 2
    for shape in range(base, 2 * base):
        assert S.tile_shape_info(3, shape)["tma_staged"]
        S.tune_record(p, shape)
        try:
            _compare(p, img)
        finally:
            S.tune_forget()


def test_static_iterate_rejects_sizes_beyond_its_array():
    import torch
    from paper_1806_08741_gb300 import sslic as S

    p = S.Params(size=(1024, 1024), grid=(4, 4), channels=3)   # K = 65536 > 16384
    img = torch.zeros((1024, 1024, 3), dtype=torch.uint8, device="cuda")
    lab = torch.empty((1024, 1024), dtype=torch.int32, device="cuda")
    cen = torch.zeros((65536, 5), dtype=torch.float32, device="cuda")
    with pytest.raises(S.SSLICError) as e:
        S.iterate_static(p, img, cen, lab, cen.clone())
    assert e.value.code == -1
