"""The oracle's region-decomposed form (the paper's multi-threaded SSLIC,
Sec. 3.1: non-overlapping regions assigned and mapped in parallel, the
per-region sums merged per label) gives the single-threaded oracle's labels,
centres, residual and label count bit for bit, for any thread count.  This
is the form bench.py times on all host cores as the CPU baseline."""
import numpy as np
import pytest

import oracle as O
from paper_1806_08741_gb300 import inputs as I


def _cases():
    rng = np.random.default_rng(3)
    rgb3d = I.make_image(I.crop_workload(I.WORKLOADS["rgb3d_2048x1216x1871"], (64, 48, 40)).image)
    return [
        ("rgb2d_conn", I.make_image(I.ImageSpec((150, 110), 3, "u8", 51, 30, 8, 20)), (16, 16),
         dict(m=10.0, max_iter=4, enforce_connectivity=True)),
        ("rgb3d_conn", rgb3d, (16, 16, 16), dict(m=10.0, max_iter=3, enforce_connectivity=True)),
        ("rgb3d_small_grid", rgb3d, (5, 6, 4), dict(m=10.0, max_iter=2)),
        ("gray3d_u16", I.make_image(I.ImageSpec((40, 36, 30), 1, "u16", 52, 12, 300)), (8, 8, 8),
         dict(m=20.0, max_iter=3, enforce_connectivity=True)),
        ("float_fp64", rng.uniform(0, 1, size=(30, 34, 5)).astype(np.float32), (6, 6),
         dict(m=0.5, max_iter=3, mode=O.FP64)),
        ("float_fp32", rng.uniform(0, 1, size=(22, 18, 16, 3)).astype(np.float32), (5, 5, 5),
         dict(m=0.5, max_iter=2, mode=O.FP32)),
        ("line_1d", I.make_image(I.ImageSpec((300,), 3, "u8", 53, 9, 8)), (7,), dict(m=10.0, max_iter=3)),
        ("vol_4d", rng.integers(0, 256, size=(6, 7, 8, 9, 2)).astype(np.uint8), (3, 3, 3, 3),
         dict(m=10.0, max_iter=2, enforce_connectivity=True)),
        ("threshold", I.make_image(I.ImageSpec((96, 80), 3, "u8", 54, 20, 6)), (8, 8),
         dict(m=10.0, max_iter=10, conv_threshold=0.05)),
    ]


@pytest.mark.parametrize("name,img,grid,kw", _cases(), ids=[c[0] for c in _cases()])
@pytest.mark.parametrize("threads", [1, 3, 8])
def test_regions_equal_single_threaded(name, img, grid, kw, threads):
    p = O.params_for(img, grid, **kw)
    ref = O.slic(p, img)
    got = O.slic_regions(p, img, threads)
    np.testing.assert_array_equal(got["labels"], ref["labels"])
    np.testing.assert_array_equal(got["centres"], ref["centres"])
    assert got["iterations"] == ref["iterations"]
    assert got["residual"] == ref["residual"]
    assert got["num_labels"] == ref["num_labels"]


def test_regions_without_openmp():
    """The plain build ignores the parallel pragmas and runs the regions one
    after another: the same results."""
    img = I.make_image(I.ImageSpec((70, 60, 20), 3, "u8", 55, 10, 6))
    p = O.params_for(img, (8, 8, 8), m=10.0, max_iter=2, enforce_connectivity=True)
    ref = O.slic(p, img)
    got = O.slic_regions(p, img, 5, openmp=False)
    np.testing.assert_array_equal(got["labels"], ref["labels"])
    np.testing.assert_array_equal(got["centres"], ref["centres"])


def test_regions_reject_zero_threads():
    img = np.zeros((8, 8, 1), np.uint8)
    with pytest.raises(RuntimeError):
        O.slic_regions(O.params_for(img, (4, 4)), img, 0)
