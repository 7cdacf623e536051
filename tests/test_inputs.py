"""The seeded synthetic generator: determinism, crops, recipe statistics,
and (GPU) byte equality of the CUDA generator with the CPU one."""
import numpy as np
import pytest

from paper_1806_08741_gb300 import inputs as I


def test_deterministic_and_crop_consistent():
    spec = I.ImageSpec((70, 45, 9), 3, "u8", seed=3, regions=40, sigma=6)
    a = I.make_image(spec)
    b = I.make_image(spec)
    assert a.shape == (9, 45, 70, 3)
    np.testing.assert_array_equal(a, b)
    c = I.make_image(spec, origin=(13, 7, 2), extent=(20, 11, 5))
    np.testing.assert_array_equal(c, a[2:7, 7:18, 13:33])


def test_region_count_and_noise_level():
    spec = I.ImageSpec((256, 256), 3, "u8", seed=11, regions=32, sigma=8)
    reg = I.make_regions(spec)
    assert len(np.unique(reg)) == int(np.prod(spec.sites())) == 36
    clean = I.make_image(I.ImageSpec((256, 256), 3, "u8", seed=11, regions=32, sigma=0))
    noisy = I.make_image(spec).astype(np.int64) - clean.astype(np.int64)
    inner = (clean > 40) & (clean < 215)
    assert abs(noisy[inner].std() - 8.0) < 0.2
    assert abs(noisy[inner].mean()) < 0.1


def test_workload_shapes():
    w = I.WORKLOADS["rgb3d_2048x1216x1871"]
    assert w.image.shape == (1871, 1216, 2048, 3)
    assert abs(np.prod(w.image.sites()) - 200000) < 10000
    assert I.WORKLOADS["rgb2d_2048x1216"].image.voxels == 2048 * 1216


def test_uint16_range():
    spec = I.ImageSpec((40, 30, 20), 1, "u16", seed=5, regions=30, sigma=300)
    a = I.make_image(spec)
    assert a.dtype == np.uint16 and a.max() > 30000


@pytest.mark.gpu
@pytest.mark.parametrize("spec", [
    I.ImageSpec((123, 77, 9), 3, "u8", seed=21, regions=50, sigma=6),
    I.ImageSpec((300, 200), 3, "u8", seed=22, regions=80, sigma=6, ramp_amp=32),
    I.ImageSpec((64, 48, 40), 1, "u16", seed=23, regions=20, sigma=300),
])
def test_gpu_generator_matches_cpu(spec):
    import torch
    out = torch.empty(spec.shape, dtype=torch.uint8 if spec.dtype == "u8" else torch.uint16,
                      device="cuda")
    I.make_image_device(spec, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), I.make_image(spec))


def test_spec_struct_matches_header():
    """The generator's ctypes spec has synth.h's fields, types and order."""
    import ctypes
    import os
    import re
    from paper_1806_08741_gb300 import inputs as Inp
    ct = {"int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64, "uint64_t": ctypes.c_uint64}
    text = open(os.path.join(os.path.dirname(Inp.__file__), "synth.h")).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    body = re.search(r"typedef\s+struct\s*\{(.*?)\}\s*synth_spec\s*;", text, flags=re.S).group(1)
    want = []
    for decl in filter(None, (d.strip() for d in body.split(";"))):
        t, name = decl.split(None, 1)
        arr = re.match(r"(\w+)\s*\[\s*(\d+)\s*\]$", name.strip())
        want.append((arr.group(1), ct[t] * int(arr.group(2))) if arr else (name.strip(), ct[t]))
    got = list(Inp._Spec._fields_)
    assert [f for f, _ in got] == [f for f, _ in want]
    for (f, a), (_, b) in zip(got, want):
        assert ctypes.sizeof(a) == ctypes.sizeof(b) and getattr(a, "_type_", a) == getattr(b, "_type_", b), f
