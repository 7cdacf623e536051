"""The C-ABI library loads and exports every entry point include/sslic.h
declares (no GPU needed; no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            names += re.findall(r"SSLIC_API\s+[\w\s\*]+?\b(sslic_\w+)\s*\(", text)
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1806_08741_gb300 import build as B
    from paper_1806_08741_gb300 import sslic as S
    B.build()
    return S.load()


def test_header_declares_entry_points():
    names = _declared()
    for n in ("sslic_create", "sslic_run", "sslic_destroy", "sslic_iterate", "sslic_seed",
              "sslic_connectivity", "sslic_run_host", "sslic_run_from"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for n in _declared():
        assert hasattr(lib, n), n
        assert ctypes.cast(getattr(lib, n), ctypes.c_void_p).value


def test_binding_names_match_header():
    from paper_1806_08741_gb300 import sslic as S
    assert sorted(S.EXPORTS) == sorted(_declared())


def test_host_only_calls(lib):
    from paper_1806_08741_gb300 import sslic as S
    p = S._Params()
    assert lib.sslic_default_params(3, ctypes.byref(p)) == 0
    assert p.ndim == 3 and p.max_iter == 5 and abs(p.m - 10.0) < 1e-6 and p.grid[0] == 16
    assert lib.sslic_default_params(2, ctypes.byref(p)) == 0 and p.max_iter == 10
    assert lib.sslic_default_params(7, ctypes.byref(p)) == -1
    assert lib.sslic_strerror(0) == b"ok"
    assert lib.sslic_strerror(-1) == b"invalid argument"
    assert lib.sslic_last_error(None) == b""


@pytest.mark.parametrize("field,value", [("ndim", 0), ("ndim", 5), ("channels", 0),
                                         ("channels", 300), ("dtype", 5), ("m", 0.0),
                                         ("m", float("nan")), ("max_iter", 0), ("perturb", 2),
                                         ("precision", 7)])
def test_create_rejects_bad_params_without_touching_the_gpu(lib, field, value):
    from paper_1806_08741_gb300 import sslic as S
    p = S.Params(size=(64, 64), grid=(8, 8)).to_c()
    setattr(p, field, value)
    out = ctypes.c_void_p(0)
    assert lib.sslic_create(ctypes.byref(p), ctypes.byref(out)) == -1
    assert not out.value


def test_create_rejects_bad_sizes(lib):
    from paper_1806_08741_gb300 import sslic as S
    out = ctypes.c_void_p(0)
    for size, grid in [((0, 4), (2, 2)), ((1 << 25, 4), (2, 2)), ((4, 4), (0, 2))]:
        p = S.Params(size=size, grid=grid).to_c()
        assert lib.sslic_create(ctypes.byref(p), ctypes.byref(out)) == -1
    # the tensor-core form: float images with 32..128 channels in 2-D / 3-D
    p = S.Params(size=(64, 64), grid=(8, 8), precision=1).to_c()           # C = 3 < 32
    assert lib.sslic_create(ctypes.byref(p), ctypes.byref(out)) == -1
    for kw in (dict(channels=64, dtype=S.U8), dict(channels=200, dtype=S.F32)):
        p = S.Params(size=(64, 64), grid=(8, 8), precision=1, **kw).to_c()
        assert lib.sslic_create(ctypes.byref(p), ctypes.byref(out)) == -6
    p = S.Params(size=(640,), grid=(8,), precision=1, channels=64, dtype=S.F32).to_c()
    assert lib.sslic_create(ctypes.byref(p), ctypes.byref(out)) == -6


def test_tile_shape_table_host_only(lib):
    from paper_1806_08741_gb300 import sslic as S
    assert S.num_tile_shapes(3) == 12 and S.num_tile_shapes(2) == 6 and S.num_tile_shapes(1) == 0
    seen = set()
    for nd in (2, 3):
        n = S.num_tile_shapes(nd)
        for s in range(n):
            info = S.tile_shape_info(nd, s)
            tx, ty, tz = info["dims"]
            assert info["voxels_per_lane"] in (2, 4)
            assert tx % 16 == 0 and (tz == 1) == (nd == 2)
            assert info["tma_staged"] == (s >= n // 2)
            if s >= n // 2:   # the TMA-staged twin of a plain shape
                twin = S.tile_shape_info(nd, s - n // 2)
                assert (twin["dims"], twin["voxels_per_lane"]) == (info["dims"], info["voxels_per_lane"])
            seen.add((nd, info["dims"], info["voxels_per_lane"], info["tma_staged"]))
    assert len(seen) == 18  # every index names a different configuration
    dims = (ctypes.c_int32 * 3)()
    assert lib.sslic_tile_shape_info(3, 12, dims, None, None) == -1
    assert lib.sslic_tile_shape_info(1, 0, dims, None, None) == -1
    assert lib.sslic_set_tile_shape(None, 0) == -1
    assert lib.sslic_autotune(None, None, None, None, 1, None, None) == -1


def test_tune_table_host_only(lib):
    from paper_1806_08741_gb300 import sslic as S
    S.tune_forget()
    p = S.Params(size=(300, 200, 100), grid=(16, 16, 16))
    assert S.tune_lookup(p) == -1
    S.tune_record(p, 7)
    assert S.tune_lookup(p) == 7
    assert S.tune_lookup(S.Params(size=(300, 200, 100), grid=(8, 8, 8))) == -1   # keyed by grid
    assert S.tune_lookup(S.Params(size=(50, 60, 70), grid=(16, 16, 16))) == 7    # not by size
    for bad in (-1, 12):
        with pytest.raises(S.SSLICError):
            S.tune_record(p, bad)
    with pytest.raises(S.SSLICError) as e:
        S.tune_record(S.Params(size=(64, 64), grid=(8, 8), channels=4, dtype=S.F32), 0)
    assert e.value.code == -6
    lab = S.Params(size=(64, 64), grid=(8, 8), channels=3, dtype=S.F32)   # 3-channel float has tiles
    S.tune_record(lab, 2)
    assert S.tune_lookup(lab) == 2
    S.tune_forget()
    assert S.tune_lookup(p) == -1


def test_srgb_to_lab_rejects_bad_arguments_without_touching_the_gpu(lib):
    # argument checks come before any CUDA call
    f = lib.sslic_srgb_to_lab
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
    assert f(None, None, 0, None) == 0                       # nothing to do
    assert f(None, None, -1, None) == -1                     # negative count
    assert f(None, 0x20000, 4, None) == -1                   # NULL input
    assert f(0x10000, None, 4, None) == -1                   # NULL output
    assert f(0x10000, 0x10000 + 8, 4, None) == -1            # output starts inside the input
    assert f(0x10000 + 40, 0x10000, 4, None) == -1           # input starts inside the output
    assert f(0x10000, 0x10000, 1 << 62, None) == -1          # byte count overflows


_CTYPES = {"int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64, "float": ctypes.c_float, "double": ctypes.c_double}


def _header_structs():
    """Every `typedef struct { ... } name;` of include/*.h as [(field, ctype), ...]."""
    out = {}
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        for body, name in re.findall(r"typedef\s+struct\s*\{(.*?)\}\s*(\w+)\s*;", text, flags=re.S):
            fields = []
            for decl in body.split(";"):
                decl = decl.strip()
                if not decl:
                    continue
                m = re.match(r"(\w+)\s+(.*)$", decl, flags=re.S)
                ctype = _CTYPES[m.group(1)]
                for part in m.group(2).split(","):
                    part = part.strip()
                    arr = re.match(r"(\w+)\s*\[\s*(\d+)\s*\]$", part)
                    if arr:
                        fields.append((arr.group(1), ctype * int(arr.group(2))))
                    else:
                        fields.append((part, ctype))
            out[name] = fields
    return out


def test_binding_structs_match_header():
    """The ctypes structures of the binding have the header's fields, types
    and order, so the layouts agree (a field added on one side only fails)."""
    from paper_1806_08741_gb300 import sslic as S
    structs = _header_structs()
    pairs = {"sslic_params": S._Params, "sslic_result": S._Result, "sslic_profile": S._Profile,
             "sslic_server_stats": S._ServerStats}
    assert set(pairs) <= set(structs)
    for name, cls in pairs.items():
        want = structs[name]
        got = list(cls._fields_)
        assert [f for f, _ in got] == [f for f, _ in want], name
        for (f, a), (_, b) in zip(got, want):
            assert ctypes.sizeof(a) == ctypes.sizeof(b) and ctypes.alignment(a) == ctypes.alignment(b), (name, f)
            assert getattr(a, "_type_", a) == getattr(b, "_type_", b) or a == b, (name, f)
