"""ctypes loader for the CPU oracle (sslic_oracle.c).

TEST INFRASTRUCTURE ONLY.  The product package never imports this module;
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` do.  The oracle is a plain single-threaded C restatement of the
paper's centre-centric SLIC/SSLIC (arXiv 1806.08741, Sec. 2.1-3.3); see the
header of ``sslic_oracle.c`` for the readings it applies where the paper is
silent.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sslic_oracle.c")
_HDR = os.path.join(_HERE, "sslic_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_LIB_OMP = os.path.join(_BUILD, "liboracle_omp.so")

U8, U16, F32 = 0, 1, 2
FP32, FP64 = 0, 1
_DTYPE_CODE = {np.dtype(np.uint8): U8, np.dtype(np.uint16): U16, np.dtype(np.float32): F32}


class _Params(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int32),
        ("size", ctypes.c_int64 * 4),
        ("channels", ctypes.c_int32),
        ("dtype", ctypes.c_int32),
        ("grid", ctypes.c_int32 * 4),
        ("m", ctypes.c_double),
        ("max_iter", ctypes.c_int32),
        ("conv_threshold", ctypes.c_double),
        ("perturb", ctypes.c_int32),
        ("enforce_connectivity", ctypes.c_int32),
        ("mode", ctypes.c_int32),
    ]


@dataclass
class Params:
    """Parameters of one oracle run; ``size`` and ``grid`` are listed with
    dimension 0 (the fastest-varying, x) first."""

    size: tuple
    grid: tuple
    channels: int = 3
    dtype: int = U8
    m: float = 10.0
    max_iter: int = 10
    conv_threshold: float = 0.0
    perturb: bool = True
    enforce_connectivity: bool = False
    mode: int = FP32

    @property
    def ndim(self) -> int:
        return len(self.size)

    def to_c(self) -> _Params:
        p = _Params()
        p.ndim = len(self.size)
        for d in range(4):
            p.size[d] = int(self.size[d]) if d < len(self.size) else 1
            p.grid[d] = int(self.grid[d]) if d < len(self.grid) else 1
        p.channels = int(self.channels)
        p.dtype = int(self.dtype)
        p.m = float(self.m)
        p.max_iter = int(self.max_iter)
        p.conv_threshold = float(self.conv_threshold)
        p.perturb = int(bool(self.perturb))
        p.enforce_connectivity = int(bool(self.enforce_connectivity))
        p.mode = int(self.mode)
        return p


def _compile(out: str, extra, force: bool) -> str:
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(out)) or force or any(
        os.path.getmtime(s) > os.path.getmtime(out) for s in (_SRC, _HDR))
    if stale:
        tmp = out + f".tmp{os.getpid()}"
        cmd = ["cc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", *extra,
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle with the system C compiler (no fast-math, no
    contraction) into ``oracle/_build/liboracle.so``, and the same source
    with OpenMP into ``liboracle_omp.so`` (the region-decomposed form of
    ``slic_regions`` then runs on several host threads)."""
    _compile(_LIB_OMP, ["-fopenmp"], force)
    return _compile(_LIB, [], force)


_lib = None


def _bind(L):
    """Declare the argument and result types of a loaded oracle library."""
    P = ctypes.POINTER(_Params)
    vp, dp = ctypes.c_void_p, ctypes.c_void_p
    L.oracle_num_clusters.argtypes = [P]
    L.oracle_num_clusters.restype = ctypes.c_int64
    L.oracle_seed.argtypes = [P, vp, dp]
    L.oracle_gradient.argtypes = [P, vp, ctypes.c_int64]
    L.oracle_gradient.restype = ctypes.c_double
    L.oracle_assign.argtypes = [P, vp, dp, ctypes.c_int64, vp]
    L.oracle_update.argtypes = [P, vp, vp, ctypes.c_int64, dp, vp, vp]
    L.oracle_distance.argtypes = [P, dp, vp, dp]
    L.oracle_distance.restype = ctypes.c_double
    L.oracle_connectivity.argtypes = [P, dp, ctypes.c_int64, vp, vp, vp]
    L.oracle_slic.argtypes = [P, vp, vp, dp, vp, vp, vp]
    L.oracle_slic_from.argtypes = [P, vp, dp, vp, dp, vp, vp, vp]
    L.oracle_srgb_to_lab.argtypes = [vp, ctypes.c_int64, dp]
    L.oracle_assign_voxels.argtypes = [P, vp, dp, ctypes.c_int64, vp, ctypes.c_int64, vp, vp, vp]
    L.oracle_assign_voxels.restype = ctypes.c_int
    L.oracle_slic_regions.argtypes = [P, vp, vp, dp, vp, vp, vp, ctypes.c_int]
    L.oracle_slic_regions.restype = ctypes.c_int
    L.oracle_threads_available.argtypes = []
    L.oracle_threads_available.restype = ctypes.c_int
    for f in ("oracle_seed", "oracle_assign", "oracle_update", "oracle_srgb_to_lab",
              "oracle_connectivity", "oracle_slic", "oracle_slic_from"):
        getattr(L, f).restype = ctypes.c_int
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = _bind(ctypes.CDLL(build()))
    return _lib


_lib_omp = None


def lib_omp():
    """The OpenMP build of the same source (region-decomposed form)."""
    global _lib_omp
    if _lib_omp is None:
        build()
        _lib_omp = _bind(ctypes.CDLL(_LIB_OMP))
    return _lib_omp


def build_variant(src_text: str, out_dir: str) -> str:
    """Compile a modified copy of the oracle source (the tests plant known
    mistakes in it to show that the pins catch them); returns the path of
    the shared library, built with the same flags as build()."""
    os.makedirs(out_dir, exist_ok=True)
    src = os.path.join(out_dir, "sslic_oracle.c")
    with open(src, "w") as f:
        f.write(src_text)
    out = os.path.join(out_dir, "liboracle_variant.so")
    cmd = ["cc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-I", _HERE,
           "-fPIC", "-shared", "-o", out, src, "-lm"]
    subprocess.run(cmd, check=True)
    return out


class use_library:
    """Context manager: route every oracle call through the library at
    ``path`` (a variant from build_variant) until the block ends."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        self.saved = lib()
        _lib = _bind(ctypes.CDLL(self.path))
        return _lib

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def params_for(image: np.ndarray, grid, **kw) -> Params:
    """Build Params from an image array shaped [N_{n-1},...,N_0, C]."""
    shape = image.shape[:-1]
    size = tuple(int(s) for s in reversed(shape))
    grid = tuple(int(g) for g in grid)
    if len(grid) == 1 and len(size) > 1:
        grid = grid * len(size)
    return Params(size=size, grid=grid, channels=int(image.shape[-1]),
                  dtype=_DTYPE_CODE[image.dtype], **kw)


def _img(image: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(image)


def num_clusters(p: Params) -> int:
    return int(lib().oracle_num_clusters(ctypes.byref(p.to_c())))


def seed(p: Params, image: np.ndarray) -> np.ndarray:
    image = _img(image)
    K = num_clusters(p)
    if K < 0:
        raise RuntimeError("oracle seed failed: invalid parameters")
    out = np.zeros((K, p.channels + p.ndim), np.float64)
    _check(lib().oracle_seed(ctypes.byref(p.to_c()), _ptr(image), _ptr(out)), "seed")
    return out


def gradient(p: Params, image: np.ndarray, q: int) -> float:
    image = _img(image)
    return float(lib().oracle_gradient(ctypes.byref(p.to_c()), _ptr(image), int(q)))


def distance(p: Params, feature, pos, centre) -> float:
    f = np.ascontiguousarray(feature, np.float64)
    x = np.ascontiguousarray(pos, np.int64)
    c = np.ascontiguousarray(centre, np.float64)
    return float(lib().oracle_distance(ctypes.byref(p.to_c()), _ptr(f), _ptr(x), _ptr(c)))


def srgb_to_lab(rgb: np.ndarray) -> np.ndarray:
    """8-bit sRGB [..., 3] -> CIE-Lab float64 [..., 3] (reading R16: sRGB,
    D65 white, CIE 1976 L*a*b*; the paper's colour space, Sec. 2.1 and 4.1)."""
    rgb = np.ascontiguousarray(rgb, np.uint8)
    if rgb.shape[-1] != 3:
        raise ValueError("srgb_to_lab wants a trailing axis of 3 channels")
    out = np.empty(rgb.shape, np.float64)
    _check(lib().oracle_srgb_to_lab(_ptr(rgb), rgb.size // 3, _ptr(out)), "srgb_to_lab")
    return out


def assign(p: Params, image: np.ndarray, centres: np.ndarray) -> np.ndarray:
    image = _img(image)
    c = np.ascontiguousarray(centres, np.float64)
    labels = np.empty(image.shape[:-1], np.int32)
    _check(lib().oracle_assign(ctypes.byref(p.to_c()), _ptr(image), _ptr(c), c.shape[0],
                               _ptr(labels)), "assign")
    return labels


def assign_voxels(p: Params, image: np.ndarray, centres: np.ndarray, q, cand_start, cand) -> np.ndarray:
    """The labels ``assign`` would give at the raster indices ``q`` only (for
    images too large to assign whole); the candidates of voxel i are
    ``cand[cand_start[i]:cand_start[i+1]]`` and must include every centre
    whose window covers it."""
    image = _img(image)
    c = np.ascontiguousarray(centres, np.float64)
    q = np.ascontiguousarray(q, np.int64)
    cs = np.ascontiguousarray(cand_start, np.int64)
    cd = np.ascontiguousarray(cand, np.int64)
    if cs.shape[0] != q.shape[0] + 1:
        raise ValueError("cand_start needs len(q) + 1 entries")
    out = np.empty(q.shape[0], np.int32)
    _check(lib().oracle_assign_voxels(ctypes.byref(p.to_c()), _ptr(image), _ptr(c), c.shape[0], _ptr(q),
                                      q.shape[0], _ptr(cs), _ptr(cd), _ptr(out)), "assign_voxels")
    return out


def update(p: Params, image: np.ndarray, labels: np.ndarray, centres: np.ndarray):
    image = _img(image)
    lab = np.ascontiguousarray(labels, np.int32)
    c = np.array(centres, np.float64, copy=True, order="C")
    counts = np.zeros(c.shape[0], np.int64)
    res = ctypes.c_double(0.0)
    _check(lib().oracle_update(ctypes.byref(p.to_c()), _ptr(image), _ptr(lab), c.shape[0],
                               _ptr(c), _ptr(counts), ctypes.byref(res)), "update")
    return c, counts, res.value


def connectivity(p: Params, centres: np.ndarray, labels: np.ndarray):
    c = np.ascontiguousarray(centres, np.float64)
    lab = np.ascontiguousarray(labels, np.int32)
    out = np.empty_like(lab)
    n = ctypes.c_int64(0)
    _check(lib().oracle_connectivity(ctypes.byref(p.to_c()), _ptr(c), c.shape[0], _ptr(lab),
                                     _ptr(out), ctypes.byref(n)), "connectivity")
    return out, int(n.value)


def slic(p: Params, image: np.ndarray, init_centres: np.ndarray | None = None) -> dict:
    """Whole method: seeding (or the given centres), ``max_iter`` assign/update
    iterations, optional connectivity.  Returns labels, centres (K x (C+n)),
    iterations done, last residual and the label count."""
    image = _img(image)
    K = num_clusters(p)
    if K < 0:
        raise RuntimeError("oracle slic failed: invalid parameters")
    labels = np.empty(image.shape[:-1], np.int32)
    centres = np.zeros((K, p.channels + p.ndim), np.float64)
    it = ctypes.c_int32(0)
    res = ctypes.c_double(0.0)
    n = ctypes.c_int64(0)
    pc = p.to_c()
    if init_centres is None:
        rc = lib().oracle_slic(ctypes.byref(pc), _ptr(image), _ptr(labels), _ptr(centres),
                               ctypes.byref(it), ctypes.byref(res), ctypes.byref(n))
    else:
        ic = np.ascontiguousarray(init_centres, np.float64)
        rc = lib().oracle_slic_from(ctypes.byref(pc), _ptr(image), _ptr(ic), _ptr(labels),
                                    _ptr(centres), ctypes.byref(it), ctypes.byref(res),
                                    ctypes.byref(n))
    _check(rc, "slic")
    return {"labels": labels, "centres": centres, "iterations": int(it.value),
            "residual": float(res.value), "num_labels": int(n.value)}


def threads_available() -> int:
    """Host threads the OpenMP build uses by default."""
    return int(lib_omp().oracle_threads_available())


def slic_regions(p: Params, image: np.ndarray, threads: int, openmp: bool = True) -> dict:
    """The whole method in the paper's multi-threaded form (Sec. 3.1): the
    image split into non-overlapping regions of planes, assigned and mapped
    per region on ``threads`` host threads (OpenMP build), the per-region
    sums merged per label.  Same results as ``slic`` bit for bit."""
    image = _img(image)
    K = num_clusters(p)
    if K < 0:
        raise RuntimeError("oracle slic_regions failed: invalid parameters")
    labels = np.empty(image.shape[:-1], np.int32)
    centres = np.zeros((K, p.channels + p.ndim), np.float64)
    it = ctypes.c_int32(0)
    res = ctypes.c_double(0.0)
    n = ctypes.c_int64(0)
    L = lib_omp() if openmp else lib()
    _check(L.oracle_slic_regions(ctypes.byref(p.to_c()), _ptr(image), _ptr(labels), _ptr(centres),
                                 ctypes.byref(it), ctypes.byref(res), ctypes.byref(n), int(threads)),
           "slic_regions")
    return {"labels": labels, "centres": centres, "iterations": int(it.value),
            "residual": float(res.value), "num_labels": int(n.value)}
