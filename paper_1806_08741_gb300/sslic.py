"""Thin Python binding of the SSLIC C ABI (include/sslic.h).

Argument marshalling only: every step of the method runs in the sm_103a
kernels of ``libsslic.so``.  Tensors are torch tensors (device memory and
streams come from PyTorch); their data pointers are handed to the library
unchanged.  There is no CPU fallback: if the library cannot be loaded, or a
call fails, an exception is raised.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsslic.so")

SSLIC_OK = 0
U8, U16, F32 = 0, 1, 2
_ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ETIMEOUT", -5: "EBUSY", -6: "EUNSUPPORTED"}

EXPORTS = ("sslic_default_params", "sslic_create", "sslic_num_clusters", "sslic_run",
           "sslic_run_from", "sslic_run_host", "sslic_run_streamed", "sslic_seed", "sslic_iterate",
           "sslic_connectivity", "sslic_iterate_static", "sslic_server_create",
           "sslic_server_submit", "sslic_server_wait", "sslic_server_stats_get",
           "sslic_server_destroy", "sslic_num_tile_shapes", "sslic_tile_shape_info",
           "sslic_set_tile_shape", "sslic_get_tile_shape", "sslic_autotune", "sslic_tune_forget",
           "sslic_tune_record", "sslic_tune_lookup", "sslic_precision_probe", "sslic_srgb_to_lab",
           "sslic_profile_enable", "sslic_profile_read", "sslic_set_loop_graph", "sslic_destroy",
           "sslic_strerror", "sslic_last_error", "sslic_shard_seed", "sslic_shard_sums_size",
           "sslic_shard_map", "sslic_shard_finalize", "sslic_conn_slabs_begin", "sslic_conn_slabs_add",
           "sslic_conn_slabs_finish", "sslic_conn_slabs_relabel")
PHASES = ("seed", "bins", "assign", "assign_voxel", "finalize", "connectivity")


class SSLICError(RuntimeError):
    def __init__(self, code: int, what: str, detail: str = ""):
        self.code = code
        super().__init__(f"{what} failed: {_ERRORS.get(code, code)} {detail}".strip())


class _Params(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int32),
        ("size", ctypes.c_int64 * 4),
        ("channels", ctypes.c_int32),
        ("dtype", ctypes.c_int32),
        ("grid", ctypes.c_int32 * 4),
        ("m", ctypes.c_float),
        ("max_iter", ctypes.c_int32),
        ("conv_threshold", ctypes.c_double),
        ("perturb", ctypes.c_int32),
        ("enforce_connectivity", ctypes.c_int32),
        ("precision", ctypes.c_int32),
    ]


class _Profile(ctypes.Structure):
    _fields_ = [
        ("ms", ctypes.c_double * 8),
        ("calls", ctypes.c_int64 * 8),
        ("kernel_launches", ctypes.c_int64),
        ("rechecks", ctypes.c_int64),
    ]


class _ServerStats(ctypes.Structure):
    _fields_ = [
        ("submitted", ctypes.c_int64),
        ("completed", ctypes.c_int64),
        ("rejected", ctypes.c_int64),
        ("rounds", ctypes.c_int64),
        ("max_active", ctypes.c_int32),
        ("status", ctypes.c_int32),
        ("peak_bytes", ctypes.c_int64),
        ("voxel_iters", ctypes.c_double),
        ("busy_s", ctypes.c_double),
        ("p50_ms", ctypes.c_double),
        ("p99_ms", ctypes.c_double),
        ("mean_ms", ctypes.c_double),
        ("graph_launches", ctypes.c_int64),
        ("graph_captures", ctypes.c_int64),
        ("eager_rounds", ctypes.c_int64),
    ]


class _Result(ctypes.Structure):
    _fields_ = [
        ("num_clusters", ctypes.c_int64),
        ("num_labels", ctypes.c_int64),
        ("iterations", ctypes.c_int32),
        ("residual", ctypes.c_double),
    ]


_lib = None


def load(path: str = LIB_PATH):
    """Load libsslic.so (built by ``paper_1806_08741_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: run __graft_entry__.build() first")
    L = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    P = ctypes.POINTER(_Params)
    R = ctypes.POINTER(_Result)
    C = ctypes.c_void_p  # sslic_ctx*
    L.sslic_default_params.argtypes = [ctypes.c_int32, P]
    L.sslic_create.argtypes = [P, ctypes.POINTER(C)]
    L.sslic_num_clusters.argtypes = [C, ctypes.POINTER(ctypes.c_int64)]
    L.sslic_run.argtypes = [C, vp, vp, vp, vp, R]
    L.sslic_run_from.argtypes = [C, vp, vp, vp, vp, vp, R]
    L.sslic_run_host.argtypes = [C, vp, vp, vp, vp, R]
    L.sslic_run_streamed.argtypes = [C, vp, vp, vp, ctypes.c_int64, vp, R]
    i64, pi64 = ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)
    L.sslic_shard_seed.argtypes = [C, vp, i64, i64, vp, vp]
    L.sslic_shard_sums_size.argtypes = [C, pi64, pi64]
    L.sslic_shard_map.argtypes = [C, vp, vp, i64, i64, vp, vp, vp]
    L.sslic_shard_finalize.argtypes = [C, vp, vp, vp, ctypes.POINTER(ctypes.c_double), vp]
    L.sslic_conn_slabs_begin.argtypes = [C, vp, vp]
    L.sslic_conn_slabs_add.argtypes = [C, vp, i64, i64, vp]
    L.sslic_conn_slabs_finish.argtypes = [C, vp, pi64]
    L.sslic_conn_slabs_relabel.argtypes = [C, vp, i64, i64, vp]
    for f in ("sslic_shard_seed", "sslic_shard_sums_size", "sslic_shard_map", "sslic_shard_finalize",
              "sslic_conn_slabs_begin", "sslic_conn_slabs_add", "sslic_conn_slabs_finish",
              "sslic_conn_slabs_relabel"):
        getattr(L, f).restype = ctypes.c_int
    L.sslic_seed.argtypes = [C, vp, vp, vp]
    L.sslic_iterate.argtypes = [C, vp, vp, vp, vp, vp, ctypes.POINTER(ctypes.c_double)]
    L.sslic_connectivity.argtypes = [C, vp, vp, vp, vp, ctypes.POINTER(ctypes.c_int64)]
    S_ = ctypes.c_void_p  # sslic_server*
    L.sslic_server_create.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(S_)]
    L.sslic_server_submit.argtypes = [S_, P, vp, vp, vp, ctypes.POINTER(ctypes.c_int64)]
    L.sslic_server_wait.argtypes = [S_, ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]
    L.sslic_server_stats_get.argtypes = [S_, ctypes.POINTER(_ServerStats)]
    L.sslic_server_destroy.argtypes = [S_]
    L.sslic_server_destroy.restype = None
    for f in ("sslic_server_create", "sslic_server_submit", "sslic_server_wait", "sslic_server_stats_get"):
        getattr(L, f).restype = ctypes.c_int
    i32p = ctypes.POINTER(ctypes.c_int32)
    L.sslic_num_tile_shapes.argtypes = [ctypes.c_int32, i32p]
    L.sslic_tile_shape_info.argtypes = [ctypes.c_int32, ctypes.c_int32, i32p, i32p, i32p]
    L.sslic_set_tile_shape.argtypes = [C, ctypes.c_int32]
    L.sslic_get_tile_shape.argtypes = [C, i32p]
    L.sslic_autotune.argtypes = [C, vp, vp, vp, ctypes.c_int32, i32p, ctypes.POINTER(ctypes.c_float)]
    L.sslic_tune_forget.argtypes = []
    L.sslic_tune_record.argtypes = [P, ctypes.c_int32]
    L.sslic_tune_lookup.argtypes = [P, i32p]
    L.sslic_precision_probe.argtypes = [C, vp, vp, ctypes.c_int64, vp, vp, vp]
    L.sslic_precision_probe.restype = ctypes.c_int
    for f in ("sslic_num_tile_shapes", "sslic_tile_shape_info", "sslic_set_tile_shape",
              "sslic_get_tile_shape", "sslic_autotune", "sslic_tune_forget", "sslic_tune_record",
              "sslic_tune_lookup"):
        getattr(L, f).restype = ctypes.c_int
    L.sslic_iterate_static.argtypes = [P, vp, vp, vp, vp, vp]
    L.sslic_srgb_to_lab.argtypes = [vp, vp, ctypes.c_int64, vp]
    L.sslic_srgb_to_lab.restype = ctypes.c_int
    L.sslic_iterate_static.restype = ctypes.c_int
    L.sslic_profile_enable.argtypes = [C, ctypes.c_int32]
    L.sslic_set_loop_graph.argtypes = [C, ctypes.c_int32]
    L.sslic_set_loop_graph.restype = ctypes.c_int
    L.sslic_profile_read.argtypes = [C, ctypes.POINTER(_Profile)]
    L.sslic_profile_enable.restype = ctypes.c_int
    L.sslic_profile_read.restype = ctypes.c_int
    L.sslic_destroy.argtypes = [C]
    L.sslic_destroy.restype = None
    L.sslic_strerror.argtypes = [ctypes.c_int]
    L.sslic_strerror.restype = ctypes.c_char_p
    L.sslic_last_error.argtypes = [C]
    L.sslic_last_error.restype = ctypes.c_char_p
    for f in ("sslic_default_params", "sslic_create", "sslic_num_clusters", "sslic_run",
              "sslic_run_from", "sslic_run_host", "sslic_seed", "sslic_iterate",
              "sslic_connectivity"):
        getattr(L, f).restype = ctypes.c_int
    _lib = L
    return L


@dataclass
class Params:
    """The paper's filter parameters (Sec. 3.2).  ``size`` and ``grid`` list
    axis 0 (x, fastest) first."""

    size: tuple
    grid: tuple
    channels: int = 3
    dtype: int = U8
    m: float = 10.0
    max_iter: int = 10
    conv_threshold: float = 0.0
    perturb: bool = True
    enforce_connectivity: bool = False
    precision: int = 0

    @property
    def ndim(self) -> int:
        return len(self.size)

    def to_c(self) -> _Params:
        p = _Params()
        p.ndim = len(self.size)
        grid = tuple(self.grid)
        if len(grid) == 1:
            grid = grid * len(self.size)
        for d in range(4):
            p.size[d] = int(self.size[d]) if d < len(self.size) else 1
            p.grid[d] = int(grid[d]) if d < len(grid) else 1
        p.channels = int(self.channels)
        p.dtype = int(self.dtype)
        p.m = float(self.m)
        p.max_iter = int(self.max_iter)
        p.conv_threshold = float(self.conv_threshold)
        p.perturb = int(bool(self.perturb))
        p.enforce_connectivity = int(bool(self.enforce_connectivity))
        p.precision = int(self.precision)
        return p


def _dtype_code(t) -> int:
    import torch
    return {torch.uint8: U8, torch.uint16: U16, torch.float32: F32}[t.dtype]


def params_for(image, grid, **kw) -> Params:
    """Params for an image tensor/array shaped [N_{n-1}, ..., N_0, C]."""
    shape = tuple(image.shape)
    size = tuple(int(s) for s in reversed(shape[:-1]))
    if isinstance(image, np.ndarray):
        dt = {np.dtype(np.uint8): U8, np.dtype(np.uint16): U16, np.dtype(np.float32): F32}[image.dtype]
    else:
        dt = _dtype_code(image)
    return Params(size=size, grid=tuple(grid), channels=int(shape[-1]), dtype=dt, **kw)


def _ptr(t) -> ctypes.c_void_p:
    if t is None:
        return ctypes.c_void_p(0)
    if isinstance(t, np.ndarray):
        return ctypes.c_void_p(t.ctypes.data)
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


class Context:
    """One SSLIC context (device workspace sized for one image shape)."""

    def __init__(self, params: Params):
        self.lib = load()
        self.params = params
        self._c = ctypes.c_void_p(0)
        rc = self.lib.sslic_create(ctypes.byref(params.to_c()), ctypes.byref(self._c))
        if rc != SSLIC_OK:
            raise SSLICError(rc, "sslic_create")
        k = ctypes.c_int64(0)
        self._check(self.lib.sslic_num_clusters(self._c, ctypes.byref(k)), "sslic_num_clusters")
        self.K = int(k.value)

    # -- helpers -----------------------------------------------------------------
    def _check(self, rc: int, what: str):
        if rc != SSLIC_OK:
            detail = self.lib.sslic_last_error(self._c) if self._c else b""
            raise SSLICError(rc, what, (detail or b"").decode())

    @property
    def centre_width(self) -> int:
        return self.params.channels + self.params.ndim

    def _need(self, t, numel, what, device=True):
        if t is None:
            return
        n = t.size if isinstance(t, np.ndarray) else t.numel()
        if n != numel:
            raise ValueError(f"{what}: expected {numel} elements, got {n}")
        if isinstance(t, np.ndarray):
            if device:
                raise ValueError(f"{what} must be a device tensor")
            if not t.flags["C_CONTIGUOUS"]:
                raise ValueError(f"{what} must be contiguous")
        else:
            if device != t.is_cuda:
                raise ValueError(f"{what} must be on the {'GPU' if device else 'host'}")
            if not t.is_contiguous():
                raise ValueError(f"{what} must be contiguous")

    def _voxels(self) -> int:
        return int(np.prod(self.params.size))

    # -- the C ABI -----------------------------------------------------------------
    def run(self, image, labels, centres=None, stream=None) -> dict:
        V = self._voxels()
        self._need(image, V * self.params.channels, "image")
        self._need(labels, V, "labels")
        self._need(centres, self.K * self.centre_width, "centres")
        r = _Result()
        self._check(self.lib.sslic_run(self._c, _ptr(image), _ptr(labels), _ptr(centres),
                                       _stream(stream), ctypes.byref(r)), "sslic_run")
        return {"num_clusters": r.num_clusters, "num_labels": r.num_labels,
                "iterations": r.iterations, "residual": r.residual}

    def run_async(self, image, labels, centres=None, stream=None) -> None:
        """sslic_run without the result read-back (stays stream ordered when
        the convergence threshold is off and connectivity is disabled)."""
        V = self._voxels()
        self._need(image, V * self.params.channels, "image")
        self._need(labels, V, "labels")
        self._need(centres, self.K * self.centre_width, "centres")
        self._check(self.lib.sslic_run(self._c, _ptr(image), _ptr(labels), _ptr(centres),
                                       _stream(stream), None), "sslic_run")

    def run_from(self, image, init_centres, labels, centres=None, stream=None) -> dict:
        V = self._voxels()
        self._need(image, V * self.params.channels, "image")
        self._need(init_centres, self.K * self.centre_width, "init_centres")
        self._need(labels, V, "labels")
        self._need(centres, self.K * self.centre_width, "centres")
        r = _Result()
        self._check(self.lib.sslic_run_from(self._c, _ptr(image), _ptr(init_centres), _ptr(labels),
                                            _ptr(centres), _stream(stream), ctypes.byref(r)),
                    "sslic_run_from")
        return {"num_clusters": r.num_clusters, "num_labels": r.num_labels,
                "iterations": r.iterations, "residual": r.residual}

    def run_host(self, image, labels, centres=None, stream=None) -> dict:
        """Host buffers (numpy arrays or CPU tensors, ideally pinned)."""
        V = self._voxels()
        self._need(image, V * self.params.channels, "image", device=False)
        self._need(labels, V, "labels", device=False)
        self._need(centres, self.K * self.centre_width, "centres", device=False)
        r = _Result()
        self._check(self.lib.sslic_run_host(self._c, _ptr(image), _ptr(labels), _ptr(centres),
                                            _stream(stream), ctypes.byref(r)), "sslic_run_host")
        return {"num_clusters": r.num_clusters, "num_labels": r.num_labels,
                "iterations": r.iterations, "residual": r.residual}

    def run_streamed(self, image, labels, centres=None, slab_planes: int = 64, stream=None) -> dict:
        """The whole method with the image in host memory, streamed through
        the GPU in slabs of slab_planes planes along the last axis every
        iteration (sslic_run_streamed; host buffers, ideally pinned)."""
        V = self._voxels()
        self._need(image, V * self.params.channels, "image", device=False)
        self._need(labels, V, "labels", device=False)
        self._need(centres, self.K * self.centre_width, "centres", device=False)
        r = _Result()
        self._check(self.lib.sslic_run_streamed(self._c, _ptr(image), _ptr(labels), _ptr(centres),
                                                int(slab_planes), _stream(stream), ctypes.byref(r)),
                    "sslic_run_streamed")
        return {"num_clusters": r.num_clusters, "num_labels": r.num_labels,
                "iterations": r.iterations, "residual": r.residual}

    # -- one image shared by several GPUs: the calls of one rank ----------------
    def _plane(self) -> int:
        return int(np.prod(self.params.size[:-1]))

    def shard_seed(self, image_halo, lo: int, hi: int, centres, stream=None) -> None:
        """Seeds of the lattice planes in [lo, hi) (sslic_shard_seed);
        image_halo holds planes [max(0, lo-2), min(N, hi+2)) of the image;
        the other rows of centres are left zero."""
        NL = self.params.size[-1]
        a, b = max(0, lo - 2), min(NL, hi + 2)
        self._need(image_halo, (b - a) * self._plane() * self.params.channels, "image slab")
        self._need(centres, self.K * self.centre_width, "centres")
        self._check(self.lib.sslic_shard_seed(self._c, _ptr(image_halo), int(lo), int(hi), _ptr(centres),
                                              _stream(stream)), "sslic_shard_seed")

    def shard_sums_size(self) -> tuple:
        """(uint64 count, double count) of one rank's sums (sslic_shard_sums_size)."""
        nu, nf = ctypes.c_int64(0), ctypes.c_int64(0)
        self._check(self.lib.sslic_shard_sums_size(self._c, ctypes.byref(nu), ctypes.byref(nf)),
                    "sslic_shard_sums_size")
        return int(nu.value), int(nf.value)

    def shard_map(self, image_slab, labels_slab, lo: int, hi: int, centres, sums, stream=None) -> None:
        """Assignment of planes [lo, hi) and the map of their sums into
        ``sums`` (a device buffer of the sslic_shard_sums_size layout)."""
        n = (hi - lo) * self._plane()
        self._need(image_slab, n * self.params.channels, "image slab")
        self._need(labels_slab, n, "label slab")
        self._need(centres, self.K * self.centre_width, "centres")
        nu, nf = self.shard_sums_size()
        if sums.numel() * sums.element_size() != 8 * (nu + nf) or not sums.is_cuda:
            raise ValueError(f"sums: expected a device buffer of {8 * (nu + nf)} bytes")
        self._check(self.lib.sslic_shard_map(self._c, _ptr(image_slab), _ptr(labels_slab), int(lo), int(hi),
                                             _ptr(centres), _ptr(sums), _stream(stream)), "sslic_shard_map")

    def shard_finalize(self, sums, centres_prev, centres_out, residual: bool = False, stream=None):
        """Centres from the sums of every rank (sslic_shard_finalize)."""
        self._need(centres_prev, self.K * self.centre_width, "centres_prev")
        self._need(centres_out, self.K * self.centre_width, "centres_out")
        res = ctypes.c_double(0.0)
        self._check(self.lib.sslic_shard_finalize(self._c, _ptr(sums), _ptr(centres_prev), _ptr(centres_out),
                                                  ctypes.byref(res) if residual else None, _stream(stream)),
                    "sslic_shard_finalize")
        return res.value if residual else None

    def conn_slabs_begin(self, centres, stream=None) -> None:
        self._need(centres, self.K * self.centre_width, "centres")
        self._check(self.lib.sslic_conn_slabs_begin(self._c, _ptr(centres), _stream(stream)),
                    "sslic_conn_slabs_begin")

    def conn_slabs_add(self, labels_slab, lo: int, hi: int, stream=None) -> None:
        self._need(labels_slab, (hi - lo) * self._plane(), "label slab")
        self._check(self.lib.sslic_conn_slabs_add(self._c, _ptr(labels_slab), int(lo), int(hi), _stream(stream)),
                    "sslic_conn_slabs_add")

    def conn_slabs_finish(self, stream=None) -> int:
        n = ctypes.c_int64(0)
        self._check(self.lib.sslic_conn_slabs_finish(self._c, _stream(stream), ctypes.byref(n)),
                    "sslic_conn_slabs_finish")
        return int(n.value)

    def conn_slabs_relabel(self, labels_out_slab, lo: int, hi: int, stream=None) -> None:
        self._need(labels_out_slab, (hi - lo) * self._plane(), "label slab")
        self._check(self.lib.sslic_conn_slabs_relabel(self._c, _ptr(labels_out_slab), int(lo), int(hi),
                                                      _stream(stream)), "sslic_conn_slabs_relabel")

    def seed(self, image, centres, stream=None) -> None:
        self._need(image, self._voxels() * self.params.channels, "image")
        self._need(centres, self.K * self.centre_width, "centres")
        self._check(self.lib.sslic_seed(self._c, _ptr(image), _ptr(centres), _stream(stream)),
                    "sslic_seed")

    def iterate(self, image, centres_in, labels, centres_out, stream=None,
                residual: bool = False):
        V = self._voxels()
        self._need(image, V * self.params.channels, "image")
        self._need(centres_in, self.K * self.centre_width, "centres_in")
        self._need(labels, V, "labels")
        self._need(centres_out, self.K * self.centre_width, "centres_out")
        res = ctypes.c_double(0.0)
        self._check(self.lib.sslic_iterate(self._c, _ptr(image), _ptr(centres_in), _ptr(labels),
                                           _ptr(centres_out), _stream(stream),
                                           ctypes.byref(res) if residual else None),
                    "sslic_iterate")
        return res.value if residual else None

    def connectivity(self, centres, labels_in, labels_out, stream=None) -> int:
        V = self._voxels()
        self._need(centres, self.K * self.centre_width, "centres")
        self._need(labels_in, V, "labels_in")
        self._need(labels_out, V, "labels_out")
        n = ctypes.c_int64(0)
        self._check(self.lib.sslic_connectivity(self._c, _ptr(centres), _ptr(labels_in),
                                                _ptr(labels_out), _stream(stream), ctypes.byref(n)),
                    "sslic_connectivity")
        return int(n.value)

    # -- launch configuration --------------------------------------------------------
    @property
    def tile_shape(self) -> int:
        """Tile shape index the next run uses (-1: per-voxel kernel)."""
        v = ctypes.c_int32(0)
        self._check(self.lib.sslic_get_tile_shape(self._c, ctypes.byref(v)), "sslic_get_tile_shape")
        return int(v.value)

    @tile_shape.setter
    def tile_shape(self, shape: int) -> None:
        self._check(self.lib.sslic_set_tile_shape(self._c, int(shape)), "sslic_set_tile_shape")

    def autotune(self, image, labels, reps: int = 3, stream=None) -> dict:
        """Time every tile shape on this image (sslic_autotune); the fastest
        becomes this context's shape.  Returns {'best': i, 'ms': [...]}."""
        V = self._voxels()
        self._need(image, V * self.params.channels, "image")
        self._need(labels, V, "labels")
        n = num_tile_shapes(self.params.ndim)
        ms = (ctypes.c_float * max(n, 1))()
        best = ctypes.c_int32(-1)
        self._check(self.lib.sslic_autotune(self._c, _ptr(image), _ptr(labels), _stream(stream), int(reps),
                                            ctypes.byref(best), ms), "sslic_autotune")
        return {"best": int(best.value), "ms": [float(ms[i]) for i in range(n)]}

    def precision_probe(self, image, centres, tile: int, stream=None) -> dict:
        """What the tensor-core form's MMA computes on one 128-voxel tile
        (sslic_precision_probe): {'dots': (128, 32), 'cand': (32,), 'mu': (C,)}."""
        V = self._voxels()
        self._need(image, V * self.params.channels, "image")
        self._need(centres, self.K * self.centre_width, "centres")
        dots = np.zeros((128, 32), np.float32)
        cand = np.zeros(32, np.int32)
        mu = np.zeros(self.params.channels, np.float32)
        self._check(self.lib.sslic_precision_probe(self._c, _ptr(image), _ptr(centres), int(tile),
                                                   _ptr(dots), _ptr(cand), _ptr(mu)), "sslic_precision_probe")
        return {"dots": dots, "cand": cand, "mu": mu}

    def profile_enable(self, on: bool = True) -> None:
        """Start (or stop) per-phase CUDA-event timing; resets the counters."""
        self._check(self.lib.sslic_profile_enable(self._c, int(bool(on))), "sslic_profile_enable")

    def set_loop_graph(self, on: bool = True) -> None:
        """Replay the iterated loop of a run from a CUDA graph (default) or launch it eagerly."""
        self._check(self.lib.sslic_set_loop_graph(self._c, int(bool(on))), "sslic_set_loop_graph")

    def profile_read(self) -> dict:
        """{phase: (ms, calls)} plus 'kernel_launches' since the last enable."""
        p = _Profile()
        self._check(self.lib.sslic_profile_read(self._c, ctypes.byref(p)), "sslic_profile_read")
        out = {name: (p.ms[i], int(p.calls[i])) for i, name in enumerate(PHASES)}
        out["kernel_launches"] = int(p.kernel_launches)
        out["rechecks"] = int(p.rechecks)
        return out

    def close(self):
        if self._c:
            self.lib.sslic_destroy(self._c)
            self._c = ctypes.c_void_p(0)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def num_tile_shapes(ndim: int) -> int:
    v = ctypes.c_int32(0)
    rc = load().sslic_num_tile_shapes(int(ndim), ctypes.byref(v))
    if rc != SSLIC_OK:
        raise SSLICError(rc, "sslic_num_tile_shapes")
    return int(v.value)


def tile_shape_info(ndim: int, shape: int) -> dict:
    dims = (ctypes.c_int32 * 3)()
    vl = ctypes.c_int32(0)
    tma = ctypes.c_int32(0)
    rc = load().sslic_tile_shape_info(int(ndim), int(shape), dims, ctypes.byref(vl), ctypes.byref(tma))
    if rc != SSLIC_OK:
        raise SSLICError(rc, "sslic_tile_shape_info")
    return {"dims": tuple(int(d) for d in dims), "voxels_per_lane": int(vl.value), "tma_staged": bool(tma.value)}


def tune_forget() -> None:
    """Forget every shape measured by autotune in this process."""
    load().sslic_tune_forget()


def tune_record(params: Params, shape: int) -> None:
    """Record a tile shape for the image type and grid of ``params`` (used
    by later contexts and servers), e.g. one measured in an earlier run."""
    rc = load().sslic_tune_record(ctypes.byref(params.to_c()), int(shape))
    if rc != SSLIC_OK:
        raise SSLICError(rc, "sslic_tune_record")


def tune_lookup(params: Params) -> int:
    """The recorded tile shape for ``params``' image type and grid, or -1."""
    v = ctypes.c_int32(-1)
    rc = load().sslic_tune_lookup(ctypes.byref(params.to_c()), ctypes.byref(v))
    if rc != SSLIC_OK:
        raise SSLICError(rc, "sslic_tune_lookup")
    return int(v.value)


def iterate_static(params: Params, image, centres_in, labels, centres_out, stream=None) -> None:
    """One assign + update iteration through sslic_iterate_static: no
    allocation at all (a fixed device array of the library holds the
    workspace; K <= 16384, C <= 4).  For callers that cannot allocate device
    memory.  Tensors as for Context.iterate."""
    L = load()
    V = int(np.prod(params.size))
    K = 1
    grid = tuple(params.grid) * (len(params.size) if len(params.grid) == 1 else 1)
    for n_d, s_d in zip(params.size, grid):
        K *= -(-int(n_d) // int(s_d))
    W = params.channels + len(params.size)
    for t, n, what in ((image, V * params.channels, "image"), (labels, V, "labels"),
                       (centres_in, K * W, "centres_in"), (centres_out, K * W, "centres_out")):
        if t.numel() != n or not t.is_cuda or not t.is_contiguous():
            raise ValueError(f"{what}: expected a contiguous device tensor of {n} elements")
    rc = L.sslic_iterate_static(ctypes.byref(params.to_c()), _ptr(image), _ptr(centres_in),
                                _ptr(labels), _ptr(centres_out), _stream(stream))
    if rc != SSLIC_OK:
        raise SSLICError(rc, "sslic_iterate_static")


def srgb_to_lab(rgb, out=None, stream=None):
    """8-bit sRGB [..., 3] device tensor -> CIE-Lab float32 [..., 3] through
    sslic_srgb_to_lab (sRGB, D65 white, CIE 1976 L*a*b*; the colour space the
    paper clusters in, Sec. 2.1, 4.1).  ``out`` (optional) receives it."""
    import torch
    if rgb.dtype != torch.uint8 or rgb.shape[-1] != 3 or not rgb.is_cuda or not rgb.is_contiguous():
        raise ValueError("rgb: expected a contiguous uint8 device tensor [..., 3]")
    if out is None:
        out = torch.empty(rgb.shape, dtype=torch.float32, device=rgb.device)
    elif out.dtype != torch.float32 or out.shape != rgb.shape or not out.is_cuda or not out.is_contiguous():
        raise ValueError("out: expected a contiguous float32 device tensor shaped like rgb")
    rc = load().sslic_srgb_to_lab(_ptr(rgb), _ptr(out), rgb.numel() // 3, _stream(stream))
    if rc != SSLIC_OK:
        raise SSLICError(rc, "sslic_srgb_to_lab")
    return out


class Server:
    """Continuous-batching server (sslic_server_*): requests of any size, grid
    and type are kept on the device and advanced together, one iteration per
    round, one launch per phase for the whole batch; admission is bounded by
    a device-memory budget.  Host buffers passed to submit() must stay alive
    until wait() returns for the ticket (this object keeps references)."""

    def __init__(self, budget_bytes: int, max_active: int = 64):
        self.lib = load()
        self._s = ctypes.c_void_p(0)
        rc = self.lib.sslic_server_create(int(budget_bytes), int(max_active), ctypes.byref(self._s))
        if rc != SSLIC_OK:
            raise SSLICError(rc, "sslic_server_create")
        self._keep = {}

    def submit(self, params: Params, image, labels, centres=None) -> int:
        t = ctypes.c_int64(0)
        rc = self.lib.sslic_server_submit(self._s, ctypes.byref(params.to_c()), _ptr(image), _ptr(labels),
                                          _ptr(centres), ctypes.byref(t))
        if rc != SSLIC_OK:
            raise SSLICError(rc, "sslic_server_submit")
        self._keep[int(t.value)] = (image, labels, centres)
        return int(t.value)

    def wait(self, ticket: int, timeout_s: float = 600.0) -> float:
        """Block until the ticket is done; returns its latency in ms."""
        lat = ctypes.c_double(0.0)
        import time
        t_end = time.monotonic() + timeout_s
        while True:
            rc = self.lib.sslic_server_wait(self._s, int(ticket), 100, ctypes.byref(lat))
            if rc == -4 and time.monotonic() < t_end:   # still running
                continue
            self._keep.pop(int(ticket), None)
            if rc != SSLIC_OK:
                raise SSLICError(rc, "sslic_server_wait")
            return lat.value

    def stats(self) -> dict:
        st = _ServerStats()
        rc = self.lib.sslic_server_stats_get(self._s, ctypes.byref(st))
        if rc != SSLIC_OK:
            raise SSLICError(rc, "sslic_server_stats_get")
        return {k: getattr(st, k) for k, _ in _ServerStats._fields_}

    def close(self):
        if self._s:
            self.lib.sslic_server_destroy(self._s)
            self._s = ctypes.c_void_p(0)
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def segment(image, grid, stream=None, **kw):
    """Convenience: labels and centres of one device image tensor
    [N_{n-1}, ..., N_0, C]; keyword arguments are Params fields."""
    import torch
    p = params_for(image, grid, **kw)
    with Context(p) as ctx:
        labels = torch.empty(tuple(image.shape[:-1]), dtype=torch.int32, device=image.device)
        centres = torch.empty((ctx.K, ctx.centre_width), dtype=torch.float32, device=image.device)
        info = ctx.run(image, labels, centres, stream=stream)
    return labels, centres, info
