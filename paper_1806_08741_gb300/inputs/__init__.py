"""Seeded synthetic inputs for the SSLIC workloads.

This module only makes images; it contains no part of the superpixel
method.  Integer images come from a counter-based generator (definition in
``synth.h``) written in plain integer arithmetic and compiled twice -- for
the host (``synth.c``) and for the GPU (``synth_gpu.cu``) -- so that a crop
regenerated on the CPU is byte-identical to the same crop of a volume made
directly in device memory.  The float hyperspectral image is made on the host
with numpy.

The workload table ``WORKLOADS`` lists the image recipes and run parameters
of the benchmark configurations (shapes and value distributions stand in for
the paper's Visible Human cryosection slice/volume and for FIB-SEM and
hyperspectral data, none of which are available here).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field, replace

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_CPU_LIB = os.path.join(_BUILD, "libsynth.so")
_GPU_LIB = os.path.join(_BUILD, "libsynth_gpu.so")
_CPU_SRC = [os.path.join(_HERE, f) for f in ("synth.c", "synth.h", "synth_impl.h")]
_GPU_SRC = [os.path.join(_HERE, f) for f in ("synth_gpu.cu", "synth.h", "synth_impl.h")]

NVCC_ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


class _Spec(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int32),
        ("size", ctypes.c_int64 * 3),
        ("channels", ctypes.c_int32),
        ("dtype", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
        ("sites", ctypes.c_int64 * 3),
        ("sigma", ctypes.c_int64),
        ("ramp_amp", ctypes.c_int64),
        ("ramp_len", ctypes.c_int64),
    ]


@dataclass(frozen=True)
class ImageSpec:
    """Recipe of one synthetic integer image.  ``size`` lists dimension 0 (x,
    fastest) first.  ``regions`` is the requested region count; the jittered
    site lattice realises the closest per-axis rounding of it."""

    size: tuple
    channels: int = 3
    dtype: str = "u8"          # "u8" or "u16"
    seed: int = 1806
    regions: int = 32
    sigma: int = 8
    ramp_amp: int = 0

    @property
    def ndim(self) -> int:
        return len(self.size)

    @property
    def np_dtype(self):
        return np.uint8 if self.dtype == "u8" else np.uint16

    @property
    def shape(self) -> tuple:
        """numpy shape [N_{n-1}, ..., N_0, C]"""
        return tuple(reversed(self.size)) + (self.channels,)

    @property
    def voxels(self) -> int:
        return int(np.prod(self.size))

    def sites(self) -> tuple:
        n = self.ndim
        t = (self.regions / self.voxels) ** (1.0 / n)
        return tuple(max(1, min(int(s), int(round(s * t)))) for s in self.size)

    def to_c(self) -> _Spec:
        s = _Spec()
        s.ndim = self.ndim
        g = self.sites()
        for d in range(3):
            s.size[d] = int(self.size[d]) if d < self.ndim else 1
            s.sites[d] = int(g[d]) if d < self.ndim else 1
        s.channels = int(self.channels)
        s.dtype = 0 if self.dtype == "u8" else 1
        s.seed = int(self.seed)
        s.sigma = int(self.sigma)
        s.ramp_amp = int(self.ramp_amp)
        s.ramp_len = int(math.ceil(self.size[0] / g[0]))
        return s


def _stale(lib, srcs):
    return (not os.path.exists(lib)) or any(os.path.getmtime(s) > os.path.getmtime(lib)
                                            for s in srcs)


def build(gpu: bool = True) -> None:
    """Compile the CPU generator (cc, OpenMP) and, if ``gpu``, the CUDA one."""
    os.makedirs(_BUILD, exist_ok=True)
    if _stale(_CPU_LIB, _CPU_SRC):
        tmp = _CPU_LIB + f".tmp{os.getpid()}"
        subprocess.run(["cc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp,
                        _CPU_SRC[0]], check=True)
        os.replace(tmp, _CPU_LIB)
    if gpu and _stale(_GPU_LIB, _GPU_SRC):
        tmp = _GPU_LIB + f".tmp{os.getpid()}"
        subprocess.run(["nvcc", *NVCC_ARCH, "-O3", "-Xcompiler", "-fPIC", "-shared",
                        "-o", tmp, _GPU_SRC[0]], check=True)
        os.replace(tmp, _GPU_LIB)


_cpu = None
_gpu = None


def _cpu_lib():
    global _cpu
    if _cpu is None:
        build(gpu=False)
        _cpu = ctypes.CDLL(_CPU_LIB)
        P = ctypes.POINTER(_Spec)
        _cpu.synth_fill.argtypes = [P, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        _cpu.synth_regions.argtypes = [P, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    return _cpu


def _gpu_lib():
    global _gpu
    if _gpu is None:
        build(gpu=True)
        _gpu = ctypes.CDLL(_GPU_LIB)
        _gpu.synth_fill_device.argtypes = [ctypes.POINTER(_Spec), ctypes.c_void_p,
                                           ctypes.c_void_p]
    return _gpu


def _box(spec: ImageSpec, origin, extent):
    o = np.zeros(3, np.int64)
    e = np.ones(3, np.int64)
    origin = origin or (0,) * spec.ndim
    extent = extent or spec.size
    o[:spec.ndim] = origin
    e[:spec.ndim] = extent
    return o, e


def make_image(spec: ImageSpec, origin=None, extent=None) -> np.ndarray:
    """CPU: the crop [origin, origin+extent) (x first) as an array shaped
    [e_{n-1}, ..., e_0, C]."""
    o, e = _box(spec, origin, extent)
    out = np.empty(tuple(int(v) for v in reversed(e[:spec.ndim])) + (spec.channels,),
                   spec.np_dtype)
    rc = _cpu_lib().synth_fill(ctypes.byref(spec.to_c()), o.ctypes.data, e.ctypes.data,
                               out.ctypes.data)
    if rc != 0:
        raise ValueError("bad image spec or crop")
    return out


def make_regions(spec: ImageSpec, origin=None, extent=None) -> np.ndarray:
    o, e = _box(spec, origin, extent)
    out = np.empty(tuple(int(v) for v in reversed(e[:spec.ndim])), np.int32)
    rc = _cpu_lib().synth_regions(ctypes.byref(spec.to_c()), o.ctypes.data, e.ctypes.data,
                                  out.ctypes.data)
    if rc != 0:
        raise ValueError("bad image spec or crop")
    return out


def make_image_device(spec: ImageSpec, out_ptr: int, stream_ptr: int = 0) -> None:
    """GPU: write the whole image into the device buffer at ``out_ptr``
    (``voxels * channels`` elements of the spec's dtype) on ``stream_ptr``."""
    rc = _gpu_lib().synth_fill_device(ctypes.byref(spec.to_c()), ctypes.c_void_p(out_ptr),
                                      ctypes.c_void_p(stream_ptr))
    if rc != 0:
        raise RuntimeError(f"synth_fill_device failed ({rc})")


def make_hyperspectral(size=(1024, 1024), bands=64, endmembers=8, regions=500,
                       alpha=0.5, sigma=0.01, seed=1811) -> np.ndarray:
    """Float32 image [N_1, N_0, bands]: per region a Dirichlet(alpha) abundance
    vector over ``endmembers`` U[0,1]^bands spectra, plus N(0, sigma) noise.
    Regions come from the integer jittered-lattice generator."""
    spec = ImageSpec(size=tuple(size), channels=1, dtype="u8", seed=seed, regions=regions,
                     sigma=0)
    reg = make_regions(spec)
    rng = np.random.Generator(np.random.PCG64(seed))
    E = rng.uniform(0.0, 1.0, size=(endmembers, bands))
    nreg = int(np.prod(spec.sites()))
    A = rng.dirichlet(np.full(endmembers, alpha), size=nreg)
    img = (A @ E)[reg]
    img = img + rng.normal(0.0, sigma, size=img.shape)
    return img.astype(np.float32)


@dataclass(frozen=True)
class Workload:
    """One benchmark/parity configuration: an image recipe plus the SSLIC run
    parameters (grid per axis, x first)."""

    name: str
    image: ImageSpec | None
    grid: tuple
    m: float
    max_iter: int
    perturb: bool
    connectivity: bool
    float_image: dict | None = None

    @property
    def size(self) -> tuple:
        if self.image is not None:
            return self.image.size
        return tuple(self.float_image["size"])

    @property
    def voxels(self) -> int:
        return int(np.prod(self.size))


WORKLOADS = {
    # 2-D RGB 256x256, 32 regions, sigma 8; S=16 (K=256), m=10, 10 iterations
    "rgb2d_256": Workload("rgb2d_256", ImageSpec((256, 256), 3, "u8", 1807, 32, 8, 0),
                          (16, 16), 10.0, 10, True, False),
    # 2-D RGB 2048x1216 (cryosection-slice shape), 2000 regions with a colour
    # ramp, sigma 6; S=16 (K=9728), m=10, 10 iterations, connectivity on
    "rgb2d_2048x1216": Workload("rgb2d_2048x1216",
                                ImageSpec((2048, 1216), 3, "u8", 1808, 2000, 6, 32),
                                (16, 16), 10.0, 10, True, True),
    # 3-D RGB 2048x1216x1871 (~14 GB, cryosection-volume shape), 200k regions,
    # sigma 6; S=16 (K=1,138,176), m=10, 10 iterations, connectivity on
    "rgb3d_2048x1216x1871": Workload("rgb3d_2048x1216x1871",
                                     ImageSpec((2048, 1216, 1871), 3, "u8", 1809, 200000, 6, 0),
                                     (16, 16, 16), 10.0, 10, True, True),
    # the same 3-D recipe on 512x512x256 (201 MB, above the L2) for kernel
    # profiling captures that must stay small
    "rgb3d_512x512x256": Workload("rgb3d_512x512x256",
                                  ImageSpec((512, 512, 256), 3, "u8", 1809, 2881, 6, 0),
                                  (16, 16, 16), 10.0, 10, True, True),
    # 64-band float 1024x1024 hyperspectral mixture; S=16, m=0.1, 10 iterations
    "hyper64_1024": Workload("hyper64_1024", None, (16, 16), 0.1, 10, True, False,
                             float_image={"size": (1024, 1024), "bands": 64}),
}


def crop_workload(w: Workload, extent: tuple, name: str | None = None) -> Workload:
    """The same recipe on a smaller domain (used for bounded CPU samples):
    the region density is kept by scaling the requested region count."""
    img = w.image
    frac = float(np.prod(extent)) / float(np.prod(img.size))
    new_img = replace(img, size=tuple(extent), regions=max(1, int(round(img.regions * frac))))
    return replace(w, name=name or f"{w.name}_crop", image=new_img)
