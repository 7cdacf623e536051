"""Host logic of the run of one image on several ranks (shard.py), on CPU.

The ranks are gloo processes; each drives a stand-in for the library
context whose arithmetic is the oracle's (seeding, assignment, the exact
integer map, the member-mean reduce of reading R9, the residual of R10,
connectivity).  The sharded run -- slab bounds, the sum of the seed tables,
one all-reduce of the integer sums per iteration, the threshold stop, the
collection of the label slabs on rank 0 for connectivity and their return --
must give every rank its slab of the single-process oracle's labels, the
same centres, iteration count, residual and label count.  The GPU form of
the same run is tests/test_gpu_shard.py.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle as O
from paper_1806_08741_gb300 import inputs as I
from paper_1806_08741_gb300 import shard as SH


class OracleCtx:
    """The context calls run_sharded makes, computed by the oracle on the
    whole image (a stand-in for the library: only the orchestration is under
    test here)."""

    def __init__(self, params, image):
        self.p = params
        self.img = image
        self.n = len(params.size)
        self.C = params.channels
        self.K = O.num_clusters(params)
        self.centre_width = self.C + self.n
        self.plane = int(np.prod(params.size[:-1]))
        self.conn = None

    def _lattice_plane(self, k):
        n, NL, S = self.n, self.p.size[-1], self.p.grid[-1]
        ns = [-(-self.p.size[d] // self.p.grid[d]) for d in range(n)]
        j = k // int(np.prod(ns[:-1]))
        return (NL - 1 - (ns[-1] - 1) * S) // 2 + j * S

    def shard_seed(self, image_halo, lo, hi, centres):
        full = O.seed(self.p, self.img)
        out = np.zeros_like(full)
        for k in range(self.K):
            if lo <= self._lattice_plane(k) < hi:
                out[k] = full[k]
        centres.copy_(torch.from_numpy(out.astype(np.float32).reshape(-1)))

    def shard_sums_size(self):
        return self.K * (self.C + 4), 0

    def shard_map(self, image_slab, labels, lo, hi, centres, sums):
        cen = centres.numpy().reshape(self.K, self.centre_width).astype(np.float64)
        lab = O.assign(self.p, self.img, cen).reshape(-1)[lo * self.plane:hi * self.plane]
        labels.copy_(torch.from_numpy(lab.astype(np.int32)))
        feat = self.img.reshape(-1, self.C)[lo * self.plane:hi * self.plane].astype(np.int64)
        q = np.arange(lo * self.plane, hi * self.plane)
        pos = []
        rem = q
        for d in range(3):
            N = self.p.size[d] if d < self.n else 1
            pos.append(rem % N)
            rem = rem // N
        s = np.zeros((self.K, self.C + 4), np.int64)
        m = lab >= 0
        for c in range(self.C):
            np.add.at(s[:, c], lab[m], feat[m, c])
        for d in range(3):
            np.add.at(s[:, self.C + d], lab[m], pos[d][m])
        np.add.at(s[:, self.C + 3], lab[m], 1)
        sums.copy_(torch.from_numpy(s.reshape(-1)))

    def shard_finalize(self, sums, prev, out, residual=False):
        s = sums.numpy().reshape(self.K, self.C + 4)
        old = prev.numpy().reshape(self.K, self.centre_width).astype(np.float64)
        new = old.copy()
        w = [self.p.m * self.p.m / (S * S) for S in self.p.grid]
        total, nonempty = 0.0, 0
        for k in range(self.K):
            n = s[k, self.C + 3]
            if n == 0:
                continue
            cols = list(range(self.C)) + [self.C + d for d in range(self.n)]
            D2 = 0.0
            for j, col in enumerate(cols):
                v = float(np.float32(np.float64(s[k, col]) / np.float64(n)))
                diff = v - old[k, j]
                D2 += diff * diff if j < self.C else w[j - self.C] * (diff * diff)
                new[k, j] = v
            total += np.sqrt(D2)
            nonempty += 1
        out.copy_(torch.from_numpy(new.astype(np.float32).reshape(-1)))
        return total / nonempty if nonempty else 0.0

    def conn_slabs_begin(self, centres):
        self.conn = {"centres": centres.numpy().reshape(self.K, self.centre_width).astype(np.float64),
                     "labels": np.full(int(np.prod(self.p.size)), -9, np.int32), "next": 0}

    def conn_slabs_add(self, labels, lo, hi):
        assert lo == self.conn["next"]
        self.conn["labels"][lo * self.plane:hi * self.plane] = labels.numpy()
        self.conn["next"] = hi

    def conn_slabs_finish(self):
        assert self.conn["next"] == self.p.size[-1]
        lab = self.conn["labels"].reshape(tuple(reversed(self.p.size)))
        out, n = O.connectivity(self.p, self.conn["centres"], lab)
        self.conn["out"] = out.reshape(-1)
        return n

    def conn_slabs_relabel(self, labels, lo, hi):
        labels.copy_(torch.from_numpy(self.conn["out"][lo * self.plane:hi * self.plane]))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, case, outdir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        img, grid, kw = case
        p = O.params_for(img, grid, **kw)
        comm = SH.Comm()
        NL = p.size[-1]
        bounds = SH.slab_bounds(NL, world, SH.slab_align(len(p.size)))
        lo, hi = bounds[rank]
        a, b = SH.halo_window(lo, hi, NL)
        plane = int(np.prod(p.size[:-1]))
        halo = torch.from_numpy(img.reshape(-1)[a * plane * p.channels:b * plane * p.channels].copy())
        r = SH.run_sharded(OracleCtx(p, img), p, halo, lo, hi, comm, bounds, "cpu")
        np.savez(os.path.join(outdir, f"r{rank}.npz"), labels=r.labels.numpy(), centres=r.centres.numpy(),
                 it=r.iterations, res=r.residual, n=r.num_labels, lo=lo, hi=hi)
    finally:
        dist.destroy_process_group()


def _cases():
    return {
        "rgb3d_conn": (I.make_image(I.ImageSpec((40, 36, 48), 3, "u8", 61, 12, 6)), (8, 8, 8),
                       dict(m=10.0, max_iter=3, enforce_connectivity=True)),
        "rgb2d_thr": (I.make_image(I.ImageSpec((70, 200), 3, "u8", 62, 16, 8)), (16, 16),
                      dict(m=10.0, max_iter=10, conv_threshold=0.2, enforce_connectivity=True)),
    }


@pytest.mark.parametrize("name", sorted(_cases()))
@pytest.mark.parametrize("world", [2, 3])
def test_sharded_run_equals_single_process(name, world, tmp_path):
    case = _cases()[name]
    img, grid, kw = case
    p = O.params_for(img, grid, **kw)
    try:
        SH.slab_bounds(p.size[-1], world, SH.slab_align(len(p.size)))
    except ValueError:
        pytest.skip("too few planes for this many ranks")
    mp.start_processes(_rank_main, args=(world, _free_port(), case, str(tmp_path)), nprocs=world,
                       start_method="spawn")
    ref = O.slic(p, img)
    plane = int(np.prod(p.size[:-1]))
    lab = np.empty(int(np.prod(p.size)), np.int32)
    for r in range(world):
        d = np.load(tmp_path / f"r{r}.npz")
        lab[int(d["lo"]) * plane:int(d["hi"]) * plane] = d["labels"]
        np.testing.assert_array_equal(d["centres"].astype(np.float64), ref["centres"])
        assert int(d["it"]) == ref["iterations"]
        assert float(d["res"]) == ref["residual"]
        assert int(d["n"]) == ref["num_labels"]
    np.testing.assert_array_equal(lab.reshape(ref["labels"].shape), ref["labels"])


def test_slab_bounds():
    for NL, world, al in [(1871, 8, 8), (1216, 4, 64), (44, 2, 8), (64, 1, 64), (200, 3, 64)]:
        b = SH.slab_bounds(NL, world, al)
        assert len(b) == world and b[0][0] == 0 and b[-1][1] == NL
        for (lo, hi), (lo2, _) in zip(b, b[1:]):
            assert hi == lo2
        for lo, hi in b:
            assert hi > lo and lo % al == 0 and (hi % al == 0 or hi == NL)
    with pytest.raises(ValueError):
        SH.slab_bounds(16, 3, 8)
    assert SH.halo_window(8, 16, 40) == (6, 18) and SH.halo_window(0, 8, 9) == (0, 9)
