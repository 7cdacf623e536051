"""One image shared by several ranks (sslic_shard_*, shard.py) and
connectivity handed over slab by slab (sslic_conn_slabs_*), on the GPU.

* The slab form of connectivity gives sslic_connectivity's labels and label
  count bit for bit, for every way of cutting the image into slabs.
* Two ranks, each a process with its own context on this one GPU, each
  holding a slab of the image, exchange their sums through gloo (host
  copies: neither rank's kernels wait on the other's) and give sslic_run's
  labels, centres, iteration count and label count bit for bit.  Across GPUs
  the same run takes NCCL on device tensors.
"""
import os
import socket

import numpy as np
import pytest

import oracle as O
from paper_1806_08741_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _synth(size, C=3, dtype="u8", sigma=6, seed=9):
    V = int(np.prod(size))
    return I.make_image(I.ImageSpec(tuple(size), C, dtype, seed, max(2, V // 4000), sigma))


def _run(img, grid, **kw):
    import torch
    from paper_1806_08741_gb300 import sslic as S
    p = S.params_for(img, grid, **kw)
    with S.Context(p) as ctx:
        lab = torch.empty(img.shape[:-1], dtype=torch.int32, device="cuda")
        cen = torch.empty((ctx.K, ctx.centre_width), dtype=torch.float32, device="cuda")
        info = ctx.run(torch.from_numpy(np.ascontiguousarray(img)).cuda(), lab, cen)
        return lab.cpu().numpy(), cen.cpu().numpy(), info


SLAB_CASES = [
    ("3d_s8", lambda: _synth((72, 40, 64)), (8, 8, 8), [(0, 8), (8, 24), (24, 32), (32, 64)]),
    ("3d_s16_ragged", lambda: _synth((50, 44, 70)), (16, 16, 16), [(0, 16), (16, 48), (48, 70)]),
    ("3d_whole", lambda: _synth((40, 30, 20)), (8, 8, 8), [(0, 20)]),
    ("3d_u16", lambda: _synth((48, 36, 40), 1, "u16", sigma=300), (8, 8, 8), [(0, 16), (16, 40)]),
    ("2d_rows", lambda: _synth((150, 300)), (16, 16), [(0, 64), (64, 192), (192, 300)]),
    ("2d_s64", lambda: _synth((90, 200)), (64, 64), [(0, 64), (64, 128), (128, 200)]),
]


@pytest.mark.parametrize("name,mk,grid,slabs", SLAB_CASES, ids=[c[0] for c in SLAB_CASES])
def test_conn_slabs_equal_connectivity(name, mk, grid, slabs):
    import torch
    from paper_1806_08741_gb300 import sslic as S
    img = mk()
    p = S.params_for(img, grid, m=10.0, max_iter=3)
    plane = int(np.prod(p.size[:-1]))
    with S.Context(p) as ctx:
        dimg = torch.from_numpy(img).cuda()
        lab = torch.empty(img.shape[:-1], dtype=torch.int32, device="cuda")
        cen = torch.empty((ctx.K, ctx.centre_width), dtype=torch.float32, device="cuda")
        ctx.run(dimg, lab, cen)                       # labels of 3 iterations, no connectivity
        ref = torch.empty_like(lab)
        n_ref = ctx.connectivity(cen, lab, ref)
        flat = lab.reshape(-1)
        for attempt in range(2):                      # twice: the context's slab state is reused
            ctx.conn_slabs_begin(cen)
            for lo, hi in slabs:
                ctx.conn_slabs_add(flat[lo * plane:hi * plane].clone(), lo, hi)
            n = ctx.conn_slabs_finish()
            out = torch.full_like(flat, -7)
            for lo, hi in reversed(slabs):
                part = torch.empty((hi - lo) * plane, dtype=torch.int32, device="cuda")
                ctx.conn_slabs_relabel(part, lo, hi)
                out[lo * plane:hi * plane] = part
            torch.cuda.synchronize()
            assert n == n_ref
            assert torch.equal(out.reshape(lab.shape), ref)


def test_conn_slabs_reject_bad_order_and_bounds():
    import torch
    from paper_1806_08741_gb300 import sslic as S
    img = _synth((40, 32, 48))
    p = S.params_for(img, (16, 16, 16), m=10.0, max_iter=1)
    plane = 40 * 32
    with S.Context(p) as ctx:
        cen = torch.zeros((ctx.K, ctx.centre_width), dtype=torch.float32, device="cuda")
        lab = torch.zeros(48 * plane, dtype=torch.int32, device="cuda")
        ctx.conn_slabs_begin(cen)
        for lo, hi in [(8, 24), (0, 4), (0, 8)]:       # not from plane 0 / not aligned / thinner than S
            with pytest.raises(S.SSLICError) as e:
                ctx.conn_slabs_add(lab[lo * plane:hi * plane], lo, hi)
            assert e.value.code == -1
        ctx.conn_slabs_add(lab[:16 * plane], 0, 16)
        with pytest.raises(S.SSLICError) as e:          # planes 16..47 missing
            ctx.conn_slabs_finish()
        assert e.value.code == -1


# ---- two ranks on this GPU -------------------------------------------------------
def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, case, outdir):
    import torch
    import torch.distributed as dist
    from paper_1806_08741_gb300 import shard as SH
    from paper_1806_08741_gb300 import sslic as S
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        img, grid, kw = case
        p = S.params_for(img, grid, **kw)
        NL = p.size[-1]
        bounds = SH.slab_bounds(NL, world, SH.slab_align(len(p.size)))
        lo, hi = bounds[rank]
        a, b = SH.halo_window(lo, hi, NL)
        plane = int(np.prod(p.size[:-1]))
        flat = img.reshape(-1)
        halo = torch.from_numpy(flat[a * plane * p.channels:b * plane * p.channels].copy()).cuda()
        with S.Context(p) as ctx:
            r = SH.run_sharded(ctx, p, halo, lo, hi, SH.Comm(), bounds, torch.device("cuda"))
            np.savez(os.path.join(outdir, f"r{rank}.npz"), labels=r.labels.cpu().numpy(),
                     centres=r.centres.cpu().numpy(), it=r.iterations, res=r.residual, n=r.num_labels,
                     lo=lo, hi=hi)
    finally:
        dist.destroy_process_group()


SHARD_CASES = {
    "3d_conn_ragged": (lambda: _synth((60, 44, 44)), (8, 8, 8),
                       dict(m=10.0, max_iter=4, enforce_connectivity=True)),
    "3d_s16": (lambda: _synth((64, 48, 80)), (16, 16, 16), dict(m=10.0, max_iter=3, enforce_connectivity=True)),
    "2d_threshold": (lambda: _synth((120, 200)), (16, 16),
                     dict(m=10.0, max_iter=10, conv_threshold=0.2, enforce_connectivity=True)),
    "3d_u16_no_conn": (lambda: _synth((40, 36, 48), 1, "u16", sigma=300), (8, 8, 8), dict(m=20.0, max_iter=3)),
}


@pytest.mark.parametrize("name", sorted(SHARD_CASES))
def test_two_ranks_equal_single_gpu_run(name, tmp_path):
    import torch.multiprocessing as mp
    mk, grid, kw = SHARD_CASES[name]
    img = mk()
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), (img, grid, kw), str(tmp_path)), nprocs=world,
                       start_method="spawn")
    ref_l, ref_c, ref_i = _run(img, grid, **kw)
    plane = int(np.prod(ref_l.shape[1:]))
    lab = np.empty(ref_l.size, np.int32)
    for r in range(world):
        d = np.load(tmp_path / f"r{r}.npz")
        lab[int(d["lo"]) * plane:int(d["hi"]) * plane] = d["labels"]
        np.testing.assert_array_equal(d["centres"], ref_c)
        assert int(d["it"]) == ref_i["iterations"]
        assert float(d["res"]) == ref_i["residual"]
        assert int(d["n"]) == ref_i["num_labels"]
    np.testing.assert_array_equal(lab.reshape(ref_l.shape), ref_l)
    o = O.slic(O.params_for(img, grid, **kw), img)
    np.testing.assert_array_equal(lab.reshape(ref_l.shape), o["labels"])
