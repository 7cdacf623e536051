"""Parity at the full size of the 3-D benchmark volume (2048 x 1216 x 1871 RGB
uint8, 4.66 G voxels, S = 16, K = 1,138,176) in the launch configuration
the benchmark times (the autotuned tile shape):

- the seeds, all K of them, bit for bit against the oracle's seeding of the
  same image (rows a1, a2);
- one assign + update iteration from those seeds (rows a3, a4), on outputs
  the oracle computes one voxel at a time: the labels of a million random
  voxels and of every voxel in the windows of 40 random clusters, and those
  clusters' updated centres (exact integer sums, reading R9);
- the whole run (10 iterations and connectivity, row a6) through properties
  that hold at any size: every voxel labelled, labels below the returned
  count, every new label used.

The image comes from the seeded input generator on the device and is copied
to the host for the oracle (the generator gives byte-identical images on both
sides; tests/test_inputs.py)."""
import numpy as np
import pytest

import oracle as O
from paper_1806_08741_gb300 import inputs as I

import _lattice

pytestmark = pytest.mark.gpu


def test_full_size_3d():
    import torch
    from paper_1806_08741_gb300 import sslic as S
    w = I.WORKLOADS["rgb3d_2048x1216x1871"]
    spec = w.image
    size = spec.size
    stream = torch.cuda.current_stream()
    img = torch.empty(spec.shape, dtype=torch.uint8, device="cuda")
    I.make_image_device(spec, img.data_ptr(), stream.cuda_stream)
    host = img.cpu().numpy()
    po = O.params_for(host, w.grid, m=w.m, max_iter=1, perturb=True)
    seeds = O.seed(po, host)
    K = seeds.shape[0]
    assert K == 1138176

    p = S.params_for(img, w.grid, m=w.m, max_iter=1, perturb=True)
    with S.Context(p) as ctx:
        labels = torch.empty(spec.shape[:-1], dtype=torch.int32, device="cuda")
        ctx.autotune(img, labels, reps=1, stream=stream)
        cs = torch.empty((K, ctx.centre_width), dtype=torch.float32, device="cuda")
        ctx.seed(img, cs)
        np.testing.assert_array_equal(cs.cpu().numpy().astype(np.float64), seeds)
        cout = torch.empty_like(cs)
        ctx.iterate(img, torch.from_numpy(seeds.astype(np.float32)).cuda(), labels, cout)
        torch.cuda.synchronize()
        got_c = cout.cpu().numpy().astype(np.float64)

        rng = np.random.default_rng(2026)
        V = int(np.prod(size))
        q_rand = rng.integers(0, V, size=1_000_000, dtype=np.int64)
        ks = rng.choice(K, size=40, replace=False)
        wins = []
        for k in ks:
            c = seeds[k, 3:]
            lo = [max(0, int(np.ceil(c[d])) - w.grid[d]) for d in range(3)]
            hi = [min(size[d] - 1, int(np.ceil(c[d])) + w.grid[d] - 1) for d in range(3)]
            zz, yy, xx = np.meshgrid(np.arange(lo[2], hi[2] + 1), np.arange(lo[1], hi[1] + 1),
                                     np.arange(lo[0], hi[0] + 1), indexing="ij")
            wins.append((xx + size[0] * (yy + size[1] * zz.astype(np.int64))).reshape(-1))
        q = np.concatenate([q_rand] + wins)
        start, cand = _lattice.seed_candidates(size, w.grid, q)
        want = O.assign_voxels(po, host, seeds, q, start, cand)
        got = labels.view(-1)[torch.from_numpy(q).cuda()].cpu().numpy()
        np.testing.assert_array_equal(got, want)

        # updated centres of the sampled clusters: every member lies in the
        # cluster's window, so its members are the window voxels labelled k
        off = q_rand.shape[0]
        flat = host.reshape(-1, 3)
        for k, wq in zip(ks, wins):
            lab_k = want[off:off + wq.shape[0]]
            off += wq.shape[0]
            mem = wq[lab_k == k]
            if mem.size == 0:
                np.testing.assert_array_equal(got_c[k], seeds[k])
                continue
            n = np.int64(mem.size)
            feat = flat[mem].astype(np.int64).sum(0)
            pos = [(mem % size[0]).sum(), ((mem // size[0]) % size[1]).sum(), (mem // (size[0] * size[1])).sum()]
            sums = np.concatenate([feat, np.asarray(pos, np.int64)])
            ref = (sums.astype(np.float64) / np.float64(n)).astype(np.float32).astype(np.float64)
            np.testing.assert_array_equal(got_c[k], ref)

    # the whole run at full size: properties
    p = S.params_for(img, w.grid, m=w.m, max_iter=w.max_iter, perturb=True, enforce_connectivity=True)
    with S.Context(p) as ctx:
        cen = torch.empty((K, ctx.centre_width), dtype=torch.float32, device="cuda")
        info = ctx.run(img, labels, cen, stream=stream)
        torch.cuda.synchronize()
        nl = info["num_labels"]
        assert info["iterations"] == w.max_iter and nl >= K
        assert int(labels.min()) >= 0 and int(labels.max()) < nl
        used = torch.bincount(labels.view(-1), minlength=nl)
        assert bool((used[K:] > 0).all())   # every new label names a relabelled component
