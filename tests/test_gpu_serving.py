"""Batched / served form: each request's result in the mix equals the same
request run alone through the single-image path (integer images: bit for
bit), under a budget small enough that requests wait for admission; and the
first small ones equal the CPU oracle."""
import numpy as np
import pytest

import oracle as O
from paper_1806_08741_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _mix(seed=3):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(10):
        side = int(rng.integers(60, 400))
        h = int(rng.integers(50, 300))
        img = I.make_image(I.ImageSpec((side, h), 3, "u8", 100 + i, max(2, side * h // 3000), 6))
        S = int(rng.choice([8, 16, 32]))
        m = float(rng.choice([5.0, 10.0, 20.0]))
        reqs.append((img, (S, S), m))
    for i in range(4):
        side = int(rng.integers(30, 72))
        img = I.make_image(I.ImageSpec((side, side + 3, side - 5), 1, "u16", 200 + i, 12, 300))
        S = int(rng.choice([8, 16]))
        reqs.append((img, (S, S, S), 10.0))
    # a type without a tile kernel (per-voxel path in the batch)
    reqs.append((I.make_image(I.ImageSpec((90, 70), 2, "u8", 300, 10, 6)), (8, 8), 10.0))
    return reqs


def _alone(img, grid, m, iters, thr=0.0, info=False):
    import torch
    from paper_1806_08741_gb300 import sslic as S
    p = S.params_for(img, grid, m=m, max_iter=iters, conv_threshold=thr)
    with S.Context(p) as ctx:
        lab = torch.empty(img.shape[:-1], dtype=torch.int32, device="cuda")
        cen = torch.empty((ctx.K, ctx.centre_width), dtype=torch.float32, device="cuda")
        r = ctx.run(torch.from_numpy(img).cuda(), lab, cen)
        if info:
            return lab.cpu().numpy(), cen.cpu().numpy(), r
        return lab.cpu().numpy(), cen.cpu().numpy()


@pytest.mark.parametrize("budget_mb", [2048, 24])
def test_served_results_equal_alone(budget_mb):
    import torch
    from paper_1806_08741_gb300 import sslic as S
    reqs = _mix()
    iters = 6
    outs = []
    with S.Server(budget_mb << 20, max_active=8) as srv:
        tickets = []
        for img, grid, m in reqs:
            p = S.params_for(img, grid, m=m, max_iter=iters)
            lab = np.empty(img.shape[:-1], np.int32)
            K = 1
            for n, g in zip(p.size, p.grid):
                K *= -(-n // g)
            cen = np.empty((K, p.channels + p.ndim), np.float32)
            tickets.append(srv.submit(p, img, lab, cen))
            outs.append((lab, cen))
        lat = [srv.wait(t) for t in tickets]
        st = srv.stats()
    assert st["completed"] == len(reqs) and st["status"] == 0
    assert all(x > 0 for x in lat)
    # a round form runs directly the first time it is met and from a captured
    # graph when it comes back
    assert st["graph_launches"] + st["eager_rounds"] == st["rounds"]
    assert st["graph_captures"] <= st["eager_rounds"] and st["graph_launches"] >= st["graph_captures"]
    if budget_mb == 24:
        assert st["max_active"] < len(reqs)   # admission had to wait for memory
    for (img, grid, m), (lab, cen) in zip(reqs, outs):
        ref_l, ref_c = _alone(img, grid, m, iters)
        np.testing.assert_array_equal(lab, ref_l)
        np.testing.assert_array_equal(cen, ref_c)


def test_recurring_round_forms_replay_captured_graphs():
    """Requests admitted together and finishing together make the same round
    form (no joiners, no finishers, the same groups) round after round: after
    its first, direct run each such form is captured once and replayed."""
    from paper_1806_08741_gb300 import sslic as S
    img = I.make_image(I.ImageSpec((200, 150), 3, "u8", 77, 10, 6))
    iters = 12
    outs = []
    with S.Server(1 << 30, max_active=8) as srv:
        p = S.params_for(img, (16, 16), m=10.0, max_iter=iters)
        tickets = []
        for _ in range(4):
            lab = np.empty(img.shape[:-1], np.int32)
            tickets.append(srv.submit(p, img, lab))
            outs.append(lab)
        for t in tickets:
            srv.wait(t)
        st = srv.stats()
    assert st["status"] == 0 and st["completed"] == 4
    assert st["graph_launches"] + st["eager_rounds"] == st["rounds"]
    assert st["graph_captures"] >= 1 and st["graph_launches"] >= st["rounds"] // 2
    ref_l, _ = _alone(img, (16, 16), 10.0, iters)
    for lab in outs:
        np.testing.assert_array_equal(lab, ref_l)


def test_served_small_requests_equal_oracle():
    from paper_1806_08741_gb300 import sslic as S
    reqs = _mix(5)[:3]
    with S.Server(512 << 20) as srv:
        res = []
        for img, grid, m in reqs:
            p = S.params_for(img, grid, m=m, max_iter=4)
            lab = np.empty(img.shape[:-1], np.int32)
            res.append((srv.submit(p, img, lab), lab, img, grid, m))
        for t, lab, img, grid, m in res:
            srv.wait(t)
            ref = O.slic(O.params_for(img, grid, m=m, max_iter=4), img)
            np.testing.assert_array_equal(lab, ref["labels"])


def test_served_requests_with_convergence_thresholds():
    """Requests with a centre-residual threshold leave after the round in
    which their residual drops below it -- the iteration at which sslic_run
    stops -- with the same labels and centres; others in the mix run all
    their iterations."""
    from paper_1806_08741_gb300 import sslic as S
    reqs = _mix(7)[:9]
    iters = 12
    # thresholds that stop runs at different iterations (from each run's own residuals)
    thr = []
    for i, (img, grid, m) in enumerate(reqs):
        if i % 3 == 2:
            thr.append(0.0)
            continue
        _, _, r_hi = _alone(img, grid, m, 3, info=True)
        thr.append(r_hi["residual"] * (1.5 if i % 3 == 0 else 1.01))
    outs = []
    with S.Server(1 << 30, max_active=6) as srv:
        tickets = []
        for (img, grid, m), t in zip(reqs, thr):
            p = S.params_for(img, grid, m=m, max_iter=iters, conv_threshold=t)
            lab = np.empty(img.shape[:-1], np.int32)
            K = 1
            for n, g in zip(p.size, p.grid):
                K *= -(-n // g)
            cen = np.empty((K, p.channels + p.ndim), np.float32)
            tickets.append(srv.submit(p, img, lab, cen))
            outs.append((lab, cen))
        for t in tickets:
            srv.wait(t)
        st = srv.stats()
    assert st["status"] == 0
    early = 0
    for (img, grid, m), t, (lab, cen) in zip(reqs, thr, outs):
        ref_l, ref_c, info = _alone(img, grid, m, iters, thr=t, info=True)
        early += info["iterations"] < iters
        np.testing.assert_array_equal(lab, ref_l)
        np.testing.assert_array_equal(cen, ref_c)
    assert early >= 3   # the thresholds did stop runs early


def test_server_rejects():
    from paper_1806_08741_gb300 import sslic as S
    img = np.zeros((512, 512, 3), np.uint8)
    lab = np.empty((512, 512), np.int32)
    with S.Server(1 << 20) as srv:
        with pytest.raises(S.SSLICError) as e:
            srv.submit(S.params_for(img, (16, 16)), img, lab)   # larger than the whole budget
        assert e.value.code == -2
        img4 = np.zeros((6, 6, 6, 6, 1), np.uint8)
        with pytest.raises(S.SSLICError) as e:   # the batched tables hold up to three axes
            srv.submit(S.params_for(img4, (3, 3, 3, 3)), img4, np.empty(img4.shape[:-1], np.int32))
        assert e.value.code == -6


def test_served_requests_with_connectivity_equal_alone():
    """Requests that enforce connectivity (Sec. 3.1 stage 3) leave the
    rounds when their iterations are done; a finisher thread relabels them
    while the rounds of the others go on.  Each result equals the request run
    alone through sslic_run bit for bit, whatever it shares the server with:
    2-D colour and 3-D grey images, with and without connectivity, sizes that
    rise and fall so that the connectivity workspace grows and is reused."""
    import torch
    from paper_1806_08741_gb300 import sslic as S
    rng = np.random.default_rng(11)
    reqs = []
    for i, (w, h) in enumerate([(80, 60), (300, 220), (120, 90), (420, 330), (64, 64), (256, 300)]):
        img = I.make_image(I.ImageSpec((w, h), 3, "u8", 400 + i, max(2, w * h // 2500), 6))
        reqs.append((img, (16, 16) if i % 2 else (8, 8), float(rng.choice([5.0, 10.0, 20.0])), i % 3 != 2))
    for i, side in enumerate([40, 72, 56]):
        img = I.make_image(I.ImageSpec((side, side + 5, side - 3), 1, "u16", 500 + i, 20, 300))
        reqs.append((img, (8, 8, 8), 10.0, True))
    iters = 5
    outs = []
    with S.Server(1 << 30, max_active=6) as srv:
        tickets = []
        for img, grid, m, conn in reqs:
            p = S.params_for(img, grid, m=m, max_iter=iters, enforce_connectivity=conn)
            lab = np.empty(img.shape[:-1], np.int32)
            K = 1
            for n, g in zip(p.size, p.grid):
                K *= -(-n // g)
            cen = np.empty((K, p.channels + p.ndim), np.float32)
            tickets.append(srv.submit(p, img, lab, cen))
            outs.append((lab, cen))
        for t in tickets:
            srv.wait(t)
        st = srv.stats()
    assert st["status"] == 0 and st["completed"] == len(reqs)
    for (img, grid, m, conn), (lab, cen) in zip(reqs, outs):
        p = S.params_for(img, grid, m=m, max_iter=iters, enforce_connectivity=conn)
        with S.Context(p) as ctx:
            rl = torch.empty(img.shape[:-1], dtype=torch.int32, device="cuda")
            rc = torch.empty((ctx.K, ctx.centre_width), dtype=torch.float32, device="cuda")
            info = ctx.run(torch.from_numpy(img).cuda(), rl, rc)
        np.testing.assert_array_equal(lab, rl.cpu().numpy())
        np.testing.assert_array_equal(cen, rc.cpu().numpy())
        if conn:
            assert lab.min() >= 0 and lab.max() < info["num_labels"]
    # the first request against the oracle's whole run, connectivity included
    img, grid, m, conn = reqs[0]
    ref = O.slic(O.params_for(img, grid, m=m, max_iter=iters, enforce_connectivity=conn), img)
    np.testing.assert_array_equal(outs[0][0], ref["labels"])


@pytest.mark.parametrize("shape", [0, 1, 2, 5, 9, 11])
def test_served_results_equal_alone_for_each_recorded_shape(shape):
    """The tile shape recorded for an image type (as by autotune) is the one
    the batched form uses; no shape changes a result."""
    from paper_1806_08741_gb300 import sslic as S
    reqs = _mix(11)[:8]
    iters = 3
    S.tune_forget()
    try:
        for img, grid, m in reqs:
            p = S.params_for(img, grid, m=m, max_iter=iters)
            if (p.dtype, p.channels) in ((S.U8, 3), (S.U8, 1), (S.U16, 1)) and shape < S.num_tile_shapes(p.ndim):
                S.tune_record(p, shape)
        outs = []
        with S.Server(1 << 30, max_active=8) as srv:
            tickets = []
            for img, grid, m in reqs:
                p = S.params_for(img, grid, m=m, max_iter=iters)
                lab = np.empty(img.shape[:-1], np.int32)
                tickets.append(srv.submit(p, img, lab))
                outs.append(lab)
            for t in tickets:
                srv.wait(t)
    finally:
        S.tune_forget()
    for (img, grid, m), lab in zip(reqs, outs):
        ref = O.slic(O.params_for(img, grid, m=m, max_iter=iters), img)
        np.testing.assert_array_equal(lab, ref["labels"])


def test_served_lab_requests_match_alone():
    """3-channel float (CIE-Lab) requests go through the batched tile kernel
    beside integer ones; each equals its run alone within the float
    tolerance, the integer ones bit for bit.  Both sides are the GPU's FP32
    path and differ only in the order of their floating-point sums, so a
    near-tie may flip: labels >= 99.99 % equal, and every cluster whose
    member set is the same on both sides within 1e-5 per element (reading
    T1; on these small images one flipped voxel moves its cluster's centre by
    more than a table-wide 1e-5)."""
    from paper_1806_08741_gb300 import sslic as S
    rng = np.random.default_rng(11)
    reqs = []
    for i in range(5):
        size = (int(rng.integers(70, 300)), int(rng.integers(60, 200)))
        rgb = I.make_image(I.ImageSpec(size, 3, "u8", 400 + i, max(2, size[0] * size[1] // 3000), 6))
        reqs.append((O.srgb_to_lab(rgb).astype(np.float32), (int(rng.choice([8, 16])),) * 2, 10.0))
    for i in range(3):
        side = int(rng.integers(40, 90))
        rgb = I.make_image(I.ImageSpec((side, side - 7, side - 20), 3, "u8", 500 + i, 20, 6))
        reqs.append((O.srgb_to_lab(rgb).astype(np.float32), (8, 8, 8), 10.0))
    reqs += _mix(13)[:3]
    iters = 5
    outs = []
    with S.Server(1 << 30, max_active=6) as srv:
        tickets = []
        for img, grid, m in reqs:
            p = S.params_for(img, grid, m=m, max_iter=iters)
            lab = np.empty(img.shape[:-1], np.int32)
            K = 1
            for n, g in zip(p.size, p.grid):
                K *= -(-n // g)
            cen = np.empty((K, p.channels + p.ndim), np.float32)
            tickets.append(srv.submit(p, img, lab, cen))
            outs.append((lab, cen))
        for t in tickets:
            srv.wait(t)
        assert srv.stats()["status"] == 0
    for (img, grid, m), (lab, cen) in zip(reqs, outs):
        ref_l, ref_c = _alone(img, grid, m, iters)
        if img.dtype == np.float32:
            assert (lab == ref_l).mean() >= 0.9999
            flip = lab != ref_l
            differ = np.unique(np.concatenate([lab[flip], ref_l[flip]]))
            same = np.setdiff1d(np.arange(cen.shape[0]), differ)
            rel = np.abs(cen[same] - ref_c[same]) / np.maximum(np.abs(ref_c[same]), 1e-3)
            assert rel.max() <= 1e-5, rel.max()
        else:
            np.testing.assert_array_equal(lab, ref_l)
            np.testing.assert_array_equal(cen, ref_c)
