"""Serving queue (wos_queue_create / wos_submit / wos_wait): every request's
counts, singular values, truncation and reconstructed Gamma_1 data equal, bit
for bit, the same request solved alone through wos_build_operator,
wos_op_svd and wos_reconstruct -- whether it runs mixed with other requests,
joins while others are walking, waits for admission behind the slot or
budget limit, and whatever the slice of walks per step.  The lone path is in
turn pinned to the oracle by the walk and SVD parity tests."""
import time

import numpy as np
import pytest
import torch

from gpu_util import ctx, gpu_build
from paper_2409_03686_gb300 import workloads as W
from paper_2409_03686_gb300 import wos

pytestmark = pytest.mark.gpu

SEED = 7


def _requests(n=10):
    insts = W.mixed_batch(n_instances=n, seed=SEED, m_lo=16, m_hi=160, n_lo=500, n_hi=6000)
    meas = [W.measurements(inst, noise=0.01, seed=q) for q, inst in enumerate(insts)]
    return insts, meas


def auto_rank(S):
    """Truncation of a request with r = 0: the first r with S[r-1]/S[r] >= 1.5
    and S[r-1]/S[0] < 1e-3, else the last such gap at any level, else k."""
    last = 0
    for r in range(1, len(S)):
        if not S[r] > 0:
            break
        if S[r - 1] / S[r] >= 1.5:
            last = r
            if S[r - 1] / S[0] < 1e-3:
                return r
    return last if last else len(S)


_alone_cache = {}


def _alone(inst, m, r=0, alpha=0.0):
    key = (inst.name, inst.M_D, inst.M_tot, inst.N, inst.stream, inst.eps, inst.fp64, r, alpha)
    if key in _alone_cache:
        return _alone_cache[key]
    dev = torch.device("cuda:0")
    g = gpu_build(inst, trace=False)
    counts = g["counts_t"]
    sigma = torch.as_tensor(wos.wos_element_measures(inst.domain, inst.partition),
                            dtype=torch.float64, device=dev)
    g1 = inst.partition.gamma1
    U, S, V, _ = wos.wos_op_svd(ctx(), counts, inst.N, g1, sigma, sync=False)
    S_h = S.cpu().numpy()
    r_use = r if r else auto_rank(S_h)
    u1, _ = wos.wos_reconstruct(ctx(), U, S, V, counts, inst.N, g1, sigma,
                                torch.as_tensor(m.uD, device=dev),
                                r_use, u0=torch.as_tensor(m.u0, device=dev),
                                tikhonov_alpha=alpha, want_uD_hat=False)
    out = dict(counts=g["counts"], S=S_h, r=r_use, u1=u1.cpu().numpy())
    _alone_cache[key] = out
    return out


def _check(t, ref, name):
    np.testing.assert_array_equal(t.S, ref["S"], err_msg=name)
    assert t.r_used.value == ref["r"], name
    np.testing.assert_array_equal(t.u_gamma1, ref["u1"], err_msg=name)
    if t.counts is not None:
        np.testing.assert_array_equal(t.counts.astype(np.int64), ref["counts"], err_msg=name)


def test_mixed_requests_equal_lone_solves():
    insts, meas = _requests()
    q = wos.wos_queue_create(ctx(), seed=SEED, slice_walks=1000)  # ragged last slice
    try:
        tickets = [wos.wos_submit(q, inst, m.uD, m.u0, want_counts=True)
                   for inst, m in zip(insts, meas)]
        for t in tickets:
            assert wos.wos_wait(q, t, 120_000)
        st = wos.wos_queue_get_stats(q)
    finally:
        wos.wos_queue_destroy(q)
    assert st["completed"] == len(insts) and st["failed"] == 0
    assert st["walks"] == sum(i.M_D * i.N for i in insts)
    assert st["slices"] >= max((i.N + 999) // 1000 for i in insts)
    for inst, m, t in zip(insts, meas, tickets):
        _check(t, _alone(inst, m), inst.name)


def test_staggered_arrivals_and_admission_limits():
    """Requests arriving while others walk join at the next slice; with two
    slots the rest wait in the queue.  Results stay identical."""
    insts, meas = _requests()
    q = wos.wos_queue_create(ctx(), seed=SEED, slice_walks=512, max_inflight=2,
                             side_streams=2)
    try:
        tickets = []
        for inst, m in zip(insts, meas):
            tickets.append(wos.wos_submit(q, inst, m.uD, m.u0, want_counts=True))
            time.sleep(0.002)
        for t in tickets:
            assert wos.wos_wait(q, t, 120_000)
        st = wos.wos_queue_get_stats(q)
        assert st["inflight"] == 0 and st["queued"] == 0
    finally:
        wos.wos_queue_destroy(q)
    for inst, m, t in zip(insts, meas, tickets):
        _check(t, _alone(inst, m), inst.name)


def test_device_budget_serialises_admission():
    """A budget that holds one or two of these requests at a time still
    completes every request."""
    insts, meas = _requests(4)
    q = wos.wos_queue_create(ctx(), seed=SEED, device_budget=1 << 20)
    try:
        tickets = [wos.wos_submit(q, inst, m.uD, m.u0) for inst, m in zip(insts, meas)]
        for t in tickets:
            assert wos.wos_wait(q, t, 120_000)
    finally:
        wos.wos_queue_destroy(q)
    for inst, m, t in zip(insts, meas, tickets):
        _check(t, _alone(inst, m), inst.name)


def test_explicit_truncation_tikhonov_and_poll():
    insts, meas = _requests(3)
    q = wos.wos_queue_create(ctx(), seed=SEED)
    try:
        t1 = wos.wos_submit(q, insts[0], meas[0].uD, meas[0].u0, r=3)
        t2 = wos.wos_submit(q, insts[1], meas[1].uD, meas[1].u0, r=4, tikhonov_alpha=1e-4)
        deadline = time.time() + 120
        while not (wos.wos_poll(q, t1) and wos.wos_poll(q, t2)):
            assert time.time() < deadline
            time.sleep(0.001)
    finally:
        wos.wos_queue_destroy(q)
    _check(t1, _alone(insts[0], meas[0], r=3), insts[0].name)
    _check(t2, _alone(insts[1], meas[1], r=4, alpha=1e-4), insts[1].name)


def test_fp64_queue():
    insts, meas = _requests(3)
    insts = [i.replace(fp64=True) for i in insts]
    q = wos.wos_queue_create(ctx(), seed=SEED, precision=1, slice_walks=700)
    try:
        tickets = [wos.wos_submit(q, inst, m.uD, m.u0, want_counts=True)
                   for inst, m in zip(insts, meas)]
        for t in tickets:
            assert wos.wos_wait(q, t, 120_000)
    finally:
        wos.wos_queue_destroy(q)
    for inst, m, t in zip(insts, meas, tickets):
        _check(t, _alone(inst, m), inst.name + "-fp64")


def test_invalid_requests_rejected_at_submit():
    insts, meas = _requests(2)
    q = wos.wos_queue_create(ctx(), seed=SEED)
    try:
        with pytest.raises(wos.WosError) as e:
            wos.wos_submit(q, insts[0].replace(eps=0.0), meas[0].uD, meas[0].u0)
        assert e.value.code == 1
        with pytest.raises(wos.WosError) as e:  # can never fit the budget
            q2 = wos.wos_queue_create(ctx(), seed=SEED, device_budget=1024)
            try:
                wos.wos_submit(q2, insts[0], meas[0].uD, meas[0].u0)
            finally:
                wos.wos_queue_destroy(q2)
        assert e.value.code == 1
        with pytest.raises(wos.WosError) as e:  # eps below the FP32 floor
            wos.wos_submit(q, insts[1].replace(eps=1e-12), meas[1].uD, meas[1].u0)
        assert e.value.code == 4
        st = wos.wos_queue_get_stats(q)
        assert st["submitted"] == 0
    finally:
        wos.wos_queue_destroy(q)
    with pytest.raises(wos.WosError):
        wos.wos_queue_create(ctx(), seed=SEED, precision=5)


def test_preconditioned_svd_requests_equal_lone_solves():
    """Requests large enough for the QR-preconditioned SVD (n >= 32)."""
    insts = [W.annulus_config(N=3000, grid=7, m_each=48).replace(stream=1, seed=SEED),
             W.square_config(N=3000, grid=7, n_side=16).replace(stream=2, seed=SEED),
             W.ball_config(N=2000, n_points=64, nb=8, ns=12).replace(stream=3, seed=SEED)]
    meas = [W.measurements(inst, noise=0.01, seed=q) for q, inst in enumerate(insts)]
    q = wos.wos_queue_create(ctx(), seed=SEED, slice_walks=800)
    try:
        tickets = [wos.wos_submit(q, inst, m.uD, m.u0, want_counts=True)
                   for inst, m in zip(insts, meas)]
        for t in tickets:
            assert wos.wos_wait(q, t, 120_000)
    finally:
        wos.wos_queue_destroy(q)
    for inst, m, t in zip(insts, meas, tickets):
        _check(t, _alone(inst, m), inst.name)


def test_served_requests_match_the_oracle():
    """Requests served in a mix, checked against the oracle itself (not only
    against the lone GPU solve): three sampled rows of every request's counts
    replayed walk by walk (the rows may differ only by the walks whose exit
    element differs, <= 0.1 % of them, each moving one count out of one
    column and into another), its singular values against the oracle's
    Jacobi SVD of the served counts (1e-10 relative, the floor rule for the
    tiny ones) and u_Gamma1 against the oracle's TSVD at the served
    truncation (1e-8 relative)."""
    from gpu_util import oracle_walks
    from oracle import oracle as O
    insts, meas = _requests(6)
    q = wos.wos_queue_create(ctx(), seed=SEED, slice_walks=1500)
    try:
        tickets = [wos.wos_submit(q, inst, m.uD, m.u0, want_counts=True)
                   for inst, m in zip(insts, meas)]
        for t in tickets:
            assert wos.wos_wait(q, t, 120_000)
    finally:
        wos.wos_queue_destroy(q)
    checked = 0
    for inst, m, t in zip(insts, meas, tickets):
        inst = inst.replace(seed=SEED)
        C = t.counts.astype(np.int64)
        assert (C.sum(1) == inst.N).all(), inst.name
        rows = sorted({0, inst.M_D // 2, inst.M_D - 1})
        el, _, _ = oracle_walks(inst, rows=rows)
        for q_, i in enumerate(rows):
            ref = np.bincount(el[q_][el[q_] >= 0], minlength=inst.M_tot)
            assert np.abs(C[i] - ref).sum() <= 2 * max(1, int(0.001 * inst.N)), (inst.name, i)
        g1 = inst.partition.gamma1
        sig = O.element_measures(inst.domain, inst.partition)
        nu = inst.nu_vec()
        Uo, so, Vo, _, ok = O.jacobi_svd(O.operator_B(C, inst.N, g1, nu, sig))
        assert ok
        big = so >= 1e-6 * so[0]
        err = np.abs(t.S - so)
        assert np.all(err[big] <= 1e-10 * so[big]), inst.name
        assert np.all(err[~big] <= 1e-10 * so[0]), inst.name
        r = t.r_used.value
        if r < len(so) and so[r - 1] / so[r] < 1.5:
            continue  # not at a gap: the r-TSVD is not stable to 1e-8
        ro, _ = O.reconstruct(Uo, so, Vo, r, C, inst.N, g1, nu, sig, m.uD, m.u0)
        assert np.linalg.norm(t.u_gamma1 - ro) <= 1e-8 * np.linalg.norm(ro), (inst.name, r)
        checked += 1
    assert checked >= 3


def test_voronoi_requests_are_served():
    """Requests on extrinsic Voronoi partitions (the cell measures come from
    the library): served in a mix with an intrinsic-cell request, each equal
    to its lone solve bit for bit."""
    insts = [W.shell_config(N=2000, n_points=40, voronoi=(300, 60), shift=0.3).replace(
                 stream=1, seed=SEED),
             W.annulus_voronoi_config(N=1500, eps=1e-5, fp64=False, n_points=30, m0=120,
                                      m1=80).replace(stream=2, seed=SEED),
             W.square_config(N=2000, grid=5, n_side=12).replace(stream=3, seed=SEED)]
    meas = [W.measurements(inst, noise=0.01, seed=q) for q, inst in enumerate(insts)]
    q = wos.wos_queue_create(ctx(), seed=SEED, slice_walks=700)
    try:
        tickets = [wos.wos_submit(q, inst, m.uD, m.u0, want_counts=True)
                   for inst, m in zip(insts, meas)]
        for t in tickets:
            assert wos.wos_wait(q, t, 120_000)
    finally:
        wos.wos_queue_destroy(q)
    for inst, m, t in zip(insts, meas, tickets):
        _check(t, _alone(inst, m), inst.name)
