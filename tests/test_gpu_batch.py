"""The batched form (mm_step_batch): many independent film pairs of uneven
sizes, each on one of a few lane streams, stepped together.

Each pair in a batch must take exactly the steps it takes alone (bit for bit:
same launches, same order on its own stream), and fixed-dt batched steps must
match the FP64 oracle's Dormand-Prince steps pair by pair (rel L2 <= 1e-5).
At the size of the 256-pair workload, sampled pairs are re-run alone and
compared bit for bit.
"""

import numpy as np
import pytest
import torch

import workloads
from paper_1801_04181_gb300 import MMError, assign_lanes, step_batch
from tests.pair_setup import gpu_pair, oracle_system, rel_l2

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _small_batch():
    specs = [((40, 24, 1), (0.25, 0.0, 0.0), 3.0, 11), ((33, 20, 2), (7.6, 0.0, 0.0), 0.4, 12),
             ((48, 16, 3), (1.9, 0.0, 0.0), 9.0, 13), ((24, 30, 4), (12.3, 0.0, 0.0), 5.5, 14)]
    out = []
    for n, u, v, seed in specs:
        fp, m0, m1 = workloads.film_pair_stick_slip(n=n, gap=5, seed=seed)
        fp.u0 = u
        fp.mech.v_drive = v
        fp.mech.x0_spring = 1e-9
        out.append((fp, m0, m1))
    return out


def _make(pairs, lanes, adaptive):
    streams = [torch.cuda.Stream() for _ in range(max(lanes) + 1)]
    return [gpu_pair(fp, m0, m1, adaptive=adaptive, rtol=1e-5, stream=streams[l])
            for (fp, m0, m1), l in zip(pairs, lanes)]


def _state(mm):
    m = [mm.get_magnetization(g).cpu().numpy() for g in (0, 1)]
    return m, mm.get_slider_state(), mm.step_stats()


def test_batch_equals_pairs_stepped_alone():
    pairs = _small_batch()
    lanes = assign_lanes([fp.cells() for fp, _, _ in pairs], 2)
    batch = _make(pairs, lanes, adaptive=True)
    t_b, dt_b = step_batch(batch, 4, [1e-14] * len(batch))
    torch.cuda.synchronize()
    got = [_state(mm) for mm in batch]
    for mm in batch:
        mm.close()
    for i, (fp, m0, m1) in enumerate(pairs):
        mm = gpu_pair(fp, m0, m1, adaptive=True, rtol=1e-5)
        t, dt = mm.step(4, 1e-14)
        ref = _state(mm)
        mm.close()
        assert t == t_b[i] and dt == dt_b[i]
        assert all(np.array_equal(a, b) for a, b in zip(got[i][0], ref[0]))
        assert got[i][1] == ref[1] and got[i][2] == ref[2]
        assert ref[2][0] == 4


def test_fixed_dt_batch_matches_oracle():
    from oracle import dynamics as D

    pairs = _small_batch()[:3]
    batch = _make(pairs, [0, 1, 0], adaptive=False)
    dt = 5e-14
    t_b, _ = step_batch(batch, 3, [dt] * len(batch))
    for (fp, m0, m1), mm, t in zip(pairs, batch, t_b):
        t_ref, y = D.run_fixed(oracle_system(fp), [m0, m1, 0.0, 0.0], dt, 3)
        assert abs(t - t_ref) < 1e-20
        x, v, _ = mm.get_slider_state()
        for g, init in ((0, m0), (1, m1)):
            got = mm.get_magnetization(g).double().cpu().numpy()
            assert rel_l2(got, y[g]) < TOL
            assert rel_l2(got - init, y[g] - init) < 1e-3
        assert abs(x - y[2]) <= 1e-5 * abs(y[2])
        assert abs(v - y[3]) <= 1e-5 * abs(y[3])
        mm.close()


def test_mixed_integrator_batch_matches_oracle():
    """A batch whose pairs step with different solvers (explicit Euler and
    DP45, Sec. III), each matching its own oracle integrator."""
    from oracle import dynamics as D

    pairs = _small_batch()[:3]
    integ = ["euler", "rk45", "euler"]
    streams = [torch.cuda.Stream() for _ in range(2)]
    batch = [gpu_pair(fp, m0, m1, adaptive=False, stream=streams[i % 2], integrator=it)
             for i, ((fp, m0, m1), it) in enumerate(zip(pairs, integ))]
    dt = 5e-14
    t_b, _ = step_batch(batch, 3, [dt] * len(batch))
    for (fp, m0, m1), mm, t, it in zip(pairs, batch, t_b, integ):
        run = D.run_euler if it == "euler" else D.run_fixed
        t_ref, y = run(oracle_system(fp), [m0, m1, 0.0, 0.0], dt, 3)
        assert abs(t - t_ref) < 1e-20
        x, v, _ = mm.get_slider_state()
        for g, init in ((0, m0), (1, m1)):
            got = mm.get_magnetization(g).double().cpu().numpy()
            assert rel_l2(got, y[g]) < TOL
            assert rel_l2(got - init, y[g] - init) < 1e-3
        assert abs(x - y[2]) <= 1e-5 * abs(y[2])
        assert abs(v - y[3]) <= 1e-5 * abs(y[3])
        mm.close()


def test_batch_rejects_repeated_context_and_bad_dt():
    pairs = _small_batch()[:2]
    batch = _make(pairs, [0, 0], adaptive=True)
    with pytest.raises(MMError):
        step_batch([batch[0], batch[0]], 1, [1e-14, 1e-14])
    with pytest.raises(MMError):
        step_batch(batch, 1, [1e-14, -1.0])
    # nothing was stepped
    assert all(mm.step_stats() == (0, 0) for mm in batch)
    for mm in batch:
        mm.close()


def test_full_size_batch_256_sampled_pairs_bitwise():
    """The 256-pair workload on 16 lanes, two batched adaptive steps; the
    largest, the smallest and a middle pair re-run alone must agree bit for bit."""
    specs = workloads.batch_pairs(256, seed=0)
    cost = [fp.n_base[0] * fp.n_base[1] * (fp.n_base[2] + 4) for fp in specs]
    lanes = assign_lanes(cost, 16)
    streams = [torch.cuda.Stream() for _ in range(16)]
    batch = []
    for fp, l in zip(specs, lanes):
        m0, m1 = workloads.batch_patterns(fp)
        batch.append(gpu_pair(fp, m0, m1, adaptive=True, rtol=1e-5, stream=streams[l]))
    t_b, dt_b = step_batch(batch, 2, [1e-13] * len(batch))
    torch.cuda.synchronize()
    order = np.argsort([fp.cells() for fp in specs])
    picks = [int(order[-1]), int(order[0]), int(order[len(order) // 2])]
    got = {i: _state(batch[i]) for i in picks}
    assert all(mm.step_stats()[0] == 2 for mm in batch)
    # every pair stayed normalised
    for i in range(0, 256, 37):
        m = batch[i].get_magnetization(0).double()
        assert float((m.pow(2).sum(0).sqrt() - 1).abs().max()) < 1e-6
    for mm in batch:
        mm.close()
    torch.cuda.synchronize()
    for i in picks:
        fp = specs[i]
        m0, m1 = workloads.batch_patterns(fp)
        mm = gpu_pair(fp, m0, m1, adaptive=True, rtol=1e-5)
        t, dt = mm.step(2, 1e-13)
        ref = _state(mm)
        mm.close()
        assert t == t_b[i] and dt == dt_b[i]
        assert all(np.array_equal(a, b) for a, b in zip(got[i][0], ref[0]))
        assert got[i][1] == ref[1] and got[i][2] == ref[2]
