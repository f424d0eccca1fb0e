"""Batched iteration (uot_sinkhorn_batched: on-chip cluster solves and the
streaming team engine) against the FP64 oracle, problem by problem, at the
FP32 tolerance (1e-5 relative per plan entry)."""

import math

import numpy as np
import pytest

import oracle
from paper_2412_11079_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5


@pytest.fixture(scope="module")
def uot():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_11079_gb300 import build, uot as u
    build.build()
    u.load()
    return u


def rel_err(got, ref):
    floor = 1e-6 * np.abs(ref).max()
    return float(np.max(np.abs(np.asarray(got, np.float64) - ref) / np.maximum(np.abs(ref), floor)))


def mixed_problems():
    shapes = [(1, 1), (3, 5), (64, 65), (17, 4096), (2000, 300), (777, 1025), (129, 2049),
              (500, 64), (63, 1000), (1024, 1024), (31, 33), (4000, 129)]
    out = []
    rng = np.random.default_rng(7)
    for k, (n, m) in enumerate(shapes):
        reg = float(rng.uniform(0.05, 0.3))
        reg_m = math.inf if k % 5 == 4 else float(np.exp(rng.uniform(np.log(0.1), np.log(10))))
        iters = [0, 1, 7, 40, 25][k % 5]
        out.append(workloads.uniform2d(seed=100 + k, n=n, m=m, reg=reg, reg_m=reg_m, iters=iters))
    return out


def check_batch(uot, problems, tuning=None, pad=0):
    from paper_2412_11079_gb300.batch import Batch
    B = Batch(problems, pad=pad)
    B.init_plans()
    B.prepare(tuning)
    B.run()
    res = B.results()
    for p, plan, r in zip(problems, B.plans, res):
        ref = oracle.sinkhorn(oracle.init_plan(p.C, p.reg), p.a, p.b, p.reg, p.reg_m, p.iters)
        assert r.iters_done == p.iters and r.dev_status == 0
        assert rel_err(plan.double().cpu().numpy(), ref.plan) <= FP32_TOL, (p.name, p.iters)
    return B


def test_mixed_batch_matches_oracle(uot):
    """Default schedule: problems that fit on chip run there (clusters of 1 to
    16 CTAs), the rest stream."""
    B = check_batch(uot, mixed_problems())
    place = B.placement()
    assert set(place) - {0} and 0 in place, place


def test_streaming_engine_only(uot):
    B = check_batch(uot, mixed_problems(), uot.batch_tuning(resident_max_cluster=0))
    assert set(B.placement()) == {0}


def test_padded_rows_streaming_and_on_chip(uot):
    """Plans that are views into wider rows (leading dimension beyond the
    16-byte rounding): per-row copies in the streaming engine, strided loads
    on chip."""
    check_batch(uot, mixed_problems(), uot.batch_tuning(resident_max_cluster=0), pad=12)
    check_batch(uot, mixed_problems(), pad=8)


@pytest.mark.parametrize("max_cluster", [0, 16])
def test_pot_rule_in_both_engines(uot, max_cluster):
    """Problems of a batch may use either rule; each matches its oracle, on
    chip and streaming."""
    from paper_2412_11079_gb300.batch import Batch
    problems = mixed_problems() + on_chip_problems()[:6]
    for k, p in enumerate(problems):
        p.rule = uot.UOT_RULE_POT if k % 2 == 0 else uot.UOT_RULE_PAPER
    B = Batch(problems)
    B.init_plans()
    B.prepare(uot.batch_tuning(resident_max_cluster=max_cluster))
    B.run()
    res = B.results()
    for p, plan, r in zip(problems, B.plans, res):
        P0 = oracle.init_plan(p.C, p.reg)
        ref = (oracle.sinkhorn_pot(P0, p.a, p.b, p.reg, p.reg_m, p.iters)
               if p.rule == uot.UOT_RULE_POT else
               oracle.sinkhorn(P0, p.a, p.b, p.reg, p.reg_m, p.iters))
        assert r.iters_done == p.iters and r.dev_status == 0
        assert rel_err(plan.double().cpu().numpy(), ref.plan) <= FP32_TOL, (p.name, p.rule)


def test_large_teams_on_small_problems(uot):
    """Tiny target work per CTA forces multi-CTA teams (software barriers,
    shared row counters) even for small problems."""
    check_batch(uot, mixed_problems(), uot.batch_tuning(stages=3, max_team=64, target_elems=1e4,
                                                        resident_max_cluster=0))


def test_single_cta_teams_only(uot):
    check_batch(uot, mixed_problems()[:8], uot.batch_tuning(stages=6, max_team=1, target_elems=1e12,
                                                            resident_max_cluster=0))


def on_chip_problems():
    """Shapes that need clusters of 1, 2, 4, 8 and 16 CTAs (shared memory of
    about 227 KB per CTA), with ragged widths, narrow and wide rows (one to
    256 threads per row) and unequal masses."""
    shapes = [(1, 1), (3, 5), (7, 4096), (200, 200), (64, 65), (300, 250), (90, 1025),
              (700, 300), (129, 2049), (1500, 250), (33, 4095), (2000, 300), (4000, 129),
              (450, 1023)]
    out = []
    rng = np.random.default_rng(11)
    for k, (n, m) in enumerate(shapes):
        reg = float(rng.uniform(0.03, 0.2))
        reg_m = math.inf if k % 4 == 3 else float(np.exp(rng.uniform(np.log(0.1), np.log(10))))
        iters = [0, 3, 30, 12][k % 4]
        out.append(workloads.uniform2d(seed=300 + k, n=n, m=m, reg=reg, reg_m=reg_m, iters=iters))
    return out


@pytest.mark.parametrize("max_cluster", [1, 2, 4, 8, 16])
def test_on_chip_cluster_sizes(uot, max_cluster):
    """Each cap on the cluster size: problems that fit run on chip in the
    smallest cluster that holds them, the others stream; all match."""
    B = check_batch(uot, on_chip_problems(), uot.batch_tuning(resident_max_cluster=max_cluster))
    place = B.placement()
    assert max(place) <= max_cluster and max_cluster in place, place
    # The smallest power-of-two cluster whose shared memory (at most 227 KB
    # per CTA) holds the rows, of padded width, beside the column arrays.
    for p, c in zip(on_chip_problems(), place):
        n, m = p.C.shape
        ldk = (m + 3) // 4 * 4
        block = lambda cs: 4 * -(-n // cs) * ldk
        if c:
            assert block(c) <= 232448 and (c == 1 or block(c // 2) > 160 * 1024), (n, m, c)
        else:
            assert block(max_cluster) > 160 * 1024, (n, m)


def test_batched_run_captured_in_graph(uot):
    from paper_2412_11079_gb300.batch import Batch
    probs = mixed_problems()[:6]
    B = Batch(probs)
    B.init_plans()
    B.prepare()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        B.run(stream=s)  # warm-up outside capture
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=s):
            B.init_plans(stream=s)
            B.run(stream=s)
    g.replay()
    torch.cuda.synchronize()
    for p, plan in zip(probs, B.plans):
        ref = oracle.sinkhorn(oracle.init_plan(p.C, p.reg), p.a, p.b, p.reg, p.reg_m, p.iters)
        assert rel_err(plan.double().cpu().numpy(), ref.plan) <= FP32_TOL


def test_prepare_rejects_unsupported(uot):
    from paper_2412_11079_gb300.batch import Batch
    p = workloads.uniform2d(seed=1, n=4, m=4100, iters=1)
    with pytest.raises(uot.UotError):
        B = Batch([p])
        B.prepare()
    q = workloads.uniform2d(seed=2, n=5, m=6, iters=1)
    B = Batch([q])
    B.descs[0].ldp = 7  # rows no longer 16-byte aligned
    with pytest.raises(uot.UotError):
        B.prepare()


def test_autotune_picks_a_working_schedule(uot):
    from paper_2412_11079_gb300.batch import Batch, autotune
    probs = mixed_problems()[:5]
    B = Batch(probs)
    cands = [uot.batch_tuning(3, 8, 1e6), uot.batch_tuning(4, 32, 4e7)]
    best, timings = autotune(B, cands)
    assert len(timings) == 2 and best is not None
    B.init_plans()
    B.run()
    for p, plan in zip(probs, B.plans):
        ref = oracle.sinkhorn(oracle.init_plan(p.C, p.reg), p.a, p.b, p.reg, p.reg_m, p.iters)
        assert rel_err(plan.double().cpu().numpy(), ref.plan) <= FP32_TOL


@pytest.mark.slow
def test_uneven_batch_full_size_sampled(uot):
    """512 problems, N and M log-uniform in [64, 4096], 200 iterations each,
    in the launch configuration the benchmark times: the schedule the
    autotuner picks from the benchmark's own candidates.  At least 32
    problems are compared with the oracle: four from every decile of size,
    and at least one of every on-chip cluster size and every streaming team
    size class that the schedule uses."""
    from paper_2412_11079_gb300.batch import Batch, autotune, candidates
    probs = workloads.batch_uneven(seed=0)
    B = Batch(probs)
    best, _ = autotune(B)
    assert any((c.stages, c.max_team, c.target_elems, c.resident_max_cluster) ==
               (best.stages, best.max_team, best.target_elems, best.resident_max_cluster)
               for c in candidates())
    B.init_plans()
    B.run()
    res = B.results()
    assert all(r.iters_done == 200 and r.dev_status == 0 for r in res)
    place, teams = B.placement(), B.teams()
    sizes = np.array([p.C.size for p in probs])
    order = np.argsort(sizes, kind="stable")
    sample = set()
    for d in range(10):
        chunk = order[d * len(order) // 10:(d + 1) * len(order) // 10]
        sample.update(int(i) for i in chunk[[0, len(chunk) // 3, 2 * len(chunk) // 3, -1]])
    for key in sorted(set(place) - {0}):
        sample.add(next(i for i in order if place[i] == key))
    for key in sorted(set(teams) - {0}):
        sample.add(next(i for i in order[::-1] if teams[i] == key))
    covered_clusters = {place[i] for i in sample} - {0}
    covered_teams = {teams[i] for i in sample} - {0}
    assert covered_clusters == set(place) - {0} and covered_teams == set(teams) - {0}
    assert len(sample) >= 32 and any(place[i] for i in sample) and \
        any(not place[i] for i in sample)
    for i in sorted(sample):
        p = probs[i]
        ref = oracle.sinkhorn(oracle.init_plan(p.C, p.reg), p.a, p.b, p.reg, p.reg_m, p.iters)
        assert rel_err(B.plans[i].double().cpu().numpy(), ref.plan) <= FP32_TOL, \
            (p.name, place[i], teams[i])