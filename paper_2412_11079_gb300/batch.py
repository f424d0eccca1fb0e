"""Batched solves: device storage for many uneven problems and the schedule
autotuner for the one-launch batched iteration (uot_sinkhorn_batched).

Plans are stored with a leading dimension rounded up to a multiple of 4 so
every row starts on a 16-byte boundary (the bulk copies need it).  The
autotuner times candidate schedules (ring depth, largest team, target work
per CTA, largest on-chip cluster) on the batch itself and keeps the fastest,
cached per batch shape.
"""

from __future__ import annotations

import torch

from . import uot

_TUNE_CACHE: dict = {}


class Batch:
    def __init__(self, problems, device=None, pad: int = 0):
        """problems: objects with C (N x M float32 numpy), a, b, reg, reg_m, iters.
        pad: extra elements per row beyond the 16-byte rounding (a multiple
        of 4), for plans that are views into wider storage."""
        self.device = torch.device(device or "cuda")
        self.problems = problems
        self.C, self.plans, self.stores, self.a, self.b = [], [], [], [], []
        for p in problems:
            n, m = p.C.shape
            ld = (m + 3) // 4 * 4 + pad
            store = torch.zeros((n, ld), dtype=torch.float32, device=self.device)
            self.stores.append(store)
            self.plans.append(store[:, :m])
            self.C.append(torch.from_numpy(p.C).to(self.device))
            self.a.append(torch.from_numpy(p.a).to(self.device))
            self.b.append(torch.from_numpy(p.b).to(self.device))
        self.descs = []
        for p, plan, a, b in zip(problems, self.plans, self.a, self.b):
            d = uot.UotProblem()
            d.plan = plan.data_ptr()
            d.ldp = plan.stride(0)
            d.n, d.m = plan.shape
            d.a = a.data_ptr()
            d.b = b.data_ptr()
            d.reg, d.reg_m, d.iters = p.reg, p.reg_m, p.iters
            d.rule = getattr(p, "rule", uot.UOT_RULE_PAPER)
            self.descs.append(d)
        self.ws = uot.workspace_bytes(uot.uot_batched_workspace_size(self.descs), self.device)
        self.tuning = None

    @property
    def elements(self) -> int:
        return sum(int(pl.numel()) for pl in self.plans)

    @property
    def element_iterations(self) -> int:
        return sum(int(pl.numel()) * p.iters for pl, p in zip(self.plans, self.problems))

    def init_plans(self, stream=None):
        for C, plan, p in zip(self.C, self.plans, self.problems):
            uot.uot_init_kernel(C, plan, p.reg, stream=stream)

    def prepare(self, tuning=None, stream=None):
        self.tuning = tuning or uot.batch_tuning()
        uot.uot_batched_prepare(self.descs, self.ws, self.tuning, stream)

    def run(self, stream=None):
        uot.uot_sinkhorn_batched(self.ws, stream)

    def placement(self):
        """On-chip cluster size per problem (0: streaming engine)."""
        return uot.uot_batched_placement(self.ws, len(self.descs))

    def teams(self):
        """Streaming team size class per problem (0: on chip)."""
        return uot.uot_batched_placement(self.ws, len(self.descs), teams=True)[1]

    def results(self, stream=None, check_status=True):
        return uot.uot_batched_results(self.ws, len(self.descs), stream, check_status)

    def key(self):
        return tuple((d.n, d.m, d.iters) for d in self.descs)


def candidates():
    """Ring depths that keep two streaming CTAs per SM, team sizes, work per
    CTA, and the largest on-chip cluster.  (On the 512-problem batch of
    uneven sizes the fastest was teams of at most 8 CTAs with an on-chip cap
    of 2: 83 ms against 91 ms for teams of 16 with a cap of 4; teams of 4
    took 136 ms, and a cap of 1 matched 2.)"""
    out = []
    for stages in (2, 3):
        for max_team in (8, 16, 32):
            for target in (1.0e7, 4.0e7):
                for cluster in (2, 4, 8):
                    out.append(uot.batch_tuning(stages, max_team, target, cluster))
    return out


def autotune(batch: Batch, cands=None, repeats: int = 1):
    """Times each candidate schedule on the batch (plans re-initialised before
    every run) and prepares the batch with the fastest.  Returns
    (best tuning, {(stages, max_team, target, cluster): ms})."""
    key = batch.key()
    if key in _TUNE_CACHE:
        batch.prepare(_TUNE_CACHE[key])
        return _TUNE_CACHE[key], {}
    timings = {}
    best, best_ms = None, float("inf")
    for t in cands or candidates():
        batch.prepare(t)
        ms = []
        for _ in range(repeats + 1):
            batch.init_plans()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            batch.run()
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        m = min(ms[1:]) if len(ms) > 1 else ms[0]
        timings[(t.stages, t.max_team, t.target_elems, t.resident_max_cluster)] = m
        if m < best_ms:
            best, best_ms = t, m
    _TUNE_CACHE[key] = best
    batch.prepare(best)
    return best, timings
