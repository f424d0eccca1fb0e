"""The C-ABI library builds, loads and exports every symbol include/uot.h
declares; host-side argument validation returns error codes without a GPU."""

import ctypes
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2412_11079_gb300 import build, uot
    build.build()
    return uot.load()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "uot.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(uot_[a-z_0-9]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    from paper_2412_11079_gb300 import uot
    names = declared_functions()
    assert "uot_sinkhorn" in names and "uot_init_kernel" in names and "uot_cost" in names
    for name in names:
        assert hasattr(lib, name), name
        assert name in uot.SIGNATURES, f"binding lacks {name}"


def test_status_strings_and_defaults(lib):
    from paper_2412_11079_gb300 import uot
    assert uot.uot_status_string(0) == "ok"
    assert "workspace" in uot.uot_status_string(uot.UOT_ERR_WORKSPACE)
    o = uot.UotOptions()
    lib.uot_default_options(ctypes.byref(o))
    assert (o.dtype, o.algo, o.check_every, o.tile, o.cluster, o.max_ctas, o.rule) == \
        (0, 0, 1, 0, 0, 0, uot.UOT_RULE_PAPER)
    assert (o.storage, o.deterministic) == (uot.UOT_STORAGE_INPLACE, 0)


def test_workspace_size(lib):
    from paper_2412_11079_gb300 import uot
    s = uot.uot_workspace_size(16384, 16384)
    assert s % 256 == 0 and s >= 3 * 16384 * 4 + 16384 * 4
    # deterministic mode: one slot of column partials per row group (304 slots)
    d = uot.uot_workspace_size(16384, 16384, uot.options(deterministic=True))
    assert d % 256 == 0 and d >= s + 304 * 16384 * 4
    assert uot.uot_workspace_size(0, 5) == 0
    assert uot.uot_workspace_size(5, -1) == 0


def test_fused_config_table(lib):
    from paper_2412_11079_gb300 import uot
    total, _ = uot.uot_fused_config(-1)
    assert total >= 7
    seen = set()
    for k in range(total):
        _, c = uot.uot_fused_config(k)
        elem = 4 if c["dtype"] == 0 else 2
        assert c["cols"] == c["threads"] * c["vecs"] * (16 // elem)
        assert c["threads"] % 32 == 0
        seen.add(c["dtype"])
    assert seen == {0, 1, 2}


def test_argument_validation_needs_no_gpu(lib):
    from paper_2412_11079_gb300 import uot
    o = uot.options()
    P = ctypes.c_void_p(4096)  # never dereferenced: validation fails first
    res = uot.UotResult()
    f = lib.uot_sinkhorn
    # NULL plan
    assert f(None, 4, P, P, 4, 4, 0.1, 1.0, 5, 0.0, P, 1 << 20, ctypes.byref(o), None,
             ctypes.byref(res)) == uot.UOT_ERR_INVALID_ARG
    # ld < m
    assert f(P, 3, P, P, 4, 4, 0.1, 1.0, 5, 0.0, P, 1 << 20, ctypes.byref(o), None,
             None) == uot.UOT_ERR_INVALID_ARG
    # reg <= 0, NaN reg, reg_m <= 0, negative iters, NaN tol
    for reg, reg_m, iters, tol in [(0.0, 1.0, 5, 0.0), (math.nan, 1.0, 5, 0.0),
                                   (0.1, 0.0, 5, 0.0), (0.1, 1.0, -1, 0.0),
                                   (0.1, 1.0, 5, math.nan)]:
        assert f(P, 4, P, P, 4, 4, reg, reg_m, iters, tol, P, 1 << 20, ctypes.byref(o), None,
                 None) == uot.UOT_ERR_INVALID_ARG
    # workspace too small / misaligned
    assert f(P, 4, P, P, 4, 4, 0.1, 1.0, 5, 0.0, P, 16, ctypes.byref(o), None,
             None) == uot.UOT_ERR_WORKSPACE
    assert f(P, 4, P, P, 4, 4, 0.1, 1.0, 5, 0.0, ctypes.c_void_p(4096 + 8), 1 << 20,
             ctypes.byref(o), None, None) == uot.UOT_ERR_WORKSPACE
    # bad dtype, nonzero reserved, cluster out of range
    for field, val in [("dtype", 7), ("cluster", 9), ("algo", 3), ("max_ctas", -1)]:
        bad = uot.options()
        setattr(bad, field, val)
        assert f(P, 4, P, P, 4, 4, 0.1, 1.0, 5, 0.0, P, 1 << 20, ctypes.byref(bad), None,
                 None) == uot.UOT_ERR_INVALID_ARG
    bad = uot.options()
    bad.reserved[0] = 1
    assert f(P, 4, P, P, 4, 4, 0.1, 1.0, 5, 0.0, P, 1 << 20, ctypes.byref(bad), None,
             None) == uot.UOT_ERR_INVALID_ARG
    # unknown rule; the scaling-vector rule needs the kernel form
    assert f(P, 4, P, P, 4, 4, 0.1, 1.0, 5, 0.0, P, 1 << 20, ctypes.byref(uot.options(rule=2)),
             None, None) == uot.UOT_ERR_INVALID_ARG
    assert f(P, 4, P, P, 4, 4, 0.1, 1.0, 5, 0.0, P, 1 << 20,
             ctypes.byref(uot.options(rule=uot.UOT_RULE_POT)), None,
             None) == uot.UOT_ERR_UNSUPPORTED
    # storage and deterministic: unknown values; neither exists for the multi-pass
    # baseline
    for field, val in [("storage", 2), ("deterministic", 2), ("storage", -1)]:
        bad = uot.options()
        setattr(bad, field, val)
        assert f(P, 4, P, P, 4, 4, 0.1, 1.0, 5, 0.0, P, 1 << 20, ctypes.byref(bad), None,
                 None) == uot.UOT_ERR_INVALID_ARG
    for kw in [dict(storage=uot.UOT_STORAGE_KFORM), dict(deterministic=True)]:
        mp = uot.options(algo=uot.UOT_ALGO_MULTIPASS, **kw)
        assert f(P, 4, P, P, 4, 4, 0.1, 1.0, 5, 0.0, P, 1 << 20, ctypes.byref(mp), None,
                 None) == uot.UOT_ERR_UNSUPPORTED
    g = lib.uot_init_kernel
    assert g(None, 4, P, 4, 4, 4, 0.1, None, None) == uot.UOT_ERR_INVALID_ARG
    assert g(P, 4, P, 4, 4, 4, -1.0, None, None) == uot.UOT_ERR_INVALID_ARG
    h = lib.uot_cost
    assert h(P, 4, P, 4, 4, 4, 0, None, None) == uot.UOT_ERR_INVALID_ARG
    assert h(P, 2, P, 4, 4, 4, 0, P, None) == uot.UOT_ERR_INVALID_ARG
    k = lib.uot_sinkhorn_kform
    # missing U, non-integer storage scale, multi-pass requested
    assert k(P, 4, P, P, 4, 4, 0.1, 1.0, 5, 0.0, 0.0, None, P, P, 1 << 20, ctypes.byref(o),
             None, None) == uot.UOT_ERR_INVALID_ARG
    assert k(P, 4, P, P, 4, 4, 0.1, 1.0, 5, 0.0, 0.5, P, P, P, 1 << 20, ctypes.byref(o),
             None, None) == uot.UOT_ERR_INVALID_ARG
    mp = uot.options(algo=uot.UOT_ALGO_MULTIPASS)
    assert k(P, 4, P, P, 4, 4, 0.1, 1.0, 5, 0.0, 0.0, P, P, P, 1 << 20, ctypes.byref(mp),
             None, None) == uot.UOT_ERR_INVALID_ARG
    assert lib.uot_init_kernel_scaled(P, 4, P, 4, 4, 4, 0.1, 0.5, None, None) == \
        uot.UOT_ERR_INVALID_ARG
    assert lib.uot_kform_plan(P, 4, 0, None, P, 4, 4, P, 4, 0, None) == uot.UOT_ERR_INVALID_ARG
    assert lib.uot_kform_cost(P, 4, 9, P, P, P, 4, 4, 4, P, None) == uot.UOT_ERR_INVALID_ARG


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2412_11079_gb300 import uot
    saved = uot._lib
    uot._lib = None
    try:
        with pytest.raises(RuntimeError, match="libuot.so not found"):
            uot.load(str(tmp_path / "missing.so"))
    finally:
        uot._lib = saved


def test_product_path_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2412_11079_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle", text, flags=re.M), f
                assert "oracle/" not in text, f


def test_batch_autotuner_candidates_keep_the_tuning_contract(lib):
    """Every schedule the autotuner may pick is one include/uot.h accepts:
    ring depth 2..6, a power-of-two team, positive work per CTA, an on-chip
    cluster cap of 0, 1, 2, 4, 8 or 16, reserved fields zero; defaults too."""
    pytest.importorskip("torch")
    from paper_2412_11079_gb300 import batch, uot
    cands = batch.candidates()
    assert len(cands) == len({(t.stages, t.max_team, t.target_elems, t.resident_max_cluster)
                              for t in cands})
    for t in cands + [uot.batch_tuning()]:
        assert 2 <= t.stages <= 6
        assert t.max_team >= 1 and t.max_team & (t.max_team - 1) == 0
        assert t.target_elems > 0
        assert t.resident_max_cluster in (0, 1, 2, 4, 8, 16)
        assert list(t.reserved) == [0, 0, 0]


def test_wait_selftest_validates_arguments_without_a_gpu(lib):
    from paper_2412_11079_gb300 import uot
    P = ctypes.c_void_p(4096)  # never dereferenced: validation fails first
    f = lib.uot_selftest_wait
    assert f(None, 1, 0, 0.1, P, None) == uot.UOT_ERR_INVALID_ARG
    assert f(P, 1, 0, 0.1, None, None) == uot.UOT_ERR_INVALID_ARG
    for bad in (0.0, -1.0, 11.0, math.nan):
        assert f(P, 1, 0, bad, P, None) == uot.UOT_ERR_INVALID_ARG
    assert f(ctypes.c_void_p(4098), 1, 0, 0.1, P, None) == uot.UOT_ERR_INVALID_ARG


def test_size_limits(lib):
    """1 <= n, m <= 2^30: the kernels' indices and row counters stay 32-bit."""
    assert lib.uot_workspace_size(1 << 30, 4, None) > 0
    assert lib.uot_workspace_size(4, 1 << 30, None) > 0
    for n, m in ((0, 4), (4, 0), ((1 << 30) + 1, 4), (4, (1 << 30) + 1), (-1, 4)):
        assert lib.uot_workspace_size(n, m, None) == 0


def test_backward_batch_validation(lib):
    """The batched adjoint refuses bad batches, overlapping problems and a
    short workspace before touching the device (fake, aligned pointers)."""
    from paper_2412_11079_gb300 import uot
    n, m, T = 64, 96, 5
    one = int(lib.uot_backward_workspace_size(n, m, T))
    assert one > 0 and int(lib.uot_backward_batch_workspace_size(3, n, m, T)) == 3 * one
    assert int(lib.uot_backward_batch_workspace_size(0, n, m, T)) == 0
    hs = (int(lib.uot_grad_hist_size(n, m, T)) + 255) // 256 * 256
    P = ctypes.c_void_p(1 << 20)  # 256-byte aligned, never dereferenced

    def call(batch, sk=n * m, sc=n * m, sd=n * m, hstride=hs, ws=3 * one):
        return lib.uot_sinkhorn_backward_batch(batch, P, m, sk, P, m, sc, P, P, n, m, 0.1, 0.7,
                                               T, P, hstride, 1.0, None, P, m, sd, P, P, P, ws,
                                               None, None)
    assert call(0) == uot.UOT_ERR_INVALID_ARG
    assert call(70000) == uot.UOT_ERR_INVALID_ARG
    assert call(3, sk=n * m - 1) == uot.UOT_ERR_INVALID_ARG       # problems overlap
    assert call(3, sd=n * m + 2) == uot.UOT_ERR_INVALID_ARG       # dC rows lose alignment
    assert call(3, hstride=hs - 256) == uot.UOT_ERR_INVALID_ARG   # history too short
    assert call(3, hstride=hs + 8) == uot.UOT_ERR_INVALID_ARG     # history misaligned
    assert call(3, ws=3 * one - 1) == uot.UOT_ERR_WORKSPACE
