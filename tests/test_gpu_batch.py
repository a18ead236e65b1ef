"""Batched W1 (pd_w1_approx_batch): every pair's result equals the one-pair
entry point and the oracle, across waves, layouts and degenerate pairs.
Runs on a GPU only."""
import numpy as np
import pytest
import torch

import oracle
from paper_2110_14734_gb300 import synth

pytestmark = pytest.mark.gpu

SAME = ("opt_quanta", "w1", "rwmd_quanta", "rwmd_A", "rwmd_B", "slack_quanta", "mass_A", "mass_B", "s",
        "coord_shift", "delta", "cell_quanta", "shift_quanta", "n_nodes", "n_arcs", "verified", "solve_method",
        "pivots", "degenerate", "arcs_priced", "cert_failures")


@pytest.fixture(scope="module")
def pd():
    from paper_2110_14734_gb300 import build
    build.build()
    from paper_2110_14734_gb300 import pdw1
    return pdw1


@pytest.fixture(scope="module")
def ctx(pd):
    c = pd.pd_create(0)
    yield c
    c.close()


def _pairs():
    u = synth.uniform_exp(500, 41)
    return [
        (synth.uniform_exp(2000, 1000), synth.uniform_exp(2000, 1001), "f32"),
        (synth.mixture_f32(5000, 7), synth.mixture_f32(4000, 8), "f32"),
        (synth.uniform_exp(4097, 11), synth.uniform_exp(33, 12), "f32"),
        (u, np.zeros((0, 2), np.float32), "f32"),
        (u, u.copy(), "f32"),
        (synth.lowerstar_u8(5000, 21), synth.lowerstar_u8(3000, 22), "u8"),
        (np.array([[0.1, 0.5]], np.float32), np.array([[0.2, 0.4], [0.3, 0.9]], np.float32), "f32"),
    ]


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("slots", [0, 3])
def test_batch_matches_single_pair_and_oracle(pd, ctx, slots):
    P = _pairs()
    eps = 0.1
    got = pd.pd_w1_approx_batch(ctx, [_cuda(a) for a, _, _ in P], [_cuda(b) for _, b, _ in P], eps,
                                pd.opts(batch_slots=slots))
    assert len(got) == len(P)
    for (A, B, dt), g in zip(P, got):
        one = pd.pd_w1_approx(ctx, _cuda(A), _cuda(B), eps, pd.opts(warm_start=0))  # the batch starts cold
        for k in SAME:
            assert g[k] == one[k], (k, g[k], one[k])
        r = oracle.w1_approx(A, B, dt, eps=eps)
        assert g["opt_quanta"] == r["opt"]
        assert (g["rwmd_A"], g["rwmd_B"]) == (r["LA"], r["LB"])
        assert g["verified"] == 1
    assert got[4]["opt_quanta"] == 0  # identical diagrams


def test_batch_host_inputs_and_global_tree_layout(pd, ctx):
    P = _pairs()[:3]
    eps = 0.05
    o = pd.opts(ns_smem=0, batch_slots=2)
    got = pd.pd_w1_approx_batch(ctx, [a for a, _, _ in P], [b for _, b, _ in P], eps, o)
    for (A, B, dt), g in zip(P, got):
        r = oracle.w1_approx(A, B, dt, eps=eps)
        assert g["opt_quanta"] == r["opt"] and g["verified"] == 1


def test_batch_of_large_pairs_is_exact(pd, ctx):
    # four 20k-point lower-star pairs in one launch (shared-memory trees)
    As = [synth.lowerstar_u8(20000, 1000 + 2 * i) for i in range(4)]
    Bs = [synth.lowerstar_u8(20000, 1001 + 2 * i) for i in range(4)]
    got = pd.pd_w1_approx_batch(ctx, [_cuda(a) for a in As], [_cuda(b) for b in Bs], 0.05)
    for A, B, g in zip(As, Bs, got):
        assert g["opt_quanta"] == pd.pd_w1_approx(ctx, _cuda(A), _cuda(B), 0.05)["opt_quanta"]
    r = oracle.w1_approx(As[0], Bs[0], "u8", eps=0.05)
    assert got[0]["opt_quanta"] == r["opt"]


def test_batch_rejects_bad_arguments(pd, ctx):
    A = _cuda(synth.uniform_exp(100, 1))
    with pytest.raises(ValueError):
        pd.pd_w1_approx_batch(ctx, [A, A], [A], 0.1)
    with pytest.raises(pd.PDError):
        pd.pd_w1_approx_batch(ctx, [A], [A], 0.1, pd.opts(solver=1))
    with pytest.raises(pd.PDError):
        pd.pd_w1_approx_batch(ctx, [A], [A], 0.0)
    assert pd.pd_w1_approx_batch(ctx, [], [], 0.1) == []


def test_batch_fallback_paths(pd, ctx):
    """Pairs solved without the transportation form (ns_transport=0: the
    sparse network in the worker) and pairs whose certificate fails on a
    coarse decomposition (small s: the sparse network after the shared
    launch) give the one-pair results and the oracle's optimum."""
    P = _pairs()[:3]
    o = pd.opts(ns_transport=0, batch_slots=2)
    got = pd.pd_w1_approx_batch(ctx, [_cuda(a) for a, _, _ in P], [_cuda(b) for _, b, _ in P], 0.1, o)
    for (A, B, dt), g in zip(P, got):
        one = pd.pd_w1_approx(ctx, _cuda(A), _cuda(B), 0.1, o)
        assert g["opt_quanta"] == one["opt_quanta"] == oracle.w1_approx(A, B, dt, eps=0.1)["opt"]
        assert g["solve_method"] == one["solve_method"] == 1
    A, B = synth.uniform_exp(700, 61), synth.uniform_exp(650, 62)
    fails = 0
    for s in (1, 2, 4, 13):
        g = pd.pd_w1_approx_batch(ctx, [_cuda(A), _cuda(B)], [_cuda(B), _cuda(A)], 0.1, pd.opts(s_override=s))
        ref = oracle.w1_approx(A, B, "f32", eps=0.1, s_override=s)["opt"]
        assert g[0]["opt_quanta"] == ref
        assert g[1]["opt_quanta"] == pd.pd_w1_approx(ctx, _cuda(B), _cuda(A), 0.1, pd.opts(s_override=s))["opt_quanta"]
        fails += sum(x["cert_failures"] > 0 for x in g)
        for x in g:
            if x["cert_failures"] > 0:
                assert x["solve_method"] == 1
    assert fails > 0  # the certificate-failure fallback of the batch ran


def test_autotuned_block_keeps_every_optimum_and_is_cached(pd, ctx, tmp_path):
    """pd_autotune times candidate (pricing block, walk limit) pairs on sample
    pairs; the choice is used by later solves of the same size class, which
    keep their optimum (the oracle's), and the cache file reproduces it
    without timing in a fresh context."""
    A, B = synth.lowerstar_u8(20000, 1000), synth.lowerstar_u8(20000, 1001)
    cache = str(tmp_path / "tune.txt")
    t = pd.pd_autotune(ctx, [_cuda(A)], [_cuda(B)], 0.05, cache_path=cache)
    assert t["pairs"] == 1 and t["from_cache"] == 0 and t["ns_block"] in (4096, 8192, 16384, 32768)
    assert t["ns_walk"] in (0, 8, 32) and t["candidates"] == 12
    assert t["best_ms"] > 0 and t["best_ms"] <= t["default_ms"] * 1.5
    r = pd.pd_w1_approx(ctx, _cuda(A), _cuda(B), 0.05)
    assert r["opt_quanta"] == oracle.w1_approx(A, B, "u8", eps=0.05)["opt"]
    line = open(cache).read().split()
    assert (int(line[-3]), int(line[-2]), int(line[-1])) == (t["size_class"], t["ns_block"], t["ns_walk"])
    c2 = pd.pd_create(0)
    try:
        t2 = pd.pd_autotune(c2, [_cuda(A)], [_cuda(B)], 0.05, cache_path=cache)
        assert t2["from_cache"] == 1 and t2["pairs"] == 0 and t2["ns_block"] == t["ns_block"]
        assert pd.pd_tuned_block(c2, 2 ** t["size_class"]) == t["ns_block"]
        assert pd.pd_tuned_block(c2, 2 ** (t["size_class"] + 3)) == 0
    finally:
        c2.close()
