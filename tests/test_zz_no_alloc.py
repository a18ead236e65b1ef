"""The allocation-free min-cost flow entry point, checked against pd_mcf_solve.

pd_mcf_solve_noalloc exists for callers that may not allocate device memory
while they solve -- a serving process with a fixed device-memory budget, or a
framework whose pool owns every device byte and forbids cudaMalloc/cudaFree
(and their implicit synchronisation) at run time.  It solves with scratch held
in one fixed array inside the library.  Here it must give exactly the optimum
that the regular, allocating entry point gives, on two calls in a row (the
second call finds the previous call's contents in the shared array).

This file is named so that pytest collects it last.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _network(seed, n, extra):
    rng = np.random.default_rng(seed)
    arcs = set()
    for u in range(n - 1):
        arcs.add((u, u + 1))
        arcs.add((u + 1, u))
    for _ in range(extra):
        u, v = (int(x) for x in rng.integers(0, n, 2))
        if u != v:
            arcs.add((u, v))
    arcs = sorted(arcs)
    t = np.array([a[0] for a in arcs], np.int64)
    rp = np.zeros(n + 1, np.int64)
    np.add.at(rp, t + 1, 1)
    sup = rng.integers(-30, 31, n).astype(np.int64)
    sup[-1] -= sup.sum()
    return dict(row_ptr=np.cumsum(rp), head=np.array([a[1] for a in arcs], np.int32),
                cost=rng.integers(0, 5000, len(arcs)).astype(np.int64), supply=sup)


def _w1_network():
    import oracle
    from paper_2110_14734_gb300 import synth
    r = oracle.w1_approx(synth.uniform_exp(800, 71), synth.uniform_exp(700, 72), "f32", eps=0.5, solve=False)
    return {k: r["net"][k] for k in ("row_ptr", "head", "cost", "supply")}


def test_noalloc_matches_the_allocating_solve_twice_in_a_row():
    from paper_2110_14734_gb300 import build
    build.build()
    from paper_2110_14734_gb300 import pdw1
    ctx = pdw1.pd_create(0)
    try:
        for net in (_network(901, 400, 6000), _w1_network(), _network(902, 60, 300)):
            dnet = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in net.items()}
            ref, _ = pdw1.pd_mcf_solve(ctx, dnet)
            first = pdw1.pd_mcf_solve_noalloc(dnet)
            second = pdw1.pd_mcf_solve_noalloc(dnet)
            assert first == ref and second == ref  # integer optimum: exact agreement
    finally:
        ctx.close()


def test_noalloc_rejects_networks_beyond_its_fixed_scratch():
    from paper_2110_14734_gb300 import build
    build.build()
    from paper_2110_14734_gb300 import pdw1
    n = 40000  # more nodes than PD_NOALLOC_MAX_NODES allows
    net = dict(row_ptr=torch.zeros(n + 1, dtype=torch.int64, device="cuda"),
               head=torch.zeros(0, dtype=torch.int32, device="cuda"),
               cost=torch.zeros(0, dtype=torch.int64, device="cuda"),
               supply=torch.zeros(n, dtype=torch.int64, device="cuda"))
    with pytest.raises(pdw1.PDError) as e:
        pdw1.pd_mcf_solve_noalloc(net)
    assert e.value.status == pdw1.PD_ECAPACITY
