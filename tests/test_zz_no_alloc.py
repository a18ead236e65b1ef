"""The allocation-free min-cost flow entry point, checked against the CPU
oracle's network simplex and against pd_mcf_solve.

pd_mcf_solve_noalloc exists for callers that may not allocate device memory
while they solve -- a serving process with a fixed device-memory budget, or a
framework whose pool owns every device byte and forbids cudaMalloc/cudaFree
(and their implicit synchronisation) at run time.  It solves with scratch held
in one fixed array inside the library.  Here it must give exactly the oracle's
optimum, and the optimum the regular, allocating entry point gives, on two
calls in a row (the second call finds the previous call's contents in the
shared array), up to the documented limits (PD_NOALLOC_MAX_NODES - 1 nodes,
PD_NOALLOC_MAX_ARCS arcs), where the last bytes of each scratch region are in
use.

This file is named so that pytest collects it last.
"""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu

MAX_NODES = 32768      # PD_NOALLOC_MAX_NODES: n_nodes + 1 may reach it
MAX_ARCS = 1 << 20     # PD_NOALLOC_MAX_ARCS


def _csr(n, arcs, sup, cost):
    """arcs: sorted unique (tail, head) rows."""
    rp = np.zeros(n + 1, np.int64)
    np.add.at(rp, arcs[:, 0] + 1, 1)
    return dict(row_ptr=np.cumsum(rp), head=arcs[:, 1].astype(np.int32), cost=cost.astype(np.int64),
                supply=sup.astype(np.int64), tails=arcs[:, 0].astype(np.int32))


def _network(seed, n, m_target, cmax=5000):
    """A connected network (both directions of a chain) plus random arcs, m_target arcs in all."""
    rng = np.random.default_rng(seed)
    keys = set(zip(range(n - 1), range(1, n))) | set(zip(range(1, n), range(n - 1)))
    need = m_target - len(keys)
    while need > 0:
        u, v = rng.integers(0, n, 2 * need), rng.integers(0, n, 2 * need)
        for a, b in zip(u.tolist(), v.tolist()):
            if a != b and (a, b) not in keys:
                keys.add((a, b))
                need -= 1
                if need == 0:
                    break
    arcs = np.array(sorted(keys), np.int64)
    sup = rng.integers(-30, 31, n).astype(np.int64)
    sup[-1] -= sup.sum()
    return _csr(n, arcs, sup, rng.integers(0, cmax, len(arcs)))


def _w1_network():
    from paper_2110_14734_gb300 import synth
    r = oracle.w1_approx(synth.uniform_exp(800, 71), synth.uniform_exp(700, 72), "f32", eps=0.5, solve=False)
    net = {k: r["net"][k] for k in ("row_ptr", "head", "cost", "supply")}
    n = len(net["supply"])
    net["tails"] = np.repeat(np.arange(n, dtype=np.int32), np.diff(net["row_ptr"]))
    return net


def _oracle_opt(net):
    st, opt, _, _ = oracle.mcf_arcs(len(net["supply"]), net["tails"], net["head"], net["cost"], net["supply"])
    assert st == 0
    return opt


def _dev(net):
    return {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in net.items() if k != "tails"}


@pytest.fixture(scope="module")
def pd():
    from paper_2110_14734_gb300 import build
    build.build()
    from paper_2110_14734_gb300 import pdw1
    return pdw1


def test_noalloc_matches_the_oracle_and_the_allocating_solve_twice_in_a_row(pd):
    ctx = pd.pd_create(0)
    try:
        for net in (_network(901, 400, 6000), _w1_network(), _network(902, 60, 300)):
            exp = _oracle_opt(net)
            dnet = _dev(net)
            ref, _ = pd.pd_mcf_solve(ctx, dnet)
            first = pd.pd_mcf_solve_noalloc(dnet)
            second = pd.pd_mcf_solve_noalloc(dnet)
            assert first == exp and second == exp and ref == exp  # integer optimum: exact agreement
    finally:
        ctx.close()


@pytest.mark.parametrize("n,m", [(MAX_NODES - 1, 2 * (MAX_NODES - 2)), (4000, MAX_ARCS)])
def test_noalloc_at_its_node_and_arc_limits(pd, n, m):
    net = _network(7, n, m)
    assert len(net["supply"]) == n and len(net["head"]) == m
    exp = _oracle_opt(net)
    dnet = _dev(net)
    assert pd.pd_mcf_solve_noalloc(dnet) == exp
    assert pd.pd_mcf_solve_noalloc(dnet) == exp


def test_noalloc_rejects_networks_beyond_its_fixed_scratch(pd):
    n = 40000  # more nodes than PD_NOALLOC_MAX_NODES allows
    net = dict(row_ptr=torch.zeros(n + 1, dtype=torch.int64, device="cuda"),
               head=torch.zeros(0, dtype=torch.int32, device="cuda"),
               cost=torch.zeros(0, dtype=torch.int64, device="cuda"),
               supply=torch.zeros(n, dtype=torch.int64, device="cuda"))
    with pytest.raises(pd.PDError) as e:
        pd.pd_mcf_solve_noalloc(net)
    assert e.value.status == pd.PD_ECAPACITY
    big = _network(8, 5000, MAX_ARCS + 1)  # one arc more than the limit
    with pytest.raises(pd.PDError) as e:
        pd.pd_mcf_solve_noalloc(_dev(big))
    assert e.value.status == pd.PD_ECAPACITY


def test_noalloc_rejects_a_malformed_network(pd):
    net = _network(9, 50, 400)
    rp = net["row_ptr"].copy()
    rp[10], rp[11] = rp[11], rp[10]  # row 10 ends before it starts; every index stays in [0, m]
    assert rp[10] > rp[11]
    bad = dict(net, row_ptr=rp)
    with pytest.raises(pd.PDError) as e:
        pd.pd_mcf_solve_noalloc(_dev(bad))
    assert e.value.status == pd.PD_EINVAL
    assert pd.pd_mcf_solve_noalloc(_dev(net)) == _oracle_opt(net)  # the next call is unaffected
