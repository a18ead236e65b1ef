"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer results must be bit-exact: condensed nodes and multiplicities, RWMD,
the CSR network (rows, heads, costs, supplies) and the optimum of the sparse
network.  Runs on a GPU only.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2110_14734_gb300 import synth

pytestmark = pytest.mark.gpu


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


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _np(t):
    return t.cpu().numpy()


def _oracle_hats(A, B, dtype, k):
    XA, YA = oracle.quantize(A, dtype, k)
    XB, YB = oracle.quantize(B, dtype, k)
    return oracle.condense0(XA, YA), oracle.condense0(XB, YB)


def _assert_nodes(got, exp):
    assert got["n_nodes"] == len(exp["X"])
    np.testing.assert_array_equal(_np(got["X"]), exp["X"])
    np.testing.assert_array_equal(_np(got["Y"]), exp["Y"])
    np.testing.assert_array_equal(_np(got["cntA"]), exp["cntA"])
    np.testing.assert_array_equal(_np(got["cntB"]), exp["cntB"])
    np.testing.assert_array_equal(_np(got["morton"]).view(np.uint64), exp["code"])


PAIRS = {
    "uniform2k": lambda: (synth.uniform_exp(2000, 1000), synth.uniform_exp(2000, 1001), "f32"),
    "lowerstar20k": lambda: (synth.lowerstar_u8(20000, 1000), synth.lowerstar_u8(20000, 1001), "u8"),
    "mixture5k": lambda: (synth.mixture_f32(5000, 7), synth.mixture_f32(4000, 8), "f32"),
    "ragged": lambda: (synth.uniform_exp(4097, 11), synth.uniform_exp(33, 12), "f32"),
}


@pytest.mark.parametrize("name", list(PAIRS))
def test_condense_matches_oracle(pd, ctx, name):
    A, B, dt = PAIRS[name]()
    k = oracle.default_shift(dt)
    Ah, Bh = _oracle_hats(A, B, dt, k)
    for (G, P, seed) in [(1, 0, 0), (4096, 0, 0), (5000, 20, 3), (77777, 300, 12345)]:
        got = pd.pd_condense(ctx, _cuda(A), _cuda(B), G, P, pd.opts(seed=seed))
        exp = oracle.condense_delta(Ah, Bh, G, P, seed)
        _assert_nodes(got, exp)


def test_condense_host_inputs_and_one_sided(pd, ctx):
    A = synth.uniform_exp(3000, 21)
    E = np.zeros((0, 2), np.float32)
    Ah, Bh = _oracle_hats(A, E, "f32", 20)
    got = pd.pd_condense(ctx, A, E, 1, 0)  # numpy -> host pointers
    _assert_nodes(got, oracle.condense_delta(Ah, Bh, 1, 0, 0))
    got = pd.pd_condense(ctx, _cuda(E), _cuda(A), 1, 0)
    _assert_nodes(got, oracle.condense_delta(Bh, Ah, 1, 0, 0))
    got = pd.pd_condense(ctx, _cuda(E), _cuda(E), 1, 0)
    assert got["n_nodes"] == 0
    D = np.array([[0.25, 0.25], [0.5, 0.5]], np.float32)  # only diagonal points
    assert pd.pd_condense(ctx, _cuda(D), _cuda(D), 1, 0)["n_nodes"] == 0


def test_invalid_inputs_are_rejected(pd, ctx):
    A = synth.uniform_exp(100, 1)
    bad = A.copy()
    bad[5, 1] = np.nan
    with pytest.raises(pd.PDError) as e:
        pd.pd_condense(ctx, _cuda(bad), _cuda(A), 1, 0)
    assert e.value.status == pd.PD_EINVAL
    big = A.copy()
    big[3, 0] = 1000.0  # 1000 * 2^20 >= 2^29
    with pytest.raises(pd.PDError):
        pd.pd_rwmd_lower_bound(ctx, _cuda(big), _cuda(A))
    with pytest.raises(pd.PDError):
        pd.pd_condense(ctx, _cuda(A), _cuda(A), 10, 5)  # 2P >= G
    # the context is still usable after errors
    assert pd.pd_rwmd_lower_bound(ctx, _cuda(A), _cuda(A)) == (0, 0, 0)


@pytest.mark.parametrize("name", list(PAIRS))
def test_rwmd_matches_oracle(pd, ctx, name):
    A, B, dt = PAIRS[name]()
    Ah, Bh = _oracle_hats(A, B, dt, oracle.default_shift(dt))
    assert pd.pd_rwmd_lower_bound(ctx, _cuda(A), _cuda(B)) == oracle.rwmd(Ah, Bh)
    E = np.zeros((0, 2), A.dtype)
    Eh = (np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int64))
    assert pd.pd_rwmd_lower_bound(ctx, _cuda(A), _cuda(E)) == oracle.rwmd(Ah, Eh)


def _upload_nodes(nodes):
    return dict(X=_cuda(nodes["X"]), Y=_cuda(nodes["Y"]), cntA=_cuda(nodes["cntA"]), cntB=_cuda(nodes["cntB"]),
                morton=_cuda(nodes["code"].view(np.int64)))


def _assert_network(got, exp):
    np.testing.assert_array_equal(_np(got["row_ptr"]), exp["row_ptr"])
    np.testing.assert_array_equal(_np(got["head"]), exp["head"])
    np.testing.assert_array_equal(_np(got["cost"]), exp["cost"])
    np.testing.assert_array_equal(_np(got["supply"]), exp["supply"])


@pytest.mark.parametrize("s", [1, 2, 5, 13, 40, 167])
def test_wspd_network_matches_oracle(pd, ctx, s):
    A, B = synth.uniform_exp(1500, 31), synth.uniform_exp(1400, 32)
    Ah, Bh = _oracle_hats(A, B, "f32", 20)
    nodes = oracle.condense_delta(Ah, Bh, 600, 2, 9)
    tree = oracle.radix_tree(nodes)
    exp = oracle.build_network(nodes, *oracle.wspd(nodes, tree, s))
    got = pd.pd_wspd_sparsify(ctx, _upload_nodes(nodes), s)
    _assert_network(got, exp)


@pytest.mark.parametrize("s", [1, 3, 13, 40, 167])
def test_split_tree_network_matches_oracle(pd, ctx, s):
    """The paper's split tree: the nodes in its leaf order and the whole CSR
    network over them, bit-exact with the oracle's sequential recursion."""
    A, B = synth.uniform_exp(1500, 33), synth.uniform_exp(1400, 34)
    Ah, Bh = _oracle_hats(A, B, "f32", 20)
    nodes = oracle.condense_delta(Ah, Bh, 600, 2, 9)
    perm, tree = oracle.split_tree(nodes)
    ordered = oracle.reorder(nodes, perm)
    exp = oracle.build_network(ordered, *oracle.wspd(ordered, tree, s))
    got, gn = pd.pd_wspd_sparsify_tree(ctx, _upload_nodes(nodes), s, 1)
    for k in ("X", "Y", "cntA", "cntB"):
        np.testing.assert_array_equal(_np(gn[k]), ordered[k])
    _assert_network(got, exp)
    assert pd.pd_wspd_count(ctx, _upload_nodes(nodes), s, 1) == int(exp["row_ptr"][-1])
    # tree = 0 is the radix tree of pd_wspd_sparsify
    got0, gn0 = pd.pd_wspd_sparsify_tree(ctx, _upload_nodes(nodes), s, 0)
    exp0 = oracle.build_network(nodes, *oracle.wspd(nodes, oracle.radix_tree(nodes), s))
    _assert_network(got0, exp0)
    assert pd.pd_wspd_count(ctx, _upload_nodes(nodes), s, 0) == int(exp0["row_ptr"][-1])


def test_split_tree_clustered_and_tiny(pd, ctx):
    rng = np.random.default_rng(15)
    ctr = rng.integers(0, 2**24, (10, 2))
    pts = np.unique(np.concatenate([c + rng.integers(0, 3000, (200, 2)) for c in ctr]), axis=0)
    Xs, Ys = pts[:, 0].astype(np.int32), pts[:, 1].astype(np.int32)
    cnt = rng.integers(1, 4, len(Xs)).astype(np.int64)
    half = len(Xs) // 2
    empty = (np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int64))
    for nodes in [oracle.condense_delta((Xs[:half], Ys[:half], cnt[:half]), (Xs[half:], Ys[half:], cnt[half:]),
                                        1, 0, 0),
                  oracle.condense_delta((Xs[:1], Ys[:1], cnt[:1]), empty, 1, 0, 0),
                  oracle.condense_delta((Xs[:2], Ys[:2], cnt[:2]), (Xs[2:3], Ys[2:3], cnt[2:3]), 1, 0, 0)]:
        perm, tree = oracle.split_tree(nodes)
        ordered = oracle.reorder(nodes, perm)
        for s in (3, 20):
            got, gn = pd.pd_wspd_sparsify_tree(ctx, _upload_nodes(nodes), s, 1)
            np.testing.assert_array_equal(_np(gn["X"]), ordered["X"])
            _assert_network(got, oracle.build_network(ordered, *oracle.wspd(ordered, tree, s)))


def test_wspd_network_clustered_and_tiny(pd, ctx):
    rng = np.random.default_rng(5)
    ctr = rng.integers(0, 2**24, (10, 2))
    pts = np.concatenate([c + rng.integers(0, 3000, (200, 2)) for c in ctr])
    pts = np.unique(pts, axis=0)
    Xs, Ys = pts[:, 0].astype(np.int32), pts[:, 1].astype(np.int32)
    cnt = rng.integers(1, 4, len(Xs)).astype(np.int64)
    half = len(Xs) // 2
    Ah = (Xs[:half], Ys[:half], cnt[:half])
    Bh = (Xs[half:], Ys[half:], cnt[half:])
    empty = (np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int64))
    for nodes in [oracle.condense_delta(Ah, Bh, 1, 0, 0),
                  oracle.condense_delta((Xs[:1], Ys[:1], cnt[:1]), empty, 1, 0, 0),
                  oracle.condense_delta((Xs[:2], Ys[:2], cnt[:2]), (Xs[2:3], Ys[2:3], cnt[2:3]), 1, 0, 0)]:
        for s in (3, 20):
            tree = oracle.radix_tree(nodes)
            exp = oracle.build_network(nodes, *oracle.wspd(nodes, tree, s))
            got = pd.pd_wspd_sparsify(ctx, _upload_nodes(nodes), s)
            _assert_network(got, exp)


def _random_network(rng, n, extra):
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
    h = np.array([a[1] for a in arcs], np.int32)
    cost = {}
    for (u, v) in arcs:  # antiparallel pairs: sometimes equal cost, sometimes not
        if (v, u) in cost and rng.random() < 0.5:
            cost[(u, v)] = cost[(v, u)]
        else:
            cost[(u, v)] = int(rng.integers(0, 1000))
    c = np.array([cost[a] for a in arcs], np.int64)
    rp = np.zeros(n + 1, np.int64)
    np.add.at(rp, t + 1, 1)
    rp = np.cumsum(rp)
    sup = rng.integers(-20, 21, n).astype(np.int64)
    sup[-1] -= sup.sum()
    return dict(row_ptr=rp, head=h, cost=c, supply=sup, tails=t.astype(np.int32))


@pytest.mark.parametrize("seed", range(6))
def test_mcf_random_networks_match_network_simplex(pd, ctx, seed):
    rng = np.random.default_rng(100 + seed)
    net = _random_network(rng, int(rng.integers(5, 300)), int(rng.integers(10, 3000)))
    st, opt, flow, pot = oracle.mcf_arcs(len(net["supply"]), net["tails"], net["head"], net["cost"], net["supply"])
    assert st == 0
    dnet = {k: _cuda(v) for k, v in net.items() if k != "tails"}
    for blk in (0, 1, 64):  # network simplex, different pricing blocks, half-cycles walked or scanned
        for walk in (0, 2, 512):
            got, stats = pd.pd_mcf_solve(ctx, dnet, pd.opts(ns_block=blk, ns_walk=walk))
            assert got == opt and stats["verified"] == 1 and stats["solve_method"] == 1
    for alpha in (2, 8, 16):  # cost scaling
        got, stats = pd.pd_mcf_solve(ctx, dnet, pd.opts(solver=1, alpha=alpha, verify=1))
        assert got == opt and stats["verified"] == 1


@pytest.mark.parametrize("name", ["uniform2k", "mixture5k", "ragged"])
def test_mcf_on_w1_networks(pd, ctx, name):
    A, B, dt = PAIRS[name]()
    r = oracle.w1_approx(A, B, dt, eps=0.5)
    net = {k: _cuda(r["net"][k]) for k in ("row_ptr", "head", "cost", "supply")}
    got, stats = pd.pd_mcf_solve(ctx, net, pd.opts(verify=1))
    assert got == r["opt"] and stats["verified"] == 1
    if name != "mixture5k":
        got, stats = pd.pd_mcf_solve(ctx, net, pd.opts(solver=1, verify=1))
        assert got == r["opt"] and stats["verified"] == 1


def _check_w1(pd, ctx, A, B, dt, eps, **kw):
    tree = kw.get("tree", "radix")
    kappa, tau = kw.get("kappa", 1), kw.get("tau", 0)
    r = oracle.w1_approx(A, B, dt, eps=eps, tree=tree, kappa=kappa, tau=tau,
                         **{k: v for k, v in kw.items() if k in ("k", "s_override", "perturb", "seed", "condense")})
    o = pd.opts(verify=1, s_override=kw.get("s_override", 0), perturb=int(kw.get("perturb", True)),
                seed=kw.get("seed", 0), condense=int(kw.get("condense", True)),
                coord_shift=kw.get("k", -1) if kw.get("k") is not None else -1, tree=int(tree == "split"),
                diag_kappa=kappa, diag_tau=tau)
    g = pd.pd_w1_approx(ctx, _cuda(A), _cuda(B), eps, o)
    assert (g["rwmd_A"], g["rwmd_B"]) == (r["LA"], r["LB"])
    # the simplex straight on the sparse network must agree as well
    g2 = pd.pd_w1_approx(ctx, _cuda(A), _cuda(B), eps, pd.opts(
        s_override=o.s_override, perturb=o.perturb, seed=o.seed, condense=o.condense, coord_shift=o.coord_shift,
        ns_transport=0, tree=o.tree, diag_kappa=kappa, diag_tau=tau))
    assert g2["opt_quanta"] == r["opt"] and g2["solve_method"] == 1
    assert g["s"] == r["s"] and g["cell_quanta"] == r["G"] and g["shift_quanta"] == r["P"]
    assert g["delta"] == r["delta"]
    assert g["n_nodes"] == len(r["nodes"]["X"]) and g["n_arcs"] == int(r["net"]["row_ptr"][-1])
    assert g["opt_quanta"] == r["opt"], (g["opt_quanta"], r["opt"])
    assert g["verified"] == 1
    assert g["w1"] == math.ldexp(r["opt"], -r["k"])
    return g, r


@pytest.mark.parametrize("eps", [0.1, 0.5, 2.0])
def test_w1_approx_uniform2k(pd, ctx, eps):
    A, B, dt = PAIRS["uniform2k"]()
    g, r = _check_w1(pd, ctx, A, B, dt, eps)
    # (1 +- eps) band against the exact FP64 W1 (Corollary, approximation bound)
    w = oracle.w1_exact(A.astype(np.float64), B.astype(np.float64))
    q = 2.0 ** -20
    slack = g["slack_quanta"] * q + (r["FA"] + r["FB"]) * q
    assert (1 - eps) * w - slack <= g["w1"] <= (1 + eps) * w + slack


@pytest.mark.parametrize("eps", [0.1, 0.05, 0.01])
def test_w1_approx_lowerstar_u8(pd, ctx, eps):
    A, B = synth.lowerstar_u8(20000, 1000), synth.lowerstar_u8(20000, 1001)
    g, r = _check_w1(pd, ctx, A, B, "u8", eps)
    # other pricing blocks and walk limits reach the same optimum
    for walk, blk in ((0, 0), (48, 32768), (512, 4096)):
        assert pd.pd_w1_approx(ctx, _cuda(A), _cuda(B), eps, pd.opts(ns_walk=walk, ns_block=blk))[
            "opt_quanta"] == r["opt"]


@pytest.mark.parametrize("name,eps", [("uniform2k", 0.1), ("lowerstar20k", 0.05), ("mixture5k", 0.1)])
def test_w1_approx_on_the_split_tree(pd, ctx, name, eps):
    """Algorithm 4 on the paper's split tree (pd_opts.tree = 1): every integer
    result bit-exact with the oracle on the same tree, both solve paths."""
    A, B, dt = PAIRS[name]()
    g, r = _check_w1(pd, ctx, A, B, dt, eps, tree="split")
    assert g["n_arcs"] == int(r["net"]["row_ptr"][-1])


@pytest.mark.parametrize("kappa,tau", [(0, 3000), (0, 200000), (1, 5000)])
def test_w1_approx_unbalanced_transport(pd, ctx, kappa, tau):
    """The Conclusion's unbalanced transport on R^2: ā and b̄ destroy and
    create units at kappa * d_diag + tau quanta.  Every integer result equals
    the oracle's (both solve paths, both trees), one-sided pairs give the sum
    of the costs, and the nearest-neighbour bounds stay below the optimum."""
    A, B = synth.uniform_exp(1500, 51), synth.uniform_exp(1200, 52)
    g, r = _check_w1(pd, ctx, A, B, "f32", 0.1, kappa=kappa, tau=tau)
    _check_w1(pd, ctx, A, B, "f32", 0.1, kappa=kappa, tau=tau, tree="split")
    g = pd.pd_w1_approx(ctx, _cuda(A), _cuda(B), 0.1, pd.opts(diag_kappa=kappa, diag_tau=tau, solver=1))
    assert g["opt_quanta"] == r["opt"]
    E = np.zeros((0, 2), np.float32)
    ge, re_ = _check_w1(pd, ctx, A, E, "f32", 0.1, kappa=kappa, tau=tau, condense=False)
    Ah = re_["Ahat"]
    assert ge["opt_quanta"] == sum(int(c) * oracle.cmake(int(x), int(y), kappa, tau) for x, y, c in zip(*Ah))
    db = [synth.uniform_exp(int(n), 60 + i) for i, n in enumerate((300, 900, 1500))]
    pd.pd_db_build(ctx, [_cuda(d) for d in db])
    nn = pd.pd_nn_search(ctx, _cuda(A), 0.1, pd.opts(diag_kappa=kappa, diag_tau=tau, nn_prune=0))
    exp = [oracle.w1_approx(A, d, "f32", eps=0.1, kappa=kappa, tau=tau)["opt"] for d in db]
    assert nn["opt"] == exp and all(lb <= o for lb, o in zip(nn["lb"], exp))
    with pytest.raises(pd.PDError):
        pd.pd_w1_approx(ctx, _cuda(A), _cuda(B), 0.1, pd.opts(diag_kappa=2))


def test_w1_approx_edge_cases(pd, ctx):
    A = synth.uniform_exp(500, 41)
    B = synth.uniform_exp(450, 42)
    E = np.zeros((0, 2), np.float32)
    _check_w1(pd, ctx, A, E, "f32", 0.1)
    g, r = _check_w1(pd, ctx, A, E, "f32", 0.1, condense=False)  # one side empty: all mass to the diagonal
    assert g["opt_quanta"] == g["rwmd_quanta"]
    g, _ = _check_w1(pd, ctx, A, A, "f32", 0.1)
    assert g["opt_quanta"] == 0
    g1, _ = _check_w1(pd, ctx, A, B, "f32", 0.1, seed=7)
    g2, _ = _check_w1(pd, ctx, B, A, "f32", 0.1, seed=7)
    assert g1["opt_quanta"] == g2["opt_quanta"]
    _check_w1(pd, ctx, A, B, "f32", 0.1, s_override=1)
    _check_w1(pd, ctx, A, B, "f32", 0.1, s_override=3, perturb=False)
    _check_w1(pd, ctx, A, B, "f32", 0.1, condense=False)
    _check_w1(pd, ctx, A, B, "f32", 0.1, k=12)
    g = pd.pd_w1_approx(ctx, _cuda(E), _cuda(E), 0.1)
    assert g["opt_quanta"] == 0 and g["n_nodes"] == 0


def test_cost_scaling_round_cap_and_time_limit_return_timeout(pd, ctx):
    """The watchdogs of both solvers end a solve early with PD_ETIMEOUT and
    leave the context usable: the cost-scaling kernel's round cap (every
    block leaves through its bounded grid barriers) and the simplex's device
    wall-clock limit (checked every 128 pivots)."""
    A, B, dt = PAIRS["uniform2k"]()
    r = oracle.w1_approx(A, B, dt, eps=0.5, solve=False)
    net = {k: _cuda(r["net"][k]) for k in ("row_ptr", "head", "cost", "supply")}
    for rounds in (1, 2, 5):
        with pytest.raises(pd.PDError) as e:
            pd.pd_mcf_solve(ctx, net, pd.opts(solver=1, max_rounds=rounds))
        assert e.value.status == pd.PD_ETIMEOUT
    L = synth.lowerstar_u8(20000, 1000), synth.lowerstar_u8(20000, 1001)
    with pytest.raises(pd.PDError) as e:
        pd.pd_w1_approx(ctx, _cuda(L[0]), _cuda(L[1]), 0.05, pd.opts(time_limit_ms=1))
    assert e.value.status == pd.PD_ETIMEOUT
    got, _ = pd.pd_mcf_solve(ctx, net, pd.opts(solver=1))
    assert got == oracle.mcf(r["net"])[0]


def test_solver_round_cap_returns_timeout(pd, ctx):
    A, B, dt = PAIRS["uniform2k"]()
    with pytest.raises(pd.PDError) as e:
        pd.pd_w1_approx(ctx, _cuda(A), _cuda(B), 0.1, pd.opts(max_rounds=3))
    assert e.value.status == pd.PD_ETIMEOUT
    # and the context keeps working
    assert pd.pd_w1_approx(ctx, _cuda(A), _cuda(B), 0.5)["opt_quanta"] > 0


@pytest.mark.parametrize("eps", [0.05, 0.1, 0.01])
def test_w1_approx_full_size_lowerstar_100k(pd, ctx, eps):
    """The benchmark workload (100k + 100k uint8 points) at every eps of the
    lower-star configuration (s = 327, 167, 1607): exact parity of every
    integer result with the oracle."""
    A, B = synth.lowerstar_u8(100000, 1000), synth.lowerstar_u8(100000, 1001)
    _check_w1(pd, ctx, A, B, "u8", eps)


@pytest.mark.parametrize("n", [5000, 10000])
def test_w1_approx_continuous_mixture(pd, ctx, n):
    """Continuous float32 coordinates with few duplicates (birth U[0,1],
    persistence 0.95 Exp(0.01) + 0.05 U[0, 0.5]) at eps = 0.1: about 2n
    condensed nodes, more than the all-shared-memory tree holds (the 5k pair
    takes the layout with pred and flow in global memory, the 10k pair keeps
    the whole tree in global memory); 10k points per diagram is the largest
    size of this shape the CPU oracle solves within a test's time.  At 5k
    the result is also checked against the exact FP64 W1 (the (1 +- eps) band
    of the approximation bound)."""
    A, B = synth.mixture_f32(n, 1000), synth.mixture_f32(n, 1001)
    g, r = _check_w1(pd, ctx, A, B, "f32", 0.1)
    assert g["n_nodes"] > 9216
    if n == 5000:
        w = oracle.w1_exact(A.astype(np.float64), B.astype(np.float64))
        q = 2.0 ** -20
        slack = g["slack_quanta"] * q + (r["FA"] + r["FB"]) * q
        assert 0.9 * w - slack <= g["w1"] <= 1.1 * w + slack


def test_w1_approx_coordinates_beyond_float32_exactness(pd, ctx):
    """Diagrams translated along (t, t) to coordinates of 2^26-2^27 quanta,
    where float32 no longer holds them exactly: the integer path must still
    be bit-exact with the oracle."""
    A, B = synth.uniform_exp(1500, 81) + 100.0, synth.uniform_exp(1400, 82) + 100.0
    assert (A * 2.0 ** 20).min() >= 2 ** 23
    _check_w1(pd, ctx, A.astype(np.float32), B.astype(np.float32), "f32", 0.1)


def test_w1_certificate_on_coarse_decompositions(pd, ctx):
    """Small s gives a sparse network that misses many direct routes: the
    transportation optimum must then fail its certificate (tree query of the
    WSPD) and the sparse network be solved instead -- the optimum always
    equals the oracle's OPT(WS)."""
    A, B = synth.uniform_exp(700, 61), synth.uniform_exp(650, 62)
    fails = 0
    for s in (1, 2, 4, 13):
        g, r = _check_w1(pd, ctx, A, B, "f32", 0.1, s_override=s)
        fails += g["cert_failures"] > 0
        if g["cert_failures"] > 0:
            assert g["solve_method"] == 1
    assert fails > 0


@pytest.mark.parametrize("kappa,tau", [(1, 0), (0, 5000), (1, 1000)])
def test_rwmd_grid_matches_oracle(pd, ctx, kappa, tau):
    """Sides whose product of node counts is at least 2^28 take the grid
    search (rings of cells, stopped by the best distance or by the diagonal
    cost); a few far outliers in both diagrams leave the rings unfinished and
    go through the all-pairs scan.  L_A, L_B are the oracle's brute force."""
    A, B = synth.mixture_f32(25000, 41), synth.mixture_f32(22000, 42)
    far = np.array([[0.9, 9.5], [0.1, 7.0], [3.0, 3.2]], np.float32)
    A = np.concatenate([A, far])
    B = np.concatenate([B, far[:2] + np.float32(0.25)])
    Ah, Bh = _oracle_hats(A, B, "f32", 20)
    assert len(Ah[0]) * len(Bh[0]) >= 1 << 28
    o = pd.opts(diag_kappa=kappa, diag_tau=tau)
    assert pd.pd_rwmd_lower_bound(ctx, _cuda(A), _cuda(B), o) == oracle.rwmd(Ah, Bh, kappa, tau)
    assert pd.pd_rwmd_lower_bound(ctx, _cuda(B), _cuda(A), o) == oracle.rwmd(Bh, Ah, kappa, tau)


def test_rwmd_grid_lowerstar_100k(pd, ctx):
    """The 100k lower-star pair of the benchmark (lattice coordinates, many
    equal distances) through whichever RWMD path its sizes select."""
    A, B = synth.lowerstar_u8(100000, 1000), synth.lowerstar_u8(100000, 1001)
    Ah, Bh = _oracle_hats(A, B, "u8", 12)
    assert pd.pd_rwmd_lower_bound(ctx, _cuda(A), _cuda(B)) == oracle.rwmd(Ah, Bh)


@pytest.mark.parametrize("tree", [0, 1])
def test_wspd_count_matches_oracle_10k_nodes(pd, ctx, tree):
    """About 10,000 continuous nodes at s = 40 (a pair frontier of about a
    million pairs at its widest level), both trees: the counted WSPD equals
    the arcs of the oracle's network."""
    A, B = synth.mixture_f32(5200, 51), synth.mixture_f32(4800, 52)
    Ah, Bh = _oracle_hats(A, B, "f32", 20)
    nodes = oracle.condense_delta(Ah, Bh, 16, 0, 3)
    assert len(nodes["X"]) > 9000
    if tree == 1:
        perm, t = oracle.split_tree(nodes)
        nodes_t = oracle.reorder(nodes, perm)
    else:
        nodes_t, t = nodes, oracle.radix_tree(nodes)
    exp = oracle.build_network(nodes_t, *oracle.wspd(nodes_t, t, 40))
    assert pd.pd_wspd_count(ctx, _upload_nodes(nodes), 40, tree) == int(exp["row_ptr"][-1])
