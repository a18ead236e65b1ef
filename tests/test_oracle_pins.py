"""Pins for the CPU oracle: each oracle function checked against something
other than itself -- library routines, closed forms, hand-derived values,
brute force on tiny inputs, and the paper's theorems as invariants.

Nothing here needs a GPU.
"""
import itertools
import json
import math
import os
from collections import Counter
from fractions import Fraction

import numpy as np
import pytest
from scipy.optimize import linear_sum_assignment, linprog
from scipy.sparse import csr_matrix
from scipy.sparse.csgraph import shortest_path

from paper_2110_14734_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SQ2 = math.sqrt(2.0)


# --------------------------------------------------------------------------
# exact integer roots and rounded-up costs (vs Python's math.isqrt)
# --------------------------------------------------------------------------

def test_isqrt_and_ceil_sqrt_vs_math_isqrt(orc):
    rng = np.random.default_rng(1)
    vals = [0, 1, 2, 3, 4, 15, 16, 17, 2**32 - 1, 2**32, 2**62, 2**63 - 1, 2**64 - 1,
            (2**32 - 1) ** 2, (2**32 - 1) ** 2 - 1]
    vals += [int(v) for v in rng.integers(0, 2**63, 300, dtype=np.uint64)]
    vals += [int(v) ** 2 + d for v in rng.integers(0, 2**31, 100) for d in (-1, 0, 1) if int(v) ** 2 + d >= 0]
    for v in vals:
        r = math.isqrt(v)
        assert orc.isqrt(v) == r
        assert orc.ceil_sqrt(v) == (r if r * r == v else r + 1)


def test_costs_are_rounded_up_l2_and_diagonal_distance(orc):
    rng = np.random.default_rng(2)
    for _ in range(500):
        x1, y1, x2, y2 = (int(v) for v in rng.integers(-(2**29), 2**29, 4))
        d2 = (x1 - x2) ** 2 + (y1 - y2) ** 2
        c = orc.cost(x1, y1, x2, y2)
        assert (c - 1) ** 2 < d2 <= c * c or (d2 == 0 and c == 0)
        t = abs(y1 - x1)
        cd = orc.cdiag(x1, y1)
        # smallest integer >= t / sqrt(2)
        assert Fraction(cd) ** 2 * 2 >= t * t and (cd == 0 or Fraction(cd - 1) ** 2 * 2 < t * t)
    assert orc.cdiag(0, 2) == 2 and orc.cdiag(0, 3) == 3 and orc.cdiag(0, 4) == 3 and orc.cdiag(5, 5) == 0


# --------------------------------------------------------------------------
# quantisation
# --------------------------------------------------------------------------

def test_quantize_known_values(orc):
    q = 2.0 ** -20
    A = np.array([[0.5, 0.25], [1 / 256, 0.0], [2.5 * q, 0.75], [3.5 * q, 0.75], [0.3, 0.3]], np.float32)
    X, Y = orc.quantize(A, "f32", 20)
    # 0.5 -> 2^19; half-quantum values round to even; the diagonal point is dropped
    assert list(X) == [2**19, 4096, 2, 4] and list(Y) == [2**18, 0, 3 * 2**18, 3 * 2**18]
    U = np.array([[255, 0], [3, 3], [0, 7]], np.uint8)
    X, Y = orc.quantize(U, "u8", 12)
    assert list(X) == [255 * 4096, 0] and list(Y) == [0, 7 * 4096]
    with pytest.raises(ValueError):
        orc.quantize(np.array([[np.nan, 1.0]], np.float32), "f32", 20)
    with pytest.raises(ValueError):
        orc.quantize(np.array([[600.0, 1.0]], np.float32), "f32", 20)  # 600 * 2^20 >= 2^29


# --------------------------------------------------------------------------
# 0-condensation (vs collections.Counter)
# --------------------------------------------------------------------------

def test_condense0_matches_counter(orc):
    rng = np.random.default_rng(3)
    X = rng.integers(-5, 5, 2000).astype(np.int32)
    Y = rng.integers(-5, 5, 2000).astype(np.int32)
    UX, UY, cnt = orc.condense0(X, Y)
    ref = Counter(zip(X.tolist(), Y.tolist()))
    assert dict(zip(zip(UX.tolist(), UY.tolist()), cnt.tolist())) == ref
    assert list(zip(UX.tolist(), UY.tolist())) == sorted(ref)


# --------------------------------------------------------------------------
# RWMD (Algorithm 1 + the diagonal arc)
# --------------------------------------------------------------------------

def _brute_rwmd(P, Q):
    def side(P, Q):
        L = 0
        for x, y, c in zip(*P):
            best = math.isqrt(((abs(int(y) - int(x)) ** 2) + 1) // 2)
            if 2 * best * best < (int(y) - int(x)) ** 2:
                best += 1
            for u, v in zip(Q[0], Q[1]):
                d2 = (int(x) - int(u)) ** 2 + (int(y) - int(v)) ** 2
                r = math.isqrt(d2)
                r += r * r < d2
                best = min(best, r)
            L += int(c) * best
        return L
    return side(P, Q), side(Q, P)


def test_rwmd_brute_force_and_closed_forms(orc):
    rng = np.random.default_rng(4)
    for trial in range(5):
        P = (rng.integers(0, 200, 30).astype(np.int32), rng.integers(0, 200, 30).astype(np.int32),
             rng.integers(1, 4, 30).astype(np.int64))
        Q = (rng.integers(0, 200, 25).astype(np.int32), rng.integers(0, 200, 25).astype(np.int32),
             rng.integers(1, 4, 25).astype(np.int64))
        LA, LB, L = orc.rwmd(P, Q)
        assert (LA, LB) == _brute_rwmd(P, Q) and L == max(LA, LB)
    # B empty: L_A is the closed-form sum of diagonal distances, L_B = 0
    LA, LB, L = orc.rwmd(P, (np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int64)))
    assert LA == sum(int(c) * orc.cdiag(int(x), int(y)) for x, y, c in zip(*P)) and LB == 0
    # identical diagrams: every node has a partner at distance 0
    assert orc.rwmd(P, P) == (0, 0, 0)


def test_rwmd_needs_the_diagonal_option(orc):
    # A = {(0, 0.1)}, B = {(100, 100.1)} in units of 0.1: RWMD without the
    # diagonal would be ~1414 > W1 ~ 1.41; with it RWMD <= W1.
    P = (np.array([0], np.int32), np.array([1], np.int32), np.array([1], np.int64))
    Q = (np.array([1000], np.int32), np.array([1001], np.int32), np.array([1], np.int64))
    LA, LB, L = orc.rwmd(P, Q)
    w1 = orc.w1_exact(np.array([[0, 1]]), np.array([[1000, 1001]]))
    assert L <= math.ceil(w1) and L == 1


# --------------------------------------------------------------------------
# eps -> s (tighter bound from the Experiments) and delta (Algorithm 2)
# --------------------------------------------------------------------------

def test_s_from_eps(orc):
    for eps, s in [(0.1, 167), (0.05, 327), (0.01, 1607)]:
        assert orc.s_from_eps(eps) == s
        assert orc.bound(s) <= 1 + eps < orc.bound(s - 1)
    # the paper's own pairings satisfy the bound: s = 40 for 0.5, s = 93 for 0.2
    assert orc.bound(40) <= 1.5 and orc.bound(93) <= 1.2
    assert orc.eps_c(12) == 1.0 and orc.eps_c(11) == 1.0 and orc.eps_c(20) == 0.5


def test_delta_params_satisfy_the_proposition(orc):
    rng = np.random.default_rng(5)
    for _ in range(200):
        FA, FB = (int(v) for v in rng.integers(0, 10**6, 2))
        LA, LB = (int(v) for v in rng.integers(0, 10**12, 2))
        s = int(rng.integers(3, 2000))
        delta, G, P = orc.delta_params(LA, LB, FA, FB, s)
        Llo = max(LA - FA, LB - FB, 0)
        ec = 8.0 / (s - 4) if s >= 12 else 1.0
        if FA + FB > 0:
            # sqrt(2) (|A|+|B|)/2 * delta <= eps_c * L_lo  (Proposition, delta-condensation)
            assert SQ2 * (FA + FB) / 2 * delta <= ec * Llo * (1 + 1e-12) + 1e-9
        assert G >= 1 and 0 <= P and 2 * P < G
        assert G == 1 or G <= 0.99 * delta
        assert P <= 0.005 * delta


def test_splitmix_finaliser_published_vector(orc):
    # SplitMix64 from state 0: first output = finaliser(0x9E3779B97F4A7C15)
    assert orc.mix64(0x9E3779B97F4A7C15) == 0xE220A8397B1DCDAF


def test_perturbation_range_and_determinism(orc):
    seen = Counter()
    for cx in range(-30, 30):
        for cy in range(0, 30):
            dx, dy = orc.perturb(7, cx, cy, 3)
            assert -3 <= dx <= 3 and -3 <= dy <= 3
            assert (dx, dy) == orc.perturb(7, cx, cy, 3)
            seen[dx] += 1
    assert len(seen) == 7 and min(seen.values()) > 150
    assert orc.perturb(7, 1, 2, 0) == (0, 0)


def test_morton_known_values(orc):
    assert [orc.morton(1, 0), orc.morton(0, 1), orc.morton(1, 1), orc.morton(2, 0), orc.morton(3, 3)] == \
        [1, 2, 3, 4, 15]
    assert orc.morton(0xFFFFFFFF, 0) == 0x5555555555555555
    assert orc.morton(0, 0xFFFFFFFF) == 0xAAAAAAAAAAAAAAAA


def _rand_hat(rng, n, lo, hi, cmax=3):
    X = rng.integers(lo, hi, n).astype(np.int32)
    Y = rng.integers(lo, hi, n).astype(np.int32)
    keep = X != Y
    return (X[keep], Y[keep], rng.integers(1, cmax + 1, keep.sum()).astype(np.int64))


def test_condense_delta_snaps_to_nearest_lattice_point(orc):
    rng = np.random.default_rng(6)
    Ah = orc.condense0(*_rand_hat(rng, 400, -300, 300)[:2])
    Bh = orc.condense0(*_rand_hat(rng, 400, -300, 300)[:2])
    for G, P in [(1, 0), (7, 0), (10, 3), (25, 12)]:
        nodes = orc.condense_delta(Ah, Bh, G, P, 99)
        X, Y = nodes["X"].astype(np.int64), nodes["Y"].astype(np.int64)
        assert nodes["cntA"].sum() == Ah[2].sum() and nodes["cntB"].sum() == Bh[2].sum()
        assert len(set(zip(X.tolist(), Y.tolist()))) == len(X)
        # every input node is at the node of its nearest lattice point (ties round up)
        where = {}
        for x, y in zip(X.tolist(), Y.tolist()):
            cx = math.floor(Fraction(x, G) + Fraction(1, 2))
            cy = math.floor(Fraction(y, G) + Fraction(1, 2))
            assert abs(x - G * cx) <= P and abs(y - G * cy) <= P
            where[(cx, cy)] = (x, y)
        totA, totB = Counter(), Counter()
        for (hx, hy, hc), tot in ((Ah, totA), (Bh, totB)):
            for x, y, c in zip(hx.tolist(), hy.tolist(), hc.tolist()):
                cell = (math.floor(Fraction(x, G) + Fraction(1, 2)), math.floor(Fraction(y, G) + Fraction(1, 2)))
                tot[where[cell]] += c
        assert totA == Counter({k: v for k, v in zip(zip(X.tolist(), Y.tolist()), nodes["cntA"].tolist()) if v})
        assert totB == Counter({k: v for k, v in zip(zip(X.tolist(), Y.tolist()), nodes["cntB"].tolist()) if v})
        # Morton order of (X - min X, Y - min Y), strictly increasing
        mx, my = X.min(), Y.min()
        codes = [orc.morton(int(x - mx), int(y - my)) for x, y in zip(X, Y)]
        assert codes == [int(c) for c in nodes["code"]] and all(a < b for a, b in zip(codes, codes[1:]))
        if G == 1 and P == 0:
            union = Counter(zip(Ah[0].tolist(), Ah[1].tolist())) | Counter(zip(Bh[0].tolist(), Bh[1].tolist()))
            assert set(zip(X.tolist(), Y.tolist())) == set(union)


# --------------------------------------------------------------------------
# hierarchical tree (radix tree over Morton codes)
# --------------------------------------------------------------------------

def _nodes_from_points(orc, X, Y):
    XY = np.unique(np.stack([X, Y], 1), axis=0)
    X, Y = XY[:, 0].astype(np.int32), XY[:, 1].astype(np.int32)
    c = np.ones(len(X), np.int64)
    z = (np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int64))
    return orc.condense_delta((X, Y, c), z, 1, 0, 0)


@pytest.mark.parametrize("clustered", [False, True])
def test_radix_tree_structure(orc, clustered):
    rng = np.random.default_rng(7 + clustered)
    if clustered:
        ctr = rng.integers(0, 10**6, (8, 2))
        pts = np.concatenate([c + rng.integers(0, 50, (60, 2)) for c in ctr])
    else:
        pts = rng.integers(0, 5000, (500, 2))
    nodes = _nodes_from_points(orc, pts[:, 0], pts[:, 1])
    N = len(nodes["X"])
    t = orc.radix_tree(nodes)
    code = [int(c) for c in nodes["code"]]
    X, Y = nodes["X"], nodes["Y"]
    leaf_seen = Counter()
    internal_seen = Counter()
    for w in range(N - 1):
        lo, hi = int(t["lo"][w]), int(t["hi"][w])
        assert w in (lo, hi)
        d = (code[lo] ^ code[hi]).bit_length() - 1
        ranges = []
        for ch in (int(t["left"][w]), int(t["right"][w])):
            if ch < 0:
                leaf_seen[~ch] += 1
                ranges.append((~ch, ~ch))
            else:
                internal_seen[ch] += 1
                ranges.append((int(t["lo"][ch]), int(t["hi"][ch])))
        (a0, a1), (b0, b1) = ranges
        assert a0 == lo and a1 + 1 == b0 and b1 == hi
        assert all(not (code[i] >> d) & 1 for i in range(a0, a1 + 1))
        assert all((code[i] >> d) & 1 for i in range(b0, b1 + 1))
        sl = slice(lo, hi + 1)
        assert list(t["bb"][w]) == [X[sl].min(), X[sl].max(), Y[sl].min(), Y[sl].max()]
        r = min(range(lo, hi + 1), key=lambda i: (int(X[i]), int(Y[i])))
        assert int(t["rep"][w]) == r
    assert sorted(leaf_seen) == list(range(N)) and max(leaf_seen.values()) == 1
    assert sorted(internal_seen) == list(range(1, N - 1)) and max(internal_seen.values()) == 1


def _tree_ranges(t, N):
    """Leaf-position range [lo, hi] of every internal node (root 0 covers all;
    the left child of a node ends at its split, which is the left child's
    number, or its position when it is a leaf)."""
    lo = np.zeros(max(N - 1, 1), np.int64)
    hi = np.zeros(max(N - 1, 1), np.int64)
    stack = [(0, 0, N - 1)]
    while stack:
        w, a, b = stack.pop()
        lo[w], hi[w] = a, b
        L, R = int(t["left"][w]), int(t["right"][w])
        sp = L if L >= 0 else ~L
        if L >= 0:
            stack.append((L, a, sp))
        if R >= 0:
            stack.append((R, sp + 1, b))
    return lo, hi


@pytest.mark.parametrize("clustered", [False, True])
def test_split_tree_structure(orc, clustered):
    """The paper's split tree: every internal node's members are cut at the
    middle of the longest side of their tight bounding box (x on ties), the
    lower half going left; leaves are a permutation; internal numbers are a
    bijection onto 0..N-2; boxes are tight and reps are the leftmost members."""
    rng = np.random.default_rng(70 + clustered)
    if clustered:
        ctr = rng.integers(0, 10**6, (8, 2))
        pts = np.concatenate([c + rng.integers(0, 50, (60, 2)) for c in ctr])
    else:
        pts = rng.integers(0, 5000, (500, 2))
    nodes = _nodes_from_points(orc, pts[:, 0], pts[:, 1])
    N = len(nodes["X"])
    perm, t = orc.split_tree(nodes)
    assert sorted(perm.tolist()) == list(range(N))
    X, Y = nodes["X"][perm].astype(np.int64), nodes["Y"][perm].astype(np.int64)
    lo, hi = _tree_ranges(t, N)
    seen = Counter()
    for w in range(N - 1):
        a, b = int(lo[w]), int(hi[w])
        L, R = int(t["left"][w]), int(t["right"][w])
        sp = L if L >= 0 else ~L
        assert a <= sp < b
        for ch in (L, R):
            if ch >= 0:
                seen[ch] += 1
        mnx, mxx, mny, mxy = X[a:b + 1].min(), X[a:b + 1].max(), Y[a:b + 1].min(), Y[a:b + 1].max()
        assert list(t["bb"][w]) == [mnx, mxx, mny, mxy]
        by_x = mxx - mnx >= mxy - mny
        C = X if by_x else Y
        mid2 = (mnx + mxx) if by_x else (mny + mxy)
        assert all(2 * C[i] < mid2 for i in range(a, sp + 1))
        assert all(2 * C[i] >= mid2 for i in range(sp + 1, b + 1))
        r = min(range(a, b + 1), key=lambda i: (int(X[i]), int(Y[i])))
        assert int(t["rep"][w]) == r
    assert sorted(seen) == list(range(1, N - 1)) and max(seen.values()) == 1


@pytest.mark.parametrize("s,clustered", [(2, False), (5, True), (13, False), (40, True)])
def test_split_tree_wspd_is_a_well_separated_pair_decomposition(orc, s, clustered):
    rng = np.random.default_rng(91 + s)
    if clustered:
        ctr = rng.integers(0, 20000, (6, 2))
        pts = np.concatenate([c + rng.integers(0, 300, (40, 2)) for c in ctr])
    else:
        pts = rng.integers(0, 3000, (220, 2))
    nodes = _nodes_from_points(orc, pts[:, 0], pts[:, 1])
    perm, t = orc.split_tree(nodes)
    nodes = orc.reorder(nodes, perm)
    X, Y = nodes["X"], nodes["Y"]
    N = len(X)
    lo, hi = _tree_ranges(t, N)
    t = dict(t, lo=lo, hi=hi)
    pu, pv = orc.wspd_pairs(nodes, t, s)
    cover = Counter()
    for u, v in zip(pu.tolist(), pv.tolist()):
        U, V = _members(t, u), _members(t, v)
        assert _ws_exact(X, Y, U, V, s)
        for p in U:
            for q in V:
                cover[(min(p, q), max(p, q))] += 1
    assert len(cover) == N * (N - 1) // 2 and set(cover.values()) == {1}


@pytest.mark.parametrize("s", [8, 13, 20])
def test_split_tree_spanner_stretch(orc, s):
    rng = np.random.default_rng(120 + s)
    pts = rng.integers(0, 10**5, (600, 2))
    nodes = _nodes_from_points(orc, pts[:, 0], pts[:, 1])
    perm, t = orc.split_tree(nodes)
    nodes = orc.reorder(nodes, perm)
    X, Y = nodes["X"].astype(float), nodes["Y"].astype(float)
    N = len(X)
    tails, heads = orc.wspd(nodes, t, s)
    w = np.hypot(X[tails] - X[heads], Y[tails] - Y[heads])
    D = shortest_path(csr_matrix((w, (tails, heads)), shape=(N, N)), method="D")
    E = np.hypot(X[:, None] - X[None, :], Y[:, None] - Y[None, :])
    iu = np.triu_indices(N, 1)
    assert (D[iu] / E[iu]).max() <= 1 + 4 / s + 4 / (s - 2) + 1e-9


# --------------------------------------------------------------------------
# s-WSPD: definition checked by brute force
# --------------------------------------------------------------------------

def _members(t, ref):
    if ref < 0:
        return range(~ref, ~ref + 1)
    return range(int(t["lo"][ref]), int(t["hi"][ref]) + 1)


def _ws_exact(X, Y, U, V, s):
    """Balls of a common radius d around the two boxes' circumscribed circles
    at distance >= s d, in exact rational arithmetic."""
    def circ(S):
        xs = [int(X[i]) for i in S]
        ys = [int(Y[i]) for i in S]
        cx, cy = Fraction(min(xs) + max(xs), 2), Fraction(min(ys) + max(ys), 2)
        r2 = Fraction((max(xs) - min(xs)) ** 2 + (max(ys) - min(ys)) ** 2, 4)
        return cx, cy, r2
    ax, ay, ar2 = circ(U)
    bx, by, br2 = circ(V)
    r2 = max(ar2, br2)
    dist2 = (ax - bx) ** 2 + (ay - by) ** 2
    # |c_u - c_v| - 2 d >= s d  <=>  |c_u - c_v| >= (s + 2) d
    return dist2 >= (s + 2) ** 2 * r2


@pytest.mark.parametrize("s,clustered", [(2, False), (5, True), (13, False), (40, True)])
def test_wspd_is_a_well_separated_pair_decomposition(orc, s, clustered):
    rng = np.random.default_rng(11 + s)
    if clustered:
        ctr = rng.integers(0, 20000, (6, 2))
        pts = np.concatenate([c + rng.integers(0, 300, (40, 2)) for c in ctr])
    else:
        pts = rng.integers(0, 3000, (220, 2))
    nodes = _nodes_from_points(orc, pts[:, 0], pts[:, 1])
    X, Y = nodes["X"], nodes["Y"]
    N = len(X)
    t = orc.radix_tree(nodes)
    pu, pv = orc.wspd_pairs(nodes, t, s)
    cover = Counter()
    for u, v in zip(pu.tolist(), pv.tolist()):
        U, V = _members(t, u), _members(t, v)
        assert _ws_exact(X, Y, U, V, s)
        for p in U:
            for q in V:
                cover[(min(p, q), max(p, q))] += 1
    # every unordered pair of distinct points is covered by exactly one pair
    assert len(cover) == N * (N - 1) // 2 and set(cover.values()) == {1}
    tails, heads = orc.wspd(nodes, t, s)
    rep = lambda r: ~r if r < 0 else int(t["rep"][r])
    expect = Counter()
    for u, v in zip(pu.tolist(), pv.tolist()):
        assert rep(u) in _members(t, u) and rep(v) in _members(t, v)
        expect[(rep(u), rep(v))] += 1
        expect[(rep(v), rep(u))] += 1
    got = Counter(zip(tails.tolist(), heads.tolist()))
    assert got == expect and set(got.values()) == {1}  # biarcs, no duplicates


@pytest.mark.parametrize("s", [8, 13, 20])
def test_wspd_spanner_stretch(orc, s):
    rng = np.random.default_rng(20 + s)
    pts = rng.integers(0, 10**5, (600, 2))
    nodes = _nodes_from_points(orc, pts[:, 0], pts[:, 1])
    X, Y = nodes["X"].astype(float), nodes["Y"].astype(float)
    N = len(X)
    t = orc.radix_tree(nodes)
    tails, heads = orc.wspd(nodes, t, s)
    w = np.hypot(X[tails] - X[heads], Y[tails] - Y[heads])
    D = shortest_path(csr_matrix((w, (tails, heads)), shape=(N, N)), method="D")
    E = np.hypot(X[:, None] - X[None, :], Y[:, None] - Y[None, :])
    iu = np.triu_indices(N, 1)
    stretch = (D[iu] / E[iu]).max()
    assert stretch <= 1 + 4 / s + 4 / (s - 2) + 1e-9


# --------------------------------------------------------------------------
# min-cost flow: network simplex vs an LP solver and vs the Hungarian method
# --------------------------------------------------------------------------

def test_network_simplex_matches_linprog(orc):
    rng = np.random.default_rng(30)
    for trial in range(12):
        n = int(rng.integers(5, 40))
        arcs = set()
        for u in range(n - 1):  # a path both ways keeps it feasible
            arcs.add((u, u + 1))
            arcs.add((u + 1, u))
        for _ in range(3 * n):
            u, v = (int(x) for x in rng.integers(0, n, 2))
            if u != v:
                arcs.add((u, v))
        arcs = sorted(arcs)
        t = np.array([a[0] for a in arcs], np.int32)
        h = np.array([a[1] for a in arcs], np.int32)
        c = rng.integers(0, 50, len(arcs)).astype(np.int64)
        sup = rng.integers(-5, 6, n).astype(np.int64)
        sup[-1] -= sup.sum()
        st, opt, flow, pot = orc.mcf_arcs(n, t, h, c, sup)
        assert st == 0
        A = np.zeros((n, len(arcs)))
        A[t, np.arange(len(arcs))] += 1
        A[h, np.arange(len(arcs))] -= 1
        lp = linprog(c.astype(float), A_eq=A, b_eq=sup.astype(float), bounds=(0, None), method="highs")
        assert lp.status == 0 and round(lp.fun) == opt
        assert np.array_equal(A @ flow, sup) and (flow >= 0).all() and int(c @ flow) == opt
        # dual feasibility: no arc with negative reduced cost
        assert (c - pot[t] + pot[h] >= 0).all()


def _augmented(A, B, cost, diag):
    """Perfect matching on Bi(A,B): A + B-projections vs B + A-projections."""
    na, nb = len(A), len(B)
    INF = 1e18
    M = np.full((na + nb, nb + na), INF)
    for i, a in enumerate(A):
        for j, b in enumerate(B):
            M[i, j] = cost(a, b)
        M[i, nb + i] = diag(a)
    for j, b in enumerate(B):
        M[na + j, j] = diag(b)
        M[na + j, nb:] = 0.0
    r, c = linear_sum_assignment(M)
    return M[r, c].sum()


def test_exact_w1_matches_hungarian(orc):
    rng = np.random.default_rng(31)
    for trial in range(8):
        A = synth.uniform_exp(int(rng.integers(1, 60)), 500 + trial).astype(np.float64)
        B = synth.uniform_exp(int(rng.integers(1, 60)), 600 + trial).astype(np.float64)
        A = A[A[:, 0] != A[:, 1]]
        B = B[B[:, 0] != B[:, 1]]
        ref = _augmented(A, B, lambda a, b: math.hypot(a[0] - b[0], a[1] - b[1]),
                         lambda a: abs(a[1] - a[0]) / SQ2)
        assert abs(orc.w1_exact(A, B) - ref) <= 1e-9 * max(1.0, ref)


def test_integer_dense_optimum_matches_hungarian(orc):
    rng = np.random.default_rng(32)
    icost = lambda a, b: float(orc.cost(int(a[0]), int(a[1]), int(b[0]), int(b[1])))
    idiag = lambda a: float(orc.cdiag(int(a[0]), int(a[1])))
    for trial in range(6):
        A = rng.integers(0, 400, (int(rng.integers(1, 40)), 2))
        B = rng.integers(0, 400, (int(rng.integers(1, 40)), 2))
        A = A[A[:, 0] != A[:, 1]]
        B = B[B[:, 0] != B[:, 1]]
        P = orc.condense0(A[:, 0].astype(np.int32), A[:, 1].astype(np.int32))
        Q = orc.condense0(B[:, 0].astype(np.int32), B[:, 1].astype(np.int32))
        assert orc.dense_opt_int(P, Q) == round(_augmented(A, B, icost, idiag))


def test_hungarian_reference_against_permutations(orc):
    # the augmented-matrix reference itself, against all bijections (n <= 6)
    rng = np.random.default_rng(33)
    A = rng.random((3, 2)) * [1, 0] + rng.random((3, 2)) * [0, 1]
    B = rng.random((3, 2))
    pts = [tuple(p) for p in A] + [tuple(p) for p in B]
    na = nb = 3
    best = math.inf
    # bijection between A + B-projections and B + A-projections
    for perm in itertools.permutations(range(na + nb)):
        tot = 0.0
        for i, j in enumerate(perm):
            if i < na and j < nb:
                tot += math.dist(A[i], B[j])
            elif i < na:
                tot += abs(A[i][1] - A[i][0]) / SQ2 if j - nb == i else math.inf
            elif j < nb:
                tot += abs(B[j][1] - B[j][0]) / SQ2 if i - na == j else math.inf
        best = min(best, tot)
    ref = _augmented(A, B, lambda a, b: math.dist(a, b), lambda a: abs(a[1] - a[0]) / SQ2)
    assert abs(ref - best) < 1e-12
    assert abs(orc.w1_exact(A, B) - best) < 1e-9


def test_hand_derived_examples(orc):
    cases = json.load(open(os.path.join(GOLDEN, "hand_examples.json")))["cases"]
    for cs in cases:
        A = np.array(cs["A"], np.float64)
        B = np.array(cs["B"], np.float64)
        assert abs(orc.w1_exact(A, B) - cs["w1"]) < 1e-12, cs["name"]
        r = orc.w1_approx(A.astype(np.uint8), B.astype(np.uint8), "u8", k=0, s_override=10**6,
                          condense=False)
        assert r["opt"] == cs["opt_int"], cs["name"]


def test_w1_closed_forms(orc):
    A = synth.uniform_exp(300, 41).astype(np.float64)
    A = A[A[:, 0] != A[:, 1]]
    B = synth.uniform_exp(250, 42).astype(np.float64)
    B = B[B[:, 0] != B[:, 1]]
    # empty diagram: sum of distances to the diagonal
    assert abs(orc.w1_exact(A, np.zeros((0, 2))) - np.abs(A[:, 1] - A[:, 0]).sum() / SQ2) < 1e-9
    assert orc.w1_exact(A, A) == 0.0
    w = orc.w1_exact(A, B)
    assert abs(orc.w1_exact(B, A) - w) < 1e-9
    # translation along (t, t) and scaling by 2
    assert abs(orc.w1_exact(A + 3.0, B + 3.0) - w) < 1e-9
    assert abs(orc.w1_exact(2 * A, 2 * B) - 2 * w) < 1e-9
    # single points: min(|a - b|, d(a) + d(b))
    for a, b in [((0.0, 1.0), (0.1, 1.2)), ((0.0, 0.2), (5.0, 5.3))]:
        ref = min(math.dist(a, b), (a[1] - a[0]) / SQ2 + (b[1] - b[0]) / SQ2)
        assert abs(orc.w1_exact(np.array([a]), np.array([b])) - ref) < 1e-12


def test_far_from_diagonal_reduces_to_emd(orc):
    # Conditional lower bound section: far from the diagonal, W1 is the EMD
    rng = np.random.default_rng(43)
    A = rng.random((40, 2)) + [0.0, 1000.0]
    B = rng.random((40, 2)) + [0.0, 1000.0]
    D = np.hypot(A[:, None, 0] - B[None, :, 0], A[:, None, 1] - B[None, :, 1])
    r, c = linear_sum_assignment(D)
    assert abs(orc.w1_exact(A, B) - D[r, c].sum()) < 1e-9


# --------------------------------------------------------------------------
# the whole pipeline: the paper's chain of bounds, exactly in integers
# --------------------------------------------------------------------------

def _small_pair(n, seed):
    return synth.uniform_exp(n, seed), synth.uniform_exp(n, seed + 1)


@pytest.mark.parametrize("eps,seed,tree", [(0.1, 100, "radix"), (0.5, 102, "radix"), (1.0, 104, "radix"),
                                           (0.1, 106, "split"), (0.5, 108, "split")])
def test_pipeline_bound_chain(orc, eps, seed, tree):
    A, B = _small_pair(400, seed)
    r = orc.w1_approx(A, B, "f32", eps=eps, k=16, tree=tree)
    # RWMD_0 <= OPT(G_0)
    opt0 = orc.dense_opt_int(r["Ahat"], r["Bhat"])
    assert r["rwmd"] <= opt0
    # RWMD_delta <= OPT(G_delta) <= OPT(WS)  (Theorem, spanner approximation, left side)
    nd = r["nodes"]
    ia, ib = nd["cntA"] > 0, nd["cntB"] > 0
    Pd = (nd["X"][ia], nd["Y"][ia], nd["cntA"][ia])
    Qd = (nd["X"][ib], nd["Y"][ib], nd["cntB"][ib])
    optd = orc.dense_opt_int(Pd, Qd)
    assert orc.rwmd(Pd, Qd)[2] <= optd <= r["opt"]
    # OPT(WS) <= (1 + 4/s + 4/(s-2)) OPT(G_delta) + rounding slack (right side)
    assert r["opt"] <= (1 + 4 / r["s"] + 4 / (r["s"] - 2)) * optd + r["slack"]
    # (1 - eps) W1 <= W1_approx <= (1 + eps) W1 + slack   vs exact FP64 W1
    w = orc.w1_exact(A.astype(np.float64), B.astype(np.float64))
    q = 2.0 ** -r["k"]
    qerr = (r["FA"] + r["FB"]) * q  # input quantisation moves each point by < q/sqrt(2)
    assert (1 - eps) * w - qerr <= r["w1"] <= (1 + eps) * w + r["slack"] * q + qerr


def test_pipeline_identity_symmetry_and_dense_limit(orc):
    A, B = _small_pair(300, 200)
    assert orc.w1_approx(A, A, "f32", eps=0.1)["opt"] == 0
    rab = orc.w1_approx(A, B, "f32", eps=0.1, seed=5)
    rba = orc.w1_approx(B, A, "f32", eps=0.1, seed=5)
    assert rab["opt"] == rba["opt"]
    # s -> infinity without condensation: the WSPD is the complete graph and
    # OPT(WS) equals the dense integer optimum on G_0
    r = orc.w1_approx(A, B, "f32", s_override=10**7, condense=False)
    assert len(r["ws_tails"]) == len(r["nodes"]["X"]) * (len(r["nodes"]["X"]) - 1)
    assert r["opt"] == orc.dense_opt_int(r["Ahat"], r["Bhat"])


def test_pipeline_empty_and_one_sided(orc):
    A, _ = _small_pair(200, 300)
    E = np.zeros((0, 2), np.float32)
    r = orc.w1_approx(A, E, "f32", eps=0.1)
    Ah = r["Ahat"]
    closed = sum(int(c) * orc.cdiag(int(x), int(y)) for x, y, c in zip(*Ah))
    assert r["rwmd"] == closed  # RWMD(B = empty) == W1 exactly
    # with no B mass every A unit goes straight to the diagonal
    r0 = orc.w1_approx(A, E, "f32", eps=0.1, condense=False)
    assert r0["opt"] == closed
    assert orc.w1_approx(E, E, "f32", eps=0.1)["opt"] == 0


@pytest.mark.parametrize("seed,eps", [(400, 0.1), (402, 0.5), (404, 2.0)])
def test_contracting_the_zero_cost_diagonal_arc_keeps_the_optimum(orc, seed, eps):
    """The GPU solver merges ā and b̄ (the zero-cost arc b̄ -> ā contracted);
    the optimum of the paper's network must be unchanged."""
    A, B = synth.uniform_exp(300, seed), synth.uniform_exp(260, seed + 1)
    r = orc.w1_approx(A, B, "f32", eps=eps)
    net = r["net"]
    N = net["n_nodes"]
    rp, head, cost, sup = net["row_ptr"], net["head"], net["cost"], net["supply"]
    tails = np.repeat(np.arange(N + 2), np.diff(rp)).astype(np.int32)
    keep = ~((tails == N + 1) & (head == N))        # drop b̄ -> ā
    t = np.where(tails[keep] == N + 1, N, tails[keep]).astype(np.int32)  # b̄ becomes the merged node
    msup = np.concatenate([sup[:N], [sup[N] + sup[N + 1]]])
    st, opt, flow, pot = orc.mcf_arcs(N + 1, t, head[keep], cost[keep], msup)
    assert st == 0 and opt == r["opt"]


def test_nn_search_ties_and_dense_limit(orc):
    """Nearest neighbour (the NN-search application): the argmin of OPT_int,
    ties to the lowest index.  In the dense limit (no condensation, s huge)
    OPT_int is the dense integer optimum on the 0-condensed diagrams, so the
    answer must match brute force over dense_opt_int."""
    db = [_small_pair(n, 700 + i)[0] for i, n in enumerate([40, 25, 60, 33, 50, 18])]
    db.append(db[2].copy())  # a duplicate of diagram 2 at a higher index
    q = db[2].copy()
    idx, opts = orc.nn_search(q, db, "f32", eps=0.1)
    assert idx == 2 and opts[2] == 0 and opts[6] == 0
    q2 = _small_pair(45, 777)[0]
    idx2, opts2 = orc.nn_search(q2, db, "f32", s_override=10**7, condense=False)
    dense = []
    for d in db:
        XA, YA = orc.quantize(q2, "f32", 20)
        XB, YB = orc.quantize(d, "f32", 20)
        dense.append(orc.dense_opt_int(orc.condense0(XA, YA), orc.condense0(XB, YB)))
    assert opts2 == dense
    assert idx2 == min(range(len(dense)), key=lambda i: (dense[i], i))
    assert orc.nn_search(q2, [], "f32") == (-1, [])


def test_warm_start_network_oracle_gradient_and_bf16():
    """The warm-start network's oracle: its gradient equals central finite
    differences of its loss (float64, no rounding), and its bf16 rounding
    equals torch's float32 -> bfloat16 conversion."""
    torch = pytest.importorskip("torch")
    from oracle import mlp
    rng = np.random.default_rng(5)
    p = (rng.standard_normal(mlp.NPARAMS) * 0.15).astype(np.float32)
    x = rng.standard_normal((24, mlp.NIN)).astype(np.float32)
    t = rng.standard_normal(24).astype(np.float32)
    m = (rng.random(24) < 0.8).astype(np.float32)
    loss, g = mlp.loss_grad(p, x, t, m, round_inputs=False)
    idx = np.concatenate([rng.choice(mlp.NPARAMS, 150, replace=False),
                          np.arange(mlp.OFF_B1, mlp.OFF_B1 + 5), np.arange(mlp.OFF_W3, mlp.OFF_W3 + 5),
                          [mlp.OFF_B3]])
    pd64 = p.astype(np.float64)

    def L(q):
        W1 = q[mlp.OFF_W1:mlp.OFF_B1].reshape(mlp.NIN, mlp.NH)
        h1 = np.maximum(x.astype(np.float64) @ W1 + q[mlp.OFF_B1:mlp.OFF_W2], 0)
        h2 = np.maximum(h1 @ q[mlp.OFF_W2:mlp.OFF_B2].reshape(mlp.NH, mlp.NH) + q[mlp.OFF_B2:mlp.OFF_W3], 0)
        y = h2 @ q[mlp.OFF_W3:mlp.OFF_B3] + q[mlp.OFF_B3]
        return np.sum(m * (y - t) ** 2) / len(y)

    assert abs(L(pd64) - loss) < 1e-12 * max(1, abs(loss))
    h = 1e-6
    for i in idx:
        e = np.zeros_like(pd64)
        e[i] = h
        fd = (L(pd64 + e) - L(pd64 - e)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd), (i, fd, g[i])
    v = rng.standard_normal(1000).astype(np.float32) * 100
    ref = torch.from_numpy(v).to(torch.bfloat16).float().numpy().astype(np.float64)
    np.testing.assert_array_equal(mlp.bf16(v), ref)


@pytest.mark.parametrize("seed,eps,kind", [(800, 0.1, "f32"), (802, 0.05, "f32"), (804, 0.5, "f32"),
                                           (806, 0.05, "u8"), (808, 2.0, "f32")])
def test_nearest_neighbour_bound_is_below_the_optimum(orc, seed, eps, kind):
    """The search's pruning bound (1 - eps_c) * RWMD of the 0-condensed
    diagrams, RWMD with real (unrounded) distances and the diagonal option,
    never exceeds OPT_int of the pair: delta-condensation moves the points by
    at most eps_c * L_lo in total and OPT_int is at least the real W1 of the
    condensed diagrams."""
    if kind == "f32":
        A, B = synth.uniform_exp(400, seed), synth.uniform_exp(330, seed + 1)
    else:
        A, B = synth.lowerstar_u8(1500, seed), synth.lowerstar_u8(1200, seed + 1)
    r = orc.w1_approx(A, B, kind, eps=eps)

    def side(P, Q):
        px, py, pc = (np.asarray(v, np.float64) for v in P)
        qx, qy = (np.asarray(v, np.float64) for v in Q[:2])
        diag = np.abs(py - px) / math.sqrt(2.0)
        if len(qx):
            d = np.sqrt((px[:, None] - qx[None, :]) ** 2 + (py[:, None] - qy[None, :]) ** 2).min(1)
            diag = np.minimum(diag, d)
        return float((pc * diag).sum())

    rwmd = max(side(r["Ahat"], r["Bhat"]), side(r["Bhat"], r["Ahat"]))
    s = r["s"]
    ec = 8.0 / (s - 4) if s >= 12 else 1.0
    assert r["opt"] >= (1.0 - ec) * rwmd - 1e-6 * max(1.0, rwmd)
    # and the movement of the condensation is within eps_c * L_lo
    G, P = r["G"], r["P"]
    moved = (r["FA"] + r["FB"]) * math.sqrt(2.0) * (G / 2 + P) if G > 1 else 0.0
    Llo = max(r["LA"] - r["FA"], r["LB"] - r["FB"], 0)
    assert moved <= ec * Llo * (1 + 1e-9) + 1e-9


def test_wcd_bound_definition_closed_form_and_below_w1(orc):
    """WCD of A + B~ against B + A~ (Appendix, WCD): equals the closed form
    |sum_A (d - b) - sum_B (d - b)| / sqrt(2) (every point minus its own
    projection is ((b - d)/2, (d - b)/2)), and half of it never exceeds the
    exact W1 (Hungarian reference) -- including one-sided and empty pairs."""
    rng = np.random.default_rng(900)
    for trial in range(12):
        nA, nB = int(rng.integers(0, 25)), int(rng.integers(0, 25))
        A = rng.random((nA, 2)) * 3.0
        B = rng.random((nB, 2)) * 3.0
        A[:, 1] = A[:, 0] + np.abs(A[:, 1] - A[:, 0])
        B[:, 1] = B[:, 0] + np.abs(B[:, 1] - B[:, 0])
        w = orc.wcd(A, B)
        closed = abs((A[:, 1] - A[:, 0]).sum() - (B[:, 1] - B[:, 0]).sum()) / math.sqrt(2.0)
        assert abs(w - closed) <= 1e-9 * max(1.0, closed)
        if nA + nB:
            w1 = _augmented(A, B, lambda a, b: math.hypot(a[0] - b[0], a[1] - b[1]),
                            lambda a: abs(a[1] - a[0]) / SQ2)
            assert w / 2 <= w1 + 1e-9
    assert orc.wcd(np.zeros((0, 2)), np.zeros((0, 2))) == 0.0
    # condensed nodes (X, Y, count) give the same value as the expanded points
    X, Y, c = np.array([1, 4]), np.array([5, 9]), np.array([3, 2])
    pts = np.array([[1, 5]] * 3 + [[4, 9]] * 2, float)
    assert orc.wcd((X, Y, c), (X[:1], Y[:1] + 1, c[:1])) == pytest.approx(orc.wcd(pts, np.array([[1, 6]] * 3, float)))


# --------------------------------------------------------------------------
# unbalanced transport (Conclusion): diagonal arcs reassigned to creation /
# destruction costs kappa * d_diag + tau
# --------------------------------------------------------------------------

@pytest.mark.parametrize("kappa,tau", [(0, 0.3), (1, 0.25), (0, 5.0)])
def test_unbalanced_exact_matches_the_augmented_assignment(orc, kappa, tau):
    """Exact FP64 optimum with creation / destruction cost kappa * d_diag + tau
    equals the optimal assignment of the augmented bipartite graph (A + B's
    creation slots against B + A's destruction slots), by scipy's Hungarian."""
    rng = np.random.default_rng(700 + int(10 * tau))
    for trial in range(5):
        A = synth.uniform_exp(int(rng.integers(1, 40)), 900 + trial).astype(np.float64)
        B = synth.uniform_exp(int(rng.integers(1, 40)), 950 + trial).astype(np.float64)
        A, B = A[A[:, 0] != A[:, 1]], B[B[:, 0] != B[:, 1]]
        dc = lambda a: kappa * abs(a[1] - a[0]) / SQ2 + tau
        ref = _augmented(A, B, lambda a, b: math.hypot(a[0] - b[0], a[1] - b[1]), dc)
        got = orc.w1_exact(A, B, kappa=kappa, tau=tau)
        assert abs(got - ref) <= 1e-9 * max(1.0, ref)


def test_unbalanced_closed_forms_and_balanced_limit(orc):
    """One side empty: every unit is destroyed (created), the sum of the
    costs.  kappa 0 with twice tau above every distance between equal-size
    sets: nothing is destroyed, the optimum is the balanced assignment (EMD)."""
    A = synth.uniform_exp(60, 31).astype(np.float64)
    A = A[A[:, 0] != A[:, 1]]
    E = np.zeros((0, 2))
    for kappa, tau in ((0, 0.5), (1, 0.125)):
        closed = sum(kappa * abs(d - b) / SQ2 + tau for b, d in A)
        assert abs(orc.w1_exact(A, E, kappa=kappa, tau=tau) - closed) <= 1e-9 * closed
        assert abs(orc.w1_exact(E, A, kappa=kappa, tau=tau) - closed) <= 1e-9 * closed
    B = synth.uniform_exp(len(A), 32).astype(np.float64)
    B = B[B[:, 0] != B[:, 1]][: len(A)]
    A = A[: len(B)]
    D = np.hypot(A[:, None, 0] - B[None, :, 0], A[:, None, 1] - B[None, :, 1])
    r, c = linear_sum_assignment(D)
    assert abs(orc.w1_exact(A, B, kappa=0, tau=float(D.max())) - D[r, c].sum()) <= 1e-9 * D[r, c].sum()
    # integer form: single points, min(l2, cost(a) + cost(b))
    for (x1, y1, x2, y2) in ((0, 10, 3, 14), (0, 1000, 900, 1000), (5, 5000, 7, 5001)):
        for kappa, tau in ((0, 40), (1, 3), (0, 0)):
            P = (np.array([x1], np.int32), np.array([y1], np.int32), np.array([1], np.int64))
            Q = (np.array([x2], np.int32), np.array([y2], np.int32), np.array([1], np.int64))
            exp = min(orc.cost(x1, y1, x2, y2), orc.cmake(x1, y1, kappa, tau) + orc.cmake(x2, y2, kappa, tau))
            assert orc.dense_opt_int(P, Q, kappa=kappa, tau=tau) == exp
            assert orc.cmake(x1, y1, kappa, tau) == kappa * orc.cdiag(x1, y1) + tau


@pytest.mark.parametrize("kappa,tau", [(0, 20000), (1, 4000)])
def test_unbalanced_pipeline_bounds(orc, kappa, tau):
    """The pipeline with creation / destruction costs: RWMD <= OPT(G_0) on
    the 0-condensed nodes, the dense limit (s large, no condensation) equals
    the dense integer optimum, and the (1 +- eps) band holds against the exact
    FP64 optimum of the same costs."""
    A, B = _small_pair(300, 410)
    q = 2.0 ** -16
    r = orc.w1_approx(A, B, "f32", eps=0.1, k=16, kappa=kappa, tau=tau)
    opt0 = orc.dense_opt_int(r["Ahat"], r["Bhat"], kappa=kappa, tau=tau)
    assert r["rwmd"] <= opt0
    rd = orc.w1_approx(A, B, "f32", k=16, s_override=10**7, condense=False, kappa=kappa, tau=tau)
    assert rd["opt"] == opt0
    w = orc.w1_exact(A.astype(np.float64), B.astype(np.float64), kappa=kappa, tau=tau * q)
    qerr = (r["FA"] + r["FB"]) * q
    assert (1 - 0.1) * w - qerr <= r["w1"] <= (1 + 0.1) * w + r["slack"] * q + qerr
    # RWMD against brute force over the 0-condensed nodes, destruction option included
    Ah, Bh = r["Ahat"], r["Bhat"]
    def side(P, Q):
        tot = 0
        for x, y, c in zip(*P):
            best = orc.cmake(int(x), int(y), kappa, tau)
            for x2, y2 in zip(Q[0], Q[1]):
                best = min(best, orc.cost(int(x), int(y), int(x2), int(y2)))
            tot += int(c) * best
        return tot
    assert (r["LA"], r["LB"]) == (side(Ah, Bh), side(Bh, Ah))
