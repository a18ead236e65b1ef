"""CPU oracle for the approximate W1 between persistence diagrams (Dey & Zhang).

TEST INFRASTRUCTURE ONLY: the plain, slow, obviously correct restatement of
the method that the CUDA library is checked against.  Only tests/, the smoke
entry point and the benchmark's CPU-baseline leg may import this package; the
product path never does.  It shares no code with the CUDA library.

The arithmetic lives in oracle.c (built by oracle/build.py); this module
marshals numpy arrays and chains the steps in the order of Algorithm 4:
delta-condensation (Algorithm 2, which runs the RWMD of Algorithm 1), the
hierarchical tree, the s-WSPD biarcs (Algorithms 6-8), the diagonal arcs
(Algorithm 9), the CSR network and the min-cost flow (network simplex).

Parity pins for every function are in tests/test_oracle_*.py.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

from . import build as _build

_lib = None

I32P = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
I64P = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
U64P = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
F64P = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.orc_isqrt.restype = C.c_uint64
        L.orc_isqrt.argtypes = [C.c_uint64]
        L.orc_ceil_sqrt.restype = C.c_uint64
        L.orc_ceil_sqrt.argtypes = [C.c_uint64]
        L.orc_cost.restype = C.c_int64
        L.orc_cost.argtypes = [C.c_int64] * 4
        L.orc_cdiag.restype = C.c_int64
        L.orc_cdiag.argtypes = [C.c_int64] * 2
        L.orc_quantize.restype = C.c_int64
        L.orc_quantize.argtypes = [C.c_void_p, C.c_int64, C.c_int, C.c_int, I32P, I32P]
        L.orc_condense0.restype = C.c_int64
        L.orc_condense0.argtypes = [I32P, I32P, C.c_int64, I32P, I32P, I64P]
        L.orc_rwmd.restype = None
        L.orc_rwmd.argtypes = [I32P, I32P, I64P, C.c_int64, I32P, I32P, I64P, C.c_int64, C.c_int64, C.c_int64, I64P]
        L.orc_bound.restype = C.c_double
        L.orc_bound.argtypes = [C.c_int64]
        L.orc_s_from_eps.restype = C.c_int64
        L.orc_s_from_eps.argtypes = [C.c_double]
        L.orc_eps_c.restype = C.c_double
        L.orc_eps_c.argtypes = [C.c_int64]
        L.orc_delta_params.restype = None
        L.orc_delta_params.argtypes = [C.c_int64] * 5 + [C.POINTER(C.c_double), C.POINTER(C.c_int64),
                                                         C.POINTER(C.c_int64)]
        L.orc_perturb.restype = None
        L.orc_perturb.argtypes = [C.c_uint64, C.c_int64, C.c_int64, C.c_int64,
                                  C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
        L.orc_morton.restype = C.c_uint64
        L.orc_morton.argtypes = [C.c_uint32, C.c_uint32]
        L.orc_condense_delta.restype = C.c_int64
        L.orc_condense_delta.argtypes = [I32P, I32P, I64P, C.c_int64, I32P, I32P, I64P, C.c_int64,
                                         C.c_int64, C.c_int64, C.c_uint64,
                                         I32P, I32P, I64P, I64P, U64P]
        L.orc_radix_tree.restype = None
        L.orc_radix_tree.argtypes = [C.c_int64, U64P, I32P, I32P, I32P, I32P, I32P, I32P, I32P, I32P]
        L.orc_split_tree.restype = None
        L.orc_split_tree.argtypes = [C.c_int64, I32P, I32P, I32P, I32P, I32P, I32P, I32P]
        L.orc_mix64.restype = C.c_uint64
        L.orc_mix64.argtypes = [C.c_uint64]
        L.orc_wspd_pairs.restype = C.c_int64
        L.orc_wspd_pairs.argtypes = [C.c_int64, I32P, I32P, I32P, I32P, I32P, I32P, C.c_int64,
                                     I32P, I32P, C.c_int64]
        L.orc_well_separated.restype = C.c_int
        L.orc_well_separated.argtypes = [C.c_int64] * 9
        L.orc_wspd.restype = C.c_int64
        L.orc_wspd.argtypes = [C.c_int64, I32P, I32P, I32P, I32P, I32P, I32P, C.c_int64,
                               I32P, I32P, C.c_int64]
        L.orc_build_network.restype = C.c_int64
        L.orc_build_network.argtypes = [C.c_int64, I32P, I32P, I64P, I64P, C.c_int64, I32P, I32P,
                                        I64P, I32P, I64P, I64P, C.c_int64, C.c_int64]
        L.orc_mcf_csr.restype = C.c_int
        L.orc_mcf_csr.argtypes = [C.c_int64, I64P, I32P, I64P, I64P, I64P, I64P,
                                  C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.c_int64]
        L.orc_mcf_arcs.restype = C.c_int
        L.orc_mcf_arcs.argtypes = [C.c_int64, C.c_int64, I32P, I32P, I64P, I64P, I64P, I64P,
                                   C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.c_int64]
        L.orc_mcf_arcs_dbl.restype = C.c_int
        L.orc_mcf_arcs_dbl.argtypes = [C.c_int64, C.c_int64, I32P, I32P, F64P, I64P, I64P, F64P,
                                       C.POINTER(C.c_double), C.POINTER(C.c_int64), C.c_int64,
                                       C.c_double]
        L.orc_dense_opt_int.restype = C.c_int
        L.orc_dense_opt_int.argtypes = [I32P, I32P, I64P, C.c_int64, I32P, I32P, I64P, C.c_int64,
                                        C.c_int64, C.c_int64, C.POINTER(C.c_int64), C.c_int64]
        L.orc_w1_exact.restype = C.c_double
        L.orc_w1_exact.argtypes = [F64P, C.c_int64, F64P, C.c_int64, C.c_double, C.c_double, C.c_int64]
        L.orc_cmake.restype = C.c_int64
        L.orc_cmake.argtypes = [C.c_int64] * 4
        _lib = L
    return _lib


# ---------------------------------------------------------------------------
# scalar helpers
# ---------------------------------------------------------------------------

def isqrt(v: int) -> int:
    return int(lib().orc_isqrt(v))


def ceil_sqrt(v: int) -> int:
    return int(lib().orc_ceil_sqrt(v))


def cost(x1, y1, x2, y2) -> int:
    return int(lib().orc_cost(x1, y1, x2, y2))


def cmake(x, y, kappa=1, tau=0) -> int:
    """Creation / destruction cost of a unit at (x, y): kappa * cdiag + tau
    (1, 0: the distance to the diagonal of persistence diagrams; the
    Conclusion's unbalanced transport otherwise)."""
    return int(lib().orc_cmake(x, y, kappa, tau))


def cdiag(x, y) -> int:
    return int(lib().orc_cdiag(x, y))


def bound(s: int) -> float:
    return float(lib().orc_bound(s))


def s_from_eps(eps: float) -> int:
    return int(lib().orc_s_from_eps(eps))


def eps_c(s: int) -> float:
    return float(lib().orc_eps_c(s))


def delta_params(LA, LB, FA, FB, s):
    d = C.c_double()
    G = C.c_int64()
    P = C.c_int64()
    lib().orc_delta_params(LA, LB, FA, FB, s, C.byref(d), C.byref(G), C.byref(P))
    return d.value, G.value, P.value


def perturb(seed, cx, cy, P):
    dx = C.c_int64()
    dy = C.c_int64()
    lib().orc_perturb(seed, cx, cy, P, C.byref(dx), C.byref(dy))
    return dx.value, dy.value


def morton(x: int, y: int) -> int:
    return int(lib().orc_morton(x, y))


def well_separated(a, b, s) -> bool:
    """a, b: (minX, maxX, minY, maxY) boxes."""
    return bool(lib().orc_well_separated(*[int(v) for v in a], *[int(v) for v in b], int(s)))


def default_shift(dtype: str) -> int:
    return 12 if dtype == "u8" else 20


# ---------------------------------------------------------------------------
# pipeline steps
# ---------------------------------------------------------------------------

def quantize(bd: np.ndarray, dtype: str, k: int):
    """bd: (n, 2) float32 or uint8 array of (birth, death).  Returns (X, Y)."""
    if dtype == "f32":
        arr = np.ascontiguousarray(bd, dtype=np.float32)
        dt = 0
    else:
        arr = np.ascontiguousarray(bd, dtype=np.uint8)
        dt = 1
    n = arr.shape[0] if arr.ndim == 2 else 0
    X = np.zeros(max(n, 1), np.int32)
    Y = np.zeros(max(n, 1), np.int32)
    kept = lib().orc_quantize(arr.ctypes.data if n else None, n, dt, k, X, Y)
    if kept < 0:
        raise ValueError("diagram has a non-finite or out-of-range coordinate")
    return X[:kept].copy(), Y[:kept].copy()


def condense0(X, Y):
    n = len(X)
    UX = np.zeros(max(n, 1), np.int32)
    UY = np.zeros(max(n, 1), np.int32)
    cnt = np.zeros(max(n, 1), np.int64)
    m = lib().orc_condense0(np.ascontiguousarray(X, np.int32) if n else UX,
                            np.ascontiguousarray(Y, np.int32) if n else UY, n, UX, UY, cnt)
    return UX[:m].copy(), UY[:m].copy(), cnt[:m].copy()


def _nz(a, dt):
    a = np.ascontiguousarray(a, dtype=dt)
    return a if a.size else np.zeros(1, dt)


def rwmd(Ahat, Bhat, kappa=1, tau=0):
    """Ahat, Bhat = (X, Y, cnt).  Returns (L_A, L_B, max).  kappa, tau: the
    creation / destruction cost kappa * d_diag + tau (see cmake)."""
    L = np.zeros(3, np.int64)
    lib().orc_rwmd(_nz(Ahat[0], np.int32), _nz(Ahat[1], np.int32), _nz(Ahat[2], np.int64), len(Ahat[0]),
                   _nz(Bhat[0], np.int32), _nz(Bhat[1], np.int32), _nz(Bhat[2], np.int64), len(Bhat[0]),
                   int(kappa), int(tau), L)
    return int(L[0]), int(L[1]), int(L[2])


def condense_delta(Ahat, Bhat, G, P, seed):
    n = len(Ahat[0]) + len(Bhat[0])
    X = np.zeros(max(n, 1), np.int32)
    Y = np.zeros(max(n, 1), np.int32)
    ca = np.zeros(max(n, 1), np.int64)
    cb = np.zeros(max(n, 1), np.int64)
    code = np.zeros(max(n, 1), np.uint64)
    N = lib().orc_condense_delta(_nz(Ahat[0], np.int32), _nz(Ahat[1], np.int32), _nz(Ahat[2], np.int64),
                                 len(Ahat[0]), _nz(Bhat[0], np.int32), _nz(Bhat[1], np.int32),
                                 _nz(Bhat[2], np.int64), len(Bhat[0]), G, P, seed, X, Y, ca, cb, code)
    return dict(X=X[:N].copy(), Y=Y[:N].copy(), cntA=ca[:N].copy(), cntB=cb[:N].copy(),
                code=code[:N].copy())


def radix_tree(nodes):
    N = len(nodes["X"])
    M = max(N - 1, 1)
    t = dict(left=np.zeros(M, np.int32), right=np.zeros(M, np.int32), lo=np.zeros(M, np.int32),
             hi=np.zeros(M, np.int32), bb=np.zeros(4 * M, np.int32), rep=np.zeros(M, np.int32))
    if N >= 2:
        lib().orc_radix_tree(N, nodes["code"], nodes["X"], nodes["Y"], t["left"], t["right"], t["lo"],
                             t["hi"], t["bb"], t["rep"])
    else:
        t = {k: v[:0] for k, v in t.items()}
    t["bb"] = t["bb"].reshape(-1, 4)
    return t


def split_tree(nodes):
    """The paper's split tree over the nodes (longest bounding-box side cut in
    the middle).  Returns (perm, tree): perm[p] = index in `nodes` of the leaf
    at position p; the tree refers to positions, so it goes with
    reorder(nodes, perm)."""
    N = len(nodes["X"])
    M = max(N - 1, 1)
    perm = np.arange(N, dtype=np.int32)
    t = dict(left=np.zeros(M, np.int32), right=np.zeros(M, np.int32), bb=np.zeros(4 * M, np.int32),
             rep=np.zeros(M, np.int32))
    if N >= 2:
        lib().orc_split_tree(N, _nz(nodes["X"], np.int32), _nz(nodes["Y"], np.int32), perm, t["left"],
                             t["right"], t["bb"], t["rep"])
    else:
        t = {k: v[:0] for k, v in t.items()}
    t["bb"] = t["bb"].reshape(-1, 4)
    return perm, t


def reorder(nodes, perm):
    """The nodes in the order perm gives (position p holds node perm[p])."""
    return {k: np.ascontiguousarray(v[perm]) for k, v in nodes.items()}


def wspd(nodes, tree, s, cap=None):
    N = len(nodes["X"])
    if N < 2:
        return np.zeros(0, np.int32), np.zeros(0, np.int32)
    bb = np.ascontiguousarray(tree["bb"].reshape(-1))
    args = (N, nodes["X"], nodes["Y"], tree["left"], tree["right"], bb, tree["rep"], int(s))
    if cap is None:
        m = lib().orc_wspd(*args, np.zeros(1, np.int32), np.zeros(1, np.int32), 0)
        cap = m
    t = np.zeros(max(cap, 1), np.int32)
    h = np.zeros(max(cap, 1), np.int32)
    m = lib().orc_wspd(*args, t, h, cap)
    if m > cap:
        raise MemoryError("WSPD arc capacity %d < %d" % (cap, m))
    return t[:m].copy(), h[:m].copy()


def wspd_pairs(nodes, tree, s):
    """The well-separated pairs (u, v) as tree references (>= 0 internal, < 0 leaf ~c)."""
    N = len(nodes["X"])
    if N < 2:
        return np.zeros(0, np.int32), np.zeros(0, np.int32)
    bb = np.ascontiguousarray(tree["bb"].reshape(-1))
    args = (N, nodes["X"], nodes["Y"], tree["left"], tree["right"], bb, tree["rep"], int(s))
    m = lib().orc_wspd_pairs(*args, np.zeros(1, np.int32), np.zeros(1, np.int32), 0)
    pu = np.zeros(max(m, 1), np.int32)
    pv = np.zeros(max(m, 1), np.int32)
    lib().orc_wspd_pairs(*args, pu, pv, m)
    return pu[:m].copy(), pv[:m].copy()


def mix64(z: int) -> int:
    return int(lib().orc_mix64(z))


def build_network(nodes, tails, heads, kappa=1, tau=0):
    N = len(nodes["X"])
    nws = len(tails)
    na = int(np.count_nonzero(nodes["cntA"] > 0))
    nb = int(np.count_nonzero(nodes["cntB"] > 0))
    m = nws + na + nb + 1
    row_ptr = np.zeros(N + 3, np.int64)
    head = np.zeros(m, np.int32)
    cst = np.zeros(m, np.int64)
    sup = np.zeros(N + 2, np.int64)
    m2 = lib().orc_build_network(N, _nz(nodes["X"], np.int32), _nz(nodes["Y"], np.int32),
                                 _nz(nodes["cntA"], np.int64), _nz(nodes["cntB"], np.int64), nws,
                                 _nz(tails, np.int32), _nz(heads, np.int32), row_ptr, head, cst, sup,
                                 int(kappa), int(tau))
    assert m2 == m
    return dict(n_nodes=N, row_ptr=row_ptr, head=head, cost=cst, supply=sup)


def mcf(net, max_pivots=0):
    """Network simplex on the CSR network.  Returns (OPT_int, flow, potentials)."""
    n = net["n_nodes"] + 2
    m = int(net["row_ptr"][-1])
    flow = np.zeros(max(m, 1), np.int64)
    pot = np.zeros(n, np.int64)
    opt = C.c_int64()
    piv = C.c_int64()
    st = lib().orc_mcf_csr(n, net["row_ptr"], _nz(net["head"], np.int32), _nz(net["cost"], np.int64),
                           net["supply"], flow, pot, C.byref(opt), C.byref(piv), max_pivots)
    if st != 0:
        raise RuntimeError("network simplex status %d" % st)
    return opt.value, flow[:m], pot


def mcf_arcs(n, tails, heads, costs, supply, max_pivots=0):
    """Network simplex on an arbitrary arc list (non-negative integer costs)."""
    m = len(tails)
    flow = np.zeros(max(m, 1), np.int64)
    pot = np.zeros(max(n, 1), np.int64)
    opt = C.c_int64()
    piv = C.c_int64()
    st = lib().orc_mcf_arcs(n, m, _nz(tails, np.int32), _nz(heads, np.int32), _nz(costs, np.int64),
                            _nz(supply, np.int64), flow, pot, C.byref(opt), C.byref(piv), max_pivots)
    return st, opt.value, flow[:m], pot[:n]


def mcf_arcs_dbl(n, tails, heads, costs, supply, tol=1e-12, max_pivots=0):
    m = len(tails)
    flow = np.zeros(max(m, 1), np.int64)
    pot = np.zeros(max(n, 1), np.float64)
    opt = C.c_double()
    piv = C.c_int64()
    st = lib().orc_mcf_arcs_dbl(n, m, _nz(tails, np.int32), _nz(heads, np.int32), _nz(costs, np.float64),
                                _nz(supply, np.int64), flow, pot, C.byref(opt), C.byref(piv), max_pivots,
                                tol)
    return st, opt.value, flow[:m], pot[:n]


def dense_opt_int(P, Q, max_pivots=0, kappa=1, tau=0):
    """Integer optimum of the dense bipartite G(A,B) between weighted node sets
    P = (X, Y, cnt) (A side) and Q (B side), rounded-up costs."""
    opt = C.c_int64()
    st = lib().orc_dense_opt_int(_nz(P[0], np.int32), _nz(P[1], np.int32), _nz(P[2], np.int64), len(P[0]),
                                 _nz(Q[0], np.int32), _nz(Q[1], np.int32), _nz(Q[2], np.int64), len(Q[0]),
                                 int(kappa), int(tau), C.byref(opt), max_pivots)
    if st != 0:
        raise RuntimeError("network simplex status %d" % st)
    return opt.value


def w1_exact(A, B, max_pivots=0, kappa=1.0, tau=0.0) -> float:
    """Exact FP64 W1 (l2 ground metric) on unquantised (n, 2) diagrams;
    kappa, tau (in the diagrams' units): creation / destruction costs."""
    a = np.ascontiguousarray(np.asarray(A, dtype=np.float64).reshape(-1, 2))
    b = np.ascontiguousarray(np.asarray(B, dtype=np.float64).reshape(-1, 2))
    v = lib().orc_w1_exact(_nz(a.reshape(-1), np.float64), a.shape[0], _nz(b.reshape(-1), np.float64),
                           b.shape[0], float(kappa), float(tau), max_pivots)
    if v < 0:
        raise RuntimeError("exact W1 solve failed")
    return float(v)


def w1_approx(A, B, dtype, eps=0.1, k=None, s_override=0, perturb=True, seed=0,
              condense=True, solve=True, tree="radix", kappa=1, tau=0):
    """Algorithm 4 end to end.  Returns a dict of every intermediate result.

    A, B: (n, 2) arrays of (birth, death), float32 (dtype "f32") or uint8 ("u8").
    W1 ~= OPT_int * 2^-k.  condense=False keeps G = 1, P = 0 (no snapping).
    tree: "radix" (Morton radix tree) or "split" (the paper's split tree).
    kappa, tau: creation / destruction cost kappa * d_diag + tau quanta of the
    diagonal arcs (1, 0 for persistence diagrams).
    """
    if k is None:
        k = default_shift(dtype)
    XA, YA = quantize(A, dtype, k)
    XB, YB = quantize(B, dtype, k)
    Ahat = condense0(XA, YA)
    Bhat = condense0(XB, YB)
    FA = int(Ahat[2].sum())
    FB = int(Bhat[2].sum())
    LA, LB, L = rwmd(Ahat, Bhat, kappa, tau)
    s = int(s_override) if s_override else s_from_eps(eps)
    if condense:
        delta, G, P = delta_params(LA, LB, FA, FB, s)
    else:
        delta, G, P = 0.0, 1, 0
    if not perturb:
        P = 0
    nodes = condense_delta(Ahat, Bhat, G, P, seed)
    if tree == "split":  # the paper's split tree: nodes renumbered in its leaf order
        perm, tr = split_tree(nodes)
        nodes = reorder(nodes, perm)
    else:
        tr = radix_tree(nodes)
    tails, heads = wspd(nodes, tr, s)
    net = build_network(nodes, tails, heads, kappa, tau)
    out = dict(k=k, Ahat=Ahat, Bhat=Bhat, FA=FA, FB=FB, LA=LA, LB=LB, rwmd=L, s=s, delta=delta, G=G,
               P=P, nodes=nodes, tree=tr, ws_tails=tails, ws_heads=heads, net=net)
    if solve:
        opt, flow, pot = mcf(net)
        out.update(opt=opt, flow=flow, pot=pot, slack=int(flow.sum()), w1=math.ldexp(opt, -k))
    return out


def wcd(P, Q):
    """Word centroid distance used as a W1 lower bound (Appendix, WCD): with
    P~ the diagonal projections ((b+d)/2, (b+d)/2) of a diagram, the two
    multisets U = P + Q~ and V = Q + P~ have the same size n, and
    WCD = n |centroid(U) - centroid(V)| (Euclidean), which is at most the
    optimal matching cost OT(U, V) <= 2 W1(P, Q); so W1 >= WCD / 2.  P, Q:
    (n, 2) arrays of (birth, death) in any units, or (X, Y, count) triples of
    condensed nodes; FP64 straight from the definition."""
    def pts(D):
        if isinstance(D, tuple):
            X = np.repeat(np.asarray(D[0], np.float64), np.asarray(D[2], np.int64))
            Y = np.repeat(np.asarray(D[1], np.float64), np.asarray(D[2], np.int64))
            return np.stack([X, Y], axis=1) if len(X) else np.zeros((0, 2))
        return np.asarray(D, np.float64).reshape(-1, 2)
    p, q = pts(P), pts(Q)
    proj = lambda a: np.repeat(((a[:, 0] + a[:, 1]) / 2.0)[:, None], 2, axis=1)
    U = np.concatenate([p, proj(q)])
    V = np.concatenate([q, proj(p)])
    n = len(U)
    if n == 0:
        return 0.0
    return float(n * np.hypot(*(U.mean(axis=0) - V.mean(axis=0))))


def nn_search(query, db, dtype, eps=0.05, **kw):
    """Nearest neighbour of `query` among the diagrams of `db` (the NN-search
    application of the experiments section): the index minimising the
    approximate W1 of w1_approx(query, db[i]) -- OPT_int, ties to the lowest
    index -- computed by solving every pair.  Returns (index, [OPT_int])."""
    opts = [w1_approx(query, d, dtype, eps=eps, **kw)["opt"] for d in db]
    if not opts:
        return -1, []
    best = min(range(len(opts)), key=lambda i: (opts[i], i))
    return best, opts
