"""Nearest-neighbour search (pd_db_build / pd_nn_search): the answer equals
the oracle's argmin over every pair, with and without pruning, and every lower
bound is below the optimum it prunes against.  Runs on a GPU only."""
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


def _db(count, seed, lo=20, hi=1500):
    sizes = synth.db_sizes(count, seed, lo, hi)
    return [synth.uniform_exp(int(n), 5000 + 7 * seed + i) for i, n in enumerate(sizes)]


def test_nn_matches_oracle_with_and_without_pruning(pd, ctx):
    db = _db(20, 3)
    q = synth.uniform_exp(800, 42)
    eps = 0.1
    pd.pd_db_build(ctx, [_cuda(d) for d in db])
    full = pd.pd_nn_search(ctx, _cuda(q), eps, pd.opts(nn_prune=0))
    idx, opts = oracle.nn_search(q, db, "f32", eps=eps)
    assert full["opt"] == opts
    assert full["nn_index"] == idx and full["nn_opt_quanta"] == opts[idx]
    assert full["solved"] == len(db) and full["pruned"] == 0
    assert all(0 <= lb <= o for lb, o in zip(full["lb"], opts))
    pr = pd.pd_nn_search(ctx, _cuda(q), eps, pd.opts(batch_slots=4))
    assert pr["nn_index"] == idx and pr["nn_opt_quanta"] == opts[idx]
    assert pr["solved"] + pr["pruned"] == len(db)
    assert all(o_p in (-1, o) for o_p, o in zip(pr["opt"], opts))
    assert pr["lb"] == full["lb"]
    # growing waves from 1 and 3 pairs (and the default 16, above 20 pairs
    # here: one wave) reach the same answer; a pair is skipped only when its
    # bound exceeds an optimum already found
    for w0 in (1, 3):
        g = pd.pd_nn_search(ctx, _cuda(q), eps, pd.opts(nn_wave0=w0, batch_slots=8))
        assert g["nn_index"] == idx and g["nn_opt_quanta"] == opts[idx]
        assert all(o_p in (-1, o) for o_p, o in zip(g["opt"], opts))
        assert all(opts[i] == g["opt"][i] or g["lb"][i] > opts[idx] for i in range(len(db)))
    with pytest.raises(pd.PDError):
        pd.pd_nn_search(ctx, _cuda(q), eps, pd.opts(nn_wave0=-1))


def test_nn_duplicate_of_the_query_wins_at_its_lowest_index(pd, ctx):
    db = _db(12, 9)
    db[8] = db[3].copy()
    pd.pd_db_build(ctx, db)  # host-memory diagrams
    r = pd.pd_nn_search(ctx, db[3].copy(), 0.05, pd.opts(batch_slots=2))
    assert r["nn_index"] == 3 and r["nn_opt_quanta"] == 0 and r["lb"][3] == 0
    assert r["opt"][3] == 0 and r["opt"][8] in (-1, 0)


def test_nn_lowerstar_u8(pd, ctx):
    sizes = synth.db_sizes(8, 21, 500, 5000)
    db = [synth.lowerstar_u8(int(n), 9000 + i) for i, n in enumerate(sizes)]
    q = synth.lowerstar_u8(3000, 8999)
    pd.pd_db_build(ctx, [_cuda(d) for d in db])
    full = pd.pd_nn_search(ctx, _cuda(q), 0.05, pd.opts(nn_prune=0))
    pr = pd.pd_nn_search(ctx, _cuda(q), 0.05)
    idx, opts = oracle.nn_search(q, db, "u8", eps=0.05)
    assert full["opt"] == opts and full["nn_index"] == idx
    assert (pr["nn_index"], pr["nn_opt_quanta"]) == (idx, opts[idx])
    assert all(lb <= o for lb, o in zip(full["lb"], opts))


def test_nn_empty_database_and_bad_queries(pd, ctx):
    pd.pd_db_build(ctx, [])
    r = pd.pd_nn_search(ctx, _cuda(synth.uniform_exp(100, 1)), 0.1)
    assert r["nn_index"] == -1 and r["solved"] == 0
    pd.pd_db_build(ctx, [_cuda(synth.uniform_exp(50, 2))])
    with pytest.raises(pd.PDError):
        pd.pd_nn_search(ctx, _cuda(synth.lowerstar_u8(100, 3)), 0.1)  # dtype differs from the database
    with pytest.raises(pd.PDError):
        pd.pd_nn_search(ctx, _cuda(synth.uniform_exp(100, 1)), 0.0)
    with pytest.raises(pd.PDError):
        pd.pd_db_build(ctx, [_cuda(synth.uniform_exp(50, 2)), _cuda(synth.lowerstar_u8(60, 3))])


def test_nn_coordinates_beyond_float32_exactness(pd, ctx):
    """Every diagram translated along (t, t) to coordinates >= 2^23 quanta,
    where float32 stops being exact: the bound takes its absolute margin and
    must stay below every optimum; the answer equals the oracle's, with and
    without pruning, and the bounds are the same bits on every call (fixed
    order of summation)."""
    db = [(d + 100.0).astype(np.float32) for d in _db(10, 17)]
    q = (synth.uniform_exp(600, 77) + 100.0).astype(np.float32)
    assert (q * 2.0 ** 20).min() >= 2 ** 23
    eps = 0.1
    pd.pd_db_build(ctx, [_cuda(d) for d in db])
    full = pd.pd_nn_search(ctx, _cuda(q), eps, pd.opts(nn_prune=0))
    idx, opts = oracle.nn_search(q, db, "f32", eps=eps)
    assert full["opt"] == opts and full["nn_index"] == idx
    assert all(0 <= lb <= o for lb, o in zip(full["lb"], opts))
    pr = pd.pd_nn_search(ctx, _cuda(q), eps, pd.opts(batch_slots=3))
    assert (pr["nn_index"], pr["nn_opt_quanta"]) == (idx, opts[idx])
    assert pr["lb"] == full["lb"]


def _hat(D, dtype):
    k = oracle.default_shift(dtype)
    return oracle.condense0(*oracle.quantize(D, dtype, k))


def test_nn_wcd_bound_matches_the_oracle_and_stays_below_the_optimum(pd, ctx):
    """The WCD bound (Appendix, WCD) of every pair equals (1 - eps_c) WCD / 2
    of the oracle's definition (centroids of A + B~ and B + A~) on the
    quantised diagrams, rounded down (within one quantum of double rounding);
    the bound used is never below it and never above the optimum."""
    db = _db(16, 23, lo=20, hi=900)
    db[5] = np.concatenate([db[5], db[5]])  # twice the total persistence: the WCD bound grows
    q = synth.uniform_exp(700, 55)
    eps = 0.1
    s = oracle.s_from_eps(eps)
    ec = oracle.eps_c(s)
    pd.pd_db_build(ctx, [_cuda(d) for d in db])
    full = pd.pd_nn_search(ctx, _cuda(q), eps, pd.opts(nn_prune=0))
    idx, opts = oracle.nn_search(q, db, "f32", eps=eps)
    assert full["opt"] == opts and full["nn_index"] == idx
    qh = _hat(q, "f32")
    for i, d in enumerate(db):
        w = oracle.wcd(qh, _hat(d, "f32"))
        exp = int(np.floor((1 - ec) * w / 2))
        assert abs(full["wcd"][i] - exp) <= 1
        assert full["wcd"][i] <= full["lb"][i] <= opts[i]
    assert 0 <= full["wcd_above"] <= sum(1 for i in range(len(db)) if full["wcd"][i] == full["lb"][i])
