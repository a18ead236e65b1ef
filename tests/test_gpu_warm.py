"""Warm start: the network's device forward and gradients equal the oracle's,
a start from any potentials keeps the optimum, exact potentials save most
pivots, and the gain of a trained network is measured on seen and unseen
pairs.  Runs on a GPU only."""
import os
import tempfile

import numpy as np
import pytest
import torch

import oracle
from oracle import mlp
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


def test_network_forward_and_gradient_match_the_oracle(pd, ctx):
    rng = np.random.default_rng(11)
    p = (rng.standard_normal(mlp.NPARAMS) * 0.12).astype(np.float32)
    x = rng.standard_normal((333, mlp.NIN)).astype(np.float32)  # 11 tiles and a ragged one
    t = rng.standard_normal(333).astype(np.float32)
    m = (rng.random(333) < 0.9).astype(np.float32)
    pd.pd_ws_set_params(ctx, p)
    np.testing.assert_array_equal(pd.pd_ws_get_params(ctx), p)
    y = pd.pd_ws_forward(ctx, x)
    y0, _ = mlp.forward(p, x)
    np.testing.assert_allclose(y, y0, rtol=1e-4, atol=1e-4 * np.abs(y0).max())
    loss, g = pd.pd_ws_grad(ctx, x, t, m)
    loss0, g0 = mlp.loss_grad(p, x, t, m)
    assert abs(loss - loss0) <= 1e-4 * abs(loss0)
    scale = np.abs(g0).max()
    np.testing.assert_allclose(g, g0, rtol=1e-3, atol=1e-4 * scale)
    # every block of the layout is exercised
    for a, b in ((mlp.OFF_W1, mlp.OFF_B1), (mlp.OFF_B1, mlp.OFF_W2), (mlp.OFF_W2, mlp.OFF_B2),
                 (mlp.OFF_B2, mlp.OFF_W3), (mlp.OFF_W3, mlp.OFF_B3)):
        assert np.abs(g0[a:b]).max() > 0


def test_save_and_load_round_trip(pd, ctx):
    p = np.random.default_rng(3).standard_normal(mlp.NPARAMS).astype(np.float32) * 0.1
    pd.pd_ws_set_params(ctx, p)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "ws.bin")
        pd.pd_ws_save(ctx, path)
        c2 = pd.pd_create(0)
        pd.pd_ws_load(c2, path)
        np.testing.assert_array_equal(pd.pd_ws_get_params(c2), p)
        c2.close()
        with open(path, "wb") as f:
            f.write(b"not a parameter file")
        with pytest.raises(pd.PDError):
            pd.pd_ws_load(ctx, path)


@pytest.mark.parametrize("name", ["uniform2k", "lowerstar20k"])
def test_exact_potentials_start_keeps_the_optimum_and_saves_pivots(pd, ctx, name):
    if name == "uniform2k":
        A, B, dt, eps = synth.uniform_exp(2000, 1000), synth.uniform_exp(2000, 1001), "f32", 0.1
    else:
        A, B, dt, eps = synth.lowerstar_u8(20000, 1000), synth.lowerstar_u8(20000, 1001), "u8", 0.05
    cold = pd.pd_w1_approx(ctx, _cuda(A), _cuda(B), eps, pd.opts(warm_start=0))
    warm = pd.pd_w1_approx(ctx, _cuda(A), _cuda(B), eps, pd.opts(warm_start=2))
    assert warm["warm_used"] == 1 and warm["verified"] == 1
    assert warm["opt_quanta"] == cold["opt_quanta"] == oracle.w1_approx(A, B, dt, eps=eps)["opt"]
    assert warm["pivots"] < 0.75 * cold["pivots"], (warm["pivots"], cold["pivots"])


def test_trained_network_start_keeps_the_optimum_and_reports_its_gain(pd, ctx):
    """Training on seeded pairs with the last ones held out keeps the weights
    of the epoch with the smallest held-out error, never worse than no
    correction; the start from the coarse solve corrected by the trained
    network keeps the optimum, saves pivots against the cold start on unseen
    pairs, and its gain over the coarse start alone is printed (the benchmark
    reports it at the full size)."""
    train = [(synth.lowerstar_u8(20000, 3000 + 2 * i), synth.lowerstar_u8(20000, 3001 + 2 * i)) for i in range(8)]
    ctx = pd.pd_create(0)  # a fresh network: earlier tests left other parameters in the module's context
    st = pd.pd_ws_train(ctx, [_cuda(a) for a, _ in train], [_cuda(b) for _, b in train], 0.05,
                        epochs=20, lr=3e-4, seed=1)
    assert st["pairs"] == 8 and st["val_pairs"] == 1 and st["rows"] > st["val_rows"] > 0
    assert st["val_loss"] <= st["val_loss_zero"] * (1 + 1e-5) + 1e-12
    assert 0 <= st["best_epoch"] <= 20
    print("held-out mse: no correction %.4g, kept weights %.4g (epoch %d)" % (
        st["val_loss_zero"], st["val_loss"], st["best_epoch"]))
    seen = train[0]
    unseen = (synth.lowerstar_u8(20000, 5000), synth.lowerstar_u8(20000, 5001))
    gains = {}
    for name, (A, B) in (("seen", seen), ("unseen", unseen)):
        cold = pd.pd_w1_approx(ctx, _cuda(A), _cuda(B), 0.05, pd.opts(warm_start=0))
        coarse = pd.pd_w1_approx(ctx, _cuda(A), _cuda(B), 0.05, pd.opts(warm_start=4))
        warm = pd.pd_w1_approx(ctx, _cuda(A), _cuda(B), 0.05, pd.opts(warm_start=1))
        assert warm["opt_quanta"] == cold["opt_quanta"] == coarse["opt_quanta"] and warm["verified"] == 1
        assert warm["warm_used"] == 1
        gains[name] = (cold["pivots"], coarse["pivots"], warm["pivots"])
    print("pivots (cold, coarse start, coarse + network): seen %s unseen %s" % (gains["seen"], gains["unseen"]))
    assert gains["unseen"][2] < gains["unseen"][0]
    # the batched solve with the same network gives the same optima
    wb = pd.pd_w1_approx_batch(ctx, [_cuda(seen[0]), _cuda(unseen[0])], [_cuda(seen[1]), _cuda(unseen[1])], 0.05,
                               pd.opts(warm_start=1))
    for (a, b), r in zip((seen, unseen), wb):
        assert r["warm_used"] == 1
        assert r["opt_quanta"] == pd.pd_w1_approx(ctx, _cuda(a), _cuda(b), 0.05)["opt_quanta"]
    ctx.close()


def test_cost_greedy_start_keeps_the_optimum(pd, ctx):
    A, B = synth.lowerstar_u8(20000, 1000), synth.lowerstar_u8(20000, 1001)
    cold = pd.pd_w1_approx(ctx, _cuda(A), _cuda(B), 0.05, pd.opts(warm_start=0))
    z = pd.pd_w1_approx(ctx, _cuda(A), _cuda(B), 0.05, pd.opts(warm_start=3))
    assert z["warm_used"] == 1 and z["opt_quanta"] == cold["opt_quanta"] and z["verified"] == 1


@pytest.mark.parametrize("name", ["uniform2k", "lowerstar20k", "mixture5k"])
def test_coarse_solve_start_keeps_the_optimum(pd, ctx, name):
    """warm_start = 4: the potentials of an exact solve of the same pair on a
    coarser lattice, mapped to the fine nodes, seed the start; the optimum is
    the oracle's (the start only changes where the simplex begins), in the
    one-pair and the batched solve."""
    if name == "uniform2k":
        A, B, dt, eps = synth.uniform_exp(2000, 1000), synth.uniform_exp(2000, 1001), "f32", 0.1
    elif name == "lowerstar20k":
        A, B, dt, eps = synth.lowerstar_u8(20000, 1000), synth.lowerstar_u8(20000, 1001), "u8", 0.05
    else:
        A, B, dt, eps = synth.mixture_f32(5000, 7), synth.mixture_f32(4000, 8), "f32", 0.1
    exp = oracle.w1_approx(A, B, dt, eps=eps)["opt"]
    cold = pd.pd_w1_approx(ctx, _cuda(A), _cuda(B), eps, pd.opts(warm_start=0))
    warm = pd.pd_w1_approx(ctx, _cuda(A), _cuda(B), eps, pd.opts(warm_start=4))
    assert warm["warm_used"] == 1 and warm["verified"] == 1
    assert warm["opt_quanta"] == cold["opt_quanta"] == exp
    print("%s pivots cold %d coarse start %d" % (name, cold["pivots"], warm["pivots"]))
    wb = pd.pd_w1_approx_batch(ctx, [_cuda(A), _cuda(B)], [_cuda(B), _cuda(A)], eps, pd.opts(warm_start=4))
    assert [r["opt_quanta"] for r in wb] == [exp, exp]


@pytest.mark.parametrize("mode,cells", [(4, 8), (4, 256)])
def test_coarse_start_cells_keep_the_optimum(pd, ctx, mode, cells):
    """warm_cells sets the coarse lattice of warm_start = 4 (node box / cells);
    any level gives the same optimum, and a value out of range is refused."""
    A, B = synth.lowerstar_u8(20000, 1002), synth.lowerstar_u8(20000, 1003)
    exp = oracle.w1_approx(A, B, "u8", eps=0.05)["opt"]
    warm = pd.pd_w1_approx(ctx, _cuda(A), _cuda(B), 0.05, pd.opts(warm_start=mode, warm_cells=cells))
    assert warm["warm_used"] == 1 and warm["verified"] == 1 and warm["opt_quanta"] == exp
    with pytest.raises(pd.PDError):
        pd.pd_w1_approx(ctx, _cuda(A), _cuda(B), 0.05, pd.opts(warm_start=4, warm_cells=5000))


def test_automatic_warm_start(pd, ctx):
    """The default warm_start (-1): pd_w1_approx starts from the coarse solve
    on an instance of at least 4,096 transportation nodes and cold below it;
    the batched solve starts cold; every optimum is the oracle's."""
    A, B = synth.lowerstar_u8(100000, 1004), synth.lowerstar_u8(100000, 1005)
    exp = oracle.w1_approx(A, B, "u8", eps=0.05)["opt"]
    auto = pd.pd_w1_approx(ctx, _cuda(A), _cuda(B), 0.05)
    cold = pd.pd_w1_approx(ctx, _cuda(A), _cuda(B), 0.05, pd.opts(warm_start=0))
    assert auto["opt_quanta"] == cold["opt_quanta"] == exp
    assert auto["warm_used"] == 1 and cold["warm_used"] == 0 and auto["pivots"] < cold["pivots"]
    small = pd.pd_w1_approx(ctx, _cuda(synth.uniform_exp(2000, 1000)), _cuda(synth.uniform_exp(2000, 1001)), 0.1)
    assert small["warm_used"] == 0
    wb = pd.pd_w1_approx_batch(ctx, [_cuda(A)], [_cuda(B)], 0.05)
    assert wb[0]["warm_used"] == 0 and wb[0]["opt_quanta"] == exp
