"""Batched persistent solves (one launch for many systems of uneven order,
each with its own butterflies) against the oracle, per system."""
import numpy as np
import pytest
import torch

import oracle
from paper_2312_09376_gb300 import _lib, inputs
from tests import _bounds

pytestmark = pytest.mark.gpu


def _make_batch(count, lo, hi, seed=7):
    ns = inputs.batch_sizes(count, lo, hi, seed=seed)
    rs = inputs.batch_nrhs(count, 1, 8, seed=seed + 1)
    As = [inputs.gaussian(int(n), seed=1000 + i) for i, n in enumerate(ns)]
    Bs = [inputs.rhs(int(n), int(r), seed=5000 + i) for i, (n, r) in enumerate(zip(ns, rs))]
    return ns, rs, As, Bs


def _run_batch(As, Bs, prec, d=2, seeds=None, tol=1e-13, refine_max=30, autotune=False, graph=False):
    opts = _lib.make_opts(depth=d, seed=1000, prec=prec, refine_max=refine_max, tol=tol)
    Ad = [_lib.to_device(a) for a in As]
    Bd = [_lib.to_device(b) for b in Bs]
    Xd = [_lib.colmajor(b.shape[0], b.shape[1]) for b in Bs]
    plan = _lib.rbt_solve_batched_plan(opts, Ad, Bd, Xd, seeds=seeds)
    if autotune:
        v, ms = _lib.rbt_solve_batched_autotune(plan)
        assert 0 <= v < 4 and ms > 0
        assert _lib.rbt_solve_batched_variant(plan)[0] == v
    if graph:
        s = torch.cuda.Stream()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            _lib.rbt_solve_batched_run(plan, stream=s)
        for X in Xd:
            X.fill_(np.nan)
        g.replay()
        g.replay()
    else:
        _lib.rbt_solve_batched_run(plan)
    torch.cuda.synchronize()
    return [_lib.to_host(x) for x in Xd], plan.infos_host()


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_batched_matches_oracle(prec):
    ns, rs, As, Bs = _make_batch(48, 1, 300)
    seeds = [1000 + i for i in range(len(ns))]
    Xs, infos = _run_batch(As, Bs, prec, seeds=seeds)
    for i, (A, B, X) in enumerate(zip(As, Bs, Xs)):
        assert infos[i]["status"] == 0, (i, ns[i], infos[i])
        berr = _bounds.berr(A, X, B)
        assert berr <= 1e-13, (i, ns[i], berr)
        assert abs(berr - infos[i]["berr"]) <= 8 * ns[i] * 2.2e-16
        if i < 6:
            Xo, st, _, bo, _ = oracle.rbt_solve(A, B, 2, seed=seeds[i], refine_max=30, tol=1e-13)
            kappa = np.linalg.cond(A, np.inf)
            assert np.abs(X - Xo).max() <= 100 * ns[i] * kappa * 2.2e-16 * np.abs(Xo).max()


@pytest.mark.parametrize("d", [2, 3])
def test_batched_unrefined_matches_oracle_factorization(d):
    """With no refinement the first backward error of each system is that of
    the same transform and GENP (oracle) up to rounding order; depth 3 takes
    the eight-lane form of the transform (one row of an 8 x 8 group per lane)."""
    ns, rs, As, Bs = _make_batch(12, 40, 200, seed=3)
    seeds = [77 + i for i in range(len(ns))]
    Xs, infos = _run_batch(As, Bs, "f64", d=d, seeds=seeds, refine_max=0, tol=0.0)
    for i, (A, B) in enumerate(zip(As, Bs)):
        Xo, st, b0, _, _ = oracle.rbt_solve(A, B, d, seed=seeds[i], refine_max=0, tol=0.0)
        g = infos[i]["berr_unrefined"]
        assert g <= 10 * b0 + 1e-15 and b0 <= 10 * g + 1e-15


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_batched_depth3_matches_oracle(prec):
    """Depth 3 (the eight-lane transform), refined: every system reaches the
    backward-error target and the first ones agree with the oracle's solution."""
    ns, rs, As, Bs = _make_batch(24, 8, 260, seed=9)
    seeds = [300 + i for i in range(len(ns))]
    Xs, infos = _run_batch(As, Bs, prec, d=3, seeds=seeds)
    for i, (A, B, X) in enumerate(zip(As, Bs, Xs)):
        assert infos[i]["status"] == 0, (i, ns[i], infos[i])
        assert _bounds.berr(A, X, B) <= 1e-13
        if i < 4:
            Xo, st, _, bo, _ = oracle.rbt_solve(A, B, 3, seed=seeds[i], refine_max=30, tol=1e-13)
            kappa = np.linalg.cond(A, np.inf)
            assert np.abs(X - Xo).max() <= 100 * ns[i] * kappa * 2.2e-16 * np.abs(Xo).max()


def test_batched_config_sizes_graph_and_autotune():
    """2048 systems, n uniform in [48, 700], 1-8 right-hand sides, float factors
    refined in double; autotuned, captured in a CUDA graph, replayed twice."""
    ns, rs, As, Bs = _make_batch(2048, 48, 700, seed=11)
    Xs, infos = _run_batch(As, Bs, "f32", autotune=True, graph=True)
    ok = infos["status"] == 0
    assert ok.mean() == 1.0, np.unique(infos["status"], return_counts=True)
    rng = np.random.default_rng(0)
    for i in rng.choice(len(ns), 12, replace=False):
        assert _bounds.berr(As[i], Xs[i], Bs[i]) <= 1e-13
    # the larger float systems whose refinement stalls are redone in double-float
    fb = np.flatnonzero(infos["fell_back"] == 1)
    assert len(fb) > 0
    for i in fb[:6]:
        assert _bounds.berr(As[i], Xs[i], Bs[i]) <= 1e-13


def test_batched_reports_zero_pivot_per_system():
    ns, rs, As, Bs = _make_batch(8, 30, 90, seed=5)
    As[3] = inputs.zero_corner(As[3])
    Xs, infos = _run_batch(As, Bs, "f64", d=0)
    assert infos[3]["status"] == 1 and infos[3]["zero_pivot"] == 0
    for i in range(8):
        if i != 3:
            assert infos[i]["status"] == 0
            assert _bounds.berr(As[i], Xs[i], Bs[i]) <= 1e-13
    # with the transform the same system is solved
    Xs, infos = _run_batch(As, Bs, "f64", d=2)
    assert infos[3]["status"] == 0


def test_batched_refines_by_stationary_steps_only():
    ns, rs, As, Bs = _make_batch(2, 20, 30, seed=2)
    opts = _lib.make_opts(depth=2, seed=1000, prec="f32", refine="gmres")
    Ad = [_lib.to_device(a) for a in As]
    Bd = [_lib.to_device(b) for b in Bs]
    Xd = [_lib.colmajor(b.shape[0], b.shape[1]) for b in Bs]
    with pytest.raises(_lib.RbtError):
        _lib.rbt_solve_batched_plan(opts, Ad, Bd, Xd)


def _adjoint_berr(A, W, Y):
    R = W - A.T @ Y
    return (np.abs(R).max(0) / (np.abs(A).sum(0).max() * np.abs(Y).max(0) + np.abs(W).max(0))).max()


@pytest.mark.parametrize("tol", [0.0, 1e-13])
def test_batched_fallback_ladder_forward_and_adjoint(tol):
    """Float systems with fallback and no refinement steps: every float attempt
    misses the tolerance, so each system is redone in double-float on the same
    A~ (fell_back = 1) and, when that misses too (always for tol = 0), by the
    double kernel's second launch (fell_back = 2), whose X is bit for bit the
    plain double batch's.  The batched adjoint (refined to 1e-13) then uses
    the factors of the rung that produced X."""
    from paper_2312_09376_gb300.autograd import solve_batched, solve_batched_backward
    ns, rs, As, Bs = _make_batch(16, 20, 200, seed=13)
    Ws = [inputs.rhs(int(n), int(r), seed=900 + i) for i, (n, r) in enumerate(zip(ns, rs))]
    seeds = [40 + i for i in range(len(ns))]
    Ad = [_lib.to_device(a) for a in As]
    Bd = [_lib.to_device(b) for b in Bs]
    Xd, plan = solve_batched(Ad, Bd, prec="f32", refine_max=0, tol=tol, seeds=seeds)
    X64, plan64 = solve_batched(Ad, Bd, prec="f64", refine_max=0, tol=tol, seeds=seeds)
    torch.cuda.synchronize()
    infos, i64 = plan.infos_host(), plan64.infos_host()
    if tol == 0.0:
        assert np.all(infos["fell_back"] == 2) and np.all(infos["status"] == 3), infos
    else:
        assert np.all(infos["fell_back"] >= 1)
        assert np.any(infos["fell_back"] == 1)
    for i, (A, B) in enumerate(zip(As, Bs)):
        if infos[i]["fell_back"] == 2:
            assert torch.equal(Xd[i], X64[i]) and infos[i]["berr"] == i64[i]["berr"], (i, ns[i])
        else:
            assert infos[i]["status"] == 0
            assert _bounds.berr(A, _lib.to_host(Xd[i]), B) <= 1e-13, (i, ns[i], infos[i])
    plan.opts.tol = 1e-13
    plan.opts.refine_max = 30
    Ys, GAs = solve_batched_backward(plan, [_lib.to_device(w) for w in Ws])
    torch.cuda.synchronize()
    adj = plan.infos_host()
    assert np.array_equal(adj["fell_back"], infos["fell_back"])
    assert np.all(adj["status"] == 0), adj
    for i, (A, W) in enumerate(zip(As, Ws)):
        Y = _lib.to_host(Ys[i])
        assert _adjoint_berr(A, W, Y) <= 1e-13, (i, ns[i])
        X = _lib.to_host(Xd[i])
        assert np.allclose(_lib.to_host(GAs[i]), -Y @ X.T, rtol=1e-12, atol=1e-12 * np.abs(Y).max() * np.abs(X).max())
