"""Batched and served LM steps (lm_batch_*, lm_server_*) on the GPU.

Each instance's result must be the same alone and in the mix: a batch or a
served request runs exactly the kernel sequence of lm_build_OG + irl_step on
its own inputs, and the products' fixed-order reductions depend only on the
pencil grid, which the engine reports. So every instance is re-run alone with
that grid and compared bit for bit; the mixed-precision eigenvalue is also
checked against the FP64 oracle (|lambda - lambda_FP64| <= 1e-9 Ha).
"""
import numpy as np
import pytest

import __graft_entry__ as entry
import synth
from oracle import lm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def abi():
    entry.build()
    from paper_2601_01437_gb300 import abi as a
    return a


@pytest.fixture(scope="module")
def ctx(abi):
    c = abi.Context(0)
    yield c
    c.close()


INSTANCES = synth.batched_instances(64)
SMALL = [0, 2, 11, 18, 27, 48, 9]  # 784 .. 3,136 determinants, P+1 289 .. 646


def _inputs(w):
    h, eri, th, _, _ = w.inputs()
    return h, eri, th


def _solo(abi, ctx, w, theta, grid, prec):
    h, eri, _ = _inputs(w)
    sysd = ctx.system(w.n_orb, w.n_alpha, w.n_beta, w.n_hidden, h, eri)
    pen = ctx.build_OG(sysd, theta, prec=prec)
    pen.set_grid(grid)
    dth = np.zeros(w.n_params)
    res = pen.irl_step(m=w.m, k=w.k, tol=w.tol, max_restarts=200, prec=prec, dtheta_out=dth)
    pen.free()
    return res, dth


def _items(abi, ctx, idx, prec):
    items = []
    for i in idx:
        w = INSTANCES[i]
        h, eri, th = _inputs(w)
        items.append({"sys": ctx.system(w.n_orb, w.n_alpha, w.n_beta, w.n_hidden, h, eri),
                      "theta": th, "precision": prec,
                      "irl": abi.irl_settings(m=w.m, k=w.k, tol=w.tol, prec=prec),
                      "dtheta_out": np.zeros(w.n_params), "_keep": (h, eri)})
    return items


def test_batch_equals_solo_and_oracle(abi, ctx):
    """Seven uneven instances on four streams (so some share a stream), autotuned grids."""
    b = abi.Batch(ctx, n_streams=4, autotune=True)
    items = _items(abi, ctx, SMALL, abi.LM_FP32)
    res, grids = b.run(items)
    for k, i in enumerate(SMALL):
        w = INSTANCES[i]
        assert res[k].status in (abi.IRL_OK, abi.IRL_BREAKDOWN_INVARIANT), (w.name, res[k].status)
        assert 1 <= grids[k] <= 1024
        solo, dth = _solo(abi, ctx, w, items[k]["theta"], grids[k], abi.LM_FP32)
        assert solo.lambda_ == res[k].lambda_, w.name
        assert np.array_equal(dth, items[k]["dtheta_out"]), w.name
        h, eri, th = _inputs(w)
        ref = lm.lm_step(w.n_orb, w.n_alpha, w.n_beta, w.n_hidden, h, eri, th, None, None)
        assert abs(res[k].lambda_ - ref["lam"]) <= 1e-9, w.name
        assert res[k].n_matvec_lowp > 0
    # a second run reuses the resident pencils and reproduces the first
    again = _items(abi, ctx, SMALL, abi.LM_FP32)
    res2, grids2 = b.run(again)
    assert grids2 == grids
    for k in range(len(SMALL)):
        assert res2[k].lambda_ == res[k].lambda_
        assert np.array_equal(again[k]["dtheta_out"], items[k]["dtheta_out"])
    b.free()


def test_batch_restarts_replay_captured_cycles(abi, ctx):
    """Short Krylov spaces (m = 8, k = 3) force implicit restarts: the batch engine runs
    every cycle as a captured CUDA graph (the first cycle from j = 0, restarted ones from
    j = k), replayed across cycles and across two runs. Results are bit-identical to the
    same instance solved alone by direct launches, restarts and all."""
    idx = SMALL[:3]
    b = abi.Batch(ctx, n_streams=2, autotune=False)
    results = []
    for _ in range(2):
        items = _items(abi, ctx, idx, abi.LM_FP64)
        for it in items:
            it["irl"] = abi.irl_settings(m=8, k=3, tol=1e-12, prec=abi.LM_FP64)
        res, grids = b.run(items)
        results.append((res, items, grids))
    for k, i in enumerate(idx):
        w = INSTANCES[i]
        r1, r2 = results[0][0][k], results[1][0][k]
        assert r1.status in (abi.IRL_OK, abi.IRL_BREAKDOWN_INVARIANT), (w.name, r1.status)
        assert r1.n_restart >= 1, w.name
        assert r2.lambda_ == r1.lambda_ and r2.n_restart == r1.n_restart
        h, eri, th = _inputs(w)
        sysd = ctx.system(w.n_orb, w.n_alpha, w.n_beta, w.n_hidden, h, eri)
        pen = ctx.build_OG(sysd, th, prec=abi.LM_FP64)
        pen.set_grid(results[0][2][k])
        dth = np.zeros(w.n_params)
        solo = pen.irl_step(m=8, k=3, tol=1e-12, max_restarts=200, prec=abi.LM_FP64,
                            dtheta_out=dth)
        pen.free()
        assert solo.lambda_ == r1.lambda_ and solo.n_restart == r1.n_restart, w.name
        assert np.array_equal(dth, results[0][1][k]["dtheta_out"]), w.name
        ref = lm.lm_step(w.n_orb, w.n_alpha, w.n_beta, w.n_hidden, h, eri, th, None, None)
        assert abs(r1.lambda_ - ref["lam"]) <= 1e-10 * max(1.0, abs(ref["lam"])), w.name
    b.free()


def test_batch_fp64_storage_matches_oracle(abi, ctx):
    b = abi.Batch(ctx, n_streams=2, autotune=False)
    items = _items(abi, ctx, SMALL[:3], abi.LM_FP64)
    res, grids = b.run(items)
    for k, i in enumerate(SMALL[:3]):
        w = INSTANCES[i]
        h, eri, th = _inputs(w)
        ref = lm.lm_step(w.n_orb, w.n_alpha, w.n_beta, w.n_hidden, h, eri, th, None, None)
        assert res[k].lambda_ == pytest.approx(ref["lam"], rel=1e-10)
        assert np.linalg.norm(items[k]["dtheta_out"] - ref["dtheta"]) <= \
            1e-8 * np.linalg.norm(ref["dtheta"])
    b.free()


def _serve(abi, ctx, srv, idx, n_rounds=2):
    """Register the instances, submit n_rounds requests each (perturbed theta), drain."""
    sids, thetas, outs, tickets = {}, {}, {}, {}
    for i in idx:
        w = INSTANCES[i]
        h, eri, th = _inputs(w)
        sids[i] = srv.add_system(ctx.system(w.n_orb, w.n_alpha, w.n_beta, w.n_hidden, h, eri),
                                 precision=abi.LM_FP32)
    rng = np.random.default_rng(3)
    for r in range(n_rounds):
        for i in idx:
            w = INSTANCES[i]
            th = _inputs(w)[2] + (0 if r == 0 else 1e-3 * rng.standard_normal(w.n_params))
            out = np.zeros(w.n_params)
            t = srv.submit(sids[i], th, abi.irl_settings(m=w.m, k=w.k, tol=w.tol,
                                                         prec=abi.LM_FP32), out)
            thetas[t], outs[t], tickets[t] = th, out, i
    got = []
    for _ in range(200000):
        got += srv.poll()
        if len(got) == len(tickets):
            break
    assert len(got) == len(tickets)
    assert srv.pending() == 0
    return got, thetas, outs, tickets


def test_server_results_equal_solo(abi, ctx):
    srv = abi.Server(ctx, hbm_budget_bytes=150 << 30, n_streams=3, autotune=True)
    got, thetas, outs, tickets = _serve(abi, ctx, srv, SMALL[:4])
    for r in got:
        assert r.status == abi.LM_OK
        assert r.t_submit_ms <= r.t_admit_ms <= r.t_done_ms
        w = INSTANCES[tickets[r.ticket]]
        solo, dth = _solo(abi, ctx, w, thetas[r.ticket], r.grid, abi.LM_FP32)
        assert solo.lambda_ == r.result.lambda_
        assert np.array_equal(dth, outs[r.ticket])
    srv.free()


def test_server_budget_forces_eviction(abi, ctx):
    """A budget that holds one system at a time: every switch evicts the idle one (each
    of these systems needs an estimated 14-16 MB on the device)."""
    srv = abi.Server(ctx, hbm_budget_bytes=20 << 20, n_streams=2, autotune=False)
    idx = [0, 2, 27]  # 784 determinants each
    got, thetas, outs, tickets = _serve(abi, ctx, srv, idx)
    for r in got:
        assert r.status == abi.LM_OK
        w = INSTANCES[tickets[r.ticket]]
        solo, dth = _solo(abi, ctx, w, thetas[r.ticket], r.grid, abi.LM_FP32)
        assert solo.lambda_ == r.result.lambda_
    srv.free()


def test_server_rejects_oversized_system(abi, ctx):
    srv = abi.Server(ctx, hbm_budget_bytes=1 << 20, n_streams=1)
    w = INSTANCES[0]
    h, eri, _ = _inputs(w)
    with pytest.raises(abi.LMError) as e:
        srv.add_system(ctx.system(w.n_orb, w.n_alpha, w.n_beta, w.n_hidden, h, eri))
    assert e.value.code == abi.LM_ERR_SIZE
    srv.free()
