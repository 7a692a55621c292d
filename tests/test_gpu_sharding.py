"""Row sharding through the library (one pencil per shard, statistics and products summed
over the shards by the caller): lm_shard_build / lm_shard_sums / lm_shard_centre and
irl_step_sharded against the unsharded pencil on the same GPU.

The shards stand for GPUs of a multi-GPU run. Here they share one GPU: as K pencils in
one process (products summed on the host, IRL shards as threads whose reductions meet on
the host), and as two gloo ranks in two processes. No kernel of one shard waits on
another shard's kernels; every exchange is a host-side sum."""
import os
import threading

import numpy as np
import pytest

import __graft_entry__ as entry
import synth
from oracle import fock

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def abi():
    entry.build()
    from paper_2601_01437_gb300 import abi as a
    return a


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


def _case(name):
    if name == "f2":
        w = synth.WORKLOADS["f2_10o14e"]
        h, eri, th, _, _ = w.inputs()
        rows = fock.sector_dets(w.n_orb, w.n_alpha, w.n_beta)
        return w, h, eri, th, rows, None
    w = synth.Workload("mc", 14, 7, 7, 56, exact=False, n_samples=1500, m=20, k=1)
    h, eri, th, rows, cnt = w.inputs()
    return w, h, eri, th, rows, cnt.astype(np.float64)


def _split(n, k, seed=3):
    """Uneven contiguous shards (cut points drawn at random)."""
    rng = np.random.default_rng(seed)
    cuts = np.sort(rng.choice(np.arange(1, n), size=k - 1, replace=False))
    return np.split(np.arange(n), cuts)


def _build_shards(abi, ctxs, w, h, eri, th, rows, wts, parts, prec):
    pens, mx = [], []
    for ctx, idx in zip(ctxs, parts):
        sysd = ctx.system(w.n_orb, w.n_alpha, w.n_beta, w.n_hidden, h, eri)
        pen, m = ctx.shard_build(sysd, th, rows[idx].copy(),
                                 None if wts is None else wts[idx].copy(), prec=prec)
        pens.append(pen)
        mx.append(m)
    gmax = max(mx)
    sums = [pen.shard_sums(gmax) for pen in pens]
    total = sums[0].copy()
    for s in sums[1:]:
        total += s  # fixed shard order
    for pen in pens:
        pen.shard_centre(total)
    return pens


@pytest.mark.parametrize("name,prec", [("f2", 0), ("f2", 3), ("mc", 0), ("mc", 1)],
                         ids=["f2-fp64", "f2-df64", "mc-fp64", "mc-fp32"])
def test_shard_products_sum_to_the_unsharded_product(abi, name, prec):
    """Three uneven shards: the summed shard products equal the unsharded pencil's products
    (1e-12 relative with FP64-accurate factors; the FP32 copies at their own resolution),
    every shard reports the global energy, and the shards' centred factors are the rows of
    the unsharded ones."""
    w, h, eri, th, rows, wts = _case(name)
    ctx = abi.Context(0)
    sysd = ctx.system(w.n_orb, w.n_alpha, w.n_beta, w.n_hidden, h, eri)
    full = ctx.build_OG(sysd, th, rows=rows, weights=wts, prec=prec)
    E = full.info().energy
    parts = _split(len(rows), 3)
    pens = _build_shards(abi, [ctx] * 3, w, h, eri, th, rows, wts, parts, prec)
    for pen in pens:
        assert pen.info().energy == pytest.approx(E, rel=1e-13)
    P1 = w.n_params + 1
    Of = full.export(abi.EXPORT_O)
    Os = np.concatenate([pen.export(abi.EXPORT_O) for pen in pens])
    assert _rel(Os, Of) <= 1e-13
    rng = np.random.default_rng(11)
    tol = 2e-6 if prec == 1 else 1e-12
    for sym in (abi.LM_SYM_NONE, abi.LM_SYM_HALF):
        for _ in range(2):
            v = rng.standard_normal(P1)
            hr, sr = np.zeros(P1), np.zeros(P1)
            full.apply(v, hr, sr, sym=sym, prec=prec)
            hs, ss = np.zeros(P1), np.zeros(P1)
            for pen in pens:
                a, b = np.zeros(P1), np.zeros(P1)
                pen.apply(v, a, b, sym=sym, prec=prec)
                hs += a
                ss += b
            assert _rel(hs, hr) <= tol and _rel(ss, sr) <= tol
    # a shard between build and centring is refused by the product and the solver
    sh, m = ctx.shard_build(sysd, th, rows[parts[0]].copy(),
                            None if wts is None else wts[parts[0]].copy(), prec=prec)
    with pytest.raises(abi.LMError) as e:
        sh.apply(np.ones(P1), np.zeros(P1))
    assert e.value.code == abi.LM_ERR_ARG
    with pytest.raises(abi.LMError):
        sh.irl_step(m=10, k=1)
    for pen in pens + [full, sh]:
        pen.free()
    ctx.close()


class _HostSum:
    """Sum of one vector per shard thread, added in shard order, handed to every shard."""

    def __init__(self, k):
        self.k = k
        self.slots = [None] * k
        self.bar = threading.Barrier(k, timeout=60)

    def reduce(self, r, vec):
        self.slots[r] = np.array(vec, copy=True)
        self.bar.wait()
        tot = self.slots[0].copy()
        for s in self.slots[1:]:
            tot += s
        self.bar.wait()
        vec[:] = tot
        return 0


def _sharded_solve(abi, name, prec, k, where):
    import torch
    w, h, eri, th, rows, wts = _case(name)
    ctxs = [abi.Context(0) for _ in range(k)]
    parts = _split(len(rows), k)
    pens = _build_shards(abi, ctxs, w, h, eri, th, rows, wts, parts, prec)
    P = w.n_params
    outs = [dict() for _ in range(k)]
    hs = _HostSum(k)
    streams = [torch.cuda.Stream() for _ in range(k)]

    def dev_reduce(r):
        # sum the shards' device vectors in shard order, on this shard's stream
        def red(ptr, n, st):
            ext = torch.cuda.ExternalStream(st)
            ext.synchronize()

            class View:
                __cuda_array_interface__ = {"shape": (n,), "typestr": "<f8",
                                            "data": (ptr, False), "version": 3}
            t = torch.as_tensor(View(), device="cuda")
            hs.slots[r] = t
            hs.bar.wait()
            tot = hs.slots[0].clone()
            for s in hs.slots[1:]:
                tot += s
            torch.cuda.synchronize()
            hs.bar.wait()
            t.copy_(tot)
            torch.cuda.synchronize()
            return 0
        return red

    def run(r):
        try:
            dth = np.zeros(P)
            c = np.zeros(P + 1)
            red = (lambda vec, n, st: hs.reduce(r, vec)) if where == abi.LM_REDUCE_HOST \
                else dev_reduce(r)
            res = pens[r].irl_step_sharded(red, where=where, m=w.m, k=w.k, tol=w.tol,
                                           max_restarts=500, prec=prec, dtheta_out=dth, c_out=c,
                                           stream=streams[r])
            outs[r].update(res=res, dth=dth, c=c)
        except Exception as e:  # reported by the main thread
            outs[r]["err"] = e
            hs.bar.abort()

    ths = [threading.Thread(target=run, args=(r,)) for r in range(k)]
    for t in ths:
        t.start()
    for t in ths:
        t.join(timeout=600)
    for o in outs:
        assert "err" not in o, o.get("err")
    ctx = ctxs[0]
    sysd = ctx.system(w.n_orb, w.n_alpha, w.n_beta, w.n_hidden, h, eri)
    full = ctx.build_OG(sysd, th, rows=rows, weights=wts, prec=prec)
    dref = np.zeros(P)
    ref = full.irl_step(m=w.m, k=w.k, tol=w.tol, max_restarts=500, prec=prec, dtheta_out=dref)
    full.free()
    for pen in pens:
        pen.free()
    for c in ctxs:
        c.close()
    return outs, ref, dref


@pytest.mark.parametrize("name,prec,k", [("f2", 3, 2), ("mc", 0, 3), ("mc", 1, 2)],
                         ids=["f2-df64-2", "mc-fp64-3", "mc-fp32-2"])
def test_irl_sharded_matches_unsharded(abi, name, prec, k):
    """irl_step_sharded on K shards (threads, host-staged reduction) against irl_step on the
    unsharded pencil: the same eigenvalue (1e-10 relative), update (1e-8) and product
    count, and bitwise the same result on every shard (replicated Lanczos work)."""
    outs, ref, dref = _sharded_solve(abi, name, prec, k, abi.LM_REDUCE_HOST)
    for o in outs:
        r = o["res"]
        assert r.status in (abi.IRL_OK, abi.IRL_BREAKDOWN_INVARIANT), r.status
        assert r.lambda_ == pytest.approx(ref.lambda_, rel=1e-10)
        assert _rel(o["dth"], dref) <= 1e-8
        assert r.n_matvec == ref.n_matvec
        assert r.energy == pytest.approx(ref.energy, rel=1e-13)
    for o in outs[1:]:
        assert o["res"].lambda_ == outs[0]["res"].lambda_
        assert np.array_equal(o["c"], outs[0]["c"])


@pytest.mark.parametrize("k", [1, 2])
def test_irl_sharded_device_reduction(abi, k):
    """The device-side reduction form (the callback enqueues the sum on the solver's stream,
    as an NCCL all-reduce would): one shard with an identity reduction, and two shards
    summed on the device, against the unsharded solve."""
    outs, ref, dref = _sharded_solve(abi, "mc", 0, k, abi.LM_REDUCE_DEVICE)
    for o in outs:
        assert o["res"].lambda_ == pytest.approx(ref.lambda_, rel=1e-10)
        assert _rel(o["dth"], dref) <= 1e-8


def _gloo_rank(rank, world, port, q):
    """One rank of the world-2 run: its own context and row shard on cuda:0, statistics
    and products summed with gloo all-reduces on host tensors."""
    import torch
    import torch.distributed as dist
    try:
        os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        dist.init_process_group("gloo", rank=rank, world_size=world)
        from paper_2601_01437_gb300 import abi
        w, h, eri, th, rows, wts = _case("mc")
        idx = np.array_split(np.arange(len(rows)), world)[rank]
        ctx = abi.Context(0)
        sysd = ctx.system(w.n_orb, w.n_alpha, w.n_beta, w.n_hidden, h, eri)
        pen, m = ctx.shard_build(sysd, th, rows[idx].copy(), wts[idx].copy(), prec=abi.LM_FP64)
        t = torch.tensor([m], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        sums = torch.from_numpy(pen.shard_sums(float(t.item())))
        dist.all_reduce(sums)
        pen.shard_centre(sums.numpy())

        def red(vec, n, st):
            dist.all_reduce(torch.from_numpy(vec))
            return 0
        dth = np.zeros(w.n_params)
        res = pen.irl_step_sharded(red, m=w.m, k=w.k, tol=w.tol, max_restarts=500,
                                   dtheta_out=dth)
        pen.free()
        ctx.close()
        dist.destroy_process_group()
        q.put((rank, res.lambda_, res.energy, res.n_matvec, dth))
    except Exception as e:  # pragma: no cover - reported to the parent
        q.put((rank, repr(e)))


def test_irl_sharded_gloo_world2(abi):
    """Two processes, one row shard each, gloo all-reduces of the P+3 statistics and of
    every product: both ranks return the unsharded pencil's eigenvalue and update."""
    import torch.multiprocessing as mp
    ctxm = mp.get_context("spawn")
    q = ctxm.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctxm.Process(target=_gloo_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=600) for _ in procs]
    for p in procs:
        p.join(timeout=120)
    for g in got:
        assert len(g) == 5, g
    w, h, eri, th, rows, wts = _case("mc")
    ctx = abi.Context(0)
    full = ctx.build_OG(ctx.system(w.n_orb, w.n_alpha, w.n_beta, w.n_hidden, h, eri), th,
                        rows=rows, weights=wts)
    dref = np.zeros(w.n_params)
    ref = full.irl_step(m=w.m, k=w.k, tol=w.tol, max_restarts=500, dtheta_out=dref)
    full.free()
    ctx.close()
    for rank, lam, E, nmv, dth in got:
        assert lam == pytest.approx(ref.lambda_, rel=1e-10)
        assert E == pytest.approx(ref.energy, rel=1e-13)
        assert nmv == ref.n_matvec
        assert _rel(dth, dref) <= 1e-8
    assert got[0][1] == got[1][1]
