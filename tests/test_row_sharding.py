"""The row-sharded form of the path on CPU ranks (gloo, world size 2).

Each rank holds a contiguous share of the determinant rows (exact sector,
|psi|^2 weights) and builds their ln psi, O, E_loc and G with the oracle. The
exchange plan a multi-GPU build would follow is then carried out with
torch.distributed: one max of ln psi (the weights' shift), one sum of the
weight normaliser and the weighted sums behind E and <O> (P+3 numbers), after
which every rank centres its own rows; each pencil product is a local partial
y_H, y_S followed by one sum of a 2(P+1) vector. The result must be the
unsharded oracle pencil, and identical on every rank."""
import os
import socket
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import synth
    from oracle import fock, native

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    w = synth.WORKLOADS["tiny_6o6e"]
    h, eri, th, _, _ = w.inputs()
    dets = fock.sector_dets(w.n_orb, w.n_alpha, w.n_beta)
    mine = np.array_split(dets, world)[rank]
    lnpsi, O, eloc, G = native.rows(w.n_orb, w.n_alpha, w.n_beta, w.n_hidden, h, eri, th, mine)
    # weights exp(2 (ln psi - max)) / sum: a global max, then a global sum
    m = torch.tensor([lnpsi.max()], dtype=torch.float64)
    dist.all_reduce(m, op=dist.ReduceOp.MAX)
    e = np.exp(2.0 * (lnpsi - m.item()))
    sums = torch.from_numpy(np.concatenate([[e.sum(), e @ eloc], e @ O]))
    dist.all_reduce(sums)
    s = sums.numpy()
    E, Obar, wl = s[1] / s[0], s[2:] / s[0], e / s[0]
    # local centring with the global statistics
    Oc = O - Obar[None, :]
    Oc[:, 0] = 1.0
    Gpc = G - eloc[:, None] * Obar[None, :]
    Gpc[:, 0] = eloc
    Gpc = Gpc - E * Oc
    v = np.random.default_rng(3).standard_normal(O.shape[1])
    WO = Oc * wl[:, None]
    y = torch.from_numpy(np.concatenate([WO.T @ (Gpc @ v), WO.T @ (Oc @ v)]))
    dist.all_reduce(y)
    out.put((rank, float(E), y.numpy()))
    dist.destroy_process_group()


def test_row_sharded_pencil_gloo_world2():
    import torch.multiprocessing as mp

    import synth
    from oracle import lm

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=180) for _ in range(2)), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    w = synth.WORKLOADS["tiny_6o6e"]
    h, eri, th, _, _ = w.inputs()
    pd = lm.build_pencil(w.n_orb, w.n_alpha, w.n_beta, w.n_hidden, h, eri, th)
    v = np.random.default_rng(3).standard_normal(pd.Oc.shape[1])
    yH, yS = lm.pencil_apply(pd.Oc, pd.Gpc, pd.w, v)
    ref = np.concatenate([yH, yS])
    (_, E0, y0), (_, E1, y1) = res
    assert np.array_equal(y0, y1) and E0 == E1
    assert abs(E0 - pd.E) <= 1e-13 * abs(pd.E)
    assert np.linalg.norm(y0 - ref) <= 1e-12 * np.linalg.norm(ref)
