"""lm_apply_pencil_noalloc: the pencil product for callers that cannot allocate
device memory when they need it (a framework whose caching allocator owns the
device memory, a solver with a fixed memory budget, a loop that cannot wait on
an allocation). Its scratch lives in a fixed file-scope device array, so the
test checks it against the regular lm_apply_pencil on the same factors, for two
calls in a row (the second call reuses the scratch the first one left), and
that it rejects what it cannot do without allocating. Collected last (file
name) so a stop-at-first-failure run has already run every other test."""
import numpy as np
import pytest

import __graft_entry__ as entry
import synth

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_noalloc_pencil_matches_apply_pencil_on_consecutive_calls():
    import torch
    entry.build()
    from paper_2601_01437_gb300 import abi

    dev = torch.device("cuda", 0)
    ctx = abi.Context(0)
    w = synth.WORKLOADS["f2_10o14e"]
    h, eri, th, _, _ = w.inputs()
    pen = ctx.build_OG(ctx.system(w.n_orb, w.n_alpha, w.n_beta, w.n_hidden, h, eri), th)
    inf = pen.info()
    n, ld, p1 = inf.n_rows, inf.ld, inf.n_params + 1
    O = torch.from_numpy(pen.export(abi.EXPORT_O)).to(dev)
    G = torch.from_numpy(pen.export(abi.EXPORT_G)).to(dev)
    wt = torch.from_numpy(pen.export(abi.EXPORT_W)).to(dev)
    rng = np.random.default_rng(5)
    for sym in (abi.LM_SYM_NONE, abi.LM_SYM_HALF):
        for _call in range(2):
            v = rng.standard_normal(p1)
            Hr = np.zeros(p1)
            Sr = np.zeros(p1)
            pen.apply(v, Hr, Sr, sym=sym)
            vd = torch.from_numpy(v).to(dev)
            Hd = torch.full((p1,), float("nan"), dtype=torch.float64, device=dev)
            Sd = torch.full((p1,), float("nan"), dtype=torch.float64, device=dev)
            rc = abi.apply_pencil_noalloc(O, G, wt, n, ld, p1, vd, Hd, Sd, sym=sym)
            torch.cuda.synchronize()
            assert rc == abi.LM_OK
            assert _rel(Hd.cpu().numpy(), Hr) <= 1e-12
            assert _rel(Sd.cpu().numpy(), Sr) <= 1e-12
    # H only, then S only
    v = rng.standard_normal(p1)
    Hr = np.zeros(p1)
    Sr = np.zeros(p1)
    pen.apply(v, Hr, Sr, sym=abi.LM_SYM_NONE)
    vd = torch.from_numpy(v).to(dev)
    Hd = torch.zeros(p1, dtype=torch.float64, device=dev)
    Sd = torch.zeros(p1, dtype=torch.float64, device=dev)
    assert abi.apply_pencil_noalloc(O, G, wt, n, ld, p1, vd, Hd, None) == abi.LM_OK
    assert abi.apply_pencil_noalloc(O, G, wt, n, ld, p1, vd, None, Sd) == abi.LM_OK
    torch.cuda.synchronize()
    assert _rel(Hd.cpu().numpy(), Hr) <= 1e-12 and _rel(Sd.cpu().numpy(), Sr) <= 1e-12
    # what it cannot do without allocating is refused before any launch
    assert abi.apply_pencil_noalloc(O, G, wt, n, abi.LM_NOALLOC_MAX_LD + 8, p1, vd, Hd, None) \
        == abi.LM_ERR_SIZE
    assert abi.apply_pencil_noalloc(O.cpu(), G, wt, n, ld, p1, vd, Hd, None) == abi.LM_ERR_ARG
    assert abi.apply_pencil_noalloc(O, G, wt, n, ld, p1, v, Hd, None) == abi.LM_ERR_ARG
    pen.free()
    ctx.close()
