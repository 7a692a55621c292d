"""Streamed pencils (lm_build_streamed): O_c and G'_c rebuilt chunk by chunk inside every
product, against the resident pencil of lm_build_OG and the FP64 oracle.

Bars: the rows equal the resident pencil's; ln psi equals it to 1e-13 of max |ln psi| and
the weights to 1e-13 (a resident sector pencil takes ln psi, psi and tanh z_j from
per-determinant tables formed in double-float arithmetic, a streamed one forms them per row
and per connection in FP64 and double-float); E_loc equals it to 1e-12 of each entry's
condition scale (the same terms in another order); products equal the resident
pencil's to 1e-12 relative with FP64-accurate factors, FP32 copies to 1e-6; energy to
1e-13; the IRL
eigenvalue to 1e-10 of the oracle's (FP64-accurate factors) or within 1e-9 Ha after the
FP64 continuation (FP32 factors)."""
import numpy as np
import pytest

import __graft_entry__ as entry
import synth
from oracle import lm
from parity_tools import componentwise

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


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


CASES = {
    # 400 determinants in chunks of 97 (the last ragged)
    "tiny": (synth.WORKLOADS["tiny_6o6e"], 97),
    # 14,400 determinants in chunks of 4,000
    "f2": (synth.WORKLOADS["f2_10o14e"], 4000),
    # 1,000 LiCl-shaped MC rows with multiplicities, chunks of 300
    "mc": (synth.Workload("mc", 14, 7, 7, 56, exact=False, n_samples=1000, m=20, k=1), 300),
}


def _pair(ctx, abi, name, prec, arith=0):
    w, chunk = CASES[name]
    h, eri, th, rows, cnt = w.inputs()
    wts = None if cnt is None else cnt.astype(np.float64)
    sysd = ctx.system(w.n_orb, w.n_alpha, w.n_beta, w.n_hidden, h, eri, arith=arith)
    full = ctx.build_OG(sysd, th, rows=rows, weights=wts, prec=prec)
    st = ctx.build_streamed(sysd, th, chunk, rows=rows, weights=wts, prec=prec)
    return w, h, eri, th, rows, cnt, full, st


@pytest.mark.parametrize("name,prec,arith", [("tiny", 0, 0), ("tiny", 3, 1), ("f2", 3, 0),
                                             ("mc", 0, 0), ("mc", 1, 0)],
                         ids=["tiny-fp64", "tiny-df64-fp64build", "f2-df64", "mc-fp64",
                              "mc-fp32"])
def test_streamed_products_equal_resident(ctx, abi, name, prec, arith):
    w, h, eri, th, rows, cnt, full, st = _pair(ctx, abi, name, prec, arith)
    assert st.info().energy == pytest.approx(full.info().energy, rel=1e-13)
    assert np.array_equal(st.export(abi.EXPORT_ROWS), full.export(abi.EXPORT_ROWS))
    l_st, l_full = st.export(abi.EXPORT_LNPSI), full.export(abi.EXPORT_LNPSI)
    assert np.abs(l_st - l_full).max() <= 1e-13 * np.abs(l_full).max()
    pd = lm.build_pencil(w.n_orb, w.n_alpha, w.n_beta, w.n_hidden, h, eri, th, rows, cnt)
    AE, _, _ = lm.condition_scales(pd, w.n_orb, w.n_alpha, w.n_beta, w.n_hidden, h, eri, th,
                                   union_occ=True)
    componentwise(st.export(abi.EXPORT_ELOC), full.export(abi.EXPORT_ELOC), AE, 1e-12,
                  "E_loc, streamed vs resident")
    assert _rel(st.export(abi.EXPORT_W), full.export(abi.EXPORT_W)) <= 1e-13
    P1 = w.n_params + 1
    rng = np.random.default_rng(4)
    tol = 1e-6 if prec == abi.LM_FP32 else 1e-12
    for sym in (abi.LM_SYM_NONE, abi.LM_SYM_HALF, abi.LM_SYM_ELOC):
        for _ in range(2):
            v = rng.standard_normal(P1)
            hf, sf, hs, ss = (np.zeros(P1) for _ in range(4))
            full.apply(v, hf, sf, sym=sym, prec=prec)
            st.apply(v, hs, ss, sym=sym, prec=prec)
            assert _rel(hs, hf) <= tol and _rel(ss, sf) <= tol
    with pytest.raises(abi.LMError) as e:
        st.export(abi.EXPORT_O)
    assert e.value.code == abi.LM_ERR_ARG
    full.free()
    st.free()


@pytest.mark.parametrize("name,prec", [("tiny", 0), ("f2", 3), ("mc", 1)])
def test_streamed_irl_against_the_oracle(ctx, abi, name, prec):
    w, h, eri, th, rows, cnt, full, st = _pair(ctx, abi, name, prec)
    ref = lm.lm_step(w.n_orb, w.n_alpha, w.n_beta, w.n_hidden, h, eri, th, rows, cnt)
    dth = np.zeros(w.n_params)
    res = st.irl_step(m=w.m, k=w.k, tol=w.tol, max_restarts=500, prec=prec, dtheta_out=dth)
    rf = full.irl_step(m=w.m, k=w.k, tol=w.tol, max_restarts=500, prec=prec)
    assert res.status in (abi.IRL_OK, abi.IRL_BREAKDOWN_INVARIANT), res.status
    if prec == abi.LM_FP32:
        assert abs(res.lambda_ - ref["lam"]) <= 1e-9
    else:
        assert res.lambda_ == pytest.approx(ref["lam"], rel=1e-10)
    assert _rel(dth, ref["dtheta"]) <= (1e-6 if prec == abi.LM_FP32 else 1e-8)
    if prec != abi.LM_FP32:  # same products up to rounding: the same number of them
        assert res.n_matvec == rf.n_matvec
    full.free()
    st.free()


def test_streamed_refusals(ctx, abi):
    import torch
    w, h, eri, th, rows, cnt, full, st = _pair(ctx, abi, "tiny", abi.LM_BF16)
    V = torch.zeros((2, w.n_params + 1), dtype=torch.float64, device="cuda")
    with pytest.raises(abi.LMError) as e:
        st.apply_block(V, V.clone(), None)
    assert e.value.code == abi.LM_ERR_ARG
    with pytest.raises(abi.LMError) as e:
        ctx.build_streamed(ctx.system(6, 3, 3, 24, h, eri), th, 0)
    assert e.value.code == abi.LM_ERR_ARG
    full.free()
    st.free()
