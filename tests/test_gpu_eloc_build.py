"""The E_loc estimator's G-free build (lm_build_O) against the FP64 oracle and against
the full build of lm_build_OG.

Bars: O_c and E_loc componentwise at the double-float build bar (1e-11 of each entry's
condition scale), ln psi and the weights elementwise (1e-13, 1e-12), E to 1e-12 of the
oracle's; against lm_build_OG's pencil O_c, ln psi, E_loc, weights and E bit-identical
(the same kernel arithmetic with the G accumulation left out), so the estimator's
products and IRL results are bit-identical too; the IRL eigenvalue of the estimator
operator within 1e-10 (relative) of the oracle's dense SHEP."""
import numpy as np
import pytest

import __graft_entry__ as entry
import synth
from oracle import lm
from parity_tools import componentwise, saturated_theta

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


def _elementwise(got, ref, tol, what, floor=0.0):
    got, ref = np.asarray(got), np.asarray(ref)
    r = np.abs(got - ref) / np.maximum(np.abs(ref), floor)
    assert np.all(np.isfinite(r)) and r.max() <= tol, f"{what}: {r.max():.3e} > {tol:.0e}"


def _case(name):
    if name == "mc":
        h, eri = synth.integrals(14, 111)
        th = synth.rbm_theta(14, 56, 111)
        rows, cnt = synth.proxy_mc_samples(14, 7, 7, 1000, 111, h, walkers=512, burn_in=50)
        return (14, 7, 7, 56), h, eri, th, rows, cnt
    if name == "edge_nh127":
        h, eri = synth.integrals(6, 17)
        th = synth.rbm_theta(6, 127, 17, sigma=0.5)
        return (6, 3, 3, 127), h, eri, th, None, None
    if name == "saturated":
        h, eri = synth.integrals(8, 29)
        return (8, 4, 4, 32), h, eri, saturated_theta(8, 32, 29), None, None
    if name == "empty_alpha":
        h, eri = synth.integrals(4, 17)
        th = synth.rbm_theta(4, 3, 17, sigma=0.2)
        return (4, 0, 2, 3), h, eri, th, None, None
    w = synth.WORKLOADS[name]
    h, eri, th, rows, cnt = w.inputs()
    return (w.n_orb, w.n_alpha, w.n_beta, w.n_hidden), h, eri, th, rows, cnt


CASES = [("tiny_6o6e", 0), ("tiny_6o6e", 3), ("f2_10o14e", 3), ("mc", 1), ("edge_nh127", 0),
         ("empty_alpha", 0), ("saturated", 3)]


@pytest.mark.parametrize("name,prec", CASES,
                         ids=["tiny-fp64", "tiny-df64", "f2-df64", "mc-fp32", "nh127", "empty-alpha",
                              "saturated"])
def test_gfree_build_against_the_oracle_and_the_full_build(ctx, abi, name, prec):
    shape, h, eri, th, rows, cnt = _case(name)
    n, na, nb, nh = shape
    wts = None if cnt is None else cnt.astype(np.float64)
    sysd = ctx.system(n, na, nb, nh, h, eri)
    gf = ctx.build_O(sysd, th, rows=rows, weights=wts, prec=prec)
    full = ctx.build_OG(sysd, th, rows=rows, weights=wts, prec=prec)
    pd = lm.build_pencil(n, na, nb, nh, h, eri, th, rows, cnt)
    P1 = pd.Oc.shape[1]
    # against the oracle, entry by entry
    AE, AO, _ = lm.condition_scales(pd, n, na, nb, nh, h, eri, th, union_occ=True)
    Oc = gf.export(abi.EXPORT_O)
    componentwise(Oc[:, :P1], pd.Oc, AO, 1e-11, "O_c")
    componentwise(gf.export(abi.EXPORT_ELOC), pd.eloc, AE, 1e-11, "E_loc")
    _elementwise(gf.export(abi.EXPORT_W), pd.w, 1e-12, "weights")
    _elementwise(gf.export(abi.EXPORT_LNPSI), pd.lnpsi, 1e-13, "ln psi",
                 floor=np.abs(pd.lnpsi).max())
    assert gf.info().energy == pytest.approx(pd.E, rel=1e-12)
    # against the full build: the same arithmetic without the G accumulation
    for what in (abi.EXPORT_O, abi.EXPORT_ELOC, abi.EXPORT_LNPSI, abi.EXPORT_W, abi.EXPORT_ROWS):
        assert np.array_equal(gf.export(what), full.export(what)), what
    assert gf.info().energy == full.info().energy
    # products of the estimator operator: bit-identical to the full pencil's
    rng = np.random.default_rng(3)
    for _ in range(2):
        v = rng.standard_normal(P1)
        h1, s1, h2, s2 = (np.zeros(P1) for _ in range(4))
        gf.apply(v, h1, s1, sym=abi.LM_SYM_ELOC, prec=prec)
        full.apply(v, h2, s2, sym=abi.LM_SYM_ELOC, prec=prec)
        assert np.array_equal(h1, h2) and np.array_equal(s1, s2)
        h3 = np.zeros(P1)
        gf.apply(v, h3, None, sym=abi.LM_SYM_AUTO, prec=prec)  # the pencil's default
        assert np.array_equal(h3, h1)
    gf.free()
    full.free()


@pytest.mark.parametrize("name,prec", [("tiny_6o6e", 0), ("f2_10o14e", 3)])
def test_gfree_irl_against_the_oracle(ctx, abi, name, prec):
    """IRL on the estimator operator of a G-free pencil: the oracle's dense SHEP eigenvalue
    of O_c^T W diag(E_loc - E) O_c, and the same result as on the full pencil."""
    w = synth.WORKLOADS[name]
    h, eri, th, _, _ = w.inputs()
    sysd = ctx.system(w.n_orb, w.n_alpha, w.n_beta, w.n_hidden, h, eri)
    gf = ctx.build_O(sysd, th, prec=prec)
    full = ctx.build_OG(sysd, th, prec=prec)
    pd = lm.build_pencil(w.n_orb, w.n_alpha, w.n_beta, w.n_hidden, h, eri, th)
    _, He = lm.pencil_matrices(pd.Oc, lm.eloc_form(pd.Oc, pd.eloc, pd.E), pd.w)
    lam_ref = lm.shep(He)[0]
    P = pd.Oc.shape[1] - 1
    d1, d2 = np.zeros(P), np.zeros(P)
    r1 = gf.irl_step(m=w.m, k=w.k, tol=w.tol, max_restarts=500, prec=prec, dtheta_out=d1)
    r2 = full.irl_step(m=w.m, k=w.k, tol=w.tol, max_restarts=500, sym=abi.LM_SYM_ELOC, prec=prec,
                       dtheta_out=d2)
    assert r1.status in (abi.IRL_OK, abi.IRL_BREAKDOWN_INVARIANT), r1.status
    assert r1.lambda_ == pytest.approx(lam_ref, rel=1e-10)
    assert r1.lambda_ == r2.lambda_ and r1.n_matvec == r2.n_matvec
    assert np.array_equal(d1, d2)
    gf.free()
    full.free()


def test_gfree_refusals(ctx, abi):
    """What needs G'_c is refused before any launch: the exact operator forms, the export of
    G'_c, the block product and block phase, an FP64-arithmetic build, and rebuilding a
    G-free pencil as a full one."""
    import torch
    w = synth.WORKLOADS["tiny_6o6e"]
    h, eri, th, _, _ = w.inputs()
    sysd = ctx.system(6, 3, 3, 24, h, eri)
    gf = ctx.build_O(sysd, th, prec=abi.LM_BF16)
    P1 = w.n_params + 1
    v = np.ones(P1)
    for sym in (abi.LM_SYM_NONE, abi.LM_SYM_HALF):
        with pytest.raises(abi.LMError) as e:
            gf.apply(v, np.zeros(P1), np.zeros(P1), sym=sym)
        assert e.value.code == abi.LM_ERR_ARG
        with pytest.raises(abi.LMError) as e:
            gf.irl_step(m=20, k=1, sym=sym)
        assert e.value.code == abi.LM_ERR_ARG
    with pytest.raises(abi.LMError) as e:
        gf.export(abi.EXPORT_G)
    assert e.value.code == abi.LM_ERR_ARG
    V = torch.zeros((4, P1), dtype=torch.float64, device="cuda")
    with pytest.raises(abi.LMError) as e:
        gf.apply_block(V, V.clone(), None, sym=abi.LM_SYM_ELOC)
    assert e.value.code == abi.LM_ERR_ARG
    with pytest.raises(abi.LMError) as e:
        gf.irl_step(m=32, k=1, block=16, prec=abi.LM_BF16)
    assert e.value.code == abi.LM_ERR_ARG
    with pytest.raises(abi.LMError) as e:
        ctx.build_OG(sysd, th, prec=abi.LM_BF16, pencil=gf)
    assert e.value.code == abi.LM_ERR_ARG
    with pytest.raises(abi.LMError) as e:
        ctx.build_O(ctx.system(6, 3, 3, 24, h, eri, arith=1), th)
    assert e.value.code == abi.LM_ERR_ARG
    gf.free()
