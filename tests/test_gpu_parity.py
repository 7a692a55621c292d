"""GPU parity: the sm_103a library through its C ABI against the FP64 oracle.

Bars (stated per test): bit-exact sector enumeration, connectivity and signs;
1e-12 relative on the FP64 build (O_c, G'_c, E_loc, ln psi, weights);
1e-10 relative (2-norm) on FP64 pencil products and IRL eigenvalues;
1e-8 relative on the update Delta theta; mixed precision within 1e-9 Ha of
the FP64 eigenvalue after FP64 refinement.
"""
import numpy as np
import pytest

import __graft_entry__ as entry
import oracle
import synth
from oracle import fock, lm, native
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


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


def _mc_rows(n, na, nb, count, seed, h):
    return synth.proxy_mc_samples(n, na, nb, count, seed, h, walkers=512, burn_in=50)


# ------------------------------------------------------------------ K1
@pytest.mark.parametrize("n,na,nb", [(2, 1, 1), (6, 3, 3), (6, 2, 2), (7, 5, 5), (8, 5, 5),
                                     (10, 7, 7), (10, 6, 6), (11, 9, 9), (9, 0, 4), (32, 1, 1)])
def test_sector_enumeration_bit_exact(ctx, n, na, nb):
    got = ctx.enumerate_sector(n, na, nb)
    want = fock.sector_dets(n, na, nb)
    assert got.dtype == np.uint64 and np.array_equal(got, want)


# ------------------------------------------------------------------ K3/K4
def _check_connections(ctx, n, na, nb, h, eri, rows):
    sysd = ctx.system(n, na, nb, 1, h, eri)
    cap = 4096
    od, sg, hv, cnt = ctx.debug_connections(sysd, rows, cap)
    for i, x in enumerate(rows):
        ro_d, ro_h, ro_s = native.connections(n, na, nb, h, eri, int(x))
        assert cnt[i] == len(ro_d)
        assert od[i, 0] == x and sg[i, 0] == 1
        gi = np.argsort(od[i, :cnt[i]], kind="stable")
        oi = np.argsort(ro_d, kind="stable")
        assert np.array_equal(od[i, :cnt[i]][gi], ro_d[oi]), "connectivity differs"
        assert np.array_equal(sg[i, :cnt[i]][gi].astype(np.int32), ro_s[oi]), "sign differs"
        scale = np.abs(ro_h).max()
        assert np.abs(hv[i, :cnt[i]][gi] - ro_h[oi]).max() <= 1e-13 * scale


def test_connections_bit_exact_tiny_all_rows(ctx):
    h, eri = synth.integrals(6, 111)
    _check_connections(ctx, 6, 3, 3, h, eri, fock.sector_dets(6, 3, 3))


@pytest.mark.parametrize("n,na,nb,nrows", [(10, 7, 7, 64), (14, 7, 7, 16), (9, 0, 4, 32),
                                           (7, 7, 3, 20)])
def test_connections_bit_exact_sampled(ctx, n, na, nb, nrows):
    h, eri = synth.integrals(n, 5)
    dets = fock.sector_dets(n, na, nb) if n <= 10 else _mc_rows(n, na, nb, 400, 5, h)[0]
    rng = np.random.default_rng(0)
    rows = dets[rng.choice(len(dets), size=min(nrows, len(dets)), replace=False)]
    _check_connections(ctx, n, na, nb, h, eri, rows)


# ------------------------------------------------------------------ build
def _build_both(ctx, abi, n, na, nb, nh, h, eri, theta, rows=None, counts=None, prec=0, arith=0):
    sysd = ctx.system(n, na, nb, nh, h, eri, arith=arith)
    w = None if counts is None else counts.astype(np.float64)
    pen = ctx.build_OG(sysd, theta, rows=rows, weights=w, prec=prec)
    pd = lm.build_pencil(n, na, nb, nh, h, eri, theta, rows, counts)
    pen.sysargs = (n, na, nb, nh, h, eri, theta)
    pen.arith = arith
    return pen, pd


def _elementwise(got, ref, tol, what, floor=0.0):
    """Entry by entry: |got(x) - ref(x)| <= tol * max(|ref(x)|, floor)."""
    got = np.asarray(got)
    ref = np.asarray(ref)
    r = np.abs(got - ref) / np.maximum(np.abs(ref), floor)
    assert np.all(np.isfinite(r)) and r.max() <= tol, \
        f"{what}: entry {int(np.argmax(r))} relative error {r.max():.3e} > {tol:.0e}"


# The FP64-accurate builds' componentwise bars: |error| <= tol * (first-order rounding scale)
# per entry (lm.condition_scales). Native FP64 (unit roundoff 2^-53 = 1.1e-16) is held to
# 1e-12 (~9,000 u); the double-float build (pairs of FP32 carried through error-free
# transformations, ~2^-44 = 5.7e-14 per operation) to 1e-11 (~175 of its u).
BUILD_TOL = {0: 1e-11, 1: 1e-12}


def _check_build(abi, pen, pd):
    """The FP64-accurate build against the oracle, entry by entry: O_c, G'_c and E_loc to
    a componentwise bar relative to each entry's own condition scale (so an error confined
    to the small hidden-unit columns cannot hide behind the large ones), ln psi and the
    weights relative to their own size, plus the energy."""
    P1 = pd.Oc.shape[1]
    tol = BUILD_TOL[pen.arith]
    inf = pen.info()
    assert inf.energy == pytest.approx(pd.E, rel=1e-12)
    Oc = pen.export(abi.EXPORT_O)
    Gc = pen.export(abi.EXPORT_G)
    assert np.all(Oc[:, P1:] == 0) and np.all(Gc[:, P1:] == 0)
    # the build forms G of an orbital occupied in x as (all connections) - (connections
    # that empty it), so its rounding scales with both sums: union-occupation scale
    AE, AO, AG = lm.condition_scales(pd, *pen.sysargs, union_occ=True)
    eo = componentwise(Oc[:, :P1], pd.Oc, AO, tol, "O_c")
    eg = componentwise(Gc[:, :P1], pd.Gpc, AG, tol, "G'_c")
    ee = componentwise(pen.export(abi.EXPORT_ELOC), pd.eloc, AE, tol, "E_loc")
    print(f"\n  componentwise errors / scale: O_c {eo:.2e}, G'_c {eg:.2e}, E_loc {ee:.2e}")
    # whole-matrix norms as well (the earlier bar; kept beside the componentwise one)
    assert _rel(Oc[:, :P1], pd.Oc) <= 1e-12
    assert _rel(Gc[:, :P1], pd.Gpc) <= 1e-12
    _elementwise(pen.export(abi.EXPORT_W), pd.w, 1e-12, "weights")
    lnpsi = pen.export(abi.EXPORT_LNPSI)
    _elementwise(lnpsi, pd.lnpsi, 1e-13, "ln psi", floor=np.abs(pd.lnpsi).max())
    assert np.array_equal(pen.export(abi.EXPORT_ROWS), pd.rows)


ARITHS = pytest.mark.parametrize("arith", [0, 1], ids=["df64", "fp64"])


@ARITHS
def test_build_parity_tiny(ctx, abi, arith):
    w = synth.WORKLOADS["tiny_6o6e"]
    h, eri, th, _, _ = w.inputs()
    pen, pd = _build_both(ctx, abi, 6, 3, 3, 24, h, eri, th, arith=arith)
    _check_build(abi, pen, pd)
    pen.free()


@ARITHS
def test_build_parity_f2_full_size(ctx, abi, arith):
    """All 14,400 rows of the F2-shaped workload, element by element."""
    w = synth.WORKLOADS["f2_10o14e"]
    h, eri, th, _, _ = w.inputs()
    pen, pd = _build_both(ctx, abi, 10, 7, 7, 40, h, eri, th, arith=arith)
    _check_build(abi, pen, pd)
    pen.free()


@ARITHS
def test_build_parity_mc_rows_licl_shape(ctx, abi, arith):
    """LiCl-shaped system (28 spin orbitals, Nh=56) on 1,000 Monte Carlo rows with multiplicities."""
    h, eri = synth.integrals(14, 111)
    th = synth.rbm_theta(14, 56, 111)
    rows, cnt = _mc_rows(14, 7, 7, 1000, 111, h)
    pen, pd = _build_both(ctx, abi, 14, 7, 7, 56, h, eri, th, rows, cnt, arith=arith)
    _check_build(abi, pen, pd)
    pen.free()


@pytest.mark.parametrize("n,na,nb,nh,sigma", [(2, 1, 1, 2, 0.2), (3, 3, 1, 4, 0.2),
                                              (4, 0, 2, 3, 0.2), (32, 1, 1, 4, 0.2),
                                              (5, 2, 3, 7, 0.2), (6, 3, 3, 127, 0.02),
                                              (6, 3, 3, 127, 0.5)])
@ARITHS
def test_build_parity_edge_shapes(ctx, abi, n, na, nb, nh, sigma, arith):
    """Degenerate sectors: 4 determinants, a full spin shell, an empty spin, M = 64,
    odd P+1; the largest hidden layer (Nh = 127), where prod_j (1 + e^{-2|z_j|})
    reaches 2^127 for small theta and the cosh ratios span e^{+-70} for large theta."""
    h, eri = synth.integrals(n, 17)
    th = synth.rbm_theta(n, nh, 17, sigma=sigma)
    pen, pd = _build_both(ctx, abi, n, na, nb, nh, h, eri, th, arith=arith)
    _check_build(abi, pen, pd)
    pen.free()


@ARITHS
def test_build_parity_large_theta(ctx, abi, arith):
    """theta ~ N(0, 0.5): large pre-activations and cosh ratios far from 1."""
    h, eri = synth.integrals(10, 23)
    th = synth.rbm_theta(10, 40, 23, sigma=0.5)
    pen, pd = _build_both(ctx, abi, 10, 7, 7, 40, h, eri, th, arith=arith)
    _check_build(abi, pen, pd)
    pen.free()


@ARITHS
def test_build_parity_saturated_hidden_units(ctx, abi, arith):
    """Saturated hidden units (|z_j| near 12, 30, 48 and 66): on an enumerated sector, whose build
    reads tanh z_j and psi from the per-determinant tables, and on sampled rows of it,
    whose build forms every connection's ratios itself."""
    h, eri = synth.integrals(8, 29)
    th = saturated_theta(8, 32, 29)
    pen, pd = _build_both(ctx, abi, 8, 4, 4, 32, h, eri, th, arith=arith)
    _check_build(abi, pen, pd)
    pen.free()
    rows, cnt = _mc_rows(8, 4, 4, 300, 29, h)
    pen, pd = _build_both(ctx, abi, 8, 4, 4, 32, h, eri, th, rows, cnt, arith=arith)
    _check_build(abi, pen, pd)
    pen.free()


# ------------------------------------------------------------------ pencil
def _check_products(abi, pen, pd, mode, nvec=3, tol=1e-10, prec=0):
    S, Hp = lm.pencil_matrices(pd.Oc, pd.Gpc, pd.w)
    Hs = lm.symmetrise(Hp, "half" if mode == abi.LM_SYM_HALF else "none")
    P1 = S.shape[0]
    rng = np.random.default_rng(7)
    for _ in range(nvec):
        v = rng.standard_normal(P1)
        Hv = np.zeros(P1)
        Sv = np.zeros(P1)
        pen.apply(v, Hv, Sv, sym=mode, prec=prec)
        assert _rel(Hv, Hs @ v) <= tol
        assert _rel(Sv, S @ v) <= tol


def test_pencil_products_tiny_and_f2(ctx, abi):
    for name in ("tiny_6o6e", "f2_10o14e"):
        w = synth.WORKLOADS[name]
        h, eri, th, _, _ = w.inputs()
        pen, pd = _build_both(ctx, abi, w.n_orb, w.n_alpha, w.n_beta, w.n_hidden, h, eri, th)
        _check_products(abi, pen, pd, abi.LM_SYM_NONE)
        _check_products(abi, pen, pd, abi.LM_SYM_HALF)
        pen.free()


def test_pencil_products_mc_rows(ctx, abi):
    h, eri = synth.integrals(14, 111)
    th = synth.rbm_theta(14, 56, 111)
    rows, cnt = _mc_rows(14, 7, 7, 1000, 111, h)
    pen, pd = _build_both(ctx, abi, 14, 7, 7, 56, h, eri, th, rows, cnt)
    _check_products(abi, pen, pd, abi.LM_SYM_HALF)
    _check_products(abi, pen, pd, abi.LM_SYM_NONE)
    pen.free()


# double-float factors are the FP64-accurate storage (48-bit significand), held to
# the FP64 path's bar on pencil products (1e-10 relative)
@pytest.mark.parametrize("prec,tol", [(1, 2e-6), (2, 2e-2), (3, 1e-10)], ids=["fp32", "bf16", "df64"])
def test_pencil_products_low_precision(ctx, abi, prec, tol):
    h, eri = synth.integrals(14, 111)
    th = synth.rbm_theta(14, 56, 111)
    rows, cnt = _mc_rows(14, 7, 7, 1000, 111, h)
    pen, pd = _build_both(ctx, abi, 14, 7, 7, 56, h, eri, th, rows, cnt, prec=prec)
    _check_products(abi, pen, pd, abi.LM_SYM_HALF, tol=tol, prec=prec)
    _check_products(abi, pen, pd, abi.LM_SYM_HALF, tol=1e-10, prec=0)
    pen.free()


@pytest.mark.parametrize("n,na,nb,nh,mc", [(10, 2, 2, 41, 0), (14, 7, 7, 64, 600),
                                           (32, 1, 1, 30, 0)],
                         ids=["ldp888", "ldp1888", "ldp2016"])
@pytest.mark.parametrize("prec", [0, 3], ids=["fp64", "df64"])
def test_pencil_products_fewer_stages_than_warps(ctx, abi, n, na, nb, nh, mc, prec):
    """Row widths whose shared-memory ring holds fewer stages than the kernel has
    consumer warps (P+1 = 882, 1885, 2015 with 8-byte factors)."""
    h, eri = synth.integrals(n, 31)
    th = synth.rbm_theta(n, nh, 31, sigma=0.05)
    rows, cnt = _mc_rows(n, na, nb, mc, 31, h) if mc else (None, None)
    pen, pd = _build_both(ctx, abi, n, na, nb, nh, h, eri, th, rows, cnt, prec=prec)
    # FP64 and double-float factors: the FP64 path's 1e-10 relative bar on pencil
    # products (a pipeline fault shows up as errors of order 1 or more)
    _check_products(abi, pen, pd, abi.LM_SYM_NONE, nvec=2, tol=1e-10, prec=prec)
    _check_products(abi, pen, pd, abi.LM_SYM_HALF, nvec=2, tol=1e-10, prec=prec)
    pen.free()


@pytest.mark.parametrize("n,na,nb,nh", [(10, 7, 7, 35), (10, 3, 3, 36)], ids=["ldp760", "ldp784"])
def test_pencil_products_stage_count_multiple(ctx, abi, n, na, nb, nh):
    """FP32 rows of 760 / 784 columns: two rows per pipeline stage, and a shared-memory
    ring that holds 18 stages for 16 consumer warps unless the launch rounds it to a
    multiple of them (bulk copies land in any order). Repeated products must all match."""
    h, eri = synth.integrals(n, 41)
    th = synth.rbm_theta(n, nh, 41, sigma=0.05)
    pen, pd = _build_both(ctx, abi, n, na, nb, nh, h, eri, th, prec=abi.LM_FP32)
    for _ in range(3):
        _check_products(abi, pen, pd, abi.LM_SYM_NONE, nvec=2, tol=2e-6, prec=abi.LM_FP32)
        _check_products(abi, pen, pd, abi.LM_SYM_HALF, nvec=1, tol=2e-6, prec=abi.LM_FP32)
    pen.free()


# ------------------------------------------------------------------ IRL
def _irl_case(ctx, abi, w, theta=None, rows=None, counts=None, prec=0):
    h, eri, th, _, _ = w.inputs()
    if theta is not None:
        th = theta
    pen, pd = _build_both(ctx, abi, w.n_orb, w.n_alpha, w.n_beta, w.n_hidden, h, eri, th, rows,
                          counts, prec=prec)
    ref = lm.lm_step(w.n_orb, w.n_alpha, w.n_beta, w.n_hidden, h, eri, th, rows, counts)
    c = np.zeros(w.n_params + 1)
    dth = np.zeros(w.n_params)
    res = pen.irl_step(m=w.m, k=w.k, tol=w.tol, max_restarts=500, prec=prec, c_out=c,
                       dtheta_out=dth)
    return pen, ref, res, c, dth


# ------------------------------------------------------------ E_loc estimator
@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (3, 1e-10), (1, 2e-6)], ids=["fp64", "df64", "fp32"])
def test_pencil_products_eloc_estimator(ctx, abi, prec, tol):
    """The paper's E_loc estimator (sym = LM_SYM_ELOC): y_H = O_c^T W diag(E_loc - E) O_c v
    against the oracle's explicit matrix; y_S unchanged."""
    h, eri = synth.integrals(14, 111)
    th = synth.rbm_theta(14, 56, 111)
    rows, cnt = _mc_rows(14, 7, 7, 1000, 111, h)
    pen, pd = _build_both(ctx, abi, 14, 7, 7, 56, h, eri, th, rows, cnt, prec=prec)
    S, He = lm.pencil_matrices(pd.Oc, lm.eloc_form(pd.Oc, pd.eloc, pd.E), pd.w)
    rng = np.random.default_rng(9)
    for _ in range(3):
        v = rng.standard_normal(S.shape[0])
        Hv, Sv = np.zeros_like(v), np.zeros_like(v)
        pen.apply(v, Hv, Sv, sym=abi.LM_SYM_ELOC, prec=prec)
        assert _rel(Hv, He @ v) <= tol
        assert _rel(Sv, S @ v) <= tol
    pen.free()


@pytest.mark.parametrize("name,prec", [("tiny_6o6e", 0), ("f2_10o14e", 3)])
def test_irl_eloc_estimator(ctx, abi, name, prec):
    """IRL on the E_loc-estimator operator against the lowest eigenvalue of the
    oracle's explicit O_c^T W diag(E_loc - E) O_c."""
    w = synth.WORKLOADS[name]
    h, eri, th, _, _ = w.inputs()
    pen, pd = _build_both(ctx, abi, w.n_orb, w.n_alpha, w.n_beta, w.n_hidden, h, eri, th,
                          prec=prec)
    _, He = lm.pencil_matrices(pd.Oc, lm.eloc_form(pd.Oc, pd.eloc, pd.E), pd.w)
    lam_ref = lm.shep(He)[0]
    assert lam_ref < -1e-8  # not stationary at these parameters
    res = pen.irl_step(m=w.m, k=w.k, tol=w.tol, max_restarts=500, sym=abi.LM_SYM_ELOC, prec=prec)
    assert res.status in (abi.IRL_OK, abi.IRL_BREAKDOWN_INVARIANT), res.status
    assert res.lambda_ == pytest.approx(lam_ref, rel=1e-10)
    assert res.residual <= 1e-10
    pen.free()


def test_irl_tiny_paper_settings(ctx, abi):
    """k=1, m=20, tol=1e-12 (the paper's settings) on the 6-orbital workload."""
    w = synth.WORKLOADS["tiny_6o6e"]
    pen, ref, res, c, dth = _irl_case(ctx, abi, w)
    assert res.status in (abi.IRL_OK, abi.IRL_BREAKDOWN_INVARIANT), res.status
    assert res.lambda_ == pytest.approx(ref["lam"], rel=1e-10)
    assert _rel(dth, ref["dtheta"]) <= 1e-8
    assert abs(c @ ref["c"]) == pytest.approx(1.0, abs=1e-10)
    assert res.residual <= 1e-10
    pen.free()


def test_irl_tiny_larger_theta(ctx, abi):
    """A spread-out spectrum (theta ~ N(0, 0.3)) that needs several restarts."""
    w = synth.WORKLOADS["tiny_6o6e"]
    th = synth.rbm_theta(6, 24, 9, sigma=0.3)
    pen, ref, res, c, dth = _irl_case(ctx, abi, w, theta=th)
    assert res.status in (abi.IRL_OK, abi.IRL_BREAKDOWN_INVARIANT), res.status
    assert res.lambda_ == pytest.approx(ref["lam"], rel=1e-10)
    assert _rel(dth, ref["dtheta"]) <= 1e-8
    pen.free()


def test_irl_f2_full_size(ctx, abi):
    """F2-shaped: 14,400 determinants, P=860, m=30, k=10."""
    w = synth.WORKLOADS["f2_10o14e"]
    pen, ref, res, c, dth = _irl_case(ctx, abi, w)
    assert res.status in (abi.IRL_OK, abi.IRL_BREAKDOWN_INVARIANT), res.status
    assert res.lambda_ == pytest.approx(ref["lam"], rel=1e-10)
    assert _rel(dth, ref["dtheta"]) <= 1e-8
    assert res.lambda_gen_rq == pytest.approx(
        float(ref["c"] @ (0.5 * (ref["Hp"] + ref["Hp"].T)) @ ref["c"] / (ref["c"] @ ref["S"] @ ref["c"])),
        rel=1e-8)
    pen.free()


def test_irl_f2_full_size_df64_pencil(ctx, abi):
    """F2-shaped with double-float pencil factors in the Lanczos products."""
    w = synth.WORKLOADS["f2_10o14e"]
    pen, ref, res, c, dth = _irl_case(ctx, abi, w, prec=3)
    assert res.status in (abi.IRL_OK, abi.IRL_BREAKDOWN_INVARIANT), res.status
    assert res.lambda_ == pytest.approx(ref["lam"], rel=1e-10)
    assert _rel(dth, ref["dtheta"]) <= 1e-8
    assert res.residual <= 1e-10
    pen.free()


@pytest.mark.parametrize("name", ["tiny_6o6e", "f2_10o14e"])
def test_build_parity_df64_storage(ctx, abi, name):
    """A double-float pencil keeps its centred factors only as FP32 pairs (centred
    in double-float arithmetic); exports convert them to FP64 and must meet the
    FP64 build's bar."""
    w = synth.WORKLOADS[name]
    h, eri, th, _, _ = w.inputs()
    pen, pd = _build_both(ctx, abi, w.n_orb, w.n_alpha, w.n_beta, w.n_hidden, h, eri, th, prec=3)
    _check_build(abi, pen, pd)
    pen.free()


def test_pencil_products_f2_df64(ctx, abi):
    w = synth.WORKLOADS["f2_10o14e"]
    h, eri, th, _, _ = w.inputs()
    pen, pd = _build_both(ctx, abi, 10, 7, 7, 40, h, eri, th, prec=3)
    _check_products(abi, pen, pd, abi.LM_SYM_NONE, tol=1e-12, prec=3)
    _check_products(abi, pen, pd, abi.LM_SYM_HALF, tol=1e-12, prec=3)
    pen.free()


def test_irl_mc_rows_half(ctx, abi):
    h, eri = synth.integrals(14, 111)
    rows, cnt = _mc_rows(14, 7, 7, 2000, 111, h)
    w = synth.Workload("mc", 14, 7, 7, 56, m=20, k=1)
    pen, ref, res, c, dth = _irl_case(ctx, abi, w, rows=rows, counts=cnt)
    assert res.status in (abi.IRL_OK, abi.IRL_BREAKDOWN_INVARIANT), res.status
    assert res.lambda_ == pytest.approx(ref["lam"], rel=1e-10)
    pen.free()


LZ_CASES = {
    # exact 6-orbital sector, 25 grid rows of 13 entries
    "tiny": (synth.Workload("tiny", 6, 3, 3, 24, m=20, k=1), None),
    # 3 grid rows of 9 entries: fewer rows than cluster CTAs
    "few_rows": (synth.Workload("few", 4, 2, 2, 2, seed=5, m=12, k=3), 0.2),
    # LiCl-shaped, 57 grid rows of 29 entries on Monte Carlo rows
    "mc_licl": (synth.Workload("mc", 14, 7, 7, 56, exact=False, n_samples=1500, m=20, k=1),
                None),
    # Nh + 1 = 128 grid rows (the largest hidden layer), 6-orbital sector
    "wide_grid": (synth.Workload("wide", 6, 3, 3, 127, seed=3, m=24, k=4), 0.02),
}


@pytest.mark.parametrize("case", list(LZ_CASES))
@pytest.mark.parametrize("mode", ["cluster", "coop", "split"])
def test_irl_lanczos_launch_modes(ctx, abi, monkeypatch, mode, case):
    """The three launch forms of a Lanczos step (one thread-block cluster, one
    cooperative grid, four kernels) against the FP64 oracle."""
    monkeypatch.setenv("IRLNQS_LANCZOS", mode)
    w, sigma = LZ_CASES[case]
    h, eri, th, rows, cnt = w.inputs()
    if sigma is not None:
        th = synth.rbm_theta(w.n_orb, w.n_hidden, w.seed, sigma=sigma)
    pen, ref, res, c, dth = _irl_case(ctx, abi, w, theta=th, rows=rows, counts=cnt)
    assert res.status in (abi.IRL_OK, abi.IRL_BREAKDOWN_INVARIANT), res.status
    assert res.lambda_ == pytest.approx(ref["lam"], rel=1e-10)
    assert _rel(dth, ref["dtheta"]) <= 1e-8
    pen.free()


@pytest.mark.parametrize("prec", [1, 2])
def test_irl_mixed_precision_refined_to_fp64(ctx, abi, prec):
    """FP32 / BF16 storage with FP64 refinement: |lambda - lambda_FP64| <= 1e-9 Ha."""
    h, eri = synth.integrals(14, 111)
    rows, cnt = _mc_rows(14, 7, 7, 2000, 111, h)
    w = synth.Workload("mc", 14, 7, 7, 56, m=20, k=1)
    pen, ref, res, c, dth = _irl_case(ctx, abi, w, rows=rows, counts=cnt, prec=prec)
    assert res.status in (abi.IRL_OK, abi.IRL_BREAKDOWN_INVARIANT), res.status
    assert abs(res.lambda_ - ref["lam"]) <= 1e-9
    assert res.n_matvec_lowp > 0
    pen.free()


@pytest.mark.parametrize("sigma,seed,m,k", [(0.01, 111, 6, 2), (0.3, 9, 5, 1), (0.1, 111, 6, 2)])
def test_irl_restarts_follow_the_oracle(ctx, abi, sigma, seed, m, k):
    """Algorithm 1's implicit restart on the GPU, cycle by cycle: a small Krylov dimension
    forces several restarts (mu = m - k exact shifts each); the GPU must restart exactly as
    often as the oracle's CPU IRL (same operator, start vector, seed and null-space
    deflation) and its lowest Ritz value after every cycle must follow the oracle's."""
    from oracle import irl as oirl
    h, eri = synth.integrals(6, 111)
    th = synth.rbm_theta(6, 24, seed, sigma=sigma)
    pen, pd = _build_both(ctx, abi, 6, 3, 3, 24, h, eri, th)
    S, Hp = lm.pencil_matrices(pd.Oc, pd.Gpc, pd.w)
    Hs = 0.5 * (Hp + Hp.T)
    ref = oirl.irl_lowest(lambda v: Hs @ v, Hs.shape[0], m=m, k=k, tol=1e-12, max_restarts=200,
                          seed=111, null_basis=lm.null_vectors(6, 3, 3, 24), return_history=True)
    res = pen.irl_step(m=m, k=k, tol=1e-12, max_restarts=200, sym=abi.LM_SYM_NONE)
    lam_h, res_h, lowp_h = pen.irl_history()
    assert ref["n_restart"] >= 3  # the case exercises the restart
    assert res.status == abi.IRL_OK
    assert res.n_restart == ref["n_restart"]
    assert len(lam_h) == len(ref["history"]) == res.n_restart + 1
    assert not lowp_h.any()
    assert res.n_matvec == ref["n_matvec"] + 1  # + the explicit refinement product
    for i, (_, lam_o, res_o) in enumerate(ref["history"]):
        assert lam_h[i] == pytest.approx(lam_o, rel=1e-9), f"cycle {i}"
        # residual estimates beta_m |u_m| agree while they are above rounding level
        if res_o > 1e-9:
            assert res_h[i] == pytest.approx(res_o, rel=1e-4), f"cycle {i}"
        else:
            assert res_h[i] < 1e-7, f"cycle {i}"
    assert res.lambda_ == pytest.approx(ref["lam"], rel=1e-10)
    pen.free()


@pytest.mark.parametrize("m,k", [(20, 1), (12, 3), (6, 2)])
def test_irl_three_term_recurrence_follows_the_oracle(ctx, abi, m, k):
    """reorth = IRL_REORTH_NONE: Algorithm 2 as printed (w = A v_j - beta_{j-1} v_{j-1},
    alpha_j = <w, v_j>, w -= alpha_j v_j, no Gram-Schmidt) inside Algorithm 1's restarts,
    against the oracle's IRL with the same recurrence. Without reorthogonalisation the
    basis loses orthogonality as Ritz values converge, which amplifies rounding, so two
    correct evaluations of the same operator (the GPU's pencil and the oracle's dense
    matrix, equal to ~1e-13) may decide the convergence test one cycle apart: the restart
    counts agree within one, the Ritz history up to the last cycle both runs share, and
    the result equals the dense SHEP eigenvalue."""
    from oracle import irl as oirl
    w = synth.WORKLOADS["tiny_6o6e"]
    h, eri, th, _, _ = w.inputs()
    pen, pd = _build_both(ctx, abi, 6, 3, 3, 24, h, eri, th)
    S, Hp = lm.pencil_matrices(pd.Oc, pd.Gpc, pd.w)
    Hs = 0.5 * (Hp + Hp.T)
    ref = oirl.irl_lowest(lambda v: Hs @ v, Hs.shape[0], m=m, k=k, tol=1e-12, max_restarts=200,
                          seed=111, null_basis=lm.null_vectors(6, 3, 3, 24), return_history=True,
                          reorth="none")
    res = pen.irl_step(m=m, k=k, tol=1e-12, max_restarts=200, sym=abi.LM_SYM_NONE,
                       reorth=abi.IRL_REORTH_NONE)
    lam_h, _, _ = pen.irl_history()
    assert res.status == abi.IRL_OK
    assert abs(res.n_restart - ref["n_restart"]) <= 1
    # every cycle when the counts agree, else the cycles before the first decision
    # that went differently (the first cycle at least)
    same = res.n_restart == ref["n_restart"]
    common = min(len(lam_h), len(ref["history"])) - (0 if same else 1)
    for i, (_, lam_o, _) in enumerate(ref["history"][:max(common, 1)]):
        assert lam_h[i] == pytest.approx(lam_o, rel=1e-9), f"cycle {i}"
    assert res.lambda_ == pytest.approx(lm.shep(Hs)[0], rel=1e-10)
    pen.free()


def test_bounded_waits_time_out_and_the_context_survives(ctx, abi):
    """The timeout path of the library's bounded device waits, made to run out on purpose
    with a wait that nothing ends (a grid-barrier arrival that never comes; an mbarrier
    phase no copy completes), 1 ms limit: LM_ERR_TIMEOUT comes back instead of a hang,
    and the context then solves a normal LM step correctly."""
    import time
    for which in (0, 1):
        t0 = time.perf_counter()
        rc = ctx.debug_wait_timeout(which, 1_000_000)
        assert rc == abi.LM_ERR_TIMEOUT, rc
        assert time.perf_counter() - t0 < 1.0
    assert ctx.debug_wait_timeout(2, 1000) == abi.LM_ERR_ARG
    w = synth.WORKLOADS["tiny_6o6e"]
    pen, ref, res, c, dth = _irl_case(ctx, abi, w)
    assert res.lambda_ == pytest.approx(ref["lam"], rel=1e-10)
    pen.free()


@pytest.fixture(scope="module")
def licl_32k():
    """LiCl-shaped system (28 spin orbitals, Nh = 56, P+1 = 1,653) on 32,768 Monte Carlo rows
    with multiplicities, and the oracle's FP64 step on them (SHEP eigenvalue)."""
    h, eri = synth.integrals(14, 111)
    th = synth.rbm_theta(14, 56, 111)
    rows, cnt = _mc_rows(14, 7, 7, 32768, 111, h)
    ref = lm.lm_step(14, 7, 7, 56, h, eri, th, rows, cnt)
    return h, eri, th, rows, cnt, ref


@pytest.mark.parametrize("prec", [1, 2], ids=["fp32", "bf16"])
def test_irl_mixed_precision_32k_rows_vs_oracle(ctx, abi, licl_32k, prec):
    """The mixed-precision LM step at 32,768 LiCl-shaped rows: FP32 / BF16 factors for the
    first IRL phase, FP64 continuation and refinement, against the FP64 oracle's dense SHEP
    eigenvalue: |lambda - lambda_oracle| <= 1e-9 Ha (printed per result)."""
    h, eri, th, rows, cnt, ref = licl_32k
    sysd = ctx.system(14, 7, 7, 56, h, eri)
    pen = ctx.build_OG(sysd, th, rows=rows, weights=cnt.astype(np.float64), prec=prec)
    dth = np.zeros(th.shape[0])
    res = pen.irl_step(m=20, k=1, tol=1e-12, max_restarts=500, prec=prec, dtheta_out=dth)
    err = abs(res.lambda_ - ref["lam"])
    print(f"\n32k LiCl-shaped rows, {('FP32', 'BF16')[prec - 1]} factors: lambda = "
          f"{res.lambda_:.15f}, oracle {ref['lam']:.15f}, |error| = {err:.2e} Ha, "
          f"{res.n_matvec_lowp} low-precision + {res.n_matvec - res.n_matvec_lowp} FP64 products")
    assert res.status in (abi.IRL_OK, abi.IRL_BREAKDOWN_INVARIANT), res.status
    assert err <= 1e-9
    assert res.n_matvec_lowp > 0
    assert res.energy == pytest.approx(ref["E"], rel=1e-12)
    assert _rel(dth, ref["dtheta"]) <= 1e-6
    pen.free()


@pytest.mark.parametrize("name,prec,steps", [("tiny_6o6e", 0, 2), ("f2_10o14e", 3, 3)],
                         ids=["tiny-fp64", "f2-df64"])
def test_lm_steps_follow_the_oracle(ctx, abi, name, prec, steps):
    """theta <- theta + Delta theta, step after step; energies and eigenvalues track the
    oracle's own steps. The F2-shaped trajectory is the one bench.py times (double-float
    build and pencil, m = 30, k = 10); its second step has a gap of 0.012 between the two
    lowest eigenvalues of the symmetrised operator."""
    w = synth.WORKLOADS[name]
    h, eri, th, _, _ = w.inputs()
    sysd = ctx.system(w.n_orb, w.n_alpha, w.n_beta, w.n_hidden, h, eri)
    tg = th.copy()
    to = th.copy()
    pen = None
    for step in range(steps):
        pen = ctx.build_OG(sysd, tg, pencil=pen, prec=prec)
        res = pen.irl_step(m=w.m, k=w.k, tol=w.tol, prec=prec, theta_inout=tg)
        ref = lm.lm_step(w.n_orb, w.n_alpha, w.n_beta, w.n_hidden, h, eri, to)
        assert res.energy == pytest.approx(ref["E"], rel=1e-10)
        assert res.lambda_ == pytest.approx(ref["lam"], rel=1e-8)
        to = to + ref["dtheta"]
        assert _rel(tg, to) <= 1e-7
    pen.free()


def test_determinism_bitwise(ctx, abi):
    w = synth.WORKLOADS["tiny_6o6e"]
    h, eri, th, _, _ = w.inputs()
    out = []
    for _ in range(2):
        sysd = ctx.system(6, 3, 3, 24, h, eri)
        pen = ctx.build_OG(sysd, th)
        c = np.zeros(w.n_params + 1)
        res = pen.irl_step(m=20, k=1, c_out=c)
        out.append((res.lambda_, c.copy(), pen.export(abi.EXPORT_G)))
        pen.free()
    assert out[0][0] == out[1][0]
    assert np.array_equal(out[0][1], out[1][1]) and np.array_equal(out[0][2], out[1][2])


# ------------------------------------------------------------------ errors
def test_error_paths(ctx, abi):
    h, eri = synth.integrals(6, 1)
    th = synth.rbm_theta(6, 4, 1)
    sysd = ctx.system(6, 3, 3, 4, h, eri)
    bad_rows = np.array([0b111111, 0b111000000111], dtype=np.uint64)  # first has 6 alpha electrons
    with pytest.raises(abi.LMError) as e:
        ctx.build_OG(sysd, th, rows=bad_rows)
    assert e.value.code == abi.LM_ERR_ARG
    big = ctx.system(33, 1, 1, 4, np.zeros((33, 33)), np.zeros(33 ** 4))
    with pytest.raises(abi.LMError) as e:
        ctx.build_OG(big, np.zeros(1000))
    assert e.value.code == abi.LM_ERR_SIZE
    pen = ctx.build_OG(sysd, th)
    with pytest.raises(abi.LMError) as e:
        pen.irl_step(m=65, k=1)
    assert e.value.code == abi.LM_ERR_SIZE
    with pytest.raises(abi.LMError) as e:
        pen.irl_step(m=10, k=10)
    assert e.value.code == abi.LM_ERR_SIZE
    pen.free()


def test_context_params(abi):
    """lm_create's options: profiling from the start (the build's kernel time is recorded
    without an lm_stats_reset), the autotuner's HBM rate, and the refusals."""
    c = abi.Context(0, profile=True, hbm_gbs=6000.0)
    w = synth.WORKLOADS["tiny_6o6e"]
    h, eri, th, _, _ = w.inputs()
    pen = c.build_OG(c.system(6, 3, 3, 24, h, eri), th)
    st = c.stats()
    assert st.build_count >= 1 and st.build_ms > 0.0
    pen.free()
    c.close()
    with pytest.raises(abi.LMError) as e:
        abi.Context(0, hbm_gbs=-1.0)
    assert e.value.code == abi.LM_ERR_ARG


def test_profile_class_mask(ctx, abi):
    """lm_stats_reset with LM_PROF_ONLY | class bits times only those classes (the others
    report their launch counts and no time), 1 times every class, 0 none; other values
    are refused."""
    w = synth.WORKLOADS["tiny_6o6e"]
    h, eri, th, _, _ = w.inputs()
    sysd = ctx.system(6, 3, 3, 24, h, eri)

    def step():
        pen = ctx.build_OG(sysd, th)
        pen.irl_step(m=20, k=1, tol=1e-12)
        pen.free()

    ctx.stats_reset(abi.LM_PROF_ONLY | abi.LM_PROF_BUILD)
    step()
    st = ctx.stats()
    assert st.build_count == 1 and st.build_ms > 0.0
    assert st.pencil_count > 0 and st.pencil_ms == 0.0
    assert st.lanczos_ms == 0.0 and st.tri_ms == 0.0 and st.prep_ms == 0.0
    ctx.stats_reset(1)
    step()
    st = ctx.stats()
    assert st.build_ms > 0.0 and st.pencil_ms > 0.0 and st.tri_ms > 0.0
    counts = (st.build_count, st.pencil_count, st.lanczos_count, st.prep_count, st.tri_count)
    ctx.stats_reset(0)
    step()
    st = ctx.stats()
    assert st.build_ms == 0.0 and st.pencil_ms == 0.0
    assert (st.build_count, st.pencil_count, st.lanczos_count, st.prep_count,
            st.tri_count) == counts
    for bad in (2, 0x20 | abi.LM_PROF_ONLY, 0x200):
        with pytest.raises(abi.LMError) as e:
            ctx.stats_reset(bad)
        assert e.value.code == abi.LM_ERR_ARG
    ctx.stats_reset(0)
