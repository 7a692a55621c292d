"""The tensor-core block product (lm_apply_pencil_block: tcgen05 MMAs on the BF16 factors)
and the block-Lanczos phase of irl_step (irl_params.block = 16) against the FP64 oracle.

Bars: the block product against the oracle's explicit S~ and H~' at the BF16 storage bar
(1e-2 relative, Frobenius, as the single-vector BF16 product); against a reference that
repeats the kernel's roundings (BF16 factors and V, X' = W X rounded to BF16, exact sums)
to 1e-3; the block-Lanczos solve, after its FP64 continuation and refinement, within
1e-9 Ha of the oracle's dense SHEP eigenvalue."""
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


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def _bf16(x):
    """Round to the nearest BF16 (ties to even), returned as FP64."""
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).to(torch.float32) \
        .to(torch.bfloat16).to(torch.float64).numpy()


def _case(ctx, abi, name):
    if name == "tiny":
        w = synth.WORKLOADS["tiny_6o6e"]
        h, eri, th, rows, cnt = w.inputs()
    elif name == "f2":
        w = synth.WORKLOADS["f2_10o14e"]
        h, eri, th, rows, cnt = w.inputs()
    else:
        w = synth.Workload("mc", 14, 7, 7, 56, exact=False, n_samples=1000, m=20, k=1)
        h, eri, th, rows, cnt = w.inputs()
    wts = None if cnt is None else cnt.astype(np.float64)
    pen = ctx.build_OG(ctx.system(w.n_orb, w.n_alpha, w.n_beta, w.n_hidden, h, eri), th,
                       rows=rows, weights=wts, prec=abi.LM_BF16)
    pd = lm.build_pencil(w.n_orb, w.n_alpha, w.n_beta, w.n_hidden, h, eri, th, rows, cnt)
    return pen, pd


@pytest.mark.parametrize("name", ["tiny", "f2", "mc"])
def test_block_product_against_the_oracle(ctx, abi, name):
    """16 and 5 vectors (a ragged block), unsymmetrised and symmetrised H~', on the 6-orbital
    sector (400 rows: 7 tiles, the last ragged), the F2-shaped sector (14,400 rows) and
    1,000 LiCl-shaped MC rows (P+1 = 1,653: 13 column chunks)."""
    import torch
    pen, pd = _case(ctx, abi, name)
    P1 = pd.Oc.shape[1]
    S, Hp = lm.pencil_matrices(pd.Oc, pd.Gpc, pd.w)
    rng = np.random.default_rng(21)
    dev = torch.device("cuda", 0)
    Ob, Gb = _bf16(pd.Oc), _bf16(pd.Gpc)
    for nvec in (16, 5):
        V = rng.standard_normal((nvec, P1))
        Vd = torch.from_numpy(V).to(dev)
        Vb = _bf16(V)
        for sym in (abi.LM_SYM_NONE, abi.LM_SYM_HALF):
            HV = torch.full((nvec, P1), float("nan"), dtype=torch.float64, device=dev)
            SV = torch.full((nvec, P1), float("nan"), dtype=torch.float64, device=dev)
            pen.apply_block(Vd, HV, SV, sym=sym)
            torch.cuda.synchronize()
            hv, sv = HV.cpu().numpy(), SV.cpu().numpy()
            half = sym == abi.LM_SYM_HALF
            Hs = lm.symmetrise(Hp, "half" if half else "none")
            assert _rel(hv, (Hs @ V.T).T) <= 1e-2
            assert _rel(sv, (S @ V.T).T) <= 1e-2
            # the kernel's own roundings, repeated: X = B V (exact sums of BF16 products,
            # rounded to FP32), X' = BF16(FP32(w) X), Y = B^T X'
            w32 = pd.w.astype(np.float32).astype(np.float64)
            XO = _bf16(w32[:, None] * (Ob @ Vb.T).astype(np.float32))
            XG = _bf16(w32[:, None] * (Gb @ Vb.T).astype(np.float32))
            ys = (Ob.T @ XO).T
            yh = (Ob.T @ XG).T
            if half:
                yh = 0.5 * (yh + (Gb.T @ XO).T)
            assert _rel(sv, ys) <= 1e-3
            assert _rel(hv, yh) <= 1e-3
    # bit-reproducible (fixed-order partial sums), and H or S alone
    V = torch.from_numpy(rng.standard_normal((16, P1))).to(dev)
    outs = []
    for _ in range(2):
        HV = torch.zeros((16, P1), dtype=torch.float64, device=dev)
        pen.apply_block(V, HV, None, sym=abi.LM_SYM_HALF)
        torch.cuda.synchronize()
        outs.append(HV.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])
    SV = torch.zeros((16, P1), dtype=torch.float64, device=dev)
    pen.apply_block(V, None, SV, sym=abi.LM_SYM_HALF)
    torch.cuda.synchronize()
    assert np.isfinite(SV.cpu().numpy()).all()
    pen.free()


def test_block_product_refusals(ctx, abi):
    """A pencil without BF16 factors, more than 16 vectors and the E_loc estimator form are
    refused before any launch."""
    import torch
    w = synth.WORKLOADS["tiny_6o6e"]
    h, eri, th, _, _ = w.inputs()
    pen = ctx.build_OG(ctx.system(6, 3, 3, 24, h, eri), th, prec=abi.LM_FP32)
    V = torch.zeros((4, w.n_params + 1), dtype=torch.float64, device="cuda")
    with pytest.raises(abi.LMError) as e:
        pen.apply_block(V, V.clone(), None)
    assert e.value.code == abi.LM_ERR_ARG
    pen.free()
    pen = ctx.build_OG(ctx.system(6, 3, 3, 24, h, eri), th, prec=abi.LM_BF16)
    big = torch.zeros((17, w.n_params + 1), dtype=torch.float64, device="cuda")
    with pytest.raises(abi.LMError) as e:
        pen.apply_block(big, big.clone(), None)
    assert e.value.code == abi.LM_ERR_SIZE
    with pytest.raises(abi.LMError) as e:
        pen.apply_block(V, V.clone(), None, sym=abi.LM_SYM_ELOC)
    assert e.value.code == abi.LM_ERR_ARG
    pen.free()


@pytest.mark.parametrize("name,m", [("tiny", 32), ("mc", 64), ("f2", 48)])
def test_block_lanczos_refined_to_fp64(ctx, abi, name, m):
    """irl_step with block = 16: m / 16 block-Lanczos steps on the tensor-core product (BF16
    factors), Rayleigh-Ritz, then the FP64 continuation and refinement: the eigenvalue
    within 1e-9 Ha of the oracle's dense SHEP, the update within 1e-6 of the oracle's."""
    pen, pd = _case(ctx, abi, name)
    S, Hp = lm.pencil_matrices(pd.Oc, pd.Gpc, pd.w)
    lam, c, _ = lm.shep(0.5 * (Hp + Hp.T))
    if c[0] < 0:
        c = -c
    dref, _ = lm.update_from_c(c)
    dth = np.zeros(pd.Oc.shape[1] - 1)
    res = pen.irl_step(m=m, k=1, tol=1e-12, max_restarts=500, prec=abi.LM_BF16, block=16,
                       dtheta_out=dth)
    err = abs(res.lambda_ - lam)
    print(f"\n{name}: block Lanczos m={m}: |lambda - lambda_oracle| = {err:.2e} Ha, "
          f"{res.n_matvec_lowp} block-product vectors + {res.n_matvec - res.n_matvec_lowp} "
          f"FP64 products")
    assert res.status in (abi.IRL_OK, abi.IRL_BREAKDOWN_INVARIANT), res.status
    assert err <= 1e-9
    assert res.n_matvec_lowp == m
    assert _rel(dth, dref) <= 1e-6
    pen.free()


def test_block_lanczos_refusals(ctx, abi):
    w = synth.WORKLOADS["tiny_6o6e"]
    h, eri, th, _, _ = w.inputs()
    pen = ctx.build_OG(ctx.system(6, 3, 3, 24, h, eri), th, prec=abi.LM_BF16)
    for kw in (dict(m=20, block=16, prec=abi.LM_BF16), dict(m=32, block=16, prec=abi.LM_FP64),
               dict(m=32, block=8, prec=abi.LM_BF16)):
        with pytest.raises(abi.LMError) as e:
            pen.irl_step(k=1, **kw)
        assert e.value.code == abi.LM_ERR_ARG
    pen.free()
