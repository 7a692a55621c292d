"""Linear-method pencil of the oracle, formed explicitly (test infrastructure only).

Follows the paper's Methods section "From SR to a Stable Eigenvalue Problem":

* Basis of the linear method (linearised wavefunction, c = [1, v]):
  chi_0 = psi and chi_k = (O_k - <O_k>) psi for k >= 1 (energy-centred,
  derivative functions centred so that <chi_0|chi_k> = 0).
* VMC energy E = sum_x w(x) E_loc(x), w = |psi|^2 / sum |psi|^2 for exact
  enumeration, or multiplicity / total for a Monte Carlo row set.
* Centred Hamiltonian H' = H - E (energy-centring step); the augmented matrices
  S~_ij = <chi_i|chi_j> = (O_c^T W O_c)_ij and H~'_ij = <chi_i|H'|chi_j> =
  (O_c^T W G'_c)_ij, with O_c(x,0) = 1, G_c(x,0) = E_loc(x),
  O_c(x,k) = O_k(x) - <O_k>, G_c(x,k) = G_k(x) - <O_k> E_loc(x),
  G'_c = G_c - E O_c.
* The paper's solve: S ~ I, the standard Hermitian eigenproblem H v = lambda v
  (eq. standard_evp); the update is Delta theta = c[1:] / c[0].
* The generalised problem it approximates (eq. full_gevp), solved on the
  range of S~ (eigenvalues of S~ below 1e-12 * max dropped).

The matrices are formed explicitly with library matmuls and solved with
LAPACK (scipy.linalg.eigh): no blocking, fusion or matrix-free tricks.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla

from . import native
from .fock import sector_dets


def weights_exact(lnpsi: np.ndarray) -> np.ndarray:
    """w(x) = |psi(x)|^2 / sum_x' |psi(x')|^2 for real psi, computed with a max shift."""
    e = np.exp(2.0 * (lnpsi - lnpsi.max()))
    return e / e.sum()


def weights_counts(counts: np.ndarray) -> np.ndarray:
    c = np.asarray(counts, dtype=np.float64)
    return c / c.sum()


def centre(O, G, eloc, w):
    """Energy E, mean O, and the centred O_c, G'_c of the linear-method basis."""
    E = float(w @ eloc)
    Obar = w @ O
    Oc = O - Obar[None, :]
    Oc[:, 0] = 1.0
    Gc = G - eloc[:, None] * Obar[None, :]
    Gc[:, 0] = eloc
    Gpc = Gc - E * Oc
    return E, Obar, Oc, Gpc


def condition_scales(pd, n_orb, n_alpha, n_beta, n_hidden, h, eri, theta, union_occ=False):
    """First-order rounding scales of every entry the build produces, for componentwise
    error bars: how far a relative change u in every rounded quantity can move the entry,
    divided by u.

    Oa(x,k): |O_k(x)| on visible entries (exact 0/1); on hidden unit j,
        (|tanh z_j| + (1 - tanh^2 z_j)(|b_j| + sum_p |W_jp| x_p)) x_c (tanh's condition).
    E_loc(x) = sum_x' c_x':                        A_E(x)   = sum_x' |c_x'|
    O_c(x,k) = O_k(x) - <O_k>:                     A_O(x,k) = Oa(x,k) + <Oa_k>
    G'_c(x,k) = sum_x' c_x' O_k(x') - <O_k> E_loc(x) - E O_c(x,k):
        A_G(x,k) = sum_x' |c_x'| Oa(x',k) + |<O_k>| A_E(x) + <Oa_k> |E_loc(x)| + |E| A_O(x,k)
    column 0: O_c = 1 exactly (A_O = 1), G'_c = E_loc - E (A_G = A_E + |E|).
    (<.> is the weighted mean over the rows.)
    union_occ: the sum over x' in A_G counts every connection whose x or x' occupies the
    orbital of column k -- the scale of G formed, for orbitals occupied in x, as the sum
    over all connections minus the sum over those that empty the orbital.
    """
    ea, ga, oa = native.rows_abs(n_orb, n_alpha, n_beta, n_hidden, h, eri, theta, pd.rows,
                                 union_occ)
    ob = np.abs(pd.Obar)
    oam = pd.w @ oa
    AO = oa + oam[None, :]
    AO[:, 0] = 1.0
    AG = ga + ob[None, :] * ea[:, None] + oam[None, :] * np.abs(pd.eloc)[:, None] + \
        abs(pd.E) * AO
    AG[:, 0] = ea + abs(pd.E)
    return ea, AO, AG


def pencil_matrices(Oc, Gpc, w):
    """Explicit S~ = O_c^T W O_c and H~' = O_c^T W G'_c, both (P+1)x(P+1)."""
    WO = Oc * w[:, None]
    S = WO.T @ Oc
    Hp = WO.T @ Gpc
    return S, Hp


def symmetrise(Hp, mode: str):
    if mode == "none":
        return Hp
    if mode == "half":
        return 0.5 * (Hp + Hp.T)
    raise ValueError(mode)


def eloc_form(Oc, eloc, E):
    """G'_c of the paper's E_loc estimator (Methods, "Practical Matrix-Free
    Implementation", eq. matrix_vec_prod: [H_eff]_ij = E[O_i (E_loc - E) O_j]) on
    the centred basis: G'_c(x,k) = (E_loc(x) - E) O_c(x,k). The exact form keeps
    one more term, G'_c(x,k) = (E_loc(x) - E) O_c(x,k) + d E_loc(x) / d theta_k
    (k >= 1), which this estimator drops; column 0 is the same in both."""
    return (np.asarray(eloc) - E)[:, None] * Oc


def pencil_apply(Oc, Gpc, w, v, mode="none"):
    """y_H = O_c^T W (G'_c v) (mode none) or 1/2 (O_c^T W G'_c v + G'_c^T W O_c v)
    (mode half), y_S = O_c^T W (O_c v): the products the paper's matrix-free MVP
    (eq. matrix_vec_prod) evaluates, here through the explicit matrices."""
    S, Hp = pencil_matrices(Oc, Gpc, w)
    return symmetrise(Hp, mode) @ v, S @ v


def null_vectors(n_orb: int, n_alpha: int, n_beta: int, n_hidden: int):
    """Orthonormal basis of the particle-number null space of O_c.

    For every augmented row r of the (Nh+1)x(M+1) grid and every spin, the
    sum over that spin's visible columns of O_c equals N_spin times column 0
    of the row (r >= 1; O_c(x,0) = 1 is not centred, so for r = 0 the column-0
    term is absent). Those 2(Nh+1) vectors are exact null vectors of S~ and H~'.
    """
    m = 2 * n_orb
    m1 = m + 1
    p1 = (n_hidden + 1) * m1
    vecs = []
    for r in range(n_hidden + 1):
        blk = []
        for s, ne in ((0, n_alpha), (1, n_beta)):
            v = np.zeros(p1)
            for p in range(s * n_orb, (s + 1) * n_orb):
                v[r * m1 + p + 1] = 1.0
            if r > 0:
                v[r * m1] = -float(ne)
            blk.append(v)
        vecs.extend(blk)
    N = np.array(vecs).T
    q, _ = np.linalg.qr(N)
    return q


@dataclass
class PencilData:
    rows: np.ndarray
    w: np.ndarray
    lnpsi: np.ndarray
    eloc: np.ndarray
    E: float
    Obar: np.ndarray
    Oc: np.ndarray
    Gpc: np.ndarray
    exact: bool


def build_pencil(n_orb, n_alpha, n_beta, n_hidden, h, eri, theta, rows=None, counts=None):
    """Rows (exact sector or given samples) -> centred O_c, G'_c and weights."""
    exact = rows is None
    if exact:
        rows = sector_dets(n_orb, n_alpha, n_beta)
    lnpsi, O, eloc, G = native.rows(n_orb, n_alpha, n_beta, n_hidden, h, eri, theta, rows)
    w = weights_exact(lnpsi) if exact else weights_counts(counts)
    E, Obar, Oc, Gpc = centre(O, G, eloc, w)
    return PencilData(rows, w, lnpsi, eloc, E, Obar, Oc, Gpc, exact)


def shep(Hs):
    """Lowest eigenpair of the symmetric matrix (the paper's SHEP, eq. standard_evp)."""
    lam, vec = sla.eigh(Hs)
    return float(lam[0]), vec[:, 0], lam


def gevp_deflated(S, Hs, cutoff=1e-12):
    """Lowest eigenpair of H~ c = lambda S~ c on range(S~) (eq. full_gevp)."""
    sig, U = sla.eigh(S)
    keep = sig > cutoff * sig.max()
    X = U[:, keep] / np.sqrt(sig[keep])[None, :]
    lam, Y = sla.eigh(X.T @ Hs @ X)
    return float(lam[0]), X @ Y[:, 0]


LM_OK, LM_C0_TINY, LM_STATIONARY = 0, 1, 2


def update_from_c(c, tol=1e-12, lam=None):
    """Delta theta = c[1:]/c[0] (linearised wavefunction with c = [1, v])."""
    if lam is not None and lam > -tol:
        return None, LM_STATIONARY
    if abs(c[0]) < 1e-8 * np.linalg.norm(c):
        return None, LM_C0_TINY
    return c[1:] / c[0], LM_OK


def lm_step(n_orb, n_alpha, n_beta, n_hidden, h, eri, theta, rows=None, counts=None,
            sym="auto", tol=1e-12):
    """One oracle LM step: explicit pencil, SHEP (paper) and deflated GEVP."""
    pd = build_pencil(n_orb, n_alpha, n_beta, n_hidden, h, eri, theta, rows, counts)
    if sym == "auto":
        sym = "none" if pd.exact else "half"
    S, Hp = pencil_matrices(pd.Oc, pd.Gpc, pd.w)
    Hs = 0.5 * (Hp + Hp.T)   # the eigensolver's symmetric operator in both modes
    lam, c, spectrum = shep(Hs)
    if c[0] < 0:
        c = -c
    dtheta, status = update_from_c(c, tol, lam)
    lam_gen, cg = gevp_deflated(S, Hs)
    return dict(E=pd.E, lam=lam, c=c, dtheta=dtheta, status=status, lam_gen=lam_gen,
                c_gen=cg, S=S, Hp=Hp, spectrum=spectrum, pencil=pd, sym=sym)
