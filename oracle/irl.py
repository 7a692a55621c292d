"""Plain CPU implicitly restarted Lanczos (test infrastructure only).

Follows Algorithm 1 (IRL for NQS optimisation) and Algorithm 2 (standard
Lanczos) of the paper, with these readings where the paper is silent:

* v1 is a "random unit vector": component i is 2u-1 with u the 53-bit uniform
  of SplitMix64 (Steele, Lea & Flood 2014) at counter i for the given seed,
  then normalised (after removing optional null-space directions).
* Each new Lanczos vector is fully reorthogonalised against the basis by
  classical Gram-Schmidt applied twice (the corrections to the current
  direction are added to alpha_j).
* After a restart Lanczos resumes at step k+1 (Algorithm 1 builds steps 1..m
  in its first cycle).
* Ritz pairs come from the eigendecomposition of T_m (scipy's
  eigh_tridiagonal); the residual of the lowest pair is beta_m |e_m^T u|.
* Restart: the mu = m - k largest Ritz values are the shifts, applied by mu
  implicit shifted QR sweeps (Golub & Van Loan, Alg. 8.3.2, with a given
  shift) that accumulate Q; V_k <- V_m Q[:, :k] and the new residual is
  v_{k+1} beta_hat_k + beta_m v_{m+1} Q[m, k] (the implicit-Q restart).
* Convergence: residual < max(tol, 50 eps ||T||).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

IRL_OK, IRL_BREAKDOWN, IRL_MAX_RESTARTS = 0, 1, 2
_M64 = (1 << 64) - 1


def splitmix64_uniform(seed: int, n: int) -> np.ndarray:
    """Component i: 2u-1, u = (splitmix64 output for state seed + (i+1)*gamma) >> 11 * 2^-53."""
    out = np.empty(n)
    gamma = 0x9E3779B97F4A7C15
    for i in range(n):
        z = (seed + (i + 1) * gamma) & _M64
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        z = z ^ (z >> 31)
        u = (z >> 11) * (1.0 / 9007199254740992.0)
        out[i] = 2.0 * u - 1.0
    return out


def givens(x, z):
    r = np.hypot(x, z)
    if r == 0.0:
        return 1.0, 0.0, 0.0
    return x / r, z / r, r


def implicit_qr_sweep(a, b, nu, Q):
    """One implicit symmetric QR step with shift nu on T = tridiag(b, a, b), in place.

    Rotation p acts on indices (p, p+1): R = [[c, s], [-s, c]], T <- R T R^T,
    Q <- Q R^T; the bulge starts from the shifted first column (a0 - nu, b0).
    """
    m = a.shape[0]
    x = a[0] - nu
    z = b[0]
    for p in range(m - 1):
        c, s, r = givens(x, z)
        if p > 0:
            b[p - 1] = r
        ap, aq, bp = a[p], a[p + 1], b[p]
        a[p] = c * c * ap + 2.0 * c * s * bp + s * s * aq
        a[p + 1] = s * s * ap - 2.0 * c * s * bp + c * c * aq
        b[p] = c * s * (aq - ap) + (c * c - s * s) * bp
        if p < m - 2:
            z = s * b[p + 1]
            b[p + 1] = c * b[p + 1]
            x = b[p]
        qp = Q[:, p].copy()
        qq = Q[:, p + 1].copy()
        Q[:, p] = c * qp + s * qq
        Q[:, p + 1] = -s * qp + c * qq


def irl_lowest(matvec, n, m=20, k=1, tol=1e-12, max_restarts=200, seed=111, v0=None,
               null_basis=None, return_history=False, reorth="full"):
    """Lowest eigenpair of the symmetric operator ``matvec`` by IRL.

    reorth="full": classical Gram-Schmidt twice against the whole basis after the
    three-term step; reorth="none": Algorithm 2 as printed, w = A v_j - beta_{j-1}
    v_{j-1}, alpha_j = <w, v_j>, w = w - alpha_j v_j, and nothing else.
    Returns dict(lam, y, residual, status, n_matvec, n_restart[, history]).
    """
    if reorth not in ("full", "none"):
        raise ValueError(reorth)
    if not (1 <= k < m <= n):
        raise ValueError("need 1 <= k < m <= n")

    def proj(v):
        if null_basis is not None:
            v = v - null_basis @ (null_basis.T @ v)
        return v

    V = np.zeros((n, m + 1))
    alpha = np.zeros(m)
    beta = np.zeros(m)
    v = splitmix64_uniform(seed, n) if v0 is None else np.array(v0, dtype=float)
    v = proj(v)
    V[:, 0] = v / np.linalg.norm(v)
    j0 = 0
    n_mv = 0
    hist = []
    eps = np.finfo(float).eps
    status = IRL_MAX_RESTARTS
    lam, y, res = np.nan, None, np.inf
    for restart in range(max_restarts + 1):
        jend = m
        broke = False
        for j in range(j0, m):
            w = matvec(V[:, j])
            n_mv += 1
            if reorth == "none":
                if j > 0:
                    w = w - beta[j - 1] * V[:, j - 1]
                alpha[j] = w @ V[:, j]
                w = w - alpha[j] * V[:, j]
            else:
                alpha[j] = V[:, j] @ w
                w = w - alpha[j] * V[:, j]
                if j > 0:
                    w = w - beta[j - 1] * V[:, j - 1]
                for _ in range(2):
                    cc = V[:, :j + 1].T @ w
                    w = w - V[:, :j + 1] @ cc
                    alpha[j] += cc[j]
            w = proj(w)
            beta[j] = np.linalg.norm(w)
            tnorm = max(np.abs(alpha[:j + 1]).max(), np.abs(beta[:j + 1]).max())
            if beta[j] <= 1e-14 * max(tnorm, 1e-300):
                jend = j + 1
                broke = True
                break
            V[:, j + 1] = w / beta[j]
        if jend > 1:
            theta, U = sla.eigh_tridiagonal(alpha[:jend], beta[:jend - 1])
        else:
            theta, U = alpha[:1].copy(), np.ones((1, 1))
        lam = float(theta[0])
        u = U[:, 0]
        res = abs(beta[jend - 1] * u[jend - 1]) if not broke else 0.0
        tnorm = np.abs(theta).max()
        hist.append((restart, lam, res))
        if broke or res < max(tol, 50 * eps * tnorm):
            y = V[:, :jend] @ u
            status = IRL_BREAKDOWN if broke else IRL_OK
            break
        if restart == max_restarts:
            y = V[:, :jend] @ u
            break
        # implicit restart with the mu = m - k largest Ritz values as shifts
        a = alpha[:m].copy()
        b = beta[:m - 1].copy()
        Q = np.eye(m)
        for nu in theta[k:][::-1]:
            implicit_qr_sweep(a, b, nu, Q)
        f = V[:, :m] @ Q[:, k] * b[k - 1] + V[:, m] * beta[m - 1] * Q[m - 1, k - 1]
        Vk = V[:, :m] @ Q[:, :k]
        V[:, :k] = Vk
        alpha[:k] = a[:k]
        beta[:k - 1] = b[:k - 1]
        beta[k - 1] = np.linalg.norm(f)
        V[:, k] = f / beta[k - 1]
        j0 = k
    out = dict(lam=lam, y=y, residual=res, status=status, n_matvec=n_mv,
               n_restart=len(hist) - 1)
    if return_history:
        out["history"] = hist
    return out
