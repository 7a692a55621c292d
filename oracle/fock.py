"""Fock-space helpers of the oracle (test infrastructure only).

* ``sector_dets``: every determinant with N_alpha alpha and N_beta beta
  electrons (Methods, Fock expansion restricted to fixed N_up/N_down as the
  paper's sampler enforces), sorted ascending.
* ``jw_hamiltonian``: the second-quantised Hamiltonian (Methods, Wave Function
  Ansatz) built literally from Jordan-Wigner matrices a_p = Z x ... x Z x s- x
  I x ... (Kronecker products), summed term by term. It serves only to pin the
  Slater-Condon rules of ``og_rows.c``; it is exponential in M and meant for
  M <= 12.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp


def sector_dets(n_orb: int, n_alpha: int, n_beta: int) -> np.ndarray:
    alpha = [sum(1 << p for p in c) for c in itertools.combinations(range(n_orb), n_alpha)]
    beta = [sum(1 << (n_orb + p) for p in c) for c in itertools.combinations(range(n_orb), n_beta)]
    dets = sorted(a | b for a in alpha for b in beta)
    return np.array(dets, dtype=np.uint64)


def jw_annihilators(m: int):
    """Sparse 2^m x 2^m matrices a_p; basis index = sum_p n_p 2^p."""
    sm = sp.csr_matrix(np.array([[0.0, 1.0], [0.0, 0.0]]))   # |1> -> |0>
    z = sp.csr_matrix(np.diag([1.0, -1.0]))
    eye = sp.identity(2, format="csr")
    ops = []
    for p in range(m):
        # kron(A_{m-1}, ..., A_0): factor for bit q sits at position m-1-q
        mats = []
        for q in range(m - 1, -1, -1):
            mats.append(sm if q == p else (z if q < p else eye))
        a = mats[0]
        for f in mats[1:]:
            a = sp.kron(a, f, format="csr")
        ops.append(a)
    return ops


def jw_hamiltonian(h: np.ndarray, eri: np.ndarray) -> sp.csr_matrix:
    """H = sum_{pq,s} h_pq a+_{ps} a_{qs} + 1/2 sum_{pqrs,s,t} (pq|rs) a+_{ps} a+_{rt} a_{st} a_{qs}."""
    n = h.shape[0]
    m = 2 * n
    a = jw_annihilators(m)
    ad = [x.T.tocsr() for x in a]
    dim = 1 << m
    H = sp.csr_matrix((dim, dim))

    def so(p, s):
        return p + n * s

    for s in range(2):
        for p in range(n):
            for q in range(n):
                if h[p, q] != 0.0:
                    H = H + h[p, q] * (ad[so(p, s)] @ a[so(q, s)])
    for s in range(2):
        for t in range(2):
            for p in range(n):
                for q in range(n):
                    left = ad[so(p, s)]
                    right = a[so(q, s)]
                    for r in range(n):
                        for u in range(n):
                            v = eri[p, q, r, u]
                            if v == 0.0:
                                continue
                            H = H + (0.5 * v) * (left @ ad[so(r, t)] @ a[so(u, t)] @ right)
    return H.tocsr()


def sector_matrix_from_jw(h, eri, n_alpha, n_beta):
    n = h.shape[0]
    dets = sector_dets(n, n_alpha, n_beta).astype(np.int64)
    H = jw_hamiltonian(h, eri)
    return dets, H[dets][:, dets].toarray()
