"""Seeded generators for integrals, RBM parameters and Monte Carlo row sets.

Conventions shared by every consumer:

* Spin orbitals use the blocked order: spin orbital ``p < n_orb`` is spatial
  orbital ``p`` with spin alpha, ``p >= n_orb`` is spatial orbital ``p - n_orb``
  with spin beta. A determinant is a ``uint64`` whose bit ``p`` is the
  occupation of spin orbital ``p``.
* One-electron integrals ``h`` are a real symmetric ``n_orb x n_orb`` FP64
  array; two-electron integrals ``eri[p,q,r,s] = (pq|rs)`` are the full
  ``n_orb**4`` chemist-notation FP64 array with 8-fold symmetry.
* RBM parameters ``theta`` (length ``P = M + Nh + M*Nh``, ``M = 2*n_orb``) are
  the augmented ``(Nh+1) x (M+1)`` row-major grid without its ``(0,0)`` entry:
  row 0 holds the visible biases ``a[0..M)``, row ``j+1`` holds
  ``[b_j, W[j,0], ..., W[j,M-1]]``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def n_params(n_orb: int, n_hidden: int) -> int:
    m = 2 * n_orb
    return m + n_hidden + m * n_hidden


def integrals(n_orb: int, seed: int, hop_scale: float = 1.0):
    """Random real integrals with the symmetry of a molecular Hamiltonian.

    h = sym(X) with X_ij ~ N(0,1)/sqrt(n_orb) (upper triangle drawn, mirrored),
    plus linspace(-2, -0.5, n_orb) on the diagonal; the off-diagonal part is
    multiplied by ``hop_scale`` (weaker hopping mimics a stretched bond).
    (pq|rs) = sum_L B^L_pq B^L_rs with B^L = (Y+Y^T)/2, Y_ij ~ N(0, 1/n_orb):
    a positive-semidefinite supermatrix with the 8-fold permutational symmetry.
    """
    rng = np.random.default_rng([int(seed), 0])
    x = rng.standard_normal((n_orb, n_orb)) / math.sqrt(n_orb)
    h = np.triu(x) + np.triu(x, 1).T
    off = h - np.diag(np.diag(h))
    h = np.diag(np.diag(h)) + hop_scale * off
    h = h + np.diag(np.linspace(-2.0, -0.5, n_orb))
    b = np.empty((n_orb, n_orb, n_orb))
    for L in range(n_orb):
        y = rng.standard_normal((n_orb, n_orb)) / math.sqrt(n_orb)
        b[L] = 0.5 * (y + y.T)
    eri = np.einsum("lpq,lrs->pqrs", b, b)
    # exact 8-fold symmetry (the einsum is symmetric up to rounding order)
    eri = (eri + eri.transpose(1, 0, 2, 3)) / 2
    eri = (eri + eri.transpose(0, 1, 3, 2)) / 2
    eri = (eri + eri.transpose(2, 3, 0, 1)) / 2
    return np.ascontiguousarray(h), np.ascontiguousarray(eri)


def rbm_theta(n_orb: int, n_hidden: int, seed: int, sigma: float = 0.01):
    """RBM parameters theta_k ~ N(0, sigma) (sigma is a standard deviation)."""
    rng = np.random.default_rng([int(seed), 1])
    return rng.normal(0.0, sigma, n_params(n_orb, n_hidden))


def _bits_to_u64(occ: np.ndarray) -> np.ndarray:
    w = (np.uint64(1) << np.arange(occ.shape[1], dtype=np.uint64))
    return (occ.astype(np.uint64) * w).sum(axis=1, dtype=np.uint64)


def proxy_mc_samples(n_orb: int, n_alpha: int, n_beta: int, n_unique: int,
                     seed: int, h: np.ndarray, temperature: float = 0.6,
                     walkers: int = 4096, burn_in: int = 300,
                     max_steps: int = 20000):
    """Unique determinants with visit multiplicities from a seeded Metropolis chain.

    The chain stands in for VMC sampling. Its target weight is the
    theta-independent occupation model exp(-sum_{p occupied} h[pp]/T) over the
    (n_alpha, n_beta) sector, so that drawing it needs no wavefunction values.
    Moves swap one occupied and one empty orbital of a randomly chosen spin
    (a symmetric proposal that conserves N_alpha and N_beta). Walkers start in
    the lowest-h[pp] determinant. After ``burn_in`` steps every visited state
    is recorded; the first ``n_unique`` distinct states in visit order are kept
    with their visit counts. Returns (rows sorted ascending as uint64, counts
    as uint32).
    """
    rng = np.random.default_rng([int(seed), 2])
    m = 2 * n_orb
    eps = np.concatenate([np.diag(h), np.diag(h)]) / temperature
    order = np.argsort(np.diag(h), kind="stable")
    occ = np.zeros((walkers, m), dtype=bool)
    occ[:, order[:n_alpha]] = True
    occ[:, n_orb + order[:n_beta]] = True
    ar = np.arange(walkers)
    seen: dict[int, int] = {}
    first: list[int] = []
    for step in range(max_steps):
        spin = rng.integers(0, 2, walkers)
        nocc = np.where(spin == 0, n_alpha, n_beta)
        nvir = n_orb - nocc
        ok = (nocc > 0) & (nvir > 0)
        ki = rng.integers(0, 1 << 30, walkers) % np.maximum(nocc, 1)
        ka = rng.integers(0, 1 << 30, walkers) % np.maximum(nvir, 1)
        u = rng.random(walkers)
        base = spin * n_orb
        blk = occ[ar[:, None], base[:, None] + np.arange(n_orb)[None, :]]
        occ_rank = np.cumsum(blk, axis=1) - 1
        vir_rank = np.cumsum(~blk, axis=1) - 1
        i_loc = np.argmax(blk & (occ_rank == ki[:, None]), axis=1)
        a_loc = np.argmax((~blk) & (vir_rank == ka[:, None]), axis=1)
        i = base + i_loc
        a = base + a_loc
        d = eps[a] - eps[i]
        acc = ok & (np.log(np.maximum(u, 1e-300)) < -d)
        occ[ar[acc], i[acc]] = False
        occ[ar[acc], a[acc]] = True
        if step < burn_in:
            continue
        states = _bits_to_u64(occ)
        for s in states.tolist():
            c = seen.get(s)
            if c is None:
                seen[s] = 1
                first.append(s)
            else:
                seen[s] = c + 1
        if len(first) >= n_unique:
            break
    if len(first) < n_unique:
        raise RuntimeError("proxy chain did not reach the requested number of unique states")
    keep = first[:n_unique]
    rows = np.array(sorted(keep), dtype=np.uint64)
    counts = np.array([seen[int(s)] for s in rows], dtype=np.uint32)
    return rows, counts


@dataclass(frozen=True)
class Workload:
    """One benchmark or parity workload (sizes, seeds and IRL settings)."""

    name: str
    n_orb: int
    n_alpha: int
    n_beta: int
    n_hidden: int
    seed: int = 111
    exact: bool = True          # exact sector enumeration (else proxy MC rows)
    n_samples: int = 0          # unique MC rows when not exact
    m: int = 20                 # Krylov dimension
    k: int = 1                  # wanted (kept) Ritz pairs
    tol: float = 1e-12
    lm_steps: int = 1
    precision: str = "f64"
    extra: dict = field(default_factory=dict)

    @property
    def n_spin_orb(self) -> int:
        return 2 * self.n_orb

    @property
    def n_params(self) -> int:
        return n_params(self.n_orb, self.n_hidden)

    @property
    def n_det(self) -> int:
        return math.comb(self.n_orb, self.n_alpha) * math.comb(self.n_orb, self.n_beta)

    @property
    def n_rows(self) -> int:
        return self.n_det if self.exact else self.n_samples

    def inputs(self):
        h, eri = integrals(self.n_orb, self.seed, self.extra.get("hop_scale", 1.0))
        theta = rbm_theta(self.n_orb, self.n_hidden, self.seed)
        if self.exact:
            return h, eri, theta, None, None
        rows, counts = proxy_mc_samples(self.n_orb, self.n_alpha, self.n_beta,
                                        self.n_samples, self.seed, h)
        return h, eri, theta, rows, counts


WORKLOADS = {
    # 6 spatial orbitals, 6 electrons, 400 determinants, Nh=24, P=324
    "tiny_6o6e": Workload("tiny_6o6e", 6, 3, 3, 24, m=20, k=1, lm_steps=1),
    # F2/N2-shaped: 10 spatial orbitals, 14 electrons, 14,400 determinants, Nh=40, P=860
    "f2_10o14e": Workload("f2_10o14e", 10, 7, 7, 40, m=30, k=10, lm_steps=5),
    # LiCl-shaped: 14 spatial orbitals, 14 electrons, 262,144 unique MC rows, Nh=56, P=1652
    "licl_14o14e_mc": Workload("licl_14o14e_mc", 14, 7, 7, 56, exact=False,
                               n_samples=262144, m=20, k=1, lm_steps=1,
                               precision="f32"),
}


# Pairs (n_orb, n_electrons) with n in {8,9,10}, even N_e in [6,14] and a
# sector size between 400 and 14,400 determinants.
_BATCH_PAIRS = [(8, 6), (8, 8), (8, 10), (8, 12), (9, 6), (9, 12), (9, 14), (10, 6), (10, 14)]


def batched_instances(count: int = 64, seed: int = 111):
    """Uneven independent instances along a dissociation-curve stand-in.

    Instance i draws (n_orb, N_e) from the admissible pairs and Nh from
    [16, 40]; its integrals use seed ``seed + i`` and hop_scale
    linspace(1.0, 0.3, count)[i].
    """
    rng = np.random.default_rng([int(seed), 3])
    scales = np.linspace(1.0, 0.3, count)
    out = []
    for i in range(count):
        n, ne = _BATCH_PAIRS[int(rng.integers(0, len(_BATCH_PAIRS)))]
        nh = int(rng.integers(16, 41))
        out.append(Workload(f"inst{i:02d}_{n}o{ne}e_h{nh}", n, ne // 2, ne // 2, nh,
                            seed=seed + i, m=20, k=1, lm_steps=1, precision="f32",
                            extra={"hop_scale": float(scales[i])}))
    return out


def poisson_arrivals(rate_hz: float, duration_s: float, seed: int = 111,
                     mix=(0.6, 0.3, 0.1)):
    """Arrival times (s) and workload-class indices of a seeded Poisson stream."""
    rng = np.random.default_rng([int(seed), 4])
    t, times, cls = 0.0, [], []
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t > duration_s:
            break
        times.append(t)
        cls.append(int(rng.choice(len(mix), p=np.asarray(mix) / sum(mix))))
    return np.array(times), np.array(cls, dtype=np.int64)
