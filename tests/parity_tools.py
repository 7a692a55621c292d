"""Error bars shared by the parity tests (no GPU and no method arithmetic here)."""
import numpy as np


def componentwise(got, ref, scale, tol, what):
    """Componentwise forward error: |got - ref| <= tol * scale entry by entry, where scale
    is the sum of |terms| that forms the entry in its definition (the oracle's
    condition_scales). Entries with zero scale must match exactly. Returns the largest
    |got - ref| / scale."""
    got, ref, scale = np.asarray(got), np.asarray(ref), np.asarray(scale)
    d = np.abs(got - ref)
    z = scale == 0
    assert np.all(d[z] == 0), f"{what}: entries with zero scale differ"
    r = np.zeros_like(d)
    r[~z] = d[~z] / scale[~z]
    worst = float(r.max()) if r.size else 0.0
    if worst > tol:
        i = np.unravel_index(int(np.argmax(r)), r.shape)
        raise AssertionError(f"{what}: componentwise error {worst:.3e} > {tol:.0e} at {i}: "
                             f"got {got[i]!r}, oracle {ref[i]!r}, scale {scale[i]!r}")
    return worst


def saturated_theta(n, nh, seed):
    """RBM parameters theta ~ N(0, 0.3) with four saturated hidden units, biases
    b_j = +12, -30, +48, -66 (j = 0..3): e^{-2|z_j|} about e^-24 (2^-35, where the
    double-float e^{-2|z|} - 1 is formed as 2^k (e^r - 1) - (1 - 2^k) with k < -24), and
    e^-60, e^-96, e^-132 (the last two below FP32's range, where it is -1 to within
    2^-125). Four units keep |ln psi| near 160, where FP64 rounding of ln psi leaves the
    weights well inside their 1e-12 bar."""
    import synth
    th = synth.rbm_theta(n, nh, seed, sigma=0.3)
    M1 = 2 * n + 1
    for j, b in enumerate((12.0, -30.0, 48.0, -66.0)):
        th[(j + 1) * M1 - 1] = b
    return th
