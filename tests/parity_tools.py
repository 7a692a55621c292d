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
