"""Parity rule shared by the tests (not part of the oracle or the library).

Two backward-stable evaluations of sigma_min(zI - A) differ by about
c * u * |zI - A|; below that floor only the class "tiny" is meaningful. The
rule, per point:

    |sigma - sigma_ref| <= REL * sigma_ref + ABS * |zI - A|_1

with REL = 1e-10 (the relative bar for the path) and ABS = 1e-13 (the
absolute floor, a few hundred units of roundoff times the norm). Mask bits
must agree except at points whose reference sigma lies within
max(1e-9 * eps_l, ABS * |zI - A|_1) of the level eps_l.
"""
import numpy as np

REL = 1e-10
ABS = 1e-13


def band_norm1(bands: np.ndarray, kl: int, ku: int, z) -> np.ndarray:
    """|zI - A|_1 (largest column sum of moduli) for each point z."""
    n = bands.shape[1]
    z = np.asarray(z, dtype=np.complex128).ravel()
    best = np.zeros(z.shape[0])
    # column j collects A[i, j] for i = j - d, d in [-kl, ku]
    for j in range(n):
        off = 0.0
        diag = None
        for d in range(-kl, ku + 1):
            i = j - d
            if 0 <= i < n:
                if d == 0:
                    diag = bands[d + kl, i]
                else:
                    off += abs(bands[d + kl, i])
        col = off + np.abs(z - (diag if diag is not None else 0.0))
        best = np.maximum(best, col)
    return best


def check_sigma(sigma, ref, norm1, rel=REL, abs_=ABS):
    sigma = np.asarray(sigma, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    norm1 = np.asarray(norm1, dtype=np.float64).ravel()
    bound = rel * ref + abs_ * norm1
    err = np.abs(sigma - ref)
    bad = ~(err <= bound)
    well = (ref >= 1e-3 * norm1) & (ref > 0)
    floor = ref < 1e-3 * norm1
    info = {
        "max_rel_well": float((err[well] / ref[well]).max()) if np.any(well) else 0.0,
        "max_abs_floor": float((err[floor] / norm1[floor]).max()) if np.any(floor) else 0.0,
        "below_floor": int(np.sum((sigma <= abs_ * norm1) & (ref <= abs_ * norm1))),
        "n_bad": int(bad.sum()),
    }
    return bad, info


def mask_exclusions(ref, norm1, eps):
    """Points where a mask bit may legitimately differ (sigma_ref too close to a level)."""
    ref = np.asarray(ref, dtype=np.float64).ravel()
    norm1 = np.asarray(norm1, dtype=np.float64).ravel()
    excl = np.zeros((ref.shape[0], len(eps)), dtype=bool)
    for l, e in enumerate(eps):
        excl[:, l] = np.abs(ref - e) <= np.maximum(1e-9 * e, ABS * norm1)
    return excl


def check_masks(mask, ref_mask, ref, norm1, eps):
    mask = np.asarray(mask).astype(np.uint32).ravel()
    ref_mask = np.asarray(ref_mask).astype(np.uint32).ravel()
    excl = mask_exclusions(ref, norm1, eps)
    bad = np.zeros(mask.shape[0], dtype=bool)
    for l in range(len(eps)):
        b1 = (mask >> l) & 1
        b2 = (ref_mask >> l) & 1
        bad |= (b1 != b2) & ~excl[:, l]
    return bad, int(excl.any(axis=1).sum())
