"""Dose-comparison tools used by the tests (test infrastructure, numpy only).

* batch statistics of Sec. II.B.2 (total and its standard error from B groups)
* dose-averaged LET and its standard error from group tallies (Sec. IV)
* R80 of an integrated depth-dose curve
* per-voxel z-scores between two independent estimates
* brute-force 3-D gamma index (Low et al.), global dose criterion, on the grid
  without interpolation -- the comparison metric of Sec. II.D
"""
from __future__ import annotations

import numpy as np

MEV_TO_J = 1.602176634e-13


def batch_stats(tally: np.ndarray):
    """tally[V, B] -> (total[V], sigma[V]): sigma = sqrt(B/(B-1) * sum_b (D_b - D/B)^2)."""
    t = np.asarray(tally, dtype=np.float64)
    B = t.shape[1]
    tot = t.sum(1)
    if B < 2:
        return tot, np.zeros_like(tot)
    dev = t - tot[:, None] / B
    return tot, np.sqrt(B / (B - 1) * (dev * dev).sum(1))


def let_stats(num: np.ndarray, den: np.ndarray):
    """Dose-averaged LET from group tallies num[V, B] (sum of e L) and den[V, B] (sum of e):
    LET_d = sum num / sum den (0 where den is 0), and its standard error by the ratio
    estimator over the B groups: var = B/(B-1) sum_b (num_b - LET_d den_b)^2 / den^2."""
    num = np.asarray(num, dtype=np.float64)
    den = np.asarray(den, dtype=np.float64)
    B = num.shape[1]
    N, D = num.sum(1), den.sum(1)
    ok = D > 0
    let = np.zeros_like(N)
    let[ok] = N[ok] / D[ok]
    sig = np.zeros_like(N)
    if B > 1:
        e = num - let[:, None] * den
        sig[ok] = np.sqrt(B / (B - 1) * (e[ok] ** 2).sum(1)) / D[ok]
    return let, sig


def to_gray(energy_mev: np.ndarray, rho: np.ndarray, voxel_cm3: float) -> np.ndarray:
    """Energy (MeV) per voxel -> dose (Gy) = E * 1.602e-13 J / (rho * V * 1e-3 kg)."""
    return energy_mev * MEV_TO_J / (rho * voxel_cm3 * 1e-3)


def depth_dose(D3: np.ndarray) -> np.ndarray:
    """Integrated depth-dose (sum over each z slice) of a [nz, ny, nx] array."""
    return D3.reshape(D3.shape[0], -1).sum(1)


def r80(idd: np.ndarray, dz: float, z0: float = 0.0) -> float:
    """Depth distal to the maximum where the curve falls to 80 % of it; linear interpolation
    between voxel centres."""
    idd = np.asarray(idd, dtype=np.float64)
    k = int(np.argmax(idd))
    lvl = 0.8 * idd[k]
    zc = z0 + (np.arange(len(idd)) + 0.5) * dz
    for j in range(k, len(idd) - 1):
        if idd[j] >= lvl > idd[j + 1]:
            return float(zc[j] + (idd[j] - lvl) / (idd[j] - idd[j + 1]) * dz)
    return float(zc[-1])


def zscores(Da, sa, Db, sb, frac_of_max=0.1):
    """z = (Da - Db) / sqrt(sa^2 + sb^2) over voxels where Db exceeds frac_of_max of its max."""
    Da, sa, Db, sb = (np.asarray(x, dtype=np.float64).ravel() for x in (Da, sa, Db, sb))
    m = Db > frac_of_max * Db.max()
    den = np.sqrt(sa[m] ** 2 + sb[m] ** 2)
    den[den == 0] = np.inf
    return (Da[m] - Db[m]) / den


def gamma_index(D_ref, D_eval, voxel, dose_pct=2.0, dta_mm=2.0, threshold=0.1, search_mm=None):
    """3-D gamma index of D_eval against D_ref (Low et al.), the comparison of Sec. II.D.

    D_ref, D_eval: [nz, ny, nx]; voxel: (dx, dy, dz) in cm.  Global criterion: the dose
    tolerance is dose_pct % of max(D_ref).  For every reference voxel above
    threshold * max(D_ref), gamma^2 = min over evaluated voxels within the search radius
    (default 1.5 dta) of r^2 / dta^2 + (D_eval - D_ref)^2 / tol^2, on the grid without
    interpolation.  Returns (gamma^2 per voxel, inf where not evaluated; the mask of
    evaluated voxels)."""
    D_ref = np.asarray(D_ref, dtype=np.float64)
    D_eval = np.asarray(D_eval, dtype=np.float64)
    dx, dy, dz = (v * 10.0 for v in voxel)  # mm
    tol = dose_pct / 100.0 * D_ref.max()
    search = 1.5 * dta_mm if search_mm is None else search_mm
    # every voxel within the search sphere lies inside this box
    nx_, ny_, nz_ = (int(search // d) + 1 for d in (dx, dy, dz))
    g2 = np.full(D_ref.shape, np.inf)
    m = D_ref > threshold * D_ref.max()
    if not m.any():
        return g2, m
    nz, ny, nx = D_ref.shape
    for kz in range(-nz_, nz_ + 1):
        for ky in range(-ny_, ny_ + 1):
            for kx in range(-nx_, nx_ + 1):
                r2 = (kx * dx) ** 2 + (ky * dy) ** 2 + (kz * dz) ** 2
                if r2 > search * search:
                    continue
                zs, ze = max(0, -kz), min(nz, nz - kz)
                ys, ye = max(0, -ky), min(ny, ny - ky)
                xs, xe = max(0, -kx), min(nx, nx - kx)
                if zs >= ze or ys >= ye or xs >= xe:
                    continue
                ref = D_ref[zs:ze, ys:ye, xs:xe]
                ev = D_eval[zs + kz:ze + kz, ys + ky:ye + ky, xs + kx:xe + kx]
                val = r2 / dta_mm ** 2 + (ev - ref) ** 2 / tol ** 2
                sub = g2[zs:ze, ys:ye, xs:xe]
                np.minimum(sub, val, out=sub)
    g2[~m] = np.inf
    return g2, m


def gamma_passes(g2):
    """The pass decision gamma <= 1, with the 1e-12 allowance both implementations use."""
    return g2 <= 1.0 + 1e-12


def gamma_pass_rate(D_ref, D_eval, voxel, dose_pct=2.0, dta_mm=2.0, threshold=0.1, search_mm=None):
    """Fraction of evaluated reference voxels with gamma <= 1 (NaN if none is evaluated)."""
    g2, m = gamma_index(D_ref, D_eval, voxel, dose_pct, dta_mm, threshold, search_mm)
    if not m.any():
        return float("nan")
    return float(np.mean(gamma_passes(g2[m])))
