"""Vavilov energy-loss straggling for the oracle (test infrastructure only).

The paper uses Gaussian straggling and prints no Vavilov formula; this is the optional
Vavilov form (physics flag VAVILOV).  A proton crossing a thin layer loses energy in
collisions with free electrons whose energy transfers eps in (0, eps_max] follow the Bethe
spectrum xi (1/eps^2 - beta^2/(eps eps_max)) per unit transfer (xi = (K/2)(Z/A) rho s /
beta^2).  With x = eps/eps_max, kappa = xi/eps_max and tau conjugate to the loss in units of
eps_max, the fluctuation about the mean loss has the characteristic function

    ln phi(tau) = kappa * int_0^1 (exp(i tau x) - 1 - i tau x) (1/x^2 - beta^2/x) dx
                = kappa * (I2(tau) - beta^2 I1(tau)),
    I1 = -Cin(tau) + i (Si(tau) - tau),
    I2 = -(exp(i tau) - 1 - i tau) + i tau (-Cin(tau) + i Si(tau)),
    Cin(tau) = gamma + ln tau - Ci(tau),

(I2 by parts from I1).  The density follows by a discrete Fourier inversion on a grid wide
enough to hold all the mass; its quantiles give the table the transport samples from.

The table: ln kappa on NK nodes over [ln 0.001, ln 10], beta^2 on NB nodes over [0, 0.5], and
NU quantiles at u = U0 + i (1 - 2 U0)/(NU - 1) of z = (loss - mean loss)/xi, each node's values
shifted by their mean so that the sampled fluctuation has mean zero.  Sampling: trilinear
interpolation in (ln kappa, beta^2, u).
"""
from __future__ import annotations

import numpy as np
from scipy import special

EULER = 0.5772156649015329
NK, NB, NU = 41, 6, 513
LNK0, LNK1 = np.log(0.001), np.log(10.0)
B2MAX = 0.5
U0 = 1e-4


def log_phi(tau, kappa, b2):
    """ln of the characteristic function of the centred loss in units of eps_max."""
    tau = np.asarray(tau, dtype=np.float64)
    out = np.zeros(tau.shape, dtype=np.complex128)
    nz = tau != 0.0
    t = np.abs(tau[nz])
    si, ci = special.sici(t)
    cin = EULER + np.log(t) - ci
    i1 = -cin + 1j * (si - t)
    i2 = -(np.exp(1j * t) - 1.0 - 1j * t) + 1j * t * (-cin + 1j * si)
    v = kappa * (i2 - b2 * i1)
    out[nz] = np.where(tau[nz] < 0, np.conj(v), v)       # phi(-tau) = conj(phi(tau))
    return out


def grid_points(kappa):
    """Points of the inversion grid: the core of the distribution is about kappa wide (in units of
    eps_max) while the grid spans a few eps_max, so thin layers need a finer grid (below kappa =
    0.01 the step stays under 0.06 xi)."""
    return 1 << 14 if kappa >= 0.01 else 1 << 16


def density(kappa, b2, n=None):
    """(y, f, dy): the density f of the centred loss y (units of eps_max) on a uniform grid."""
    n = n or grid_points(kappa)
    s = np.sqrt(kappa * (1.0 - 0.5 * b2))
    ylo, yhi = -10.0 * s - 0.05, 10.0 * s + 3.0
    L = yhi - ylo
    dy = L / n
    y = ylo + dy * np.arange(n)
    tau = np.fft.fftfreq(n, d=dy) * 2.0 * np.pi
    phi = np.exp(log_phi(tau, kappa, b2)) * np.exp(-1j * tau * ylo)
    f = np.real(np.fft.fft(phi)) / L
    return y, np.maximum(f, 0.0), dy


def quantiles(kappa, b2):
    """The table row: quantiles of z = y / kappa at the NU u-nodes, shifted to mean zero."""
    y, f, dy = density(kappa, b2)
    cdf = np.concatenate([[0.0], np.cumsum(f) * dy])
    cdf /= cdf[-1]
    edges = np.concatenate([y, [y[-1] + dy]]) - 0.5 * dy
    cdf = np.maximum.accumulate(cdf)
    u = U0 + np.arange(NU) * (1.0 - 2.0 * U0) / (NU - 1)
    z = np.interp(u, cdf, edges) / kappa
    # the sampler interpolates linearly between the u-nodes: the mean of that piecewise-linear
    # quantile function is the trapezoid average
    mean = (0.5 * (z[0] + z[-1]) + z[1:-1].sum()) / (NU - 1)
    return z - mean


def table():
    """[NB][NK][NU] float64."""
    out = np.empty((NB, NK, NU))
    for ib in range(NB):
        b2 = B2MAX * ib / (NB - 1)
        for ik in range(NK):
            kappa = np.exp(LNK0 + (LNK1 - LNK0) * ik / (NK - 1))
            out[ib, ik] = quantiles(kappa, b2)
    return out


def sample_z(tab, kappa, b2, u):
    """Trilinear interpolation of the table (the sampler's definition)."""
    a = (np.log(np.clip(kappa, 0.001, 10.0)) - LNK0) / (LNK1 - LNK0) * (NK - 1)
    b = np.clip(b2, 0.0, B2MAX) / B2MAX * (NB - 1)
    c = np.asarray(u) * (NU - 1)
    ia = np.minimum(a.astype(int), NK - 2); fa = a - ia
    ib = np.minimum(np.asarray(b).astype(int), NB - 2); fb = b - ib
    ic = np.minimum(c.astype(int), NU - 2); fc = c - ic
    def at(jb, ja):
        row = tab[jb, ja]
        return row[ic] + fc * (row[ic + 1] - row[ic])
    lo = at(ib, ia) + fa * (at(ib, ia + 1) - at(ib, ia))
    hi = at(ib + 1, ia) + fa * (at(ib + 1, ia + 1) - at(ib + 1, ia))
    return lo + fb * (hi - lo)
