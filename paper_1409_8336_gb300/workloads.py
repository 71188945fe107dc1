"""Seeded synthetic inputs: nuclides, materials, phantoms and spot lists.

This module holds inputs only -- no part of the transport method's
arithmetic.  Both the CUDA path and the CPU oracle consume the `Problem`
objects built here.  Units: MeV, cm, g/cm^3.  Phantom arrays are indexed
[z, y, x] (x fastest in memory).

The workloads stand in for the paper's (Sec. II.D and III): pencil beams in
homogeneous and layered phantoms, and a multi-spot plan on a CT-like volume.
Patient CTs, nozzle phase spaces and Geant4 tables are not available; the
materials below are ICRU-like compositions restricted to H, C, N, O, P, Ca
and Ti, and the HU table is a fixed 6-bin table.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

# (Z, A, molar mass g/mol, mean excitation energy eV)
NUCLIDES = [
    (1, 1, 1.00794, 19.2),     # 0 H1
    (6, 12, 12.0107, 81.0),    # 1 C12
    (7, 14, 14.0067, 82.0),    # 2 N14
    (8, 16, 15.9994, 95.0),    # 3 O16
    (15, 31, 30.973762, 173.0),  # 4 P31
    (20, 40, 40.078, 191.0),   # 5 Ca40
    (22, 48, 47.867, 233.0),   # 6 Ti48
]
H, C, N, O, P, CA, TI = range(7)


def _norm(pairs):
    s = sum(w for _, w in pairs)
    return [i for i, _ in pairs], [w / s for _, w in pairs]


def _material(pairs, rho, I_eV=0.0, own_table=0):
    nuc, w = _norm(pairs)
    return {"nuc": nuc, "w": w, "rho": rho, "I_eV": I_eV, "own_table": own_table}


WATER = _material([(H, 0.111894), (O, 0.888106)], 1.0, I_eV=75.0)
AIR = _material([(N, 0.7553), (O, 0.2318)], 0.0012, I_eV=85.7, own_table=1)
TITANIUM = _material([(TI, 1.0)], 4.5, I_eV=233.0, own_table=1)
CORTICAL_BONE = _material([(H, 0.034), (C, 0.155), (N, 0.042), (O, 0.435), (P, 0.103), (CA, 0.225)], 1.85)
LUNG = _material([(H, 0.103), (C, 0.105), (N, 0.031), (O, 0.749), (P, 0.002)], 0.26)
BONE_LO = _material([(H, 0.070), (C, 0.200), (N, 0.040), (O, 0.530), (P, 0.050), (CA, 0.110)], 1.4)

# Flags switching physics off (used by the pin and parity tests only).
NO_STRAGGLING, NO_MCS, NO_ELASTIC, NO_INELASTIC = 1, 2, 4, 8
MOLIERE = 16                      # Moliere multiple scattering instead of Highland
VAVILOV = 32                      # Vavilov straggling where kappa <= 10 instead of Bohr's Gaussian


@dataclass
class Problem:
    nuclides: list
    materials: list                   # materials[0] is the reference water
    shape: tuple                      # (nz, ny, nx)
    voxel: tuple                      # (dx, dy, dz) cm
    origin: tuple                     # (x0, y0, z0) cm, corner of voxel (0,0,0)
    spots: np.ndarray                 # [n, 10]: E, sigma_E, x, y, sigma_x, sigma_y, u, v, w, weight
    mat: np.ndarray | None = None     # uint8 [nz, ny, nx]
    rho: np.ndarray | None = None     # float32 [nz, ny, nx]
    hu: np.ndarray | None = None      # int16 [nz, ny, nx]
    hu_bins: list = field(default_factory=list)  # (lo, hi, material, rho_a, rho_b): rho = a + b HU
    n_batches: int = 10
    flags: int = 0
    name: str = ""

    @property
    def n_voxels(self) -> int:
        return int(np.prod(self.shape))

    def with_(self, **kw) -> "Problem":
        return replace(self, **kw)


def spot_row(E, x=0.0, y=0.0, sigma=0.3, sigma_E=0.0, weight=1.0, direction=(0.0, 0.0, 1.0)):
    return [E, sigma_E, x, y, sigma, sigma, direction[0], direction[1], direction[2], weight]


def water_box(shape=(128, 64, 64), voxel=0.2, spots=None, n_batches=10, flags=0, name="water"):
    nz, ny, nx = shape
    mat = np.zeros(shape, np.uint8)
    rho = np.ones(shape, np.float32)
    if spots is None:
        spots = np.array([spot_row(150.0, sigma=0.3)])
    return Problem(NUCLIDES, [WATER], shape, (voxel, voxel, voxel),
                   (-nx * voxel / 2, -ny * voxel / 2, 0.0), np.asarray(spots, float),
                   mat=mat, rho=rho, n_batches=n_batches, flags=flags, name=name)


def config1(n_batches=10, flags=0) -> Problem:
    """150 MeV pencil beam (sigma 3 mm, zero divergence) on a 64x64x128 water box of 2 mm voxels."""
    return water_box((128, 64, 64), 0.2, np.array([spot_row(150.0, sigma=0.3)]), n_batches, flags,
                     name="water-64x64x128-2mm-150MeV")


def slab_phantom(n=128, voxel=0.15, energies=(70.0, 150.0, 230.0), sigma=0.4, n_batches=10, flags=0,
                 ti_insert=True) -> Problem:
    """Layered phantom: water 0-3 cm, cortical bone 3-5 cm, lung 5-9 cm, water beyond, with a
    1 cm titanium cube centred on the beam axis at depth 10-11 cm."""
    nz = ny = nx = n
    mats = [WATER, CORTICAL_BONE, LUNG, TITANIUM]
    z = (np.arange(nz) + 0.5) * voxel
    y = -ny * voxel / 2 + (np.arange(ny) + 0.5) * voxel
    x = -nx * voxel / 2 + (np.arange(nx) + 0.5) * voxel
    layer = np.zeros(nz, np.uint8)
    layer[(z >= 3.0) & (z < 5.0)] = 1
    layer[(z >= 5.0) & (z < 9.0)] = 2
    mat = np.broadcast_to(layer[:, None, None], (nz, ny, nx)).copy()
    if ti_insert:
        Zc, Yc, Xc = np.meshgrid((z >= 10.0) & (z < 11.0), np.abs(y) < 0.5, np.abs(x) < 0.5, indexing="ij")
        mat[Zc & Yc & Xc] = 3
    dens = np.array([m["rho"] for m in mats], np.float32)
    rho = dens[mat]
    spots = np.array([spot_row(E, sigma=sigma) for E in energies])
    return Problem(NUCLIDES, mats, (nz, ny, nx), (voxel, voxel, voxel), (-nx * voxel / 2, -ny * voxel / 2, 0.0),
                   spots, mat=mat, rho=rho, n_batches=n_batches, flags=flags,
                   name="slab-%d^3-%.1fmm" % (n, voxel * 10))


def config2(n_batches=10, flags=0) -> Problem:
    """128^3 voxels of 1.5 mm: water / cortical bone / lung / water with a Ti insert; 70/150/230 MeV
    pencil beams of sigma 4 mm, equal weights."""
    return slab_phantom(128, 0.15, (70.0, 150.0, 230.0), 0.4, n_batches, flags)


# (lo, hi, material index in the config-3 material list, rho_a, rho_b): rho = rho_a + rho_b * HU
HU_BINS = [
    (-32768, -950, 1, 0.0012, 0.0),   # air (own table)
    (-950, -200, 2, 1.0, 0.001),      # lung, rho = 1 + HU/1000
    (-200, 300, 0, 1.0, 0.001),       # water-like, rho = 1 + HU/1000
    (300, 1000, 3, 1.0, 0.0006),      # low-density bone, rho = 1 + 0.6 HU/1000
    (1000, 3060, 4, 1.0, 0.0006),     # cortical bone, rho = 1 + 0.6 HU/1000
    (3060, 32768, 5, 4.5, 0.0),       # titanium implant (own table)
]


def ct_phantom(shape=(160, 256, 256), voxel=0.1, seed=3):
    """Seeded ellipsoid CT: air outside, a soft-tissue body (0 HU), two lungs (-800 HU) and
    bones (700-1400 HU)."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    z = (np.arange(nz) + 0.5) * voxel
    y = -ny * voxel / 2 + (np.arange(ny) + 0.5) * voxel
    x = -nx * voxel / 2 + (np.arange(nx) + 0.5) * voxel
    Zg, Yg, Xg = np.meshgrid(z, y, x, indexing="ij", sparse=True)
    Lz, Ly, Lx = nz * voxel, ny * voxel, nx * voxel
    hu = np.full(shape, -1000, np.int16)

    def ell(c, a):
        return ((Xg - c[0]) / a[0]) ** 2 + ((Yg - c[1]) / a[1]) ** 2 + ((Zg - c[2]) / a[2]) ** 2 <= 1.0

    body = ell((0.0, 0.0, Lz / 2), (0.45 * Lx, 0.40 * Ly, 0.49 * Lz))
    hu[body] = 0
    for side in (-1, 1):
        c = (side * 0.2 * Lx, rng.uniform(-0.05, 0.05) * Ly, rng.uniform(0.45, 0.6) * Lz)
        a = (0.12 * Lx, 0.2 * Ly, 0.25 * Lz)
        hu[ell(c, a) & body] = -800
    for _ in range(6):
        c = (rng.uniform(-0.3, 0.3) * Lx, rng.uniform(-0.3, 0.3) * Ly, rng.uniform(0.2, 0.8) * Lz)
        a = tuple(rng.uniform(0.5, 2.0, size=3))
        hu[ell(c, a) & body] = int(rng.uniform(700, 1400))
    return hu


def config3(n_batches=10, flags=0, shape=(160, 256, 256), voxel=0.1, n_layers=40, seed=3) -> Problem:
    """Synthetic CT plan: int16 HU volume, 40 energy layers 70-180 MeV, 50 spots per layer on a
    10x5 grid of 5 mm pitch, lognormal(0, 0.5) weights."""
    nz, ny, nx = shape
    hu = ct_phantom(shape, voxel, seed)
    rng = np.random.default_rng(seed)
    rows = []
    for E in np.linspace(70.0, 180.0, n_layers):
        for iy in range(5):
            for ix in range(10):
                rows.append(spot_row(float(E), x=(ix - 4.5) * 0.5, y=(iy - 2) * 0.5, sigma=0.3,
                                     weight=float(rng.lognormal(0.0, 0.5))))
    mats = [WATER, AIR, LUNG, BONE_LO, CORTICAL_BONE, TITANIUM]
    bins = list(HU_BINS)
    return Problem(NUCLIDES, mats, shape, (voxel, voxel, voxel), (-nx * voxel / 2, -ny * voxel / 2, 0.0),
                   np.array(rows), hu=hu, hu_bins=bins, n_batches=n_batches, flags=flags,
                   name="ct-%dx%dx%d-%.0fmm-%dspots" % (nx, ny, nz, voxel * 10, len(rows)))


def config5(n_plans=64, n_phantoms=8, n_batches=10, flags=0, seed=5, scale=1.0):
    """Multi-plan stream: n_plans synthetic CT plans, each on one of n_phantoms seeded CT
    phantoms of 1 mm voxels from 128x128x96 to 320x320x200 (shared between plans), with
    50-3000 spots (log-uniform) in energy layers within 70-230 MeV on a 5 mm grid,
    lognormal(0, 0.5) weights, and 1e6-1e7 histories (log-uniform; times `scale`).
    Returns [(Problem, n_histories, seed)]."""
    rng = np.random.default_rng(seed)
    phantoms = []
    for k in range(n_phantoms):
        nxy = int(rng.integers(8, 21)) * 16            # 128 .. 320
        nz = int(rng.integers(12, 26)) * 8              # 96 .. 200
        if k == 0:
            nxy, nz = 128, 96
        if k == n_phantoms - 1:
            nxy, nz = 320, 200
        phantoms.append(ct_phantom((nz, nxy, nxy), 0.1, seed * 1000 + k))
    mats = [WATER, AIR, LUNG, BONE_LO, CORTICAL_BONE, TITANIUM]
    plans = []
    for i in range(n_plans):
        hu = phantoms[int(rng.integers(n_phantoms))]
        nz, ny, nx = hu.shape
        n_spots = int(round(np.exp(rng.uniform(np.log(50), np.log(3000)))))
        n_layers = int(np.clip(round(n_spots / 50), 1, 60))
        per_layer = max(1, n_spots // n_layers)
        e_lo = rng.uniform(70.0, 150.0)
        e_hi = min(230.0, e_lo + rng.uniform(20.0, 80.0))
        side = int(np.ceil(np.sqrt(per_layer)))
        rows = []
        for E in np.linspace(e_lo, e_hi, n_layers):
            for j in range(per_layer):
                iy, ix = divmod(j, side)
                rows.append(spot_row(float(E), x=(ix - (side - 1) / 2) * 0.5, y=(iy - (side - 1) / 2) * 0.5,
                                     sigma=0.3, weight=float(rng.lognormal(0.0, 0.5))))
        n_hist = int(round(np.exp(rng.uniform(np.log(1e6), np.log(1e7))) * scale))
        prob = Problem(NUCLIDES, mats, hu.shape, (0.1, 0.1, 0.1), (-nx * 0.05, -ny * 0.05, 0.0), np.array(rows),
                       hu=hu, hu_bins=list(HU_BINS), n_batches=n_batches, flags=flags,
                       name="plan%02d-ct-%dx%dx%d-%dspots" % (i, nx, ny, nz, len(rows)))
        plans.append((prob, max(n_hist, 1), seed * 100003 + i))
    return plans


CONFIG_HISTORIES = {1: 20000, 2: 1000000, 3: 10000000}


def config(k: int, **kw) -> Problem:
    return {1: config1, 2: config2, 3: config3}[k](**kw)
