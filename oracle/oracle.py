"""ctypes wrapper of the FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the CPU
baseline leg of the benchmark are the only callers.  Nothing in the product
package imports this module, and this module imports nothing from the
product package: problems arrive as plain `Problem` objects built by the
seeded input generators.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MAX_NUC_PER_MAT = 12
NO_STRAGGLING, NO_MCS, NO_ELASTIC, NO_INELASTIC = 1, 2, 4, 8


def build(force: bool = False) -> str:
    """Compiles oracle.c into liboracle.so (plain gcc, -O2, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Nuclide(C.Structure):
    _fields_ = [("Z", C.c_int), ("A", C.c_int), ("mass_u", C.c_double), ("I_eV", C.c_double)]


class Material(C.Structure):
    _fields_ = [("n", C.c_int), ("nuc", C.c_int * MAX_NUC_PER_MAT), ("w", C.c_double * MAX_NUC_PER_MAT),
                ("rho", C.c_double), ("I_eV", C.c_double), ("own_table", C.c_int)]


class HuBin(C.Structure):
    _fields_ = [("lo", C.c_int), ("hi", C.c_int), ("material", C.c_int), ("rho_a", C.c_double), ("rho_b", C.c_double)]


class Spot(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("E", "sigma_E", "x", "y", "sigma_x", "sigma_y", "u", "v", "w", "weight")]


class OrProblem(C.Structure):
    _fields_ = [("n_nuc", C.c_int), ("nuc", C.POINTER(Nuclide)),
                ("n_mat", C.c_int), ("mat", C.POINTER(Material)),
                ("n_hu", C.c_int), ("hu", C.POINTER(HuBin)),
                ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("x0", C.c_double), ("y0", C.c_double), ("z0", C.c_double),
                ("hu_vol", C.POINTER(C.c_int16)), ("mat_vol", C.POINTER(C.c_uint8)), ("rho_vol", C.POINTER(C.c_float)),
                ("n_spots", C.c_int), ("spots", C.POINTER(Spot)),
                ("n_batches", C.c_int), ("flags", C.c_uint)]


class OrTotals(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("incident", "deposited", "escaped", "binding", "steps", "elastic",
                                          "inelastic", "secondaries", "transparent", "inc_retries", "errors")]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            d, u64, i, u32 = C.c_double, C.c_uint64, C.c_int, C.c_uint32
            pd = C.POINTER(C.c_double)
            L.or_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
            L.or_draw4.argtypes = [u64, u64, u32, u32, pd]
            L.or_child_pid.argtypes = [u64, u64, u32]
            L.or_child_pid.restype = u64
            for f in ("or_binding_energy", "or_nuclear_mass"):
                getattr(L, f).argtypes = [i, i]
                getattr(L, f).restype = d
            L.or_mass_stopping_power.argtypes = [d, d, d]
            L.or_mass_stopping_power.restype = d
            L.or_radiation_length_element.argtypes = [i, d]
            L.or_radiation_length_element.restype = d
            L.or_highland_theta0.argtypes = [d, d, d]
            L.or_highland_theta0.restype = d
            L.or_bohr_variance.argtypes = [d, d, d, d]
            L.or_bohr_variance.restype = d
            L.or_sigma_nn.argtypes = [d, i]
            L.or_sigma_nn.restype = d
            L.or_sigma_inelastic.argtypes = [i, i, d]
            L.or_sigma_inelastic.restype = d
            L.or_sigma_elastic.argtypes = [i, i, d]
            L.or_sigma_elastic.restype = d
            L.or_elastic_kinematics.argtypes = [i, i, d, pd, pd, pd, pd, pd, pd]
            L.or_evap_integral.argtypes = [d, d]
            L.or_evap_integral.restype = d
            L.or_evap_sample_batch.argtypes = [d, d, u64, u64, i, pd]
            L.or_range_roundtrip.argtypes = [d, d, i, pd, pd, pd]
            L.or_moliere_F.argtypes = [d, i]
            L.or_moliere_F.restype = d
            L.or_moliere_params.argtypes = [C.POINTER(OrProblem), i, d, d, pd, pd]
            L.or_moliere_theta.argtypes = [d, d, d]
            L.or_moliere_theta.restype = d
            L.or_set_vavilov.argtypes = [pd]
            L.or_vavilov_params.argtypes = [d, d, d, d, pd, pd]
            L.or_vavilov_z.argtypes = [d, d, d]
            L.or_vavilov_z.restype = d
            L.or_range_csda.argtypes = [C.POINTER(OrProblem), i, d]
            L.or_range_csda.restype = d
            L.or_material_info.argtypes = [C.POINTER(OrProblem), i, pd]
            L.or_allocate_histories.argtypes = [C.POINTER(OrProblem), u64, C.POINTER(C.c_uint64)]
            L.or_run.argtypes = [C.POINTER(OrProblem), u64, u64, u64, u64, pd, pd, C.POINTER(OrTotals)]
            L.or_run_esc.argtypes = [C.POINTER(OrProblem), u64, u64, u64, u64, pd, pd, C.POINTER(OrTotals),
                                     pd, C.c_long, C.POINTER(C.c_long)]
            L.or_run_full.argtypes = [C.POINTER(OrProblem), u64, u64, u64, u64, pd, pd, C.POINTER(OrTotals),
                                      pd, C.c_long, C.POINTER(C.c_long), pd, pd]
            L.or_evap_batch.argtypes = [i, i, d, u64, u64, i, pd]
            L.or_inc_batch.argtypes = [i, i, d, u64, u64, i, i, pd, pd, pd]
            L.or_set_trap_rule.argtypes = [i]
            L.or_set_trap_rule.restype = None
            L.or_nucleus_info.argtypes = [i, i, pd]
            L.or_batch_stats.argtypes = [pd, C.c_long, i, pd, pd]
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


VAVILOV = 32
_vav_ready = False


def _ensure_vavilov(L):
    """Hands the Vavilov table (oracle/vavilov.py) to the C oracle, once per process."""
    global _vav_ready
    with _lock:
        if not _vav_ready:
            from oracle import vavilov as V

            tab = np.ascontiguousarray(V.table(), dtype=np.float64)
            L.or_set_vavilov(_dp(tab))
            _vav_ready = True


class _Marshalled:
    """Keeps the ctypes arrays of one problem alive."""

    def __init__(self, prob):
        if int(prob.flags) & VAVILOV:
            _ensure_vavilov(lib())
        self.nuc = (Nuclide * len(prob.nuclides))(*[Nuclide(*n) for n in prob.nuclides])
        mats = []
        for m in prob.materials:
            M = Material()
            M.n = len(m["nuc"])
            for k, (ni, w) in enumerate(zip(m["nuc"], m["w"])):
                M.nuc[k] = ni
                M.w[k] = w
            M.rho, M.I_eV, M.own_table = m["rho"], m.get("I_eV", 0.0), int(m.get("own_table", 0))
            mats.append(M)
        self.mat = (Material * len(mats))(*mats)
        self.hu = (HuBin * max(1, len(prob.hu_bins)))(*[HuBin(*b) for b in prob.hu_bins])
        self.spots_np = np.ascontiguousarray(prob.spots, dtype=np.float64)
        self.spots = self.spots_np.ctypes.data_as(C.POINTER(Spot))
        P = OrProblem()
        P.n_nuc, P.nuc = len(prob.nuclides), self.nuc
        P.n_mat, P.mat = len(mats), self.mat
        P.n_hu, P.hu = len(prob.hu_bins), self.hu
        P.nx, P.ny, P.nz = prob.shape[2], prob.shape[1], prob.shape[0]
        P.dx, P.dy, P.dz = prob.voxel
        P.x0, P.y0, P.z0 = prob.origin
        self.arrays = []
        if prob.hu is not None:
            a = np.ascontiguousarray(prob.hu, dtype=np.int16)
            self.arrays.append(a)
            P.hu_vol = a.ctypes.data_as(C.POINTER(C.c_int16))
        else:
            a = np.ascontiguousarray(prob.mat, dtype=np.uint8)
            r = np.ascontiguousarray(prob.rho, dtype=np.float32)
            self.arrays += [a, r]
            P.mat_vol = a.ctypes.data_as(C.POINTER(C.c_uint8))
            P.rho_vol = r.ctypes.data_as(C.POINTER(C.c_float))
        P.n_spots, P.spots = len(self.spots_np), self.spots
        P.n_batches, P.flags = prob.n_batches, prob.flags
        self.P = P


def run(prob, n_hist: int, seed: int, h_begin: int = 0, h_end: int | None = None, ledger: bool = False,
        escapes: int = 0):
    """Runs the oracle.  Returns (tally[V, B] MeV, totals dict, per-history ledger or None), plus
    the escaping protons [n, 8] (E, x, y, z, u, v, w, root) when escapes > 0 (buffer capacity)."""
    L = lib()
    m = _Marshalled(prob)
    nv = int(np.prod(prob.shape))
    tally = np.zeros((nv, prob.n_batches), dtype=np.float64)
    hl = np.zeros((n_hist, 4), dtype=np.float64) if ledger else None
    tot = OrTotals()
    h_end = n_hist if h_end is None else h_end
    esc = np.zeros((max(escapes, 1), 8))
    n_esc = C.c_long(0)
    rc = L.or_run_esc(C.byref(m.P), n_hist, h_begin, h_end, seed, _dp(tally),
                      _dp(hl) if hl is not None else None, C.byref(tot),
                      _dp(esc) if escapes else None, escapes, C.byref(n_esc))
    if rc != 0:
        raise RuntimeError("oracle run failed (%d)" % rc)
    totals = {k: getattr(tot, k) for k, _ in OrTotals._fields_}
    if escapes:
        return tally, totals, hl, esc[:n_esc.value]
    return tally, totals, hl


_PROBLEM_FIELDS = ("nuclides", "materials", "hu_bins", "spots", "shape", "voxel", "origin", "hu", "mat", "rho",
                   "n_batches", "flags")


def run_let(prob, n_hist: int, seed: int, h_begin: int = 0, h_end: int | None = None):
    """Runs the oracle with dose-averaged LET scoring.  Returns (tally[V, B] MeV,
    let_num[V, B] MeV keV/um, let_den[V, B] MeV, totals dict): LET_d = sum num / sum den."""
    L = lib()
    m = _Marshalled(prob)
    nv = int(np.prod(prob.shape))
    tally = np.zeros((nv, prob.n_batches), dtype=np.float64)
    num = np.zeros_like(tally)
    den = np.zeros_like(tally)
    tot = OrTotals()
    h_end = n_hist if h_end is None else h_end
    rc = L.or_run_full(C.byref(m.P), n_hist, h_begin, h_end, seed, _dp(tally), None, C.byref(tot), None, 0, None,
                       _dp(num), _dp(den))
    if rc != 0:
        raise RuntimeError("oracle run failed (%d)" % rc)
    return tally, num, den, {k: getattr(tot, k) for k, _ in OrTotals._fields_}


def _run_range(job):
    import types

    fields, n_hist, seed, h0, h1, let = job
    prob = types.SimpleNamespace(**fields)
    if let:
        tally, num, den, tot = run_let(prob, n_hist, seed, h_begin=h0, h_end=h1)
        return tally, tot, num, den
    tally, tot, _ = run(prob, n_hist, seed, h_begin=h0, h_end=h1)
    return tally, tot


def run_parallel(prob, n_hist: int, seed: int, procs: int | None = None, let: bool = False):
    """The same computation as run() (run_let() with let=True), split over history ranges in
    spawned worker processes (each range is an independent set of histories; tallies are
    summed in range order).  Returns (tally, totals) or (tally, totals, let_num, let_den)."""
    import multiprocessing as mp

    procs = procs or os.cpu_count() or 1
    procs = max(1, min(procs, n_hist // 200 or 1))
    fields = {k: getattr(prob, k) for k in _PROBLEM_FIELDS}
    cuts = [n_hist * i // procs for i in range(procs + 1)]
    jobs = [(fields, n_hist, seed, cuts[i], cuts[i + 1], let) for i in range(procs)]
    sums, totals = None, None

    def add(part):
        nonlocal sums, totals
        if sums is None:
            sums = [np.zeros_like(part[0]) for _ in range(3 if let else 1)]
            totals = {k: 0.0 for k in part[1]}
        sums[0] += part[0]
        if let:
            sums[1] += part[2]
            sums[2] += part[3]
        for k in totals:
            totals[k] += part[1][k]

    if procs == 1:
        add(_run_range(jobs[0]))
    else:
        # parts arrive in range order and are summed as they come (one large tally in flight
        # at a time, not one per worker)
        with mp.get_context("spawn").Pool(procs) as pool:
            for part in pool.imap(_run_range, jobs):
                add(part)
    if let:
        return sums[0], totals, sums[1], sums[2]
    return sums[0], totals


def moliere_params(prob, m: int, E: float, x: float):
    """(chi_c^2, B) of a proton of energy E (MeV) over x g/cm^2 of material m."""
    L = lib()
    mm = _Marshalled(prob)
    c2, B = C.c_double(0), C.c_double(0)
    L.or_moliere_params(C.byref(mm.P), m, E, x, C.byref(c2), C.byref(B))
    return c2.value, B.value


def material_info(prob, m: int):
    L = lib()
    mm = _Marshalled(prob)
    out = np.zeros(5)
    L.or_material_info(C.byref(mm.P), m, _dp(out))
    return {"ZA": out[0], "I_eV": out[1], "f": out[2], "X0mass": out[3]}


def allocate_histories(prob, n: int):
    L = lib()
    mm = _Marshalled(prob)
    cnt = np.zeros(len(prob.spots), dtype=np.uint64)
    L.or_allocate_histories(C.byref(mm.P), n, cnt.ctypes.data_as(C.POINTER(C.c_uint64)))
    return cnt


def range_csda(prob, m: int, E: float) -> float:
    mm = _Marshalled(prob)
    return lib().or_range_csda(C.byref(mm.P), m, E)


def range_roundtrip(ZA, I_eV, E):
    E = np.ascontiguousarray(E, dtype=np.float64)
    R = np.zeros_like(E)
    Eb = np.zeros_like(E)
    lib().or_range_roundtrip(ZA, I_eV, len(E), _dp(E), _dp(R), _dp(Eb))
    return R, Eb


def philox(ctr, key):
    c = (C.c_uint32 * 4)(*ctr)
    k = (C.c_uint32 * 2)(*key)
    o = (C.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return list(o)


def draw4(seed, pid, word2, tag):
    u = np.zeros(4)
    lib().or_draw4(seed, pid, word2, tag, _dp(u))
    return u


def elastic(Z, A, E, u):
    u = np.ascontiguousarray(u, dtype=np.float64)
    o = [C.c_double() for _ in range(5)]
    lib().or_elastic_kinematics(Z, A, E, _dp(u), *[C.byref(x) for x in o])
    return [x.value for x in o]  # T1, cos1, T2, cos2, cos_cm


def inc_batch(Z, A, E, seed, pid0, n, cap=160):
    summ = np.zeros((n, 8))
    prod = np.zeros((n, cap, 5))
    extra = np.zeros((n, 3))
    lib().or_inc_batch(Z, A, E, seed, pid0, n, cap, _dp(summ), _dp(prod), _dp(extra))
    return summ, prod, extra


def set_trap_rule(on: bool):
    """Switches the cascade's trapped-nucleon rule (on by default; off = only the crossing cap)."""
    lib().or_set_trap_rule(1 if on else 0)


def nucleus_info(Z, A):
    out = np.zeros(3 + 16 + 6 * 15)
    lib().or_nucleus_info(Z, A, _dp(out))
    o = out[3:]
    return {"Rout": out[0], "S_n": out[1], "S_p": out[2], "r": o[:16], "rho_p": o[16:31], "rho_n": o[31:46],
            "TF_p": o[46:61], "TF_n": o[61:76], "V_p": o[76:91], "V_n": o[91:106]}


def evap_batch(Z, A, Ex, seed, pid0, n):
    """First emission of n evaporations of (Z, A) at rest: [n, 4] = species (-1 none), T, cos, n_products."""
    out = np.zeros((n, 4))
    lib().or_evap_batch(Z, A, Ex, seed, pid0, n, _dp(out))
    return out


def evap_samples(X, a, seed, pid, n):
    z = np.zeros(n)
    lib().or_evap_sample_batch(X, a, seed, pid, n, _dp(z))
    return z


def batch_stats(tally):
    tally = np.ascontiguousarray(tally, dtype=np.float64)
    nv, B = tally.shape
    tot = np.zeros(nv)
    sig = np.zeros(nv)
    lib().or_batch_stats(_dp(tally), nv, B, _dp(tot), _dp(sig))
    return tot, sig


def f(name):
    """Direct access to a scalar oracle routine by name (argtypes set in lib())."""
    return getattr(lib(), name)
