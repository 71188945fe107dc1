"""Python binding of the engine's C ABI (include/pmc.h): argument marshalling only.

Every step of the transport runs in the CUDA library libpmc.so built in-tree
by build.py.  There is no CPU fallback: if the library is missing, loading it
raises.  PyTorch is used only as plumbing: optionally its caching allocator
for the library's device memory and its current CUDA stream for launches.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpmc.so")
LIB_FAST_PATH = os.path.join(HERE, "libpmc_fast.so")   # the -use_fast_math build

PMC_OK = 0
ERRORS = {-1: "PMC_E_INVALID", -2: "PMC_E_OOM", -3: "PMC_E_QUEUE_OVERFLOW", -4: "PMC_E_TIMEOUT", -5: "PMC_E_CUDA"}
NO_STRAGGLING, NO_MCS, NO_ELASTIC, NO_INELASTIC, MOLIERE, VAVILOV = 1, 2, 4, 8, 16, 32
FULL_CASCADE, SURROGATE = 0, 1
MAX_NUC_PER_MAT = 12

EXPORTS = [
    "pmc_create", "pmc_destroy", "pmc_last_error", "pmc_load_materials", "pmc_load_phantom", "pmc_add_spots",
    "pmc_clear_spots", "pmc_transport", "pmc_read_dose", "pmc_read_tally", "pmc_read_ledger",
    "pmc_enable_history_ledger", "pmc_read_history_ledger", "pmc_enable_escape_record", "pmc_read_escape_record",
    "pmc_enable_let", "pmc_read_let", "pmc_read_let_tally", "pmc_nonelastic_events", "pmc_plans_create",
    "pmc_plans_destroy", "pmc_plans_last_error", "pmc_plans_load_materials", "pmc_plans_load_surrogate",
    "pmc_plans_bytes", "pmc_plans_run",
    "pmc_set_launch", "pmc_autotune", "pmc_transport_noalloc", "pmc_surrogate_dataset", "pmc_train_surrogate",
    "pmc_surrogate_params", "pmc_surrogate_load", "pmc_surrogate_grad", "pmc_surrogate_infer", "pmc_gamma_plan_bytes", "pmc_gamma_plan", "pmc_gamma_device",
    "pmc_gamma_index", "pmc_enable_profile", "pmc_read_profile", "pmc_debug_philox", "pmc_debug_tables",
    "pmc_debug_inc", "pmc_debug_elastic", "pmc_debug_surrogate_waits", "pmc_debug_drain_waits",
    "pmc_debug_vavilov_table",
    "pmc_enable_deposit_log", "pmc_read_deposit_log", "pmc_debug_event_stage",
]

AllocFn = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FreeFn = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class Options(C.Structure):
    _fields_ = [("device", C.c_int), ("n_batches", C.c_int), ("physics_flags", C.c_uint), ("block_size", C.c_int),
                ("chunk", C.c_int64), ("alloc", AllocFn), ("free", FreeFn), ("alloc_user", C.c_void_p)]


class Nuclide(C.Structure):
    _fields_ = [("Z", C.c_int), ("A", C.c_int), ("mass_u", C.c_double), ("I_eV", C.c_double)]


class Material(C.Structure):
    _fields_ = [("n", C.c_int), ("nuc", C.c_int * MAX_NUC_PER_MAT), ("w", C.c_double * MAX_NUC_PER_MAT),
                ("rho", C.c_double), ("I_eV", C.c_double), ("own_table", C.c_int)]


class HuBin(C.Structure):
    _fields_ = [("lo", C.c_int), ("hi", C.c_int), ("material", C.c_int), ("rho_a", C.c_double), ("rho_b", C.c_double)]


class Spot(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("E", "sigma_E", "x", "y", "sigma_x", "sigma_y", "u", "v", "w", "weight")]


SURROGATE_PARAMS = 209936
SURROGATE_FEATURES = 12


class TrainOpts(C.Structure):
    _fields_ = [("n_events", C.c_uint64), ("epochs", C.c_int), ("batch", C.c_int), ("lr", C.c_double),
                ("weight_decay", C.c_double), ("seed", C.c_uint64)]


class TrainResult(C.Structure):
    _fields_ = [("first_loss", C.c_double), ("last_loss", C.c_double), ("steps", C.c_int64)]


class Ledger(C.Structure):
    _fields_ = [(n, C.c_int64) for n in ("incident", "deposited", "escaped", "binding", "histories", "steps",
                                         "elastic", "inelastic", "secondaries", "transparent", "inc_retries",
                                         "queue_high_water", "generations", "dropped", "errors",
                                         "surrogate_events")]


class EventYields(C.Structure):
    _fields_ = [("events", C.c_uint64), ("transparent", C.c_uint64), ("retries", C.c_uint64),
                ("count", C.c_uint64 * 6), ("energy", C.c_double * 6), ("residual_T", C.c_double),
                ("excitation_left", C.c_double), ("binding", C.c_double), ("ms", C.c_double)]


class Plan(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("dx", C.c_double), ("dy", C.c_double),
                ("dz", C.c_double), ("x0", C.c_double), ("y0", C.c_double), ("z0", C.c_double),
                ("hu", C.c_void_p), ("mat", C.c_void_p), ("rho", C.c_void_p), ("spots", C.c_void_p),
                ("n_spots", C.c_int), ("n_histories", C.c_uint64), ("seed", C.c_uint64),
                ("dose_gy", C.c_void_p), ("sigma_gy", C.c_void_p)]


class PlanResult(C.Structure):
    _fields_ = [("status", C.c_int), ("slot", C.c_int), ("device_bytes", C.c_uint64), ("t_admit_ms", C.c_double),
                ("t_end_ms", C.c_double), ("gpu_ms", C.c_double), ("ledger", Ledger)]


SPECIES = ("n", "p", "d", "t", "He3", "alpha")
# pmc_deposit: tally entry [voxel][group] received llrint(e0 2^24) - llrint(e1 2^24) - llrint(e2 2^24)
DEPOSIT_DTYPE = np.dtype([("voxel", np.int32), ("group", np.int32), ("e", np.float64, 3)])

_libs = {}
_lock = threading.Lock()


def lib(path: str = LIB_PATH):
    """Loads the engine library (raises if it has not been built: there is no fallback)."""
    with _lock:
        if path not in _libs:
            if not os.path.exists(path):
                raise ImportError("%s not built: run `python -m paper_1409_8336_gb300.build` "
                                  "(or __graft_entry__.build())" % os.path.basename(path))
            L = C.CDLL(path)
            vp, i, u64, d = C.c_void_p, C.c_int, C.c_uint64, C.c_double
            pd, pi64, pf = C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_float)
            L.pmc_create.argtypes = [C.POINTER(vp), C.POINTER(Options)]
            L.pmc_destroy.argtypes = [vp]
            L.pmc_destroy.restype = None
            L.pmc_last_error.argtypes = [vp]
            L.pmc_last_error.restype = C.c_char_p
            L.pmc_load_materials.argtypes = [vp, C.POINTER(Nuclide), i, C.POINTER(Material), i, C.POINTER(HuBin), i]
            L.pmc_load_phantom.argtypes = [vp, i, i, i, d, d, d, d, d, d, vp, vp, vp]
            L.pmc_add_spots.argtypes = [vp, C.POINTER(Spot), i]
            L.pmc_clear_spots.argtypes = [vp]
            L.pmc_transport.argtypes = [vp, u64, u64, i, vp]
            L.pmc_read_dose.argtypes = [vp, vp, vp, C.c_size_t]
            L.pmc_read_tally.argtypes = [vp, pi64, C.c_size_t]
            L.pmc_read_ledger.argtypes = [vp, C.POINTER(Ledger)]
            L.pmc_enable_history_ledger.argtypes = [vp, u64]
            L.pmc_read_history_ledger.argtypes = [vp, pi64, u64]
            L.pmc_enable_escape_record.argtypes = [vp, u64]
            L.pmc_read_escape_record.argtypes = [vp, C.POINTER(C.c_float), u64, C.POINTER(C.c_uint64)]
            L.pmc_enable_let.argtypes = [vp, i]
            L.pmc_enable_deposit_log.argtypes = [vp, u64]
            L.pmc_read_deposit_log.argtypes = [vp, vp, u64, C.POINTER(C.c_uint64)]
            L.pmc_nonelastic_events.argtypes = [vp, i, d, u64, u64, u64, C.POINTER(EventYields)]
            L.pmc_plans_create.argtypes = [C.POINTER(vp), C.POINTER(Options), i, u64]
            L.pmc_plans_destroy.argtypes = [vp]
            L.pmc_plans_destroy.restype = None
            L.pmc_plans_last_error.argtypes = [vp]
            L.pmc_plans_last_error.restype = C.c_char_p
            L.pmc_plans_load_materials.argtypes = [vp, C.POINTER(Nuclide), i, C.POINTER(Material), i,
                                                   C.POINTER(HuBin), i]
            L.pmc_plans_load_surrogate.argtypes = [vp, pf, C.c_size_t]
            L.pmc_plans_bytes.argtypes = [vp, C.POINTER(Plan), i, C.POINTER(C.c_uint64)]
            L.pmc_plans_run.argtypes = [vp, C.POINTER(Plan), i, i, C.POINTER(PlanResult)]
            L.pmc_read_let.argtypes = [vp, vp, vp, C.c_size_t]
            L.pmc_read_let_tally.argtypes = [vp, pi64, pi64, C.c_size_t]
            L.pmc_set_launch.argtypes = [vp, i, C.c_int64]
            L.pmc_autotune.argtypes = [vp, u64, u64, C.POINTER(C.c_int), C.POINTER(C.c_int64)]
            L.pmc_surrogate_dataset.argtypes = [vp, u64, u64, pf]
            L.pmc_train_surrogate.argtypes = [vp, C.POINTER(TrainOpts), C.POINTER(TrainResult)]
            L.pmc_surrogate_params.argtypes = [vp, pf, C.c_size_t]
            L.pmc_surrogate_load.argtypes = [vp, pf, C.c_size_t]
            L.pmc_surrogate_grad.argtypes = [vp, pf, pf, pf, pf, pf, i, pf, pf, pf]
            L.pmc_surrogate_infer.argtypes = [vp, pf, i, pf]
            L.pmc_debug_surrogate_waits.argtypes = [vp]
            L.pmc_debug_drain_waits.argtypes = [vp, u64, u64]
            L.pmc_debug_vavilov_table.argtypes = [pf, C.c_size_t]
            L.pmc_gamma_plan_bytes.argtypes = [d, d, d, d, d, C.POINTER(C.c_size_t)]
            L.pmc_gamma_plan.argtypes = [d, d, d, d, d, vp, C.c_size_t, vp]
            L.pmc_gamma_device.argtypes = [vp, vp, vp, i, i, i, d, d, vp, vp]
            L.pmc_gamma_index.argtypes = [pd, pd, i, i, i, d, d, d, d, d, d, d, pf, pd]
            L.pmc_transport_noalloc.argtypes = [vp, u64, u64, vp, vp, vp, vp]
            L.pmc_enable_profile.argtypes = [vp, i]
            L.pmc_read_profile.argtypes = [vp, pd, pi64, pi64]
            L.pmc_debug_philox.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), i]
            L.pmc_debug_tables.argtypes = [vp, i, pd, pd, pd, i]
            L.pmc_debug_inc.argtypes = [vp, i, d, u64, u64, i, pd, pd, i]
            L.pmc_debug_elastic.argtypes = [vp, i, d, pd, pd, i]
            L.pmc_debug_event_stage.argtypes = [vp, i, vp, pd, i, u64, pf, u64, C.POINTER(C.c_uint64), pd]
            _libs[path] = L
    return _libs[path]


class PmcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _fp(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def _torch_allocator(device):
    import torch

    def alloc(n, _user):
        try:
            return torch.cuda.caching_allocator_alloc(int(n), device=device)
        except Exception:  # noqa: BLE001 - reported to the library as a NULL allocation
            return None

    def free(p, _user):
        torch.cuda.caching_allocator_delete(int(p))

    return AllocFn(alloc), FreeFn(free)


def _material_args(nuclides, materials, hu_bins):
    nuc = (Nuclide * len(nuclides))(*[Nuclide(*n) for n in nuclides])
    mats = []
    for m in materials:
        M = Material()
        M.n = len(m["nuc"])
        for k, (ni, w) in enumerate(zip(m["nuc"], m["w"])):
            M.nuc[k], M.w[k] = ni, w
        M.rho, M.I_eV, M.own_table = m["rho"], m.get("I_eV", 0.0), int(m.get("own_table", 0))
        mats.append(M)
    mat = (Material * len(mats))(*mats)
    hu = (HuBin * max(1, len(hu_bins)))(*[HuBin(*b) for b in hu_bins])
    return nuc, len(nuclides), mat, len(mats), hu, len(hu_bins)


class Engine:
    """One engine context on one GPU.  Method names follow the C ABI."""

    def __init__(self, device: int = 0, n_batches: int = 10, physics_flags: int = 0, block_size: int = 0,
                 chunk: int = 0, torch_allocator: bool = False, fast_math: bool = False, library: str | None = None):
        self._L = lib(library or (LIB_FAST_PATH if fast_math else LIB_PATH))
        self.fast_math = fast_math
        opt = Options()
        opt.device, opt.n_batches, opt.physics_flags = device, n_batches, physics_flags
        opt.block_size, opt.chunk = block_size, chunk
        self._keep = None
        if torch_allocator:
            self._keep = _torch_allocator(device)
            opt.alloc, opt.free = self._keep
        self._ctx = C.c_void_p()
        rc = self._L.pmc_create(C.byref(self._ctx), C.byref(opt))
        if rc != PMC_OK:
            raise PmcError(rc, "pmc_create failed")
        self.n_batches = n_batches
        self.shape = None

    def close(self):
        if self._ctx:
            self._L.pmc_destroy(self._ctx)
            self._ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def _check(self, rc):
        if rc != PMC_OK:
            raise PmcError(rc, self._L.pmc_last_error(self._ctx).decode())

    # --- inputs ---------------------------------------------------------
    def load_materials(self, nuclides, materials, hu_bins=()):
        self._check(self._L.pmc_load_materials(self._ctx, *_material_args(nuclides, materials, hu_bins)))

    def load_phantom(self, shape, voxel, origin, hu=None, mat=None, rho=None):
        """shape (nz, ny, nx); arrays [nz, ny, nx] in host memory (pinned or pageable)."""
        nz, ny, nx = shape
        self._arrays = []

        def ptr(a, dt):
            if a is None:
                return None
            if hasattr(a, "data_ptr"):          # a pinned torch tensor
                assert a.is_contiguous() and not a.is_cuda
                return a.data_ptr()
            a = np.ascontiguousarray(a, dtype=dt)
            self._arrays.append(a)
            return a.ctypes.data

        self._check(self._L.pmc_load_phantom(self._ctx, nx, ny, nz, *voxel, *origin, ptr(hu, np.int16),
                                             ptr(mat, np.uint8), ptr(rho, np.float32)))
        self.shape = tuple(shape)

    def add_spots(self, spots):
        s = np.ascontiguousarray(spots, dtype=np.float64).reshape(-1, 10)
        self._check(self._L.pmc_add_spots(self._ctx, s.ctypes.data_as(C.POINTER(Spot)), len(s)))

    def clear_spots(self):
        self._check(self._L.pmc_clear_spots(self._ctx))

    def load_problem(self, prob):
        """Loads a workloads.Problem (materials, phantom, spots)."""
        self.load_materials(prob.nuclides, prob.materials, prob.hu_bins)
        self.load_phantom(prob.shape, prob.voxel, prob.origin, hu=prob.hu, mat=prob.mat, rho=prob.rho)
        self.clear_spots()
        self.add_spots(prob.spots)

    def set_launch(self, block_size=0, chunk=0):
        self._check(self._L.pmc_set_launch(self._ctx, block_size, chunk))

    def autotune(self, n_histories: int, seed: int = 12345):
        """Times the candidate launch shapes on full transports and keeps the fastest."""
        b, c = C.c_int(0), C.c_int64(0)
        self._check(self._L.pmc_autotune(self._ctx, n_histories, seed, C.byref(b), C.byref(c)))
        return b.value, c.value

    # --- run ------------------------------------------------------------
    def transport(self, n_histories: int, seed: int, mode: int = FULL_CASCADE, stream=None):
        s = None
        if stream is not None:
            s = stream if isinstance(stream, int) else stream.cuda_stream
        self._check(self._L.pmc_transport(self._ctx, n_histories, seed, mode, s))

    def transport_noalloc(self, n_histories: int, seed: int, tally_ptr: int, dose_ptr=None, sigma_ptr=None,
                          stream=None):
        """Transport that allocates no device memory; outputs go to caller-owned device arrays
        (pointers: tally [n_voxels * n_batches] int64, dose and sigma [n_voxels] float64)."""
        s = None
        if stream is not None:
            s = stream if isinstance(stream, int) else stream.cuda_stream
        self._check(self._L.pmc_transport_noalloc(self._ctx, n_histories, seed, tally_ptr, dose_ptr, sigma_ptr, s))

    # --- outputs --------------------------------------------------------
    @property
    def n_voxels(self):
        return int(np.prod(self.shape))

    def read_dose(self, dose=None, sigma=None):
        n = self.n_voxels
        dose = np.empty(n) if dose is None else dose
        sigma = np.empty(n) if sigma is None else sigma

        def ptr(a):
            return a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data

        self._check(self._L.pmc_read_dose(self._ctx, ptr(dose), ptr(sigma), n))
        return dose, sigma

    def read_tally(self):
        t = np.empty((self.n_voxels, self.n_batches), dtype=np.int64)
        self._check(self._L.pmc_read_tally(self._ctx, t.ctypes.data_as(C.POINTER(C.c_int64)), t.size))
        return t

    def read_ledger(self):
        led = Ledger()
        self._check(self._L.pmc_read_ledger(self._ctx, C.byref(led)))
        return {k: getattr(led, k) for k, _ in Ledger._fields_}

    def enable_history_ledger(self, n):
        self._check(self._L.pmc_enable_history_ledger(self._ctx, n))
        self._hist_n = n

    def read_history_ledger(self, n):
        out = np.empty((n, 4), dtype=np.int64)
        self._check(self._L.pmc_read_history_ledger(self._ctx, out.ctypes.data_as(C.POINTER(C.c_int64)), n))
        return out

    def enable_escape_record(self, cap):
        self._check(self._L.pmc_enable_escape_record(self._ctx, cap))
        self._esc_cap = cap

    def read_escape_record(self):
        cap = self._esc_cap
        out = np.empty((cap, 8), dtype=np.float32)
        n = C.c_uint64(0)
        self._check(self._L.pmc_read_escape_record(self._ctx, out.ctypes.data_as(C.POINTER(C.c_float)), cap,
                                                   C.byref(n)))
        return out[: n.value]

    def enable_deposit_log(self, cap):
        """Debug: log every deposit of the next transports (cap records; 0 switches it off)."""
        self._check(self._L.pmc_enable_deposit_log(self._ctx, cap))
        self._dlog_cap = cap

    def read_deposit_log(self):
        """The last transport's deposits: structured array (voxel, group, e[3])."""
        out = np.empty(self._dlog_cap, dtype=DEPOSIT_DTYPE)
        n = C.c_uint64(0)
        self._check(self._L.pmc_read_deposit_log(self._ctx, out.ctypes.data, self._dlog_cap, C.byref(n)))
        return out[: n.value]

    def enable_let(self, on=True):
        """Scores the dose-averaged LET beside the dose in the next transports."""
        self._check(self._L.pmc_enable_let(self._ctx, 1 if on else 0))

    def read_let(self):
        """(LET_d, its standard error) per voxel in keV/um."""
        n = self.n_voxels
        let, sig = np.empty(n), np.empty(n)
        self._check(self._L.pmc_read_let(self._ctx, let.ctypes.data, sig.ctypes.data, n))
        return let, sig

    def read_let_tally(self):
        """Raw LET group tallies [V, B]: numerator (2^-24 MeV keV/um), weights (2^-24 MeV)."""
        num = np.empty((self.n_voxels, self.n_batches), dtype=np.int64)
        den = np.empty_like(num)
        p = C.POINTER(C.c_int64)
        self._check(self._L.pmc_read_let_tally(self._ctx, num.ctypes.data_as(p), den.ctypes.data_as(p), num.size))
        return num, den

    def enable_profile(self, on=True, primary_only=False):
        """Kernel timing events inside the run's graph: around every launch, or around the
        primary-transport launches only (primary_only, the lightest)."""
        self._check(self._L.pmc_enable_profile(self._ctx, (2 if primary_only else 1) if on else 0))

    def read_profile(self):
        """Per kernel kind (primary transport, secondary transport, cascade, statistics):
        summed ms, launch groups and kernels of the last transport, and the primary-transport
        step count."""
        ms = np.zeros(8)
        n = np.zeros(8, dtype=np.int64)
        steps = C.c_int64(0)
        self._check(self._L.pmc_read_profile(self._ctx, _dp(ms), n.ctypes.data_as(C.POINTER(C.c_int64)),
                                             C.byref(steps)))
        # the primaries (phase space + transport), the drain of all later generations (their
        # transport and cascades), the event stage of the primaries' non-elastic collisions
        # (cascade + evaporation, or the learned stand-in), the dose statistics
        kinds = ("transport_primary", "drain", "cascade", "stats")
        return {k: {"ms": float(ms[i]), "span_ms": float(ms[4 + i]), "launches": int(n[i]), "kernels": int(n[4 + i])}
                for i, k in enumerate(kinds)}, int(steps.value)

    # --- learned stand-in of the event generator --------------------------
    def surrogate_dataset(self, n_events: int, seed: int):
        out = np.empty((n_events, SURROGATE_FEATURES), dtype=np.float32)
        self._check(self._L.pmc_surrogate_dataset(self._ctx, n_events, seed, _fp(out)))
        return out

    def train_surrogate(self, n_events=10_000_000, epochs=3, batch=8192, lr=1e-3, weight_decay=1e-5, seed=4):
        o = TrainOpts(n_events, epochs, batch, lr, weight_decay, seed)
        r = TrainResult()
        self._check(self._L.pmc_train_surrogate(self._ctx, C.byref(o), C.byref(r)))
        return {"first_loss": r.first_loss, "last_loss": r.last_loss, "steps": r.steps}

    def surrogate_params(self):
        out = np.empty(SURROGATE_PARAMS, dtype=np.float32)
        self._check(self._L.pmc_surrogate_params(self._ctx, _fp(out), out.size))
        return out

    def surrogate_load(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        self._check(self._L.pmc_surrogate_load(self._ctx, _fp(p), p.size))

    def surrogate_grad(self, params, x, y, tau, mask):
        f = lambda a: np.ascontiguousarray(a, dtype=np.float32)  # noqa: E731
        params, x, y, tau, mask = f(params), f(x), f(y), f(tau), f(mask)
        rows = x.shape[0]
        loss = np.zeros(1, dtype=np.float32)
        grad = np.empty(SURROGATE_PARAMS, dtype=np.float32)
        yhat = np.empty((rows, 16), dtype=np.float32)
        self._check(self._L.pmc_surrogate_grad(self._ctx, _fp(params), _fp(x), _fp(y), _fp(tau), _fp(mask), rows,
                                               _fp(loss), _fp(grad), _fp(yhat)))
        return float(loss[0]), grad, yhat

    def surrogate_infer(self, x):
        """The loaded network on the tensor cores (as in the transport's event stage):
        rows x[n][32] -> outputs [n][16]."""
        x = np.ascontiguousarray(x, dtype=np.float32)
        y = np.empty((x.shape[0], 16), dtype=np.float32)
        self._check(self._L.pmc_surrogate_infer(self._ctx, _fp(x), x.shape[0], _fp(y)))
        return y

    # --- single-routine device checks ------------------------------------
    def debug_drain_waits(self, n_histories: int, seed: int):
        """A full-cascade transport whose drain never sees its work finished, so that every
        warp's bounded wait runs out; returns the library's status (PMC_E_TIMEOUT expected)."""
        return int(self._L.pmc_debug_drain_waits(self._ctx, n_histories, seed))

    def debug_surrogate_waits(self):
        """Runs the tensor-core network with its MMAs withheld so every wait runs out;
        returns the library's status (PMC_E_TIMEOUT expected)."""
        return int(self._L.pmc_debug_surrogate_waits(self._ctx))

    def debug_tables(self, material, E):
        E = np.ascontiguousarray(E, dtype=np.float64)
        r, e = np.empty_like(E), np.empty_like(E)
        self._check(self._L.pmc_debug_tables(self._ctx, material, _dp(E), _dp(r), _dp(e), len(E)))
        return r, e

    def nonelastic_events(self, nuclide, E, n, seed, pid0=0):
        """n non-elastic events of a proton of energy E (MeV) on the loaded nuclide index
        `nuclide`, on the device.  Returns the totals: events, transparent, retries,
        count[species], energy[species] (MeV), residual_T, excitation_left, binding, ms."""
        y = EventYields()
        self._check(self._L.pmc_nonelastic_events(self._ctx, nuclide, E, n, seed, pid0, C.byref(y)))
        out = {k: getattr(y, k) for k, _ in EventYields._fields_ if k not in ("count", "energy")}
        out["count"] = dict(zip(SPECIES, list(y.count)))
        out["energy"] = dict(zip(SPECIES, list(y.energy)))
        return out

    def debug_inc(self, nuclide, E, seed, pid0, n, cap=160):
        summ = np.zeros((n, 8))
        prod = np.zeros((n, cap, 5))
        self._check(self._L.pmc_debug_inc(self._ctx, nuclide, E, seed, pid0, n, _dp(summ), _dp(prod), cap))
        return summ, prod

    def debug_elastic(self, nuclide, E, u):
        u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1, 3)
        out = np.empty((len(u), 5))
        self._check(self._L.pmc_debug_elastic(self._ctx, nuclide, E, _dp(u), _dp(out), len(u)))
        return out


    def debug_event_stage(self, mode, nuclide, E, seed, cap=None):
        """The event stage alone on n events: (protons [k, 3] = event, T, cos; local [n] MeV)."""
        nuc = np.ascontiguousarray(nuclide, dtype=np.int32)
        E = np.ascontiguousarray(E, dtype=np.float64)
        n = len(E)
        cap = cap or 32 * n + 1024
        out = np.empty((cap, 3), dtype=np.float32)
        loc = np.empty(n)
        k = C.c_uint64(0)
        self._check(self._L.pmc_debug_event_stage(self._ctx, mode, nuc.ctypes.data, _dp(E), n, seed,
                                                  out.ctypes.data_as(C.POINTER(C.c_float)), cap, C.byref(k), _dp(loc)))
        return out[: k.value], loc


class PlanStream:
    """Many plans through one GPU, several at a time, admitted by a device-memory budget
    (pmc_plans_* of the C ABI).  Plans are workloads.Problem-like objects (shape, voxel,
    origin, hu or mat/rho, spots) with a history count and a seed."""

    def __init__(self, device=0, slots=4, budget_bytes=64 << 30, n_batches=10, physics_flags=0, block_size=0,
                 chunk=0, fast_math=False):
        self._L = lib(LIB_FAST_PATH if fast_math else LIB_PATH)
        opt = Options()
        opt.device, opt.n_batches, opt.physics_flags = device, n_batches, physics_flags
        opt.block_size, opt.chunk = block_size, chunk
        self._s = C.c_void_p()
        rc = self._L.pmc_plans_create(C.byref(self._s), C.byref(opt), slots, budget_bytes)
        if rc != PMC_OK:
            raise PmcError(rc, "pmc_plans_create failed")
        self.n_batches = n_batches

    def close(self):
        if self._s:
            self._L.pmc_plans_destroy(self._s)
            self._s = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def _check(self, rc):
        if rc != PMC_OK:
            raise PmcError(rc, self._L.pmc_plans_last_error(self._s).decode())

    def load_materials(self, nuclides, materials, hu_bins=()):
        self._check(self._L.pmc_plans_load_materials(self._s, *_material_args(nuclides, materials, hu_bins)))

    def load_surrogate(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        self._check(self._L.pmc_plans_load_surrogate(self._s, _fp(p), p.size))

    @staticmethod
    def _plan(prob, n, seed, keep, outputs=True):
        nz, ny, nx = prob.shape
        pl = Plan()
        pl.nx, pl.ny, pl.nz = nx, ny, nz
        pl.dx, pl.dy, pl.dz = prob.voxel
        pl.x0, pl.y0, pl.z0 = prob.origin

        def arr(a, dt):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dtype=dt)
            keep.append(a)
            return a.ctypes.data

        pl.hu = arr(prob.hu, np.int16)
        if prob.hu is None:
            pl.mat, pl.rho = arr(prob.mat, np.uint8), arr(prob.rho, np.float32)
        pl.spots = arr(prob.spots, np.float64)
        pl.n_spots = len(prob.spots)
        pl.n_histories, pl.seed = n, seed
        dose = sigma = None
        if outputs:
            dose = np.empty(nx * ny * nz)
            keep.append(dose)
            pl.dose_gy = dose.ctypes.data
            if outputs != "dose":
                sigma = np.empty(nx * ny * nz)
                keep.append(sigma)
                pl.sigma_gy = sigma.ctypes.data
        return pl, dose, sigma

    def plan_bytes(self, prob, n, mode=0):
        keep = []
        pl, _, _ = self._plan(prob, n, 0, keep, outputs=False)
        b = C.c_uint64(0)
        self._check(self._L.pmc_plans_bytes(self._s, C.byref(pl), mode, C.byref(b)))
        return b.value

    def run(self, plans, mode=0, outputs=True):
        """plans: list of (problem, n_histories, seed); outputs True (dose and sigma), "dose"
        or False.  Returns (status, one dict per plan: status, slot, device_bytes,
        t_admit_ms, t_end_ms, gpu_ms, ledger, dose / sigma in Gy)."""
        keep, arr, outs = [], (Plan * max(1, len(plans)))(), []
        for i, (prob, n, seed) in enumerate(plans):
            pl, dose, sigma = self._plan(prob, n, seed, keep, outputs)
            arr[i] = pl
            outs.append((dose, sigma))
        res = (PlanResult * max(1, len(plans)))()
        rc = self._L.pmc_plans_run(self._s, arr, len(plans), mode, res)
        out = []
        for i in range(len(plans)):
            r = res[i]
            out.append({"status": r.status, "slot": r.slot, "device_bytes": r.device_bytes,
                        "t_admit_ms": r.t_admit_ms, "t_end_ms": r.t_end_ms, "gpu_ms": r.gpu_ms,
                        "ledger": {k: getattr(r.ledger, k) for k, _ in Ledger._fields_},
                        "dose": outs[i][0], "sigma": outs[i][1]})
        return rc, out


def gamma_index(ref, ev, voxel, dose_pct=2.0, dta_mm=2.0, threshold=0.1, search_mm=0.0, fast_math=False,
                want_map=True):
    """3-D gamma index on the GPU from host arrays (global criterion, on the grid).
    ref, ev: [nz, ny, nx] doses; voxel (dx, dy, dz) in cm; search_mm 0 means 1.5 dta.
    Returns (gamma per voxel as float32, -1 where not evaluated, or None; pass rate)."""
    ref = np.ascontiguousarray(ref, dtype=np.float64)
    ev = np.ascontiguousarray(ev, dtype=np.float64)
    if ref.ndim != 3 or ev.shape != ref.shape:
        raise ValueError("ref and ev must be [nz, ny, nx] arrays of one shape")
    nz, ny, nx = ref.shape
    g = np.empty(ref.shape, dtype=np.float32) if want_map else None
    rate = C.c_double(0.0)
    rc = lib(LIB_FAST_PATH if fast_math else LIB_PATH).pmc_gamma_index(
        _dp(ref), _dp(ev), nx, ny, nz, voxel[0], voxel[1], voxel[2], dose_pct, dta_mm, threshold, search_mm,
        _fp(g) if want_map else None, C.byref(rate))
    if rc != PMC_OK:
        raise PmcError(rc, "pmc_gamma_index failed")
    return g, rate.value


class GammaIndex:
    """3-D gamma index of device-resident doses (torch CUDA tensors of float64, [nz, ny, nx]),
    asynchronous on a stream.  The plan (the sorted search sphere) is made once per voxel
    size and distance criteria."""

    def __init__(self, voxel, dose_pct=2.0, dta_mm=2.0, threshold=0.1, search_mm=0.0, fast_math=False,
                 stream=None):
        import torch

        self.L = lib(LIB_FAST_PATH if fast_math else LIB_PATH)
        self.voxel = tuple(float(v) for v in voxel)
        self.dose_pct, self.threshold = dose_pct, threshold
        nb = C.c_size_t(0)
        rc = self.L.pmc_gamma_plan_bytes(*self.voxel, dta_mm, search_mm, C.byref(nb))
        if rc != PMC_OK:
            raise PmcError(rc, "pmc_gamma_plan_bytes failed")
        self.plan_bytes = nb.value
        self.buf = torch.empty((nb.value + 255) // 8 + 32, dtype=torch.float64, device="cuda")
        self.plan = (self.buf.data_ptr() + 255) // 256 * 256
        s = stream if stream is not None else torch.cuda.current_stream()
        rc = self.L.pmc_gamma_plan(*self.voxel, dta_mm, search_mm, self.plan, self.plan_bytes, s.cuda_stream)
        if rc != PMC_OK:
            raise PmcError(rc, "pmc_gamma_plan failed")

    def __call__(self, ref, ev, gamma=None, stream=None):
        """Launches on `stream` (torch stream or None for the current one).  counts() then
        gives (evaluated, passed) once the stream has reached it."""
        import torch

        assert ref.is_cuda and ev.is_cuda and ref.dtype == torch.float64 and ev.dtype == torch.float64
        assert ref.is_contiguous() and ev.is_contiguous() and ref.shape == ev.shape and ref.dim() == 3
        if gamma is not None:
            assert gamma.is_cuda and gamma.dtype == torch.float32 and gamma.is_contiguous()
            assert gamma.shape == ref.shape
        nz, ny, nx = ref.shape
        s = stream if stream is not None else torch.cuda.current_stream()
        rc = self.L.pmc_gamma_device(self.plan, ref.data_ptr(), ev.data_ptr(), nx, ny, nz, self.dose_pct,
                                     self.threshold, gamma.data_ptr() if gamma is not None else None, s.cuda_stream)
        if rc != PMC_OK:
            raise PmcError(rc, "pmc_gamma_device failed")

    def counts(self):
        import torch

        off = (self.plan - self.buf.data_ptr()) // 8
        c = self.buf[off:off + 2].view(torch.int64).cpu().numpy()
        return int(c[0]), int(c[1])


def debug_philox(ctr, key, fast_math=False):
    """Philox4x32-10 on the device: ctr [n, 4] uint32, key (2,) -> [n, 4] uint32."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.empty_like(ctr)
    P = C.POINTER(C.c_uint32)
    rc = lib(LIB_FAST_PATH if fast_math else LIB_PATH).pmc_debug_philox(ctr.ctypes.data_as(P), key.ctypes.data_as(P), out.ctypes.data_as(P), len(ctr))
    if rc != PMC_OK:
        raise PmcError(rc, "pmc_debug_philox failed")
    return out


def debug_vavilov_table(library: str | None = None):
    """The Vavilov straggling table as built by the library's host code [6][41][513] (no device)."""
    L = lib(library or LIB_PATH)
    out = np.empty((6, 41, 513), dtype=np.float32)
    rc = L.pmc_debug_vavilov_table(_fp(out), out.size)
    if rc != PMC_OK:
        raise PmcError(rc, "bad table size")
    return out
