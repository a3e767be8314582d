"""Thin ctypes binding of the C ABI in ``include/atm3.h`` (libatm3.so).

Argument marshalling only: every step of the computation runs in the CUDA
kernels behind the C ABI.  Host arrays are NumPy float64 SoA ``[3, n]``;
device arrays may be given as CUDA tensors (any object with ``data_ptr()``),
in which case the ``_dev`` entry points are used.  If the shared library is
missing, loading raises: there is no CPU fallback.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libatm3.so")

TRAVERSALS = {"3c01": 0, "3c18": 1, "3c08": 2, "3cw": 3, "3c08a": 4}
TRUNCATIONS = {"pair": 0, "product": 1}
PRECISIONS = {"fp64": 0, "fp32c": 1, "surrogate": 2}
FORCES = {"total": 0, "lj": 1, "atm": 2}

STATUS = {0: "ok", 1: "invalid argument", 2: "box smaller than three cells", 3: "CUDA error",
          4: "device wait timed out", 5: "non-finite input", 6: "call out of order",
          7: "capacity exceeded", 8: "fixed-point range exceeded"}

ABI_VERSION = 3  # ATM3_ABI_VERSION of include/atm3.h
EXPORTED = ["atm_abi_version", "atm_create", "atm_batch_create", "atm_batch_size", "atm_destroy",
            "atm_last_error", "atm_set_state", "atm_set_state_dev", "atm_build_cells",
            "atm_get_cells", "atm_compute_forces", "atm_get_results", "atm_get_forces",
            "atm_get_forces_dev", "atm_get_state", "atm_step", "atm_step_host", "atm_set_options",
            "atm_autotune",
            "atm_density_accumulate", "atm_density_get", "atm_density_reset",
            "atm_set_profiling", "atm_get_profile", "atm_compute_forces_noalloc",
            "atm_surrogate_set_model", "atm_surrogate_get_model", "atm_surrogate_init",
            "atm_surrogate_save", "atm_surrogate_load", "atm_surrogate_descriptors",
            "atm_surrogate_mlp", "atm_surrogate_loss_grad", "atm_surrogate_add_frame",
            "atm_surrogate_add_rows", "atm_surrogate_dataset", "atm_surrogate_clear",
            "atm_surrogate_train", "atm_surrogate_options", "atm_surrogate_error",
            "atm_measure_fma_peak", "atm_rdf_accumulate", "atm_rdf_get", "atm_rdf_reset",
            "atm_lj_tail", "atm_thermostat", "atm_measure_rsqrt_peak", "atm_set_forces",
            "atm_set_unit_classes", "atm_batch_cells", "atm_cell_grid", "atm_set_deterministic",
            "atm_set_pair_masks",
            "atm_surrogate_training_arithmetic", "atm_set_owned_layers"]

SUR_NDESC, SUR_NVEC, SUR_NOUT, SUR_NPARAM = 32, 48, 16, 7312


class Params(ctypes.Structure):
    _fields_ = [("box", ctypes.c_double * 3), ("rc", ctypes.c_double), ("nu", ctypes.c_double),
                ("lj_eps", ctypes.c_double), ("lj_sigma", ctypes.c_double),
                ("dt", ctypes.c_double), ("lj_shift", ctypes.c_int), ("device", ctypes.c_int),
                ("cuda_stream", ctypes.c_void_p)]


class Result(ctypes.Structure):
    _fields_ = [("e2", ctypes.c_double), ("e3", ctypes.c_double), ("w2", ctypes.c_double),
                ("w3", ctypes.c_double), ("ekin", ctypes.c_double),
                ("n_cand3", ctypes.c_uint64), ("n_int3", ctypes.c_uint64),
                ("n_cand2", ctypes.c_uint64), ("n_int2", ctypes.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Profile(ctypes.Structure):
    _fields_ = [("ms_cells", ctypes.c_double), ("ms_lj", ctypes.c_double),
                ("ms_atm", ctypes.c_double), ("ms_md", ctypes.c_double),
                ("n_launches", ctypes.c_int64), ("n_atm_launches", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Tuning(ctypes.Structure):
    _fields_ = [("persistent", ctypes.c_int), ("nwarps", ctypes.c_int),
                ("ms_per_eval", ctypes.c_double), ("nclass", ctypes.c_int),
                ("cut", ctypes.c_int * 2)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "cut"}
        d["cuts"] = [int(self.cut[i]) for i in range(max(0, self.nclass - 1))]
        return d


class AtmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s (%d): %s" % (STATUS.get(status, "?"), status, msg))
        self.status = status


_lib = None


def load():
    """Load libatm3.so (must have been built; see ``build.py``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libatm3.so is not built (%s); run paper_2510_21230_gb300.build.build()"
                           % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    P, i32, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
    sig = {
        "atm_abi_version": [],
        "atm_create": [ctypes.POINTER(Params), i64, ctypes.POINTER(P)],
        "atm_batch_create": [ctypes.POINTER(Params), P, i32, ctypes.POINTER(P)],
        "atm_batch_size": [P, P, P],
        "atm_batch_cells": [P, P],
        "atm_cell_grid": [ctypes.POINTER(Params), P],
        "atm_destroy": [P],
        "atm_set_state": [P, P, P],
        "atm_set_state_dev": [P, P, P],
        "atm_build_cells": [P],
        "atm_get_cells": [P, P, P, P, P],
        "atm_compute_forces": [P, i32, i32, i32, ctypes.POINTER(Result)],
        "atm_get_results": [P, ctypes.POINTER(Result)],
        "atm_get_forces": [P, P, i32],
        "atm_get_forces_dev": [P, P, i32],
        "atm_get_state": [P, P, P],
        "atm_step": [P, i32, i32, i32, i32, ctypes.POINTER(Result)],
        "atm_step_host": [P, i32, i32, i32, i32, P, P, P, ctypes.POINTER(Result)],
        "atm_set_options": [P, i32, i32, i32],
        "atm_set_unit_classes": [P, i32, P],
        "atm_set_deterministic": [P, i32],
        "atm_set_pair_masks": [P, i32],
        "atm_set_owned_layers": [P, i32, i32, i32],
        "atm_autotune": [P, i32, i32, i32, i32, ctypes.POINTER(Tuning)],
        "atm_density_accumulate": [P, i32, i32],
        "atm_density_get": [P, P, P],
        "atm_density_reset": [P],
        "atm_set_profiling": [P, i32],
        "atm_get_profile": [P, ctypes.POINTER(Profile)],
        "atm_compute_forces_noalloc": [ctypes.POINTER(Params), i64, P, i32, i32, i32, P,
                                       ctypes.POINTER(Result)],
        "atm_surrogate_set_model": [P, P, P, P],
        "atm_surrogate_get_model": [P, P, P, P],
        "atm_surrogate_init": [P, ctypes.c_uint64],
        "atm_surrogate_save": [P, ctypes.c_char_p],
        "atm_surrogate_load": [P, ctypes.c_char_p],
        "atm_surrogate_descriptors": [P, P, P],
        "atm_surrogate_mlp": [P, i64, P, P, P, P],
        "atm_surrogate_loss_grad": [P, i64, P, P, P, ctypes.c_double, P, P],
        "atm_surrogate_add_frame": [P, i32, i32, i32],
        "atm_surrogate_add_rows": [P, i64, P, P, P],
        "atm_surrogate_dataset": [P, P, P],
        "atm_surrogate_clear": [P],
        "atm_surrogate_train": [P, i64, i64, ctypes.c_double, ctypes.c_uint64, P],
        "atm_surrogate_options": [P, i32],
        "atm_surrogate_training_arithmetic": [P, i32],
        "atm_surrogate_error": [P, P, P, P, i32],
        "atm_measure_fma_peak": [i32, i32, P],
        "atm_rdf_accumulate": [P, ctypes.c_double, i32],
        "atm_rdf_get": [P, P, P],
        "atm_rdf_reset": [P],
        "atm_lj_tail": [ctypes.POINTER(Params), i64, P, P],
        "atm_thermostat": [P, P],
        "atm_measure_rsqrt_peak": [i32, P],
        "atm_set_forces": [P, P, i32, i32, i32],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.restype = i32
        fn.argtypes = args
    L.atm_last_error.restype = ctypes.c_char_p
    L.atm_last_error.argtypes = [P]
    if L.atm_abi_version() != ABI_VERSION:  # the structures above must match the library's
        raise RuntimeError("libatm3.so has ABI version %d, this binding %d"
                           % (L.atm_abi_version(), ABI_VERSION))
    _lib = L
    return L


def _host_ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _is_device(a):
    return hasattr(a, "data_ptr") and getattr(a, "is_cuda", False)


def make_params(box, rc=2.5, nu=0.073, lj_eps=1.0, lj_sigma=1.0, dt=0.002, lj_shift=False,
                device=0, stream=None):
    box = np.broadcast_to(np.asarray(box, dtype=np.float64), (3,))
    p = Params()
    for d in range(3):
        p.box[d] = float(box[d])
    p.rc, p.nu, p.lj_eps, p.lj_sigma, p.dt = rc, nu, lj_eps, lj_sigma, dt
    p.lj_shift = 1 if lj_shift else 0
    p.device = int(device)
    p.cuda_stream = stream
    return p


def cell_grid(box, rc=2.5):
    """Linked-cell grid (n_x, n_y, n_z) of one system, as the library forms it
    (``atm_cell_grid``)."""
    L = load()
    nc = np.zeros(3, dtype=np.int32)
    st = L.atm_cell_grid(ctypes.byref(make_params(box, rc)), _host_ptr(nc))
    if st != 0:
        raise AtmError(st, "atm_cell_grid failed")
    return nc


class AtmSystem:
    """One periodic LJ+ATM system, or a batch of independent replicas, on one
    GPU (wraps an ``atm_ctx``).  For a batch, ``n`` is a list, ``box`` a list
    of boxes and the other per-replica keyword arguments may be lists; state
    arrays are the replicas' SoA arrays back to back (shape ``[3, sum(n)]``)."""

    def __init__(self, box, n, rc=2.5, nu=0.073, lj_eps=1.0, lj_sigma=1.0, dt=0.002,
                 lj_shift=False, device=0, stream=None):
        self._lib = load()
        self._ctx = None
        ns = [int(v) for v in np.atleast_1d(n)]
        R = len(ns)
        boxes = np.asarray(box, dtype=np.float64)
        if boxes.ndim == 0:
            boxes = np.full((R, 3), float(boxes))
        elif boxes.ndim == 1:
            boxes = np.broadcast_to(boxes, (R, 3))

        def per(v, r):
            return v[r] if isinstance(v, (list, tuple, np.ndarray)) else v

        arr = (Params * R)()
        for r in range(R):
            arr[r] = make_params(boxes[r], per(rc, r), per(nu, r), per(lj_eps, r),
                                 per(lj_sigma, r), per(dt, r), per(lj_shift, r), device, stream)
        self.params = arr
        self.replicas = R
        self.ns = ns
        self.n = int(sum(ns))
        self.box = np.array(boxes[0])
        ctx = ctypes.c_void_p()
        nn = np.asarray(ns, dtype=np.int64)
        st = self._lib.atm_batch_create(arr, _host_ptr(nn), R, ctypes.byref(ctx))
        if st != 0:
            raise AtmError(st, "atm_batch_create failed")
        self._ctx = ctx
        nc = ctypes.c_int64()
        self._check(self._lib.atm_batch_cells(self._ctx, ctypes.byref(nc)))
        self.ncell_total = int(nc.value)

    # -- helpers
    def _check(self, st):
        if st != 0:
            raise AtmError(st, self._lib.atm_last_error(self._ctx).decode())

    def close(self):
        if getattr(self, "_ctx", None):
            self._lib.atm_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- state
    def set_state(self, x, v=None):
        if _is_device(x):
            assert tuple(x.shape) == (3, self.n) and x.is_contiguous()
            vp = None
            if v is not None:
                assert tuple(v.shape) == (3, self.n) and v.is_contiguous()
                vp = v.data_ptr()
            self._check(self._lib.atm_set_state_dev(self._ctx, x.data_ptr(), vp))
            return
        x = np.ascontiguousarray(x, dtype=np.float64)
        assert x.shape == (3, self.n)
        vp = None
        if v is not None:
            v = np.ascontiguousarray(v, dtype=np.float64)
            assert v.shape == (3, self.n)
            vp = _host_ptr(v)
        self._check(self._lib.atm_set_state(self._ctx, _host_ptr(x), vp))

    def set_forces(self, f, trav="3c08", trunc="pair", prec="fp32c"):
        """Total force of the state just set (original order), as computed with
        (trav, trunc, prec): the next step with that combination starts from it."""
        f = np.ascontiguousarray(f, dtype=np.float64)
        assert f.shape == (3, self.n)
        self._check(self._lib.atm_set_forces(self._ctx, _host_ptr(f), TRAVERSALS[trav],
                                             TRUNCATIONS[trunc], PRECISIONS[prec]))

    def step_host(self, x, v, f=None, nsteps=1, trav="3c08", trunc="pair", prec="fp32c"):
        """One host round trip (atm_step_host): x, v (and f, when given) are the
        state and its total force; they are overwritten in place with the state
        and total force after nsteps steps.  Returns the scalars."""
        for a in (x, v) + ((f,) if f is not None else ()):
            assert a.shape == (3, self.n) and a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
        r = Result()
        self._check(self._lib.atm_step_host(self._ctx, int(nsteps), TRAVERSALS[trav],
                                            TRUNCATIONS[trunc], PRECISIONS[prec], _host_ptr(x),
                                            _host_ptr(v), _host_ptr(f) if f is not None else None,
                                            ctypes.byref(r)))
        return r.as_dict()

    def get_state(self, x=None, v=None):
        x = np.zeros((3, self.n)) if x is None else x
        v = np.zeros((3, self.n)) if v is None else v
        self._check(self._lib.atm_get_state(self._ctx, _host_ptr(x), _host_ptr(v)))
        return x, v

    # -- cells
    def build_cells(self):
        self._check(self._lib.atm_build_cells(self._ctx))

    def get_cells(self):
        """Cell arrays (for a batch in the global cell numbering; ncell is replica 0's grid)."""
        nc = np.zeros(3, dtype=np.int32)
        cell_of = np.zeros(self.n, dtype=np.int32)
        start = np.zeros(self.ncell_total + 1, dtype=np.int32)
        perm = np.zeros(self.n, dtype=np.int32)
        self._check(self._lib.atm_get_cells(self._ctx, _host_ptr(cell_of), _host_ptr(start),
                                            _host_ptr(perm), _host_ptr(nc)))
        return dict(cell_of=cell_of, cell_start=start, perm=perm, ncell=nc)

    # -- forces
    def compute_forces(self, trav="3c18", trunc="pair", prec="fp64", sync=True):
        r = Result()
        self._check(self._lib.atm_compute_forces(
            self._ctx, TRAVERSALS[trav], TRUNCATIONS[trunc], PRECISIONS[prec],
            ctypes.byref(r) if sync else None))
        return r.as_dict() if sync else None

    def results(self):
        """Scalars of the last evaluation, one dict per replica."""
        out = (Result * self.replicas)()
        self._check(self._lib.atm_get_results(self._ctx, out))
        return [out[r].as_dict() for r in range(self.replicas)]

    def get_forces(self, which="total", out=None):
        if out is not None and _is_device(out):
            assert tuple(out.shape) == (3, self.n) and out.is_contiguous()
            self._check(self._lib.atm_get_forces_dev(self._ctx, out.data_ptr(), FORCES[which]))
            return out
        f = np.zeros((3, self.n)) if out is None else out
        self._check(self._lib.atm_get_forces(self._ctx, _host_ptr(f), FORCES[which]))
        return f

    def step(self, nsteps=1, trav="3c18", trunc="pair", prec="fp64", sync=True):
        r = Result()
        self._check(self._lib.atm_step(self._ctx, int(nsteps), TRAVERSALS[trav],
                                       TRUNCATIONS[trunc], PRECISIONS[prec],
                                       ctypes.byref(r) if sync else None))
        return r.as_dict() if sync else None

    # -- launch options, autotuning
    def set_options(self, persistent=False, nwarps=0, graph=False):
        self._check(self._lib.atm_set_options(self._ctx, int(bool(persistent)), int(nwarps),
                                              int(bool(graph))))

    def set_owned_layers(self, z_lo, z_hi, replica=0):
        """Domain decomposition: the replica owns cell layers [z_lo, z_hi)
        (``atm_set_owned_layers``)."""
        self._check(self._lib.atm_set_owned_layers(self._ctx, int(replica), int(z_lo), int(z_hi)))

    def set_pair_masks(self, on=True):
        """FP32C pair rule of the block traversals: pairs decided once per
        evaluation into per-molecule bitmaps (on, the default) or by each unit."""
        self._check(self._lib.atm_set_pair_masks(self._ctx, int(bool(on))))

    def set_deterministic(self, on=True):
        """Deterministic mode (``atm_set_deterministic``): repeated runs give
        bit-identical forces, energies, virials and counts."""
        self._check(self._lib.atm_set_deterministic(self._ctx, 1 if on else 0))

    def set_unit_classes(self, cuts=()):
        """Unit size classes of the block traversals: cuts = () for one
        launch, else 1 or 2 rising bounds (staged molecules)."""
        cuts = [int(c) for c in cuts]
        arr = (ctypes.c_int * max(1, len(cuts)))(*cuts) if cuts else None
        self._check(self._lib.atm_set_unit_classes(self._ctx, len(cuts) + 1, arr))

    def autotune(self, trav="3c08", trunc="pair", prec="fp32c", reps=3):
        t = Tuning()
        self._check(self._lib.atm_autotune(self._ctx, TRAVERSALS[trav], TRUNCATIONS[trunc],
                                           PRECISIONS[prec], int(reps), ctypes.byref(t)))
        return t.as_dict()

    # -- density profile
    def density_accumulate(self, axis=2, nbins=600):
        self._check(self._lib.atm_density_accumulate(self._ctx, int(axis), int(nbins)))

    def density_get(self, nbins):
        counts = np.zeros((self.replicas, nbins), dtype=np.uint64)
        samples = np.zeros(1, dtype=np.int64)
        self._check(self._lib.atm_density_get(self._ctx, _host_ptr(counts), _host_ptr(samples)))
        return counts, int(samples[0])

    def thermostat(self, temperature):
        """Rescale velocities so that each replica's kinetic temperature is
        ``temperature`` (a number or one value per replica)."""
        t = np.ascontiguousarray(np.broadcast_to(np.asarray(temperature, dtype=np.float64),
                                                 (self.replicas,)))
        self._check(self._lib.atm_thermostat(self._ctx, _host_ptr(t)))

    def rdf_accumulate(self, r_max=2.5, nbins=250):
        self._check(self._lib.atm_rdf_accumulate(self._ctx, float(r_max), int(nbins)))

    def rdf_get(self, nbins):
        counts = np.zeros((self.replicas, nbins), dtype=np.uint64)
        samples = np.zeros(1, dtype=np.int64)
        self._check(self._lib.atm_rdf_get(self._ctx, _host_ptr(counts), _host_ptr(samples)))
        return counts, int(samples[0])

    def rdf_reset(self):
        self._check(self._lib.atm_rdf_reset(self._ctx))

    def density_reset(self):
        self._check(self._lib.atm_density_reset(self._ctx))

    # -- profiling (device time of the library's kernels, launch counts)
    def set_profiling(self, on=True, forces_only=False):
        """Device-time profile of the library's launch groups; forces_only
        times the force evaluations alone (fewer timestamps in a step)."""
        self._check(self._lib.atm_set_profiling(self._ctx, (2 if forces_only else 1) if on else 0))

    def get_profile(self):
        p = Profile()
        self._check(self._lib.atm_get_profile(self._ctx, ctypes.byref(p)))
        return p.as_dict()


    # ------------------------------------------------------- surrogate

    def surrogate_set_model(self, params, mean, scale):
        params = np.ascontiguousarray(params, dtype=np.float32)
        mean = np.ascontiguousarray(mean, dtype=np.float32)
        scale = np.ascontiguousarray(scale, dtype=np.float32)
        assert params.size == SUR_NPARAM and mean.size == SUR_NDESC and scale.size == SUR_NDESC
        self._check(self._lib.atm_surrogate_set_model(self._ctx, _host_ptr(params), _host_ptr(mean),
                                                    _host_ptr(scale)))

    def surrogate_get_model(self):
        params = np.zeros(SUR_NPARAM, dtype=np.float32)
        mean = np.zeros(SUR_NDESC, dtype=np.float32)
        scale = np.zeros(SUR_NDESC, dtype=np.float32)
        self._check(self._lib.atm_surrogate_get_model(self._ctx, _host_ptr(params), _host_ptr(mean),
                                                    _host_ptr(scale)))
        return params, mean, scale

    def surrogate_init(self, seed=0):
        self._check(self._lib.atm_surrogate_init(self._ctx, int(seed)))

    def surrogate_save(self, path):
        self._check(self._lib.atm_surrogate_save(self._ctx, os.fsencode(path)))

    def surrogate_load(self, path):
        self._check(self._lib.atm_surrogate_load(self._ctx, os.fsencode(path)))

    def surrogate_descriptors(self):
        """Descriptors ``[n, 32]`` and vectors ``[n, 48]`` (float32, original order)."""
        D = np.zeros((self.n, SUR_NDESC), dtype=np.float32)
        V = np.zeros((self.n, SUR_NVEC), dtype=np.float32)
        self._check(self._lib.atm_surrogate_descriptors(self._ctx, _host_ptr(D), _host_ptr(V)))
        return D, V

    def surrogate_mlp(self, D, V):
        """Tensor-core inference on given rows: ``(w [rows, 3], F [rows, 3])``."""
        D = np.ascontiguousarray(D, dtype=np.float32).reshape(-1, SUR_NDESC)
        V = np.ascontiguousarray(V, dtype=np.float32).reshape(-1, SUR_NVEC)
        n = D.shape[0]
        w = np.zeros((n, SUR_NOUT), dtype=np.float32)
        F = np.zeros((n, 3), dtype=np.float32)
        self._check(self._lib.atm_surrogate_mlp(self._ctx, n, _host_ptr(D), _host_ptr(V),
                                              _host_ptr(w), _host_ptr(F)))
        return w, F

    def surrogate_loss_grad(self, D, V, T, sigma2):
        D = np.ascontiguousarray(D, dtype=np.float32).reshape(-1, SUR_NDESC)
        V = np.ascontiguousarray(V, dtype=np.float32).reshape(-1, SUR_NVEC)
        T = np.ascontiguousarray(T, dtype=np.float32).reshape(-1, 3)
        loss = ctypes.c_double(0.0)
        g = np.zeros(SUR_NPARAM, dtype=np.float32)
        self._check(self._lib.atm_surrogate_loss_grad(self._ctx, D.shape[0], _host_ptr(D),
                                                    _host_ptr(V), _host_ptr(T), float(sigma2),
                                                    ctypes.byref(loss), _host_ptr(g)))
        return loss.value, g

    def surrogate_add_frame(self, trav="3c08", trunc="pair", prec="fp32c"):
        self._check(self._lib.atm_surrogate_add_frame(self._ctx, TRAVERSALS[trav],
                                                    TRUNCATIONS[trunc], PRECISIONS[prec]))

    def surrogate_add_rows(self, D, V, T):
        D = np.ascontiguousarray(D, dtype=np.float32).reshape(-1, SUR_NDESC)
        V = np.ascontiguousarray(V, dtype=np.float32).reshape(-1, SUR_NVEC)
        T = np.ascontiguousarray(T, dtype=np.float32).reshape(-1, 3)
        self._check(self._lib.atm_surrogate_add_rows(self._ctx, D.shape[0], _host_ptr(D),
                                                   _host_ptr(V), _host_ptr(T)))

    def surrogate_dataset(self):
        """``(rows, sigma2)`` of the device-side training set."""
        rows = ctypes.c_int64(0)
        s2 = ctypes.c_double(0.0)
        self._check(self._lib.atm_surrogate_dataset(self._ctx, ctypes.byref(rows), ctypes.byref(s2)))
        return rows.value, s2.value

    def surrogate_clear(self):
        self._check(self._lib.atm_surrogate_clear(self._ctx))

    def surrogate_train(self, steps, batch=0, lr=1e-3, seed=0):
        """Adam steps on the data set; returns the per-step minibatch losses."""
        loss = np.zeros(max(0, int(steps)), dtype=np.float64)
        self._check(self._lib.atm_surrogate_train(self._ctx, int(steps), int(batch), float(lr),
                                                int(seed), _host_ptr(loss)))
        return loss

    def surrogate_training_arithmetic(self, tensor_cores=True):
        """Gradients on the tensor cores (bfloat16 operands, FP32 sums; the
        default) or in FP32 on the CUDA cores."""
        self._check(self._lib.atm_surrogate_training_arithmetic(self._ctx, 1 if tensor_cores else 0))

    def surrogate_options(self, exact_every=50):
        self._check(self._lib.atm_surrogate_options(self._ctx, int(exact_every)))

    def surrogate_error(self, reset=False):
        """``(rms_diff, rms_exact, checks)`` of the interleaved exact steps."""
        d = ctypes.c_double(0.0)
        e = ctypes.c_double(0.0)
        k = ctypes.c_int64(0)
        self._check(self._lib.atm_surrogate_error(self._ctx, ctypes.byref(d), ctypes.byref(e),
                                                ctypes.byref(k), 1 if reset else 0))
        return d.value, e.value, k.value


def lj_tail(box, n, rc=2.5, lj_eps=1.0, lj_sigma=1.0):
    """Long-range corrections (total energy, pressure) of truncated LJ."""
    L = load()
    p = make_params(box, rc=rc, lj_eps=lj_eps, lj_sigma=lj_sigma)
    e = ctypes.c_double(0.0)
    pt = ctypes.c_double(0.0)
    st = L.atm_lj_tail(ctypes.byref(p), int(n), ctypes.byref(e), ctypes.byref(pt))
    if st != 0:
        raise AtmError(st, "atm_lj_tail failed")
    return e.value, pt.value


def measure_rsqrt_peak(device=0):
    """Measured FP32 rsqrt throughput of the device in G operations/s."""
    L = load()
    g = ctypes.c_double(0.0)
    st = L.atm_measure_rsqrt_peak(int(device), ctypes.byref(g))
    if st != 0:
        raise AtmError(st, "atm_measure_rsqrt_peak failed")
    return g.value


def measure_fma_peak(device=0, fp64=False):
    """Measured FMA throughput of the device in TFLOP/s (FP32 or FP64)."""
    L = load()
    t = ctypes.c_double(0.0)
    st = L.atm_measure_fma_peak(int(device), 1 if fp64 else 0, ctypes.byref(t))
    if st != 0:
        raise AtmError(st, "atm_measure_fma_peak failed")
    return t.value


def compute_forces_noalloc(box, x_dev, f_dev, trav="3c18", trunc="pair", prec="fp64", rc=2.5,
                           nu=0.073, lj_eps=1.0, lj_sigma=1.0, lj_shift=False, device=0,
                           stream=None):
    """One force evaluation through ``atm_compute_forces_noalloc``: no device
    memory is allocated by the library (for callers that cannot allocate);
    ``x_dev`` and ``f_dev`` are caller-owned [3, n] float64 CUDA tensors.
    Returns the scalars of the evaluation."""
    L = load()
    n = int(x_dev.shape[1])
    assert tuple(x_dev.shape) == (3, n) and tuple(f_dev.shape) == (3, n)
    assert x_dev.is_contiguous() and f_dev.is_contiguous()
    p = make_params(box, rc, nu, lj_eps, lj_sigma, 0.0, lj_shift, device, stream)
    r = Result()
    st = L.atm_compute_forces_noalloc(ctypes.byref(p), n, x_dev.data_ptr(), TRAVERSALS[trav],
                                      TRUNCATIONS[trunc], PRECISIONS[prec], f_dev.data_ptr(),
                                      ctypes.byref(r))
    if st != 0:
        raise AtmError(st, "atm_compute_forces_noalloc failed")
    return r.as_dict()
