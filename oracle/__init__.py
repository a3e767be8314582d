"""CPU oracle for the ATM linked-cell method (arXiv 2510.21230) and for the
learned force surrogate that can stand in for its triplet sum.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It wraps the plain C
oracles in ``atm_oracle.c`` and ``sur_oracle.c`` through ctypes and shares nothing with the CUDA
library.

Every array argument is a NumPy array; 3-vectors are SoA ``[3, n]`` (x row,
y row, z row) in float64.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "atm_oracle.c"), os.path.join(_HERE, "sur_oracle.c")]
_HDRS = [os.path.join(_HERE, "atm_oracle.h"), os.path.join(_HERE, "sur_oracle.h")]
_LIB = os.path.join(_HERE, "libatm_oracle.so")

TRAV = {"3c01": 0, "3c18": 1, "3c08": 2, "3cw": 3, "3c08a": 4}
TRUNC = {"pair": 0, "product": 1}
PREC = {"fp64": 0, "fp32": 1}

GCC_FLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
             "-fno-fast-math", "-Wall"]


def build(force=False):
    """Compile the oracle with gcc (no contraction of multiply-adds)."""
    newest = max(os.path.getmtime(f) for f in _SRCS + _HDRS)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    subprocess.check_call(["gcc", *GCC_FLAGS, "-o", tmp, *_SRCS, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        d, i64, i32, ci = ctypes.c_double, ctypes.c_int64, ctypes.c_int32, ctypes.c_int
        P = ctypes.c_void_p
        L.orc_atm_u.restype = d
        L.orc_atm_u.argtypes = [d, d, d, d]
        L.orc_atm_du_dsq.restype = None
        L.orc_atm_du_dsq.argtypes = [d, d, d, d, P]
        L.orc_atm_dudr_paper.restype = d
        L.orc_atm_dudr_paper.argtypes = [d, d, d, d]
        L.orc_cell_grid.restype = ci
        L.orc_cell_grid.argtypes = [P, P, P]
        L.orc_build_cells.restype = ci
        L.orc_build_cells.argtypes = [P, i64, P, P, P, P, P, P, P]
        L.orc_atm_brute.restype = ci
        L.orc_atm_brute.argtypes = [P, i64, P, ci, ci, P, P, P]
        L.orc_atm_cells.restype = ci
        L.orc_atm_cells.argtypes = [P, i64, P, ci, ci, ci, i64, i64, P, P, P]
        L.orc_atm_cells_units.restype = ci
        L.orc_atm_cells_units.argtypes = [P, i64, P, ci, ci, ci, P, i64, P, P, P]
        L.orc_lj_brute.restype = ci
        L.orc_lj_brute.argtypes = [P, i64, P, P, P, P]
        L.orc_lj_cells.restype = ci
        L.orc_lj_cells.argtypes = [P, i64, P, ci, P, P, P]
        L.orc_md_run.restype = ci
        L.orc_md_run.argtypes = [P, i64, P, P, ci, d, ci, ci, ci, P, P]
        L.orc_rdf.restype = ci
        L.orc_rdf.argtypes = [P, i64, P, d, ci, P]
        L.orc_lj_tail.restype = ci
        L.orc_lj_tail.argtypes = [P, i64, ci, P]
        L.orc_rescale.restype = ci
        L.orc_rescale.argtypes = [i64, P, d]
        L.orc_num_threads.restype = ci
        L.orc_num_threads.argtypes = []
        L.orc_sur_basis.restype = None
        L.orc_sur_basis.argtypes = [d, P, P, P, P]
        L.orc_sur_fcut.restype = d
        L.orc_sur_fcut.argtypes = [d, d]
        L.orc_sur_descriptors.restype = ci
        L.orc_sur_descriptors.argtypes = [P, P, i64, P, i64, P, P]
        L.orc_bf16.restype = d
        L.orc_bf16.argtypes = [d]
        L.orc_sur_mlp.restype = None
        L.orc_sur_mlp.argtypes = [P, P, P, i64, P, P, ci, P, P]
        L.orc_sur_loss_grad.restype = None
        L.orc_sur_loss_grad.argtypes = [P, P, P, i64, P, P, P, d, P, P]
        L.orc_sur_adam.restype = None
        L.orc_sur_adam.argtypes = [P, P, P, P, i64, i64, d, d, d, d]
        L.orc_sur_stats.restype = None
        L.orc_sur_stats.argtypes = [i64, P, P, P, P, P]
        _lib = L
    return _lib


class OracleError(RuntimeError):
    pass


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(st):
    if st != 0:
        raise OracleError({1: "invalid argument", 2: "box smaller than 3 cells"}.get(st, str(st)))


def params(box, rc, nu, lj_eps=1.0, lj_sigma=1.0, lj_shift=False):
    b = np.broadcast_to(np.asarray(box, dtype=np.float64), (3,))
    return np.array([b[0], b[1], b[2], rc, nu, lj_eps, lj_sigma, 1.0 if lj_shift else 0.0],
                    dtype=np.float64)


def _soa(x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    assert x.ndim == 2 and x.shape[0] == 3
    return x


def atm_u(a, b, c, nu):
    return lib().orc_atm_u(a, b, c, nu)


def atm_du_dsq(a, b, c, nu):
    out = np.zeros(3)
    lib().orc_atm_du_dsq(a, b, c, nu, _p(out))
    return out


def atm_dudr_paper(rij, rik, rjk, nu):
    return lib().orc_atm_dudr_paper(rij, rik, rjk, nu)


def cell_grid(prm):
    nc = np.zeros(3, dtype=np.int32)
    w = np.zeros(3)
    _check(lib().orc_cell_grid(_p(prm), _p(nc), _p(w)))
    return nc, w


def build_cells(prm, x):
    x = _soa(x)
    n = x.shape[1]
    nc, _ = cell_grid(prm)
    ncell = int(np.prod(nc.astype(np.int64)))
    xw = np.zeros((3, n))
    cell_of = np.zeros(n, dtype=np.int32)
    start = np.zeros(ncell + 1, dtype=np.int32)
    perm = np.zeros(n, dtype=np.int32)
    xl = np.zeros((3, n))
    xl32 = np.zeros((3, n), dtype=np.float32)
    _check(lib().orc_build_cells(_p(prm), n, _p(x), _p(xw), _p(cell_of), _p(start), _p(perm),
                                 _p(xl), _p(xl32)))
    return dict(xw=xw, cell_of=cell_of, cell_start=start, perm=perm, xl=xl, xl32=xl32,
                ncell=nc)


def atm_brute(prm, x, trunc="pair", member=None):
    x = _soa(x)
    n = x.shape[1]
    f = np.zeros((3, n))
    ew = np.zeros(2)
    cnt = np.zeros(1, dtype=np.uint64)
    m = -1 if member is None else TRAV[member]
    _check(lib().orc_atm_brute(_p(prm), n, _p(x), TRUNC[trunc], m, _p(f), _p(ew), _p(cnt)))
    return dict(f=f, e3=ew[0], w3=ew[1], n_int3=int(cnt[0]))


def atm_cells(prm, x, trav="3c18", trunc="pair", prec="fp64", unit_lo=-1, unit_hi=-1):
    x = _soa(x)
    n = x.shape[1]
    f = np.zeros((3, n))
    ew = np.zeros(2)
    cnt = np.zeros(2, dtype=np.uint64)
    _check(lib().orc_atm_cells(_p(prm), n, _p(x), TRAV[trav], TRUNC[trunc], PREC[prec],
                               unit_lo, unit_hi, _p(f), _p(ew), _p(cnt)))
    return dict(f=f, e3=ew[0], w3=ew[1], n_cand3=int(cnt[0]), n_int3=int(cnt[1]))


def atm_cells_units(prm, x, units, trav="3c18", trunc="pair", prec="fp64"):
    """Linked-cell ATM restricted to the listed units (base cells / block anchors)."""
    x = _soa(x)
    n = x.shape[1]
    u = np.ascontiguousarray(units, dtype=np.int64)
    f = np.zeros((3, n))
    ew = np.zeros(2)
    cnt = np.zeros(2, dtype=np.uint64)
    _check(lib().orc_atm_cells_units(_p(prm), n, _p(x), TRAV[trav], TRUNC[trunc], PREC[prec],
                                     _p(u), u.size, _p(f), _p(ew), _p(cnt)))
    return dict(f=f, e3=ew[0], w3=ew[1], n_cand3=int(cnt[0]), n_int3=int(cnt[1]))


def lj_brute(prm, x):
    x = _soa(x)
    n = x.shape[1]
    f = np.zeros((3, n))
    ew = np.zeros(2)
    cnt = np.zeros(1, dtype=np.uint64)
    _check(lib().orc_lj_brute(_p(prm), n, _p(x), _p(f), _p(ew), _p(cnt)))
    return dict(f=f, e2=ew[0], w2=ew[1], n_int2=int(cnt[0]))


def lj_cells(prm, x, prec="fp64"):
    x = _soa(x)
    n = x.shape[1]
    f = np.zeros((3, n))
    ew = np.zeros(2)
    cnt = np.zeros(2, dtype=np.uint64)
    _check(lib().orc_lj_cells(_p(prm), n, _p(x), PREC[prec], _p(f), _p(ew), _p(cnt)))
    return dict(f=f, e2=ew[0], w2=ew[1], n_cand2=int(cnt[0]), n_int2=int(cnt[1]))


def md_run(prm, x, v, nsteps, dt, trav="3c18", trunc="pair", prec="fp64"):
    """Velocity-Verlet NVE; returns final x, v, f and per-step energies
    ``[nsteps+1, 4]`` = (E2, E3, Ekin, W2+W3)."""
    x = _soa(x).copy()
    v = _soa(v).copy()
    n = x.shape[1]
    f = np.zeros((3, n))
    en = np.zeros((nsteps + 1, 4))
    _check(lib().orc_md_run(_p(prm), n, _p(x), _p(v), nsteps, dt, TRAV[trav], TRUNC[trunc],
                            PREC[prec], _p(f), _p(en)))
    return dict(x=x, v=v, f=f, energies=en)


def rdf_counts(prm, x, r_max, nbins):
    """Pair-distance histogram (every pair once) over [0, r_max) in nbins bins."""
    x = _soa(x)
    counts = np.zeros(nbins, dtype=np.uint64)
    _check(lib().orc_rdf(_p(prm), x.shape[1], _p(x), float(r_max), int(nbins), _p(counts)))
    return counts


def rdf_normalise(counts, samples, n, volume, r_max):
    """g(r) at the bin centres from pair counts: counts / (samples N/2 rho dV)."""
    counts = np.asarray(counts, dtype=np.float64)
    nb = counts.shape[-1]
    edges = np.linspace(0.0, r_max, nb + 1)
    shell = 4.0 / 3.0 * np.pi * (edges[1:] ** 3 - edges[:-1] ** 3)
    rho = n / volume
    return 0.5 * (edges[1:] + edges[:-1]), counts / (samples * 0.5 * n * rho * shell)


def lj_tail(prm, n, intervals=20000):
    """(E_tail, P_tail) of truncated LJ by quadrature of the tail integrals."""
    out = np.zeros(2)
    _check(lib().orc_lj_tail(_p(prm), int(n), int(intervals), _p(out)))
    return out[0], out[1]


def rescale(v, temperature):
    """Velocities scaled to kinetic temperature ``temperature`` (a copy)."""
    v = _soa(v).copy()
    _check(lib().orc_rescale(v.shape[1], _p(v), float(temperature)))
    return v


def num_threads():
    return lib().orc_num_threads()


# ---------------------------------------------------------------- surrogate

SUR_ND, SUR_NH, SUR_NO, SUR_NV = 32, 64, 16, 48
SUR_NP = SUR_ND * SUR_NH + SUR_NH + SUR_NH * SUR_NH + SUR_NH + SUR_NH * SUR_NO + SUR_NO


def sur_basis(rc):
    mu_g = np.zeros(16)
    mu_v = np.zeros(4)
    eg = np.zeros(1)
    ev = np.zeros(1)
    lib().orc_sur_basis(rc, _p(mu_g), _p(eg), _p(mu_v), _p(ev))
    return mu_g, float(eg[0]), mu_v, float(ev[0])


def sur_fcut(r, rc):
    return lib().orc_sur_fcut(r, rc)


def sur_descriptors(prm, x, rows=None):
    """Descriptors ``[nrows, 32]`` and vectors ``[nrows, 48]`` (v_0 .. v_15) of
    the molecules ``rows`` (default all), brute force over all molecules."""
    x = _soa(x)
    n = x.shape[1]
    r = np.arange(n, dtype=np.int64) if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    D = np.zeros((r.size, SUR_ND))
    V = np.zeros((r.size, SUR_NV))
    st = lib().orc_sur_descriptors(_p(prm), _p(x), n, _p(r), r.size, _p(D), _p(V))
    if st != 0:
        raise OracleError("surrogate descriptors need rc > 0.8 and every box side >= 2 rc")
    return D, V


def bf16(x):
    return lib().orc_bf16(float(x))


def sur_mlp(P, mean, scale, D, V, bf16_=False):
    """MLP weights ``w [n, 3]`` and forces ``F [n, 3]`` (row per molecule)."""
    P = np.ascontiguousarray(P, dtype=np.float64)
    assert P.size == SUR_NP
    mean = np.ascontiguousarray(mean, dtype=np.float64)
    scale = np.ascontiguousarray(scale, dtype=np.float64)
    D = np.ascontiguousarray(D, dtype=np.float64).reshape(-1, SUR_ND)
    V = np.ascontiguousarray(V, dtype=np.float64).reshape(-1, SUR_NV)
    n = D.shape[0]
    w = np.zeros((n, SUR_NO))
    F = np.zeros((n, 3))
    lib().orc_sur_mlp(_p(P), _p(mean), _p(scale), n, _p(D), _p(V), 1 if bf16_ else 0, _p(w), _p(F))
    return w, F


def sur_loss_grad(P, mean, scale, D, V, Fref, sigma2):
    P = np.ascontiguousarray(P, dtype=np.float64)
    mean = np.ascontiguousarray(mean, dtype=np.float64)
    scale = np.ascontiguousarray(scale, dtype=np.float64)
    D = np.ascontiguousarray(D, dtype=np.float64).reshape(-1, SUR_ND)
    V = np.ascontiguousarray(V, dtype=np.float64).reshape(-1, SUR_NV)
    Fref = np.ascontiguousarray(Fref, dtype=np.float64).reshape(-1, 3)
    n = D.shape[0]
    loss = np.zeros(1)
    g = np.zeros(SUR_NP)
    lib().orc_sur_loss_grad(_p(P), _p(mean), _p(scale), n, _p(D), _p(V), _p(Fref), sigma2,
                            _p(loss), _p(g))
    return float(loss[0]), g


def sur_adam(P, m, v, g, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step in place on float64 arrays P, m, v."""
    lib().orc_sur_adam(_p(P), _p(m), _p(v), _p(np.ascontiguousarray(g, dtype=np.float64)),
                       P.size, t, lr, beta1, beta2, eps)


def sur_stats(D, F):
    D = np.ascontiguousarray(D, dtype=np.float64).reshape(-1, SUR_ND)
    F = np.ascontiguousarray(F, dtype=np.float64).reshape(-1, 3)
    mean = np.zeros(SUR_ND)
    scale = np.zeros(SUR_ND)
    s2 = np.zeros(1)
    lib().orc_sur_stats(D.shape[0], _p(D), _p(F), _p(mean), _p(scale), _p(s2))
    return mean, scale, float(s2[0])
