"""The C ABI library builds for sm_103a, loads, and exports every entry point
that include/atm3.h declares (no GPU needed: nothing is computed)."""
import ctypes
import os
import re

import pytest

from paper_2510_21230_gb300 import atm3, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    with open(os.path.join(ROOT, "include", "atm3.h")) as fh:
        text = fh.read()
    for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(atm_[a-z0-9_]+)\s*\(",
                         text, re.M):
        names.add(m.group(1))
    return names


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    declared = _declared()
    assert "atm_compute_forces" in declared and "atm_step" in declared
    for name in sorted(declared):
        assert hasattr(lib, name), name
    assert set(atm3.EXPORTED) <= declared
    assert atm3.load().atm_abi_version() == 3


def test_invalid_arguments_are_rejected_without_a_gpu():
    lib = atm3.load()
    p = atm3.Params()
    for d in range(3):
        p.box[d] = 10.0
    p.rc, p.nu, p.lj_eps, p.lj_sigma, p.dt = 2.5, 0.073, 1.0, 1.0, 0.002
    ctx = ctypes.c_void_p()
    assert lib.atm_create(ctypes.byref(p), -1, ctypes.byref(ctx)) == 1
    p.box[0] = 7.0  # two cells of 3.5 along x
    assert lib.atm_create(ctypes.byref(p), 10, ctypes.byref(ctx)) == 2
    p.box[0] = 10.0
    p.rc = -1.0
    assert lib.atm_create(ctypes.byref(p), 10, ctypes.byref(ctx)) == 1
    assert lib.atm_destroy(None) == 0
    assert lib.atm_compute_forces(None, 0, 0, 0, None) == 1


@pytest.mark.parametrize("box,rc", [((10.77, 10.77, 10.77), 2.5), ((30.0, 30.0, 120.0), 2.5),
                                    ((37.5, 37.5, 37.5), 2.5), ((7.5, 7.5, 7.5), 2.5),
                                    ((9.0, 12.0, 40.0), 3.0)])
def test_cell_grid_query_matches_the_oracle(box, rc):
    """atm_cell_grid (host arithmetic) gives the oracle's cell grid: n_d the
    largest k with L_d / k >= r_c (37.5 / 2.5 is not binary-exact; 7.5 / 2.5
    lands on exactly 3 cells)."""
    import oracle
    nc = atm3.cell_grid(box, rc)
    assert list(nc) == list(oracle.cell_grid(oracle.params(box, rc, 0.0))[0])
    with pytest.raises(atm3.AtmError) as ei:
        atm3.cell_grid((7.4, 10.0, 10.0), 2.5)
    assert ei.value.status == 2


@pytest.mark.parametrize("rc,rho,eps,sig", [(2.5, 0.8, 1.0, 1.0), (3.0, 0.65, 1.0, 1.0),
                                            (5.0, 0.1, 2.0, 1.7)])
def test_lj_tail_matches_the_oracle_quadrature(rc, rho, eps, sig):
    """atm_lj_tail is host arithmetic: checked here against the oracle's
    numerical tail integrals."""
    import oracle
    n = 2000
    box = (n / rho) ** (1.0 / 3.0)
    e, p = atm3.lj_tail(box, n, rc=rc, lj_eps=eps, lj_sigma=sig)
    eo, po = oracle.lj_tail(oracle.params(box, rc, 0.0, lj_eps=eps, lj_sigma=sig), n)
    assert e == pytest.approx(eo, rel=1e-11)
    assert p == pytest.approx(po, rel=1e-11)
    with pytest.raises(atm3.AtmError):
        atm3.lj_tail(box, n, rc=0.0)
