"""Deterministic mode (atm_set_deterministic) through the C ABI.

With the mode on, repeated evaluations of one state give bit-identical
forces, energies, virials and counts, in the same context and in a fresh
one; the block traversals' forces are also bit-identical across launch forms
(their terms are summed as 64-bit integers, so the order of the additions
does not matter); graph-captured steps repeat bit for bit; and the results
still match the oracle within the parity tolerances (FP64 1e-10, FP32C 2e-5
relative per component, floor of the same size times the RMS force).
"""
import numpy as np
import pytest

import oracle
from paper_2510_21230_gb300 import synth

pytestmark = pytest.mark.gpu

NU = 0.073
RTOL = {"fp64": 1e-10, "fp32c": 2e-5}
ORC_PREC = {"fp64": "fp64", "fp32c": "fp32"}
KEYS = ("e2", "e3", "w2", "w3", "n_cand3", "n_int3", "n_cand2", "n_int2")


@pytest.fixture(scope="module")
def atm3():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_21230_gb300 import atm3 as m, build
    build.build()
    return m


def close(got, ref, rtol):
    scale = np.sqrt(np.mean(ref * ref)) if ref.size else 0.0
    return np.all(np.abs(got - ref) <= rtol * np.abs(ref) + rtol * scale)


def evaluate(atm3, cfg, trav, trunc, prec, det=True, opts=None, classes=None, twice=False):
    n = cfg["x"].shape[1]
    out = []
    with atm3.AtmSystem(cfg["box"], n, nu=NU) as s:
        if opts:
            s.set_options(**opts)
        if classes:
            s.set_unit_classes(classes)
        s.set_deterministic(det)
        s.set_state(cfg["x"], cfg.get("v"))
        s.build_cells()
        for _ in range(2 if twice else 1):
            r = s.compute_forces(trav, trunc, prec)
            out.append((r, s.get_forces("total"), s.get_forces("atm")))
    return out


def same(a, b):
    ra, fa, xa = a
    rb, fb, xb = b
    for k in KEYS:
        assert ra[k] == rb[k], k
    assert np.array_equal(fa, fb) and np.array_equal(xa, xb)


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
@pytest.mark.parametrize("trunc", ["pair", "product"])
@pytest.mark.parametrize("trav", ["3c01", "3c18", "3c08", "3c08a"])
def test_repeatable_and_matches_oracle(atm3, trav, trunc, prec):
    cfg = synth.homogeneous(1000, 0.8, 1.0, seed=1000)
    a, b = evaluate(atm3, cfg, trav, trunc, prec, twice=True)
    (c,) = evaluate(atm3, cfg, trav, trunc, prec)
    same(a, b)
    same(a, c)
    ref = oracle.atm_cells(oracle.params(cfg["box"], 2.5, NU), cfg["x"], trav, trunc, ORC_PREC[prec])
    r, _, f_atm = a
    assert r["n_cand3"] == ref["n_cand3"] and r["n_int3"] == ref["n_int3"]
    assert r["e3"] == pytest.approx(ref["e3"], rel=RTOL[prec])
    assert r["w3"] == pytest.approx(ref["w3"], rel=RTOL[prec])
    assert close(f_atm, ref["f"], RTOL[prec])


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
@pytest.mark.parametrize("trav,trunc", [("3c08", "pair"), ("3c18", "pair"), ("3c08", "product")])
def test_block_forces_do_not_depend_on_the_launch_form(atm3, trav, trunc, prec):
    """32,000 molecules (2197 units): one CTA per unit, a persistent grid, 8
    warps per CTA and two unit size classes give the same forces bit for bit."""
    cfg = synth.homogeneous(32000, 0.8, 1.0, seed=2000)
    base = evaluate(atm3, cfg, trav, trunc, prec)[0]
    for opts, classes in ((dict(persistent=True), None), (dict(nwarps=8), None),
                          (None, [64]), (dict(persistent=True, nwarps=4), [48, 96])):
        got = evaluate(atm3, cfg, trav, trunc, prec, opts=opts, classes=classes)[0]
        for k in ("n_cand3", "n_int3", "n_cand2", "n_int2"):
            assert got[0][k] == base[0][k], (opts, classes, k)
        assert np.array_equal(got[2], base[2]), (opts, classes)
        for k in ("e3", "w3"):
            assert got[0][k] == pytest.approx(base[0][k], rel=RTOL[prec]), (opts, classes, k)


def test_graph_steps_repeat_bit_for_bit(atm3):
    """Twenty graph-captured FP32C velocity-Verlet steps of a batch of six
    uneven replicas (LJ inside the 3c08 units), run twice from the same state."""
    reps = synth.replicas(count=6, n_lo=500, n_hi=3000)
    x = np.ascontiguousarray(np.concatenate([r["x"] for r in reps], axis=1))
    v = np.ascontiguousarray(np.concatenate([r["v"] for r in reps], axis=1))
    runs = []
    for _ in range(2):
        with atm3.AtmSystem([r["box"] for r in reps], [r["n"] for r in reps], nu=NU,
                            dt=0.002) as b:
            b.set_options(graph=True)
            b.set_deterministic(True)
            b.set_state(x, v)
            b.step(20, "3c08", "pair", "fp32c")
            xs, vs = b.get_state()
            runs.append((xs, vs, b.get_forces("total"), b.results()))
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])
    assert np.array_equal(runs[0][2], runs[1][2])
    for ra, rb in zip(runs[0][3], runs[1][3]):
        for k in KEYS + ("ekin",):
            assert ra[k] == rb[k], k


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_fallback_accumulators(atm3, prec):
    """Units whose edges overflow the pair-scalar table (rho* = 1.4) and units
    too large for the product rule's dense tables (per-molecule accumulators):
    repeatable and equal to the oracle."""
    for cfg, trunc in ((synth.homogeneous(2000, 1.4, 1.0, seed=77, jitter=0.02), "pair"),
                       (synth.homogeneous(1500, 0.8, 1.0, seed=1001), "product")):
        a, b = evaluate(atm3, cfg, "3c08", trunc, prec, twice=True)
        same(a, b)
        ref = oracle.atm_cells(oracle.params(cfg["box"], 2.5, NU), cfg["x"], "3c08", trunc,
                               ORC_PREC[prec])
        assert a[0]["n_int3"] == ref["n_int3"]
        assert close(a[2], ref["f"], RTOL[prec]), trunc


def test_full_size_repeatable(atm3):
    """The N = 256,000 liquid, 3c08 pair FP32C: two evaluations agree bit for
    bit, and the invariants hold (W3 = 9 E3, zero net force)."""
    cfg = synth.homogeneous(256000, 0.8, 1.0, seed=5000)
    a, b = evaluate(atm3, cfg, "3c08", "pair", "fp32c", twice=True)
    same(a, b)
    r, _, f = a
    assert r["w3"] == pytest.approx(9 * r["e3"], rel=1e-5)
    assert np.abs(f.sum(axis=1)).max() < 1e-3 * np.abs(f).max() * 10


def test_a_term_beyond_the_fixed_point_range_is_reported(atm3):
    """FP64 terms must stay below 2^14: a pair 0.1 sigma apart (a triplet
    scalar of about 2e4) makes the evaluation fail with ATM_E_RANGE; the
    context stays usable."""
    box = np.array([9.0, 9.0, 9.0])
    x = np.array([[1.0, 1.1, 1.0, 5.0], [1.0, 1.0, 2.0, 5.0], [1.0, 1.0, 1.0, 5.0]])
    with atm3.AtmSystem(box, 4, nu=NU) as s:
        s.set_deterministic(True)
        s.set_state(x)
        s.build_cells()
        with pytest.raises(atm3.AtmError) as ei:
            s.compute_forces("3c08", "pair", "fp64")
        assert ei.value.status == 8
        s.set_deterministic(False)
        r = s.compute_forces("3c08", "pair", "fp64")
        assert r["n_int3"] == 1
