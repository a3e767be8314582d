"""Velocity-Verlet NVE through the C ABI against the CPU oracle.

Short run, FP64: the GPU trajectory follows the oracle's step by step (the two
differ only by the rounding order of the force sums, which the chaotic
dynamics amplify slowly over a few dozen steps).  Long run (N = 32,000,
200 steps, dt = 0.002): the total-energy drift of the FP64 and FP32C GPU runs
matches the oracle's drift, and both stay small.
"""
import numpy as np
import pytest

import oracle
from paper_2510_21230_gb300 import synth

pytestmark = pytest.mark.gpu

NU = 0.073


@pytest.fixture(scope="module")
def atm3():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_21230_gb300 import atm3 as m, build
    build.build()
    return m


def test_fp64_trajectory_follows_oracle(atm3):
    cfg = synth.homogeneous(1000, 0.8, 1.0, seed=1000)
    nsteps, dt = 20, 0.002
    prm = oracle.params(cfg["box"], 2.5, NU)
    ref = oracle.md_run(prm, cfg["x"], cfg["v"], nsteps, dt, "3c18", "pair", "fp64")
    en = []
    with atm3.AtmSystem(cfg["box"], 1000, nu=NU, dt=dt) as s:
        s.set_state(cfg["x"], cfg["v"])
        r = s.step(0, "3c18", "pair", "fp64")
        en.append([r["e2"], r["e3"], r["ekin"]])
        for _ in range(nsteps):
            r = s.step(1, "3c18", "pair", "fp64")
            en.append([r["e2"], r["e3"], r["ekin"]])
        x, v = s.get_state()
    en = np.array(en)
    assert np.allclose(en, ref["energies"][:, :3], rtol=1e-8, atol=1e-9)
    d = x - ref["x"]
    d -= np.rint(d / cfg["box"][:, None]) * cfg["box"][:, None]
    assert np.abs(d).max() < 1e-9
    assert np.abs(v - ref["v"]).max() < 1e-7


def _drift(e):
    tot = e[:, 0] + e[:, 1] + e[:, 2]
    return tot[-1] - tot[0], np.abs(tot - tot[0]).max()


def _pressure(en, n, vol):
    """Virial pressure rho T + (W2 + W3) / (3V), T = 2K / (3N - 3), per record."""
    return n / vol * (2.0 * en[:, 2] / (3 * n - 3)) + en[:, 3] / (3.0 * vol)


def _gpu_nve(atm3, cfg, trav, trunc, prec, nsteps, every, dt=0.002):
    """Energies (E2, E3, K, W2 + W3) of the start and of every `every`-th step,
    and the final state."""
    en = []
    with atm3.AtmSystem(cfg["box"], cfg["n"], nu=NU, dt=dt) as s:
        s.set_state(cfg["x"], cfg["v"])
        r = s.step(0, trav, trunc, prec)
        en.append([r["e2"], r["e3"], r["ekin"], r["w2"] + r["w3"]])
        for _ in range(nsteps // every):
            r = s.step(every, trav, trunc, prec)
            en.append([r["e2"], r["e3"], r["ekin"], r["w2"] + r["w3"]])
        x, v = s.get_state()
    return np.array(en), x, v


@pytest.fixture(scope="module")
def liquid_32k():
    return synth.homogeneous(32000, 0.8, 1.0, seed=2000)


@pytest.fixture(scope="module")
def nve_ref_pair(liquid_32k):
    """The oracle's 200-step FP64 run under the pair rule (every traversal sums
    the same triplets under it, so one run serves all of them)."""
    cfg = liquid_32k
    prm = oracle.params(cfg["box"], 2.5, NU)
    return oracle.md_run(prm, cfg["x"], cfg["v"], 200, 0.002, "3c18", "pair", "fp64")


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
@pytest.mark.parametrize("trav", ["3c01", "3c18", "3c08"])
def test_nve_drift_32k_matches_oracle(atm3, liquid_32k, nve_ref_pair, trav, prec):
    """N = 32,000, 200 steps of dt = 0.002 under the pair rule: the energy
    records follow the oracle's every 10 steps, the drift matches the
    oracle's, and the ensemble averages of U / N and P agree."""
    cfg = liquid_32k
    n = cfg["n"]
    vol = float(np.prod(cfg["box"]))
    ref = nve_ref_pair["energies"]
    d_ref, m_ref = _drift(ref)
    en, _, _ = _gpu_nve(atm3, cfg, trav, "pair", prec, 200, 10)
    d, m = _drift(en)
    # same dynamics: the energy records agree with the oracle's every 10 steps
    assert np.allclose(en[:, 1], ref[::10, 1], rtol=1e-3), (trav, prec)
    assert np.allclose(en[:, 0] + en[:, 2], ref[::10, 0] + ref[::10, 2], rtol=1e-4), (trav, prec)
    # drift per molecule as small as the oracle's (the truncated potentials
    # make the total energy jump at every cutoff crossing on both sides)
    assert abs(d - d_ref) / n < 1e-4, (trav, prec, d, d_ref)
    assert m <= 1.2 * m_ref + 1e-3 * n, (trav, prec, m, m_ref)
    # ensemble averages over the run
    u, u_ref = (en[:, 0] + en[:, 1]).mean() / n, (ref[::10, 0] + ref[::10, 1]).mean() / n
    assert u == pytest.approx(u_ref, rel=1e-4), (trav, prec)
    p, p_ref = _pressure(en, n, vol).mean(), _pressure(ref[::10], n, vol).mean()
    assert p == pytest.approx(p_ref, abs=1e-3 * abs(p_ref) + 1e-4), (trav, prec)


@pytest.mark.parametrize("trav", ["3c01", "3c18", "3c08"])
def test_nve_product_rule_32k(atm3, liquid_32k, trav):
    """N = 32,000, 200 steps of dt = 0.002 under the product rule, FP64 and
    FP32C (each traversal sums its own triplet set, so each is checked on its
    own; a 200-step oracle run of the product rule is minutes of CPU per
    traversal): the first three steps follow the oracle's trajectory, the
    oracle's evaluation of the FP64 run's final state equals what the run
    reported there (counts exact), and the FP32C run's drift and averages
    match the FP64 run's.  (The oracle-anchored drift of the product rule is
    the next test, at a size the oracle steps 200 times in about a minute.)"""
    cfg = liquid_32k
    n = cfg["n"]
    vol = float(np.prod(cfg["box"]))
    prm = oracle.params(cfg["box"], 2.5, NU)
    short = oracle.md_run(prm, cfg["x"], cfg["v"], 3, 0.002, trav, "product", "fp64")
    en1, _, _ = _gpu_nve(atm3, cfg, trav, "product", "fp64", 3, 1)
    assert np.allclose(en1, short["energies"], rtol=1e-8, atol=1e-9), trav
    en64, x64, _ = _gpu_nve(atm3, cfg, trav, "product", "fp64", 200, 10)
    ref_end = oracle.atm_cells(prm, x64, trav, "product", "fp64")
    with atm3.AtmSystem(cfg["box"], n, nu=NU) as s:
        s.set_state(x64)
        s.build_cells()
        r_end = s.compute_forces(trav, "product", "fp64")
    assert r_end["e3"] == pytest.approx(en64[-1, 1], rel=1e-12), trav
    assert r_end["n_int3"] == ref_end["n_int3"] and r_end["n_cand3"] == ref_end["n_cand3"], trav
    assert r_end["e3"] == pytest.approx(ref_end["e3"], rel=1e-10), trav
    en32, _, _ = _gpu_nve(atm3, cfg, trav, "product", "fp32c", 200, 10)
    d64, m64 = _drift(en64)
    d32, m32 = _drift(en32)
    assert abs(d32 - d64) / n < 1e-4, (trav, d32, d64)
    assert m32 <= 1.2 * m64 + 1e-3 * n, (trav, m32, m64)
    u64, u32 = [(e[:, 0] + e[:, 1]).mean() / n for e in (en64, en32)]
    assert u32 == pytest.approx(u64, rel=1e-4), trav
    p64, p32 = [_pressure(e, n, vol).mean() for e in (en64, en32)]
    assert p32 == pytest.approx(p64, abs=1e-3 * abs(p64) + 1e-4), trav


def test_nve_product_rule_drift_matches_oracle(atm3):
    """Product rule, 3c08, N = 4000 (6 cells per axis), 200 steps of dt =
    0.002, FP64 and FP32C against the oracle's own 200-step run: energy
    records every 10 steps, the drift (the product rule's set of found
    triplets changes whenever a molecule changes cell, so its energy jumps
    far more than the pair rule's) and the averages of U / N and P."""
    cfg = synth.homogeneous(4000, 0.8, 1.0, seed=2100)
    n = cfg["n"]
    vol = float(np.prod(cfg["box"]))
    prm = oracle.params(cfg["box"], 2.5, NU)
    ref = oracle.md_run(prm, cfg["x"], cfg["v"], 200, 0.002, "3c08", "product", "fp64")["energies"]
    d_ref, m_ref = _drift(ref)
    for prec in ("fp64", "fp32c"):
        en, _, _ = _gpu_nve(atm3, cfg, "3c08", "product", prec, 200, 10)
        d, m = _drift(en)
        assert np.allclose(en[:, 1], ref[::10, 1], rtol=1e-3), prec
        assert np.allclose(en[:, 0] + en[:, 2], ref[::10, 0] + ref[::10, 2], rtol=1e-4), prec
        assert abs(d - d_ref) / n < 1e-4, (prec, d, d_ref)
        assert m <= 1.2 * m_ref + 1e-3 * n, (prec, m, m_ref)
        u, u_ref = (en[:, 0] + en[:, 1]).mean() / n, (ref[::10, 0] + ref[::10, 1]).mean() / n
        assert u == pytest.approx(u_ref, rel=1e-4), prec
        p, p_ref = _pressure(en, n, vol).mean(), _pressure(ref[::10], n, vol).mean()
        assert p == pytest.approx(p_ref, abs=1e-3 * abs(p_ref) + 1e-4), prec


@pytest.mark.parametrize("trav,prec", [("3c08", "fp32c"), ("3c08", "fp64"), ("3c08a", "fp32c"),
                                       ("3c18", "fp32c"), ("3c18", "fp64")])
def test_step_with_lj_inside_the_units_equals_separate_kernels(atm3, trav, prec):
    """A step under the 3c08 or 3c18 pair rule evaluates LJ inside the ATM
    units (the c08 cell pairs of each block; the base cell's half-shell pairs
    of each 3c18 unit): same counts, energies and total force as the separate
    LJ and ATM kernels on the same state; asking for the LJ or ATM part
    afterwards re-evaluates them apart."""
    rtol = 1e-10 if prec == "fp64" else 2e-5
    cfg = synth.homogeneous(4000, 0.8, 1.0, seed=1100)
    with atm3.AtmSystem(cfg["box"], cfg["n"], nu=NU, dt=0.002) as s:
        s.set_state(cfg["x"], cfg["v"])
        s.step(3, trav, "pair", prec)
        fused = s.step(0, trav, "pair", prec)   # forces of this state, fused
        f_tot = s.get_forces("total")
        f_lj = s.get_forces("lj")              # re-evaluated apart
        f_atm = s.get_forces("atm")
        sep = s.compute_forces(trav, "pair", prec)
        f_tot2 = s.get_forces("total")
        f_lj2 = s.get_forces("lj")
    for k in ("n_cand2", "n_int2", "n_cand3", "n_int3"):
        assert fused[k] == sep[k], k
    for k in ("e2", "w2", "e3", "w3"):
        assert fused[k] == pytest.approx(sep[k], rel=rtol), k
    scale = np.sqrt(np.mean(f_tot2 ** 2))
    assert np.abs(f_tot - f_tot2).max() <= rtol * 4 * scale
    assert np.allclose(f_lj, f_lj2, rtol=0, atol=1e-12 * scale)
    assert np.abs(f_lj + f_atm - f_tot2).max() <= 1e-12 * scale + rtol * scale


def test_fused_batch_step_equals_oracle_energies(atm3):
    """Uneven replicas stepped together with LJ inside the 3c08 units: per
    replica the energies after two FP64 steps match the oracle's run."""
    reps = synth.replicas(count=3, n_lo=800, n_hi=2500)
    x = np.ascontiguousarray(np.concatenate([r["x"] for r in reps], axis=1))
    v = np.ascontiguousarray(np.concatenate([r["v"] for r in reps], axis=1))
    with atm3.AtmSystem([r["box"] for r in reps], [r["n"] for r in reps], nu=NU, dt=0.002) as s:
        s.set_state(x, v)
        s.step(2, "3c08", "pair", "fp64")
        res = s.results()
    for r, rep in enumerate(reps):
        prm = oracle.params(rep["box"], 2.5, NU)
        ref = oracle.md_run(prm, rep["x"], rep["v"], 2, 0.002, "3c08", "pair", "fp64")
        e2, e3, ek = ref["energies"][-1][:3]
        assert res[r]["e2"] == pytest.approx(e2, rel=1e-9), r
        assert res[r]["e3"] == pytest.approx(e3, rel=1e-9), r
        assert res[r]["ekin"] == pytest.approx(ek, rel=1e-9), r


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_host_round_trips_with_forces_equal_continuous_steps(atm3, prec):
    """A caller that keeps the state on the host between steps gives the
    state's force back with it (atm_set_forces): each step then evaluates the
    forces once, and the run follows the continuous device run (to the
    rounding of the force sums, whose atomic accumulation order varies from
    evaluation to evaluation)."""
    cfg = synth.homogeneous(2000, 0.8, 1.0, seed=1300)
    with atm3.AtmSystem(cfg["box"], cfg["n"], nu=NU, dt=0.002) as a:
        a.set_state(cfg["x"], cfg["v"])
        a.step(0, "3c08", "pair", prec)
        ra = a.step(4, "3c08", "pair", prec)
        xa, va = a.get_state()
    with atm3.AtmSystem(cfg["box"], cfg["n"], nu=NU, dt=0.002) as b:
        b.set_state(cfg["x"], cfg["v"])
        b.step(0, "3c08", "pair", prec)
        x, v = b.get_state()          # wrapped by the cell build, as on the device
        f = b.get_forces("total")
        for _ in range(4):
            b.set_state(x, v)
            b.set_forces(f, "3c08", "pair", prec)
            rb = b.step(1, "3c08", "pair", prec)
            x, v = b.get_state()
            f = b.get_forces("total")
        with pytest.raises(atm3.AtmError):
            b.set_forces(f, "3c08", "pair", "surrogate")
    tol = {"fp64": (1e-12, 1e-12, 1e-10), "fp32c": (1e-9, 1e-7, 1e-6)}[prec]
    d = x - xa
    d -= np.rint(d / cfg["box"][:, None]) * cfg["box"][:, None]
    assert np.abs(d).max() <= tol[0]
    assert np.abs(v - va).max() <= tol[1]
    for k in ("n_int3", "n_int2"):
        assert rb[k] == ra[k], k
    for k in ("e2", "e3", "ekin"):
        assert rb[k] == pytest.approx(ra[k], rel=tol[2]), k


def test_forces_are_forgotten_with_a_new_state(atm3):
    cfg = synth.homogeneous(1000, 0.8, 1.0, seed=1301)
    with atm3.AtmSystem(cfg["box"], cfg["n"], nu=NU) as s:
        with pytest.raises(atm3.AtmError):
            s.set_forces(np.zeros((3, cfg["n"])))       # no state yet
        s.set_state(cfg["x"], cfg["v"])
        s.set_forces(np.zeros((3, cfg["n"])), "3c08", "pair", "fp32c")
        s.set_state(cfg["x"], cfg["v"])                 # forgets the forces above
        r1 = s.step(1, "3c08", "pair", "fp32c")
    with atm3.AtmSystem(cfg["box"], cfg["n"], nu=NU) as t:
        t.set_state(cfg["x"], cfg["v"])
        r2 = t.step(1, "3c08", "pair", "fp32c")
    # zero forces in the first half kick would change the kinetic energy by far more
    assert r1["e3"] == pytest.approx(r2["e3"], rel=1e-6)
    assert r1["ekin"] == pytest.approx(r2["ekin"], rel=1e-9)


@pytest.mark.parametrize("prec,graph", [("fp64", False), ("fp32c", False), ("fp32c", True)])
def test_step_host_equals_the_separate_calls(atm3, prec, graph):
    """atm_step_host (state and force in from host memory, steps, state and
    force out, one synchronisation at the end; the last step's positions
    copied out beside its force evaluation) gives what the separate calls
    give: bit for bit in deterministic mode, where the force sums do not
    depend on the order of the atomic additions.  Also without given forces,
    with two steps per round trip, and with graph steps."""
    cfg = synth.homogeneous(2000, 0.8, 1.0, seed=1302)
    runs = []
    for api in ("separate", "host"):
        with atm3.AtmSystem(cfg["box"], cfg["n"], nu=NU, dt=0.002) as s:
            s.set_deterministic(True)
            s.set_options(graph=graph)
            s.set_state(cfg["x"], cfg["v"])
            s.step(0, "3c08", "pair", prec)
            x, v = s.get_state()
            f = s.get_forces("total")
            res = []
            for nsteps in (1, 1, 2):
                if api == "separate":
                    s.set_state(x, v)
                    s.set_forces(f, "3c08", "pair", prec)
                    res.append(s.step(nsteps, "3c08", "pair", prec))
                    x, v = s.get_state()
                    f = s.get_forces("total")
                else:
                    res.append(s.step_host(x, v, f, nsteps, "3c08", "pair", prec))
            if api == "separate":
                s.set_state(x, v)
                res.append(s.step(1, "3c08", "pair", prec))
                x, v = s.get_state()
            else:
                res.append(s.step_host(x, v, None, 1, "3c08", "pair", prec))
            runs.append((x.copy(), v.copy(), f.copy(), res))
    (xa, va, fa, ra), (xb, vb, fb, rb) = runs
    assert np.array_equal(xa, xb) and np.array_equal(va, vb) and np.array_equal(fa, fb)
    for a, b in zip(ra, rb):
        for k in ("n_int3", "n_int2", "n_cand3"):
            assert a[k] == b[k], k
        for k in ("e2", "e3", "ekin", "w3"):
            assert b[k] == pytest.approx(a[k], rel=1e-12), k


def test_step_host_rejects_non_finite_input(atm3):
    cfg = synth.homogeneous(1000, 0.8, 1.0, seed=1303)
    with atm3.AtmSystem(cfg["box"], cfg["n"], nu=NU) as s:
        for which in ("x", "v", "f"):
            x, v = cfg["x"].copy(), cfg["v"].copy()
            f = np.zeros((3, cfg["n"]))
            {"x": x, "v": v, "f": f}[which][1, 7] = np.nan
            with pytest.raises(atm3.AtmError, match="NONFINITE|non-finite"):
                s.step_host(x, v, f, 1, "3c08", "pair", "fp32c")
            with pytest.raises(atm3.AtmError):
                s.step(1, "3c08", "pair", "fp32c")         # no state after the rejection
        with pytest.raises(atm3.AtmError):                  # given forces need an exact mode
            s.step_host(cfg["x"].copy(), cfg["v"].copy(), np.zeros((3, cfg["n"])), 1,
                        "3c08", "pair", "surrogate")
        x, v = cfg["x"].copy(), cfg["v"].copy()
        r = s.step_host(x, v, None, 0, "3c08", "pair", "fp32c")   # zero steps: forces of the state
        assert r["n_int3"] > 0
