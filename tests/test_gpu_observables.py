"""Observables of the validation runs through the C ABI: the pair-distance
histogram behind the radial distribution functions (section 5.1, Fig. rdfs).

The histogram is integer work decided on the FP64 canonical displacement the
oracle computes the same way, so every count must equal the oracle's bit for
bit: one system, a batch of uneven replicas, states along an MD run, and the
full 256,000-molecule liquid.
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


def _rdf(atm3, box, n, x, r_max, nbins):
    with atm3.AtmSystem(box, n, nu=NU) as s:
        s.set_state(x)
        s.build_cells()
        s.rdf_accumulate(r_max, nbins)
        counts, samples = s.rdf_get(nbins)
    assert samples == 1
    return counts


@pytest.mark.parametrize("nbins", [1, 7, 250, 4096])
def test_rdf_counts_equal_the_oracle(atm3, nbins):
    cfg = synth.config("liquid_n1000")
    r_max = 2.5
    got = _rdf(atm3, cfg["box"], cfg["n"], cfg["x"], r_max, nbins)[0]
    ref = oracle.rdf_counts(oracle.params(cfg["box"], 2.5, NU), cfg["x"], r_max, nbins)
    assert np.array_equal(got, ref)


def test_rdf_range_at_the_cell_edge_of_an_anisotropic_box(atm3):
    box = (9.0, 10.0, 11.5)
    x = synth.uniform_positions(700, box, np.random.default_rng(71))
    prm = oracle.params(box, 2.5, NU)
    _, w = oracle.cell_grid(prm)
    r_max = float(min(w))
    got = _rdf(atm3, box, 700, x, r_max, 33)[0]
    assert np.array_equal(got, oracle.rdf_counts(prm, x, r_max, 33))


def test_rdf_of_a_batch_equals_the_oracle_replica_by_replica(atm3):
    reps = synth.replicas(count=6, n_lo=300, n_hi=2500)
    x = np.ascontiguousarray(np.concatenate([r["x"] for r in reps], axis=1))
    with atm3.AtmSystem([r["box"] for r in reps], [r["n"] for r in reps], nu=NU) as s:
        s.set_state(x)
        s.build_cells()
        s.rdf_accumulate(2.5, 100)
        counts, samples = s.rdf_get(100)
    assert samples == 1 and counts.shape == (6, 100)
    for r, rep in enumerate(reps):
        ref = oracle.rdf_counts(oracle.params(rep["box"], 2.5, NU), rep["x"], 2.5, 100)
        assert np.array_equal(counts[r], ref), r


def test_rdf_accumulates_along_an_md_run(atm3):
    cfg = synth.config("liquid_n1000")
    prm = oracle.params(cfg["box"], 2.5, NU)
    ref = np.zeros(120, dtype=np.uint64)
    with atm3.AtmSystem(cfg["box"], cfg["n"], nu=NU, dt=0.002) as s:
        s.set_state(cfg["x"], cfg["v"])
        for _ in range(3):
            s.step(2, "3c08", "pair", "fp32c")
            s.rdf_accumulate(2.5, 120)
            xw, _ = s.get_state()
            ref += oracle.rdf_counts(prm, xw, 2.5, 120)
        counts, samples = s.rdf_get(120)
        assert samples == 3
        assert np.array_equal(counts[0], ref)
        s.rdf_reset()
        counts, samples = s.rdf_get(120)
        assert samples == 0 and counts.sum() == 0


def test_rdf_rejects_bad_ranges_and_mixed_accumulation(atm3):
    cfg = synth.config("liquid_n1000")
    with atm3.AtmSystem(cfg["box"], cfg["n"], nu=NU) as s:
        s.set_state(cfg["x"])
        with pytest.raises(atm3.AtmError):
            s.rdf_accumulate(2.5, 50)          # cells not built
        s.build_cells()
        for r_max, nb in ((0.0, 10), (2.5, 0), (2.5, 4097), (5.0, 10)):
            with pytest.raises(atm3.AtmError):
                s.rdf_accumulate(r_max, nb)
        s.rdf_accumulate(2.5, 50)
        with pytest.raises(atm3.AtmError):
            s.rdf_accumulate(2.0, 50)          # another range without a reset
        s.rdf_reset()
        s.rdf_accumulate(2.0, 50)


def test_rdf_full_size_liquid_equals_the_oracle(atm3):
    """The 256,000-molecule liquid (rho 0.8): every bin bit-exact."""
    cfg = synth.config("liquid_n256k")
    got = _rdf(atm3, cfg["box"], cfg["n"], cfg["x"], 2.5, 250)[0]
    ref = oracle.rdf_counts(oracle.params(cfg["box"], 2.5, NU), cfg["x"], 2.5, 250)
    assert np.array_equal(got, ref)


# ---------------------------------------------------------------- thermostat

def test_thermostat_equals_the_oracle_rescaling(atm3):
    cfg = synth.homogeneous(1000, 0.8, 1.7, seed=1000)
    with atm3.AtmSystem(cfg["box"], cfg["n"], nu=NU) as s:
        s.set_state(cfg["x"], cfg["v"])
        s.thermostat(0.746)
        _, v = s.get_state()
        r = s.results()[0]
    ref = oracle.rescale(cfg["v"], 0.746)
    assert np.allclose(v, ref, rtol=1e-13, atol=1e-15)
    assert r["ekin"] == pytest.approx(0.746 * (3 * cfg["n"] - 3) / 2, rel=1e-12)


def test_thermostat_per_replica_targets_and_a_resting_replica(atm3):
    reps = synth.replicas(count=4, n_lo=300, n_hi=1500)
    reps[2]["v"] = np.zeros_like(reps[2]["v"])
    targets = [0.746, 1.033, 2.0, 0.9]
    x = np.ascontiguousarray(np.concatenate([r["x"] for r in reps], axis=1))
    v = np.ascontiguousarray(np.concatenate([r["v"] for r in reps], axis=1))
    with atm3.AtmSystem([r["box"] for r in reps], [r["n"] for r in reps], nu=NU) as s:
        s.set_state(x, v)
        s.thermostat(targets)
        _, vg = s.get_state()
        res = s.results()
    off = 0
    for r, rep in enumerate(reps):
        ref = oracle.rescale(rep["v"], targets[r])
        assert np.allclose(vg[:, off:off + rep["n"]], ref, rtol=1e-13, atol=1e-15), r
        off += rep["n"]
        want = 0.0 if r == 2 else targets[r] * (3 * rep["n"] - 3) / 2
        assert res[r]["ekin"] == pytest.approx(want, rel=1e-12, abs=1e-12), r
    with atm3.AtmSystem([r["box"] for r in reps], [r["n"] for r in reps], nu=NU) as s:
        s.set_state(x, v)
        with pytest.raises(atm3.AtmError):
            s.thermostat([1.0, -1.0, 1.0, 1.0])


def test_nvt_run_follows_the_oracle(atm3):
    """Alternating four FP64 velocity-Verlet steps and a rescale to T = 0.746
    tracks the oracle doing the same, step for step."""
    cfg = synth.homogeneous(1000, 0.817, 1.2, seed=1000)
    prm = oracle.params(cfg["box"], 2.5, NU)
    x, v = cfg["x"], cfg["v"]
    with atm3.AtmSystem(cfg["box"], cfg["n"], nu=NU, dt=0.002) as s:
        s.set_state(x, v)
        for _ in range(4):
            s.step(4, "3c18", "pair", "fp64")
            s.thermostat(0.746)
            ref = oracle.md_run(prm, x, v, 4, 0.002, "3c18", "pair", "fp64")
            x, v = ref["x"], oracle.rescale(ref["v"], 0.746)
        xg, vg = s.get_state()
    d = xg - x
    d -= np.rint(d / cfg["box"][:, None]) * cfg["box"][:, None]
    assert np.abs(d).max() < 1e-9
    assert np.abs(vg - v).max() < 1e-7


# ---------------------------------------------------------------- peak probes

def test_measured_peaks_are_plausible(atm3):
    """The roofline denominators measured by the library: FP32 / FP64 FMA
    throughput and FP32 rsqrt throughput, positive and below the nominal
    rates derived from unit counts (152 SMs at 2.07 GHz: FP32 80.5 TFLOP/s;
    16 rsqrt per SM per clock, 5.0 T/s)."""
    f32 = atm3.measure_fma_peak(0, fp64=False)
    f64 = atm3.measure_fma_peak(0, fp64=True)
    rs = atm3.measure_rsqrt_peak(0)
    assert 10.0 < f32 < 90.0
    assert 0.1 < f64 < f32
    assert 100.0 < rs < 6000.0
