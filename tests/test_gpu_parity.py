"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Bars: cell arrays and every count bit-exact; FP64 forces within 1e-10
relative per component, FP32C forces within 2e-5 relative per component,
each with an absolute floor of the same relative size times the RMS force of
the configuration (components that cancel to near zero are judged against the
force scale, not against themselves).  Energies and virials to the same
relative tolerances.  The FP32C path is compared with the oracle's FP32
decision mode, so that both sides sum the same triplet set.
"""
import numpy as np
import pytest

import oracle
from paper_2510_21230_gb300 import synth

pytestmark = pytest.mark.gpu

NU = 0.073
RTOL = {"fp64": 1e-10, "fp32c": 2e-5}
ORC_PREC = {"fp64": "fp64", "fp32c": "fp32"}


@pytest.fixture(scope="module")
def atm3():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_21230_gb300 import atm3 as m, build
    build.build()
    return m


def assert_forces_close(got, ref, rtol, what=""):
    scale = np.sqrt(np.mean(ref * ref)) if ref.size else 0.0
    err = np.abs(got - ref)
    tol = rtol * np.abs(ref) + rtol * scale
    bad = err > tol
    if bad.any():
        q = np.argmax(err - tol)
        d, i = np.unravel_index(q, ref.shape)
        raise AssertionError("%s: %d components off; worst [%d,%d] got %.17g ref %.17g (scale %.3g)"
                             % (what, bad.sum(), d, i, got[d, i], ref[d, i], scale))


def run_gpu(atm3, cfg, trav, trunc, prec, rc=2.5):
    n = cfg["x"].shape[1]
    with atm3.AtmSystem(cfg["box"], n, rc=rc, nu=NU) as s:
        s.set_state(cfg["x"], cfg.get("v"))
        s.build_cells()
        r = s.compute_forces(trav, trunc, prec)
        return r, s.get_forces("atm"), s.get_forces("lj"), s.get_cells()


def small_liquid():
    return synth.homogeneous(1000, 0.8, 1.0, seed=1000)


# ------------------------------------------------------------------ cells

@pytest.mark.parametrize("maker", ["liquid", "slab_like", "three_cells"])
def test_cells_bit_exact(atm3, maker):
    rng = np.random.default_rng(77)
    if maker == "liquid":
        cfg = small_liquid()
    elif maker == "slab_like":
        box = np.array([9.0, 8.0, 21.0])
        x = synth.uniform_positions(900, box, rng)
        x[:, :50] += np.array([[9.0], [-16.0], [42.0]])  # images outside the box
        cfg = dict(x=x, box=box)
    else:
        box = np.array([7.6, 7.6, 7.6])
        cfg = dict(x=synth.uniform_positions(300, box, rng), box=box)
    n = cfg["x"].shape[1]
    prm = oracle.params(cfg["box"], 2.5, NU)
    ref = oracle.build_cells(prm, cfg["x"])
    with atm3.AtmSystem(cfg["box"], n) as s:
        s.set_state(cfg["x"])
        s.build_cells()
        c = s.get_cells()
        xw, _ = s.get_state()
    assert np.array_equal(c["ncell"], ref["ncell"])
    assert np.array_equal(c["cell_of"], ref["cell_of"])
    assert np.array_equal(c["cell_start"], ref["cell_start"])
    assert np.array_equal(c["perm"], ref["perm"])
    assert np.array_equal(xw, ref["xw"])


def test_cells_bit_exact_many_cells(atm3):
    """A dilute gas over 68^3 = 314,432 cells: the scan of the cell counts runs
    over segments of many 32-cell chunks per warp; cell arrays bit-exact
    against the oracle's cell build."""
    rng = np.random.default_rng(78)
    n, box = 100000, 171.0
    x = rng.uniform(0.0, box, size=(3, n))
    prm = oracle.params(np.array([box, box, box]), 2.5, 0.073)
    ref = oracle.build_cells(prm, x)
    with atm3.AtmSystem(np.array([box, box, box]), n) as s:
        s.set_state(x)
        s.build_cells()
        c = s.get_cells()
    assert int(np.prod(c["ncell"])) == 68 ** 3
    assert np.array_equal(c["cell_start"], ref["cell_start"])
    assert np.array_equal(c["perm"], ref["perm"])


# ------------------------------------------------------------------ forces, small liquid

@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
@pytest.mark.parametrize("trunc", ["pair", "product"])
@pytest.mark.parametrize("trav", ["3c01", "3c18", "3c08", "3c08a"])
def test_atm_parity_small_liquid(atm3, trav, trunc, prec):
    cfg = small_liquid()
    prm = oracle.params(cfg["box"], 2.5, NU)
    ref = oracle.atm_cells(prm, cfg["x"], trav, trunc, ORC_PREC[prec])
    r, f_atm, _, _ = run_gpu(atm3, cfg, trav, trunc, prec)
    assert r["n_cand3"] == ref["n_cand3"]
    assert r["n_int3"] == ref["n_int3"]
    rtol = RTOL[prec]
    assert r["e3"] == pytest.approx(ref["e3"], rel=rtol)
    assert r["w3"] == pytest.approx(ref["w3"], rel=rtol)
    assert_forces_close(f_atm, ref["f"], rtol, "%s/%s/%s" % (trav, trunc, prec))


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_lj_parity_small_liquid(atm3, prec):
    cfg = small_liquid()
    prm = oracle.params(cfg["box"], 2.5, NU)
    ref = oracle.lj_cells(prm, cfg["x"], ORC_PREC[prec])
    r, _, f_lj, _ = run_gpu(atm3, cfg, "3c18", "pair", prec)
    assert r["n_cand2"] == ref["n_cand2"]
    assert r["n_int2"] == ref["n_int2"]
    rtol = RTOL[prec]
    assert r["e2"] == pytest.approx(ref["e2"], rel=rtol)
    assert r["w2"] == pytest.approx(ref["w2"], rel=rtol)
    assert_forces_close(f_lj, ref["f"], rtol, "lj/" + prec)


def test_fp64_matches_brute_force_pair_rule(atm3):
    """Independent of the linked-cell oracle: the O(N^3) minimum-image brute force."""
    rng = np.random.default_rng(5)
    box = np.array([8.1, 8.1, 8.1])
    x = np.ascontiguousarray(
        synth.random_sequential(300, [0, 0, 0], box, 0.85, rng, box=box).T)
    cfg = dict(x=x, box=box)
    bf = oracle.atm_brute(oracle.params(box, 2.5, NU), x, "pair")
    for trav in ["3c18", "3c08"]:
        r, f, _, _ = run_gpu(atm3, cfg, trav, "pair", "fp64")
        assert r["n_int3"] == bf["n_int3"]
        assert r["e3"] == pytest.approx(bf["e3"], rel=1e-10)
        assert_forces_close(f, bf["f"], 1e-10, trav)


# ------------------------------------------------------------------ edge cases

def test_empty_and_tiny_systems(atm3):
    box = np.array([8.0, 8.0, 8.0])
    for n in [0, 1, 2, 3]:
        x = np.full((3, n), 1.0) + np.arange(n)[None, :] * 0.9
        with atm3.AtmSystem(box, n) as s:
            s.set_state(x)
            s.build_cells()
            for trav in ["3c01", "3c18", "3c08", "3c08a"]:
                r = s.compute_forces(trav, "product", "fp64")
                ref = oracle.atm_cells(oracle.params(box, 2.5, NU), x, trav, "product")
                assert r["n_int3"] == ref["n_int3"] and r["n_cand3"] == ref["n_cand3"]
                assert r["e3"] == pytest.approx(ref["e3"], rel=1e-12, abs=1e-300)


@pytest.mark.parametrize("trav", ["3c01", "3c18", "3c08", "3c08a"])
def test_crowded_cell_and_ragged_occupancy(atm3, trav):
    """One cell holds far more molecules than the rest (ragged staging tails)."""
    rng = np.random.default_rng(9)
    box = np.array([10.2, 7.7, 12.9])
    x = synth.uniform_positions(400, box, rng)
    x[:, :70] = rng.uniform(0.1, 2.4, size=(3, 70))
    cfg = dict(x=x, box=box)
    prm = oracle.params(box, 2.5, NU)
    for prec in ["fp64", "fp32c"]:
        ref = oracle.atm_cells(prm, x, trav, "pair", ORC_PREC[prec])
        r, f, _, _ = run_gpu(atm3, cfg, trav, "pair", prec)
        assert r["n_int3"] == ref["n_int3"] and r["n_cand3"] == ref["n_cand3"]
        assert_forces_close(f, ref["f"], RTOL[prec], trav + prec)


def test_nonfinite_input_is_rejected(atm3):
    box = np.array([8.0, 8.0, 8.0])
    x = np.ones((3, 10))
    x[1, 3] = np.nan
    with atm3.AtmSystem(box, 10) as s:
        with pytest.raises(atm3.AtmError) as ei:
            s.set_state(x)
        assert ei.value.status == 5


def test_call_order_is_checked(atm3):
    box = np.array([8.0, 8.0, 8.0])
    with atm3.AtmSystem(box, 10) as s:
        with pytest.raises(atm3.AtmError) as ei:
            s.compute_forces()
        assert ei.value.status == 6


# ------------------------------------------------------------------ medium size: many units, ragged tails

@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
@pytest.mark.parametrize("trav", ["3c18", "3c08", "3c08a"])
def test_atm_parity_32k_pair(atm3, trav, prec):
    cfg = synth.homogeneous(32000, 0.8, 1.0, seed=2000)
    prm = oracle.params(cfg["box"], 2.5, NU)
    ref = oracle.atm_cells(prm, cfg["x"], trav, "pair", ORC_PREC[prec])
    r, f, _, _ = run_gpu(atm3, cfg, trav, "pair", prec)
    assert r["n_cand3"] == ref["n_cand3"]
    assert r["n_int3"] == ref["n_int3"]
    assert r["e3"] == pytest.approx(ref["e3"], rel=RTOL[prec])
    assert_forces_close(f, ref["f"], RTOL[prec], trav + prec)


@pytest.fixture(scope="module")
def liquid_32k():
    return synth.homogeneous(32000, 0.8, 1.0, seed=2000)


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
@pytest.mark.parametrize("trav", ["3c18", "3c08", "3c08a"])
def test_atm_parity_32k_product(atm3, liquid_32k, trav, prec):
    """Product rule on the N = 32,000 liquid (2197 units of 13 cells per axis):
    the plans the benchmark times on the 256k liquid (dense distance and
    pair-scalar tables, the task cursor crossing rows, 16 warps for 3c18 in
    FP32) over many units, element by element against the oracle."""
    cfg = liquid_32k
    prm = oracle.params(cfg["box"], 2.5, NU)
    ref = oracle.atm_cells(prm, cfg["x"], trav, "product", ORC_PREC[prec])
    r, f, _, _ = run_gpu(atm3, cfg, trav, "product", prec)
    assert r["n_cand3"] == ref["n_cand3"]
    assert r["n_int3"] == ref["n_int3"]
    assert r["e3"] == pytest.approx(ref["e3"], rel=RTOL[prec])
    assert r["w3"] == pytest.approx(ref["w3"], rel=RTOL[prec])
    assert_forces_close(f, ref["f"], RTOL[prec], "32k product " + trav + prec)


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
@pytest.mark.parametrize("trunc", ["pair", "product"])
def test_atm_parity_32k_3c01(atm3, liquid_32k, trunc, prec):
    """3c01 (owner computes over 27 cells) on the N = 32,000 liquid."""
    cfg = liquid_32k
    prm = oracle.params(cfg["box"], 2.5, NU)
    ref = oracle.atm_cells(prm, cfg["x"], "3c01", trunc, ORC_PREC[prec])
    r, f, _, _ = run_gpu(atm3, cfg, "3c01", trunc, prec)
    assert r["n_cand3"] == ref["n_cand3"]
    assert r["n_int3"] == ref["n_int3"]
    assert r["e3"] == pytest.approx(ref["e3"], rel=RTOL[prec])
    assert r["w3"] == pytest.approx(ref["w3"], rel=RTOL[prec])
    assert_forces_close(f, ref["f"], RTOL[prec], "32k 3c01 " + trunc + prec)


# ------------------------------------------------------------------ full size, sampled

def _units_touching(cells_nc, cell_ids, trav):
    """Units whose staged cells include any of cell_ids (all contributors to
    the forces on molecules in those cells)."""
    nx, ny, nz = [int(v) for v in cells_nc]
    out = set()
    for c in cell_ids:
        cx, cy, cz = c % nx, (c // nx) % ny, c // (nx * ny)
        rng = range(-1, 2) if trav != "3c08" else range(-1, 1)
        for dz in rng:
            for dy in rng:
                for dx in rng:
                    out.add(((cz + dz) % nz * ny + (cy + dy) % ny) * nx + (cx + dx) % nx)
    return np.array(sorted(out), dtype=np.int64)


@pytest.fixture(scope="module")
def liquid_256k():
    return synth.homogeneous(256000, 0.8, 1.0, seed=5000)


@pytest.mark.parametrize("trunc", ["pair", "product"])
@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
@pytest.mark.parametrize("trav", ["3c01", "3c18", "3c08"])
def test_full_size_256k_sampled(atm3, liquid_256k, trav, trunc, prec):
    """N = 256,000 liquid in the benchmark's launch configuration: the forces
    of molecules in sampled cells are recomputed by the oracle from every unit
    that touches those cells; the totals are checked by invariants."""
    cfg = liquid_256k
    prm = oracle.params(cfg["box"], 2.5, NU)
    r, f, _, cells = run_gpu(atm3, cfg, trav, trunc, prec)
    rng = np.random.default_rng(1)
    ncell = len(cells["cell_start"]) - 1
    sample = rng.choice(ncell, size=6, replace=False)
    # 3c01 writes F_i of its own base cell only
    units = np.sort(sample).astype(np.int64) if trav == "3c01" else \
        _units_touching(cells["ncell"], sample, trav)
    ref = oracle.atm_cells_units(prm, cfg["x"], units, trav, trunc, ORC_PREC[prec])
    mol = np.concatenate([cells["perm"][cells["cell_start"][c]:cells["cell_start"][c + 1]]
                          for c in sample])
    assert_forces_close(f[:, mol], ref["f"][:, mol], RTOL[prec], "sampled " + trav + trunc)
    # invariants at full size: W3 = 9 E3, zero net force (Newton-3 traversals),
    # counts of the order the liquid's density gives
    assert r["w3"] == pytest.approx(9 * r["e3"], rel=1e-9 if prec == "fp64" else 1e-5)
    if trav != "3c01":
        net = np.abs(f.sum(axis=1)).max()
        assert net < (1e-9 if prec == "fp64" else 1e-3) * np.abs(f).max() * 10
    assert r["n_int3"] > (0.5e7 if trunc == "pair" else 2.5e8)


# ------------------------------------------------------------------ capacity fallbacks

@pytest.mark.parametrize("trav", ["3c18", "3c08", "3c08a"])
@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_large_units_product_rule(atm3, trav, prec):
    """Units too large for the dense pair tables (N = 1500 in a 4-cell box,
    ~23 molecules per cell) take the per-molecule accumulator path."""
    cfg = synth.homogeneous(1500, 0.8, 1.0, seed=1001)
    prm = oracle.params(cfg["box"], 2.5, NU)
    ref = oracle.atm_cells(prm, cfg["x"], trav, "product", ORC_PREC[prec])
    r, f, _, _ = run_gpu(atm3, cfg, trav, "product", prec)
    assert r["n_cand3"] == ref["n_cand3"] and r["n_int3"] == ref["n_int3"]
    assert r["e3"] == pytest.approx(ref["e3"], rel=RTOL[prec])
    assert_forces_close(f, ref["f"], RTOL[prec], "large units " + trav + prec)


@pytest.mark.parametrize("trav", ["3c18", "3c08", "3c08a"])
@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_product_rule_at_the_256k_cell_edge(atm3, trav, prec):
    """The cell edge of the 256,000-molecule liquid (2.53 sigma, about 13
    molecules per cell; here 829 molecules, 4 cells per axis): the product
    rule's dense distance and pair-scalar tables fit shared memory, 3c18's
    units (up to 199 molecules) leave one CTA per SM and run 16 warps in FP32,
    3c08's (up to 117) run 8 warps -- the plans the benchmark times, with the
    candidate tasks spanning row ends and several rows."""
    cfg = synth.homogeneous(829, 0.8, 1.0, seed=1003)
    prm = oracle.params(cfg["box"], 2.5, NU)
    ref = oracle.atm_cells(prm, cfg["x"], trav, "product", ORC_PREC[prec])
    r, f, _, _ = run_gpu(atm3, cfg, trav, "product", prec)
    assert r["n_cand3"] == ref["n_cand3"] and r["n_int3"] == ref["n_int3"]
    assert r["e3"] == pytest.approx(ref["e3"], rel=RTOL[prec])
    assert r["w3"] == pytest.approx(ref["w3"], rel=RTOL[prec])
    assert_forces_close(f, ref["f"], RTOL[prec], "256k cell edge " + trav + prec)


@pytest.mark.parametrize("trav", ["3c18", "3c08", "3c08a"])
@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_dense_liquid_edge_table_overflow(atm3, trav, prec):
    """At rho* = 1.4 units have more pair-rule edges than the per-unit edge table
    holds and fall back to per-molecule accumulators; results are unchanged."""
    cfg = synth.homogeneous(2000, 1.4, 1.0, seed=77, jitter=0.02)
    prm = oracle.params(cfg["box"], 2.5, NU)
    ref = oracle.atm_cells(prm, cfg["x"], trav, "pair", ORC_PREC[prec])
    r, f, _, _ = run_gpu(atm3, cfg, trav, "pair", prec)
    assert r["n_cand3"] == ref["n_cand3"] and r["n_int3"] == ref["n_int3"]
    assert r["e3"] == pytest.approx(ref["e3"], rel=RTOL[prec])
    assert_forces_close(f, ref["f"], RTOL[prec], "dense " + trav + prec)


@pytest.mark.parametrize("trav", ["3c18", "3c08", "3c08a"])
@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_edge_table_follows_the_recorded_need(atm3, trav, prec):
    """Outside the deterministic mode the pair rule's edge table is sized from
    the needs the units recorded in earlier evaluations of the context.  A
    liquid at rho* 0.5 sets a small capacity; the same context then evaluates
    a state whose molecules are packed into one corner region at rho* 0.8:
    its first evaluation overflows the small table (those units fall back to
    per-molecule accumulators), the second sizes the table from the new need.
    Both equal the oracle, with the same counts."""
    cfg = synth.homogeneous(2000, 0.5, 1.0, seed=1004)
    box = np.broadcast_to(np.asarray(cfg["box"], dtype=np.float64), (3,))
    packed = np.ascontiguousarray(np.mod(cfg["x"], box[:, None]) * (0.5 / 0.8) ** (1.0 / 3.0))
    prm = oracle.params(cfg["box"], 2.5, NU)
    ref = oracle.atm_cells(prm, packed, trav, "pair", ORC_PREC[prec])
    got = []
    with atm3.AtmSystem(cfg["box"], cfg["n"], nu=NU) as s:
        s.set_state(cfg["x"])
        s.build_cells()
        for _ in range(2):
            s.compute_forces(trav, "pair", prec)
        s.set_state(packed)
        s.build_cells()
        for _ in range(2):
            r = s.compute_forces(trav, "pair", prec)
            got.append((r, s.get_forces("atm")))
    for r, f in got:
        assert r["n_cand3"] == ref["n_cand3"] and r["n_int3"] == ref["n_int3"]
        assert r["e3"] == pytest.approx(ref["e3"], rel=RTOL[prec])
        assert_forces_close(f, ref["f"], RTOL[prec], "recorded need " + trav + prec)


# ------------------------------------------------------------------ wide traversal

def _wide_liquid():
    # rho 0.5, 12.6-sigma box: 5 cells per axis
    return synth.homogeneous(1000, 0.5, 1.0, seed=77)


@pytest.mark.parametrize("trunc", ["pair", "product"])
@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_wide_traversal_matches_oracle(atm3, trunc, prec):
    cfg = _wide_liquid()
    prm = oracle.params(cfg["box"], 2.5, NU)
    r, f, _, _ = run_gpu(atm3, cfg, "3cw", trunc, prec)
    ref = oracle.atm_cells(prm, cfg["x"], "3cw", trunc, ORC_PREC[prec])
    assert r["n_int3"] == ref["n_int3"] and r["n_cand3"] == ref["n_cand3"]
    assert_forces_close(f, ref["f"], RTOL[prec], "3cw " + trunc)
    assert abs(r["e3"] - ref["e3"]) <= RTOL[prec] * abs(ref["e3"]) * 10
    assert abs(r["w3"] - ref["w3"]) <= RTOL[prec] * abs(ref["w3"]) * 10


def test_wide_traversal_finds_what_the_paper_traversals_miss(atm3):
    # product rule: the wide traversal equals the brute force over all triplets
    # (its completeness bound holds here), the paper's traversals find fewer
    cfg = _wide_liquid()
    prm = oracle.params(cfg["box"], 2.5, NU)
    bf = oracle.atm_brute(prm, cfg["x"], "product")
    r, f, _, _ = run_gpu(atm3, cfg, "3cw", "product", "fp64")
    assert r["n_int3"] == 3 * bf["n_int3"]
    assert abs(r["e3"] - bf["e3"]) <= 1e-10 * abs(bf["e3"])
    assert_forces_close(f, bf["f"], 1e-10, "3cw vs brute force")
    for trav in ("3c18", "3c08"):
        rt, _, _, _ = run_gpu(atm3, cfg, trav, "product", "fp64")
        assert rt["n_int3"] < bf["n_int3"]


def test_wide_traversal_needs_five_cells(atm3):
    cfg = small_liquid()  # 4 cells per axis
    with atm3.AtmSystem(cfg["box"], 1000, nu=NU) as s:
        s.set_state(cfg["x"])
        s.build_cells()
        with pytest.raises(atm3.AtmError) as e:
            s.compute_forces("3cw", "product", "fp64")
        assert e.value.status == 2


def test_wide_traversal_32k_sampled(atm3):
    """N = 32,000 liquid (13 cells per axis): the owner forces of molecules in
    sampled base cells against the oracle run on those units alone."""
    cfg = synth.config("liquid_n32k")
    prm = oracle.params(cfg["box"], 2.5, NU)
    r, f, _, cells = run_gpu(atm3, cfg, "3cw", "product", "fp32c")
    rng = np.random.default_rng(2)
    ncell = len(cells["cell_start"]) - 1
    sample = rng.choice(ncell, size=8, replace=False)
    ref = oracle.atm_cells_units(prm, cfg["x"], sample, "3cw", "product", "fp32")
    mol = np.concatenate([cells["perm"][cells["cell_start"][c]:cells["cell_start"][c + 1]]
                          for c in sample])
    assert_forces_close(f[:, mol], ref["f"][:, mol], RTOL["fp32c"], "sampled 3cw")
    assert r["n_int3"] > 0 and r["w3"] == pytest.approx(9 * r["e3"], rel=1e-5)


# ------------------------------------------------------------------ corner-anchored 3c08

@pytest.mark.parametrize("trunc", ["pair", "product"])
def test_corner_anchored_3c08_equals_the_filtered_brute_force(atm3, trunc):
    """The corner-anchored 3c08 (every task holds the block's corner cell)
    finds exactly the brute-force triplets whose cell triple contains its own
    bounding-box corner (6 cells per axis, so the product rule's base-frame
    displacements are minimum images), fewer than the complete 3c08."""
    rng = np.random.default_rng(44)
    box = np.array([15.3, 15.3, 15.3])
    x = np.ascontiguousarray(
        synth.random_sequential(1100, [0, 0, 0], box, 0.85, rng, box=box).T)
    cfg = dict(x=x, box=box)
    prm = oracle.params(box, 2.5, NU)
    bf = oracle.atm_brute(prm, x, trunc, member="3c08a")
    r, f, _, _ = run_gpu(atm3, cfg, "3c08a", trunc, "fp64")
    assert r["n_int3"] == bf["n_int3"]
    assert r["e3"] == pytest.approx(bf["e3"], rel=1e-10)
    assert_forces_close(f, bf["f"], 1e-10, "3c08a/" + trunc)
    full, _, _, _ = run_gpu(atm3, cfg, "3c08", trunc, "fp64")
    assert r["n_int3"] < full["n_int3"]
