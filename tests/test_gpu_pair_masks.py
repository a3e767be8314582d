"""Pair bitmaps of the FP32C pair rule (atm_set_pair_masks) through the C ABI.

With the bitmaps the 3c18 / 3c08 / 3c08a units take their pair decisions from
one kernel that decides every pair of neighbouring cells once; without them
each unit decides its own pairs.  Both use the same FP32 arithmetic, so in
deterministic mode (force sums independent of the order of the additions) the
forces must agree bit for bit and the counts exactly, on a single system, a
batch of uneven replicas and in steps.  A system with a cell of more than 32
molecules runs without bitmaps and still matches the oracle; graph steps
whose cells fill beyond 32 during the replay restart and end where plain
steps end.
"""
import numpy as np
import pytest

import oracle
from paper_2510_21230_gb300 import synth

pytestmark = pytest.mark.gpu

NU = 0.073
KEYS = ("n_cand3", "n_int3", "n_cand2", "n_int2")


@pytest.fixture(scope="module")
def atm3():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_21230_gb300 import atm3 as m, build
    build.build()
    return m


def _occupancy(box, x, rc=2.5):
    box = np.broadcast_to(np.asarray(box, dtype=np.float64), (3,))
    nc = np.floor(box / rc).astype(int)
    w = box / nc
    ci = np.floor(np.mod(x.T, box) / w).astype(int) % nc
    return np.bincount((ci[:, 2] * nc[1] + ci[:, 1]) * nc[0] + ci[:, 0], minlength=int(np.prod(nc)))


def _evaluate(atm3, boxes, ns, x, trav, masks, persistent=False):
    with atm3.AtmSystem(boxes, ns, nu=NU) as s:
        s.set_deterministic(True)
        s.set_pair_masks(masks)
        s.set_options(persistent=persistent)
        s.set_state(x)
        s.build_cells()
        s.compute_forces(trav, "pair", "fp32c")
        res = s.results()
        f = s.get_forces("total")
    return res, f


@pytest.mark.parametrize("trav", ["3c08", "3c18", "3c08a"])
@pytest.mark.parametrize("persistent", [False, True])
def test_bitmaps_equal_unit_decisions_32k(atm3, trav, persistent):
    cfg = synth.homogeneous(32000, 0.8, 1.0, seed=2000)
    assert _occupancy(cfg["box"], cfg["x"]).max() <= 32
    on = _evaluate(atm3, cfg["box"], cfg["n"], cfg["x"], trav, True, persistent)
    off = _evaluate(atm3, cfg["box"], cfg["n"], cfg["x"], trav, False, persistent)
    for a, b in zip(on[0], off[0]):
        for k in KEYS:
            assert a[k] == b[k], k
        assert a["e3"] == pytest.approx(b["e3"], rel=1e-12)
    assert np.array_equal(on[1], off[1])


@pytest.mark.parametrize("trav", ["3c08", "3c18"])
def test_bitmaps_equal_unit_decisions_batch(atm3, trav):
    reps = synth.replicas(count=6, n_lo=500, n_hi=3000)
    ns = [r["n"] for r in reps]
    boxes = [r["box"] for r in reps]
    x = np.ascontiguousarray(np.concatenate([r["x"] for r in reps], axis=1))
    on = _evaluate(atm3, boxes, ns, x, trav, True)
    off = _evaluate(atm3, boxes, ns, x, trav, False)
    for a, b in zip(on[0], off[0]):
        for k in KEYS:
            assert a[k] == b[k], k
    assert np.array_equal(on[1], off[1])


def test_bitmap_steps_equal_unit_decision_steps(atm3):
    """Steps with LJ inside the 3c08 units (the benchmark's step), graph
    steps included: bit-identical trajectories with and without bitmaps."""
    cfg = synth.homogeneous(4000, 0.8, 1.0, seed=2001)
    out = []
    for masks in (True, False):
        for graph in (False, True):
            with atm3.AtmSystem(cfg["box"], cfg["n"], nu=NU, dt=0.002) as s:
                s.set_deterministic(True)
                s.set_pair_masks(masks)
                s.set_options(graph=graph)
                s.set_state(cfg["x"], cfg["v"])
                r = s.step(10, "3c08", "pair", "fp32c")
                xs, vs = s.get_state()
                out.append((r, xs, vs))
    for r, xs, vs in out[1:]:
        assert r["n_int3"] == out[0][0]["n_int3"] and r["n_int2"] == out[0][0]["n_int2"]
        assert np.array_equal(xs, out[0][1]) and np.array_equal(vs, out[0][2])


def test_cells_above_32_run_without_bitmaps(atm3):
    """A dense liquid (rho 2.3, about 37 molecules per cell) cannot use the
    bitmaps: the units decide their pairs and the counts equal the oracle's
    FP32-decision counts."""
    cfg = synth.homogeneous(1000, 2.3, 1.0, seed=2002)
    assert _occupancy(cfg["box"], cfg["x"]).max() > 32
    prm = oracle.params(cfg["box"], 2.5, NU)
    for trav in ("3c08", "3c18"):
        ref = oracle.atm_cells(prm, cfg["x"], trav, "pair", "fp32")
        res, f = _evaluate(atm3, cfg["box"], cfg["n"], cfg["x"], trav, True)
        assert res[0]["n_int3"] == ref["n_int3"] and res[0]["n_cand3"] == ref["n_cand3"]


def test_graph_restarts_when_a_cell_fills_beyond_32(atm3):
    """Free flight (no LJ, nu = 0) under a compressing velocity field: the
    graph is captured with bitmaps (every cell within 32), the central cells
    then fill beyond 32 during the replayed steps; the run must restart
    without the graph and end with the plain steps' positions and counts."""
    cfg = synth.homogeneous(8000, 0.9, 1.0, seed=2003)
    box = cfg["box"]
    x = np.ascontiguousarray(cfg["x"])
    v = np.ascontiguousarray(-4.0 * (np.mod(x, box[:, None]) - 0.5 * box[:, None]))
    assert _occupancy(box, x).max() <= 32
    out = []
    for graph in (False, True):
        with atm3.AtmSystem(box, cfg["n"], nu=0.0, lj_eps=0.0, dt=0.002) as s:
            s.set_deterministic(True)
            s.set_options(graph=graph)
            s.set_state(x, v)
            r = s.step(40, "3c08", "pair", "fp32c")
            xs, _ = s.get_state()
            out.append((r, xs))
    assert _occupancy(box, out[0][1]).max() > 32
    assert out[0][0]["n_int3"] == out[1][0]["n_int3"]
    assert np.array_equal(out[0][1], out[1][1])
