"""Batches of independent replicas, launch options, autotuning and the density
profile, through the C ABI.

A batch must give, replica by replica, exactly what separate single-system
runs give (counts bit-exact, forces within the parity tolerances), whatever
the launch form (one CTA per unit or persistent, 4 or 8 warps, CUDA-graph
steps).  The density profile is an integer histogram and must equal the
histogram of the wrapped positions bit for bit.
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


def close(got, ref, rtol):
    scale = np.sqrt(np.mean(ref * ref)) if ref.size else 0.0
    return np.all(np.abs(got - ref) <= rtol * np.abs(ref) + rtol * scale)


@pytest.fixture(scope="module")
def ensemble():
    """Six replicas with uneven N, density and temperature (the batched-ensemble recipe)."""
    return synth.replicas(count=6, n_lo=500, n_hi=3000)


def _concat(reps, key):
    return np.ascontiguousarray(np.concatenate([r[key] for r in reps], axis=1))


@pytest.mark.parametrize("trav,trunc,prec", [("3c08", "pair", "fp32c"), ("3c18", "pair", "fp64"),
                                             ("3c08", "product", "fp64"), ("3c01", "pair", "fp32c")])
def test_batch_equals_separate_runs(atm3, ensemble, trav, trunc, prec):
    ns = [r["n"] for r in ensemble]
    boxes = [r["box"] for r in ensemble]
    x = _concat(ensemble, "x")
    with atm3.AtmSystem(boxes, ns, nu=NU) as b:
        b.set_state(x)
        b.build_cells()
        b.compute_forces(trav, trunc, prec)
        res = b.results()
        f = b.get_forces("total")
    off = 0
    for r, rep in enumerate(ensemble):
        with atm3.AtmSystem(rep["box"], rep["n"], nu=NU) as s:
            s.set_state(rep["x"])
            s.build_cells()
            one = s.compute_forces(trav, trunc, prec)
            f1 = s.get_forces("total")
        for k in ("n_cand3", "n_int3", "n_cand2", "n_int2"):
            assert res[r][k] == one[k], (r, k)
        for k in ("e2", "e3", "w2", "w3"):
            assert res[r][k] == pytest.approx(one[k], rel=RTOL[prec], abs=1e-12), (r, k)
        assert close(f[:, off:off + rep["n"]], f1, RTOL[prec]), r
        off += rep["n"]


def test_batch_matches_oracle(atm3, ensemble):
    ns = [r["n"] for r in ensemble]
    with atm3.AtmSystem([r["box"] for r in ensemble], ns, nu=NU) as b:
        b.set_state(_concat(ensemble, "x"))
        b.build_cells()
        b.compute_forces("3c08", "pair", "fp64")
        res = b.results()
        f = b.get_forces("atm")
    off = 0
    for r, rep in enumerate(ensemble):
        ref = oracle.atm_cells(oracle.params(rep["box"], 2.5, NU), rep["x"], "3c08", "pair")
        assert res[r]["n_int3"] == ref["n_int3"] and res[r]["n_cand3"] == ref["n_cand3"]
        assert res[r]["e3"] == pytest.approx(ref["e3"], rel=1e-10)
        assert close(f[:, off:off + rep["n"]], ref["f"], 1e-10)
        off += rep["n"]


@pytest.mark.parametrize("persistent,nwarps", [(True, 0), (False, 8), (True, 8), (True, 4)])
def test_launch_forms_agree(atm3, ensemble, persistent, nwarps):
    ns = [r["n"] for r in ensemble]
    x = _concat(ensemble, "x")
    out = []
    for opts in [dict(), dict(persistent=persistent, nwarps=nwarps)]:
        with atm3.AtmSystem([r["box"] for r in ensemble], ns, nu=NU) as b:
            if opts:
                b.set_options(**opts)
            b.set_state(x)
            b.build_cells()
            b.compute_forces("3c08", "pair", "fp32c")
            out.append((b.results(), b.get_forces("total")))
    # FP32 pair scalars are summed by shared-memory atomics whose order depends
    # on warp scheduling: the FP32C tolerance applies between launch forms
    for ra, rb in zip(out[0][0], out[1][0]):
        assert ra["n_int3"] == rb["n_int3"] and ra["n_cand3"] == rb["n_cand3"]
        assert rb["e3"] == pytest.approx(ra["e3"], rel=RTOL["fp32c"])
    assert close(out[1][1], out[0][1], RTOL["fp32c"])


def test_graph_steps_equal_plain_steps(atm3, ensemble):
    ns = [r["n"] for r in ensemble]
    x, v = _concat(ensemble, "x"), _concat(ensemble, "v")
    final = []
    for graph in (False, True):
        with atm3.AtmSystem([r["box"] for r in ensemble], ns, nu=NU, dt=0.002) as b:
            b.set_options(graph=graph)
            b.set_state(x, v)
            b.step(8, "3c08", "pair", "fp64")
            res = b.results()
            xs, vs = b.get_state()
            final.append((res, xs, vs))
    (ra, xa, va), (rb, xb, vb) = final
    for a, c in zip(ra, rb):
        assert a["n_int3"] == c["n_int3"]
        assert c["e3"] == pytest.approx(a["e3"], rel=1e-9)
    assert np.abs(xa - xb).max() < 1e-10 and np.abs(va - vb).max() < 1e-9


@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
def test_graph_steps_restart_when_a_unit_outgrows_the_capacity(atm3, prec):
    """A graph sizes its kernels for the largest unit at capture plus at most a
    quarter of it (at least 8) of headroom.  Under a compressing velocity
    field v = -k (x - centre) the central units of a dilute liquid fill up
    during the replayed steps beyond that capacity: the run must detect it,
    restart from its snapshot without the graph, and end where plain steps
    end.  In deterministic mode the forces do not depend on the launch form,
    so positions and velocities must agree bit for bit."""
    cfg = synth.homogeneous(2000, 0.25, 1.0, seed=1300)  # 20-sigma box, 8 cells per axis
    box = cfg["box"]
    x = np.ascontiguousarray(cfg["x"])
    v = np.ascontiguousarray(cfg["v"] - 4.0 * (np.mod(x, box[:, None]) - 0.5 * box[:, None]))
    m0 = int(_unit_sizes(dict(box=box, x=x), "3c08").max())
    final = []
    for graph in (False, True):
        with atm3.AtmSystem(box, cfg["n"], nu=NU, dt=0.002) as s:
            s.set_deterministic(True)
            s.set_options(graph=graph)
            s.set_state(x, v)
            res = s.step(40, "3c08", "pair", prec)
            xs, vs = s.get_state()
            final.append((res, xs, vs))
    m1 = int(_unit_sizes(dict(box=box, x=final[0][1]), "3c08").max())
    assert m1 > m0 + max(8, m0 // 4), (m0, m1)  # the graph's capacity was exceeded
    (ra, xa, va), (rb, xb, vb) = final
    assert ra["n_int3"] == rb["n_int3"] and ra["n_int2"] == rb["n_int2"]
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)


def test_autotune_keeps_results(atm3, ensemble):
    ns = [r["n"] for r in ensemble]
    with atm3.AtmSystem([r["box"] for r in ensemble], ns, nu=NU) as b:
        b.set_state(_concat(ensemble, "x"))
        b.build_cells()
        b.compute_forces("3c08", "pair", "fp32c")
        before = b.results()
        t = b.autotune("3c08", "pair", "fp32c", reps=2)
        assert t["persistent"] in (0, 1) and t["nwarps"] in (4, 8) and t["ms_per_eval"] > 0
        b.compute_forces("3c08", "pair", "fp32c")
        after = b.results()
    for a, c in zip(before, after):
        assert a["n_int3"] == c["n_int3"]
        assert c["e3"] == pytest.approx(a["e3"], rel=RTOL["fp32c"])


def test_density_profile_is_the_histogram_of_wrapped_positions(atm3):
    cfg = synth.slab(box=(12.0, 12.0, 40.0), thickness=12.0, seed=3001)
    nb = 600
    with atm3.AtmSystem(cfg["box"], cfg["n"], nu=NU) as s:
        s.set_state(cfg["x"], cfg["v"])
        s.build_cells()
        s.density_accumulate(2, nb)
        counts, samples = s.density_get(nb)
        xw, _ = s.get_state()
    h = cfg["box"][2] / nb
    b = np.clip(np.floor(xw[2] / h).astype(np.int64), 0, nb - 1)
    ref = np.bincount(b, minlength=nb)
    assert samples == 1
    assert np.array_equal(counts[0].astype(np.int64), ref)
    assert counts.sum() == cfg["n"]


def test_contexts_of_different_unit_sizes_interleave(atm3):
    """Contexts in one process share the kernels' shared-memory limit: a
    context with small units launched after one with large units must not
    lower it under the large one's next launch (steps and graph steps)."""
    big = synth.homogeneous(4000, 0.95, 1.0, seed=1200)
    small = synth.homogeneous(600, 0.3, 1.0, seed=1201)
    with atm3.AtmSystem(big["box"], big["n"], nu=NU) as a, \
            atm3.AtmSystem(small["box"], small["n"], nu=NU) as b:
        a.set_state(big["x"], big["v"])
        b.set_state(small["x"], small["v"])
        for prec in ("fp32c", "fp64"):
            ra = a.step(2, "3c08", "pair", prec)
            rb = b.step(2, "3c08", "pair", prec)
            ra2 = a.step(2, "3c08", "pair", prec)
            assert ra["n_int3"] > 0 and rb["n_int3"] > 0 and ra2["n_int3"] > 0
        a.set_options(graph=True)
        b.set_options(graph=True)
        for _ in range(2):
            a.step(3, "3c08", "pair", "fp32c")
            b.step(3, "3c08", "pair", "fp32c")


def _unit_sizes(rep, trav):
    """Staged molecules of every unit of one replica (8 cells of the 2x2x2
    block for 3c08 / 3c08a, the base cell and its 13 forward neighbours for
    3c18), from the cell counts."""
    box = np.broadcast_to(np.asarray(rep["box"], dtype=np.float64), (3,))
    nc = np.floor(box / 2.5).astype(int)
    w = box / nc
    ci = np.floor(np.mod(rep["x"].T, box) / w).astype(int) % nc
    cnt = np.bincount((ci[:, 0] * nc[1] + ci[:, 1]) * nc[2] + ci[:, 2],
                      minlength=int(np.prod(nc))).reshape(tuple(nc))
    if trav == "3c18":
        offs = [(0, 0, 0)] + [o for o in np.ndindex(3, 3, 3)
                              if (o[0] - 1, o[1] - 1, o[2] - 1) > (0, 0, 0)]
        offs = [(0, 0, 0)] + [(a - 1, b - 1, c - 1) for a, b, c in offs[1:]]
    else:
        offs = [(a, b, c) for a in (0, 1) for b in (0, 1) for c in (0, 1)]
    return sum(np.roll(cnt, (-a, -b, -c), axis=(0, 1, 2)) for a, b, c in offs).ravel()


@pytest.mark.parametrize("trav,trunc,prec", [("3c08", "pair", "fp32c"), ("3c08", "pair", "fp64"),
                                             ("3c18", "pair", "fp32c"), ("3c08a", "pair", "fp32c"),
                                             ("3c08", "product", "fp32c"),
                                             ("3c18", "product", "fp64")])
def test_unit_size_classes_equal_one_launch(atm3, ensemble, trav, trunc, prec):
    """Units run in size classes (2 or 3 launches with their own shared-memory
    plans) give the one-launch results: counts exactly, energies and forces to
    rounding (FP64: the order of the additions; FP32C: also the warps and
    pair-scalar tables of the class plans, within the parity tolerance).  The
    bounds are chosen from the ensemble's unit sizes so that every class
    holds units."""
    ns = [r["n"] for r in ensemble]
    sizes = np.concatenate([_unit_sizes(r, trav) for r in ensemble])
    q = [int(np.percentile(sizes, p)) for p in (30, 70)]
    assert sizes.min() <= q[0] < q[1] < sizes.max()
    with atm3.AtmSystem([r["box"] for r in ensemble], ns, nu=NU) as b:
        b.set_state(_concat(ensemble, "x"))
        b.build_cells()
        b.compute_forces(trav, trunc, prec)
        ref = b.results()
        fref = b.get_forces("atm")
        for cuts in ((q[0],), (q[0], q[1]), (64,), (48, 96)):
            b.set_unit_classes(cuts)
            b.compute_forces(trav, trunc, prec)
            got = b.results()
            f = b.get_forces("atm")
            tol = 1e-12 if prec == "fp64" else RTOL["fp32c"]
            for a, c in zip(ref, got):
                assert a["n_int3"] == c["n_int3"] and a["n_cand3"] == c["n_cand3"]
                assert c["e3"] == pytest.approx(a["e3"], rel=tol, abs=1e-12)
                assert c["w3"] == pytest.approx(a["w3"], rel=tol, abs=1e-12)
            assert close(f, fref, 1e-10 if prec == "fp64" else RTOL["fp32c"])
        b.set_unit_classes(())
        b.compute_forces(trav, trunc, prec)
        assert [r["n_int3"] for r in b.results()] == [r["n_int3"] for r in ref]


def test_unit_size_classes_in_graph_steps(atm3, ensemble):
    """Graph steps with three size classes follow the one-launch steps."""
    ns = [r["n"] for r in ensemble]
    boxes = [r["box"] for r in ensemble]
    x, v = _concat(ensemble, "x"), _concat(ensemble, "v")
    sizes = np.concatenate([_unit_sizes(r, "3c08") for r in ensemble])
    cuts = (int(np.percentile(sizes, 30)), int(np.percentile(sizes, 70)))
    out = []
    for classes in ((), cuts):
        with atm3.AtmSystem(boxes, ns, nu=NU, dt=0.002) as b:
            b.set_state(x, v)
            b.set_options(graph=True)
            b.set_unit_classes(classes)
            b.step(20, "3c08", "pair", "fp64")
            out.append((b.results(), b.get_state()))
    (ra, (xa, va)), (rb, (xb, vb)) = out
    for a, c in zip(ra, rb):
        assert a["n_int3"] == c["n_int3"]
        assert c["e3"] == pytest.approx(a["e3"], rel=1e-9)
    assert np.abs(xa - xb).max() < 1e-10 and np.abs(va - vb).max() < 1e-9


def test_unit_size_class_arguments(atm3, ensemble):
    ns = [r["n"] for r in ensemble]
    with atm3.AtmSystem([r["box"] for r in ensemble], ns, nu=NU) as b:
        for bad in ((0,), (64, 32), (64, 64), (10, 20, 30), (4096,)):
            with pytest.raises(atm3.AtmError):
                b.set_unit_classes(bad)
        b.set_unit_classes((40,))
        b.set_unit_classes(())


@pytest.fixture(scope="module")
def ensemble64():
    """The batched-ensemble workload as benchmarked: 64 replicas, N
    log-uniform in [500, 20000], rho U(0.1, 0.85), T U(0.7, 1.3)."""
    return synth.replicas(count=64)


def test_batch_of_64_replicas_as_benchmarked(atm3, ensemble64):
    """The 64-replica batch in the benchmark's launch configuration (graph
    steps, autotuned launch form with unit size classes on a side stream)
    equals the same replicas as 64 separate contexts (counts bit-exact,
    energies and forces within the FP32C tolerance), and three sampled
    replicas equal the oracle."""
    reps = ensemble64
    ns = [r["n"] for r in reps]
    x, v = _concat(reps, "x"), _concat(reps, "v")
    with atm3.AtmSystem([r["box"] for r in reps], ns, nu=NU, dt=0.002) as b:
        b.set_state(x, v)
        b.build_cells()
        b.set_options(graph=True)
        b.autotune("3c08", "pair", "fp32c", reps=2)
        b.step(3, "3c08", "pair", "fp32c")
        xs, vs = b.get_state()
        # forces of the stepped state, with the tuned launch form
        b.set_state(xs, vs)
        b.build_cells()
        b.compute_forces("3c08", "pair", "fp32c")
        res = b.results()
        f = b.get_forces("total")
        fa = b.get_forces("atm")
    off = 0
    for r, rep in enumerate(reps):
        sl = slice(off, off + rep["n"])
        with atm3.AtmSystem(rep["box"], rep["n"], nu=NU) as s:
            s.set_state(np.ascontiguousarray(xs[:, sl]))
            s.build_cells()
            one = s.compute_forces("3c08", "pair", "fp32c")
            f1 = s.get_forces("total")
        for k in ("n_cand3", "n_int3", "n_cand2", "n_int2"):
            assert res[r][k] == one[k], (r, k)
        for k in ("e2", "e3", "w2", "w3"):
            assert res[r][k] == pytest.approx(one[k], rel=RTOL["fp32c"], abs=1e-12), (r, k)
        assert close(f[:, sl], f1, RTOL["fp32c"]), r
        off += rep["n"]
    # oracle parity on three replicas: the smallest, the largest and the densest
    pick = {int(np.argmin(ns)), int(np.argmax(ns)), int(np.argmax([r["rho"] for r in reps]))}
    starts = np.concatenate([[0], np.cumsum(ns)])
    for r in sorted(pick):
        sl = slice(starts[r], starts[r + 1])
        ref = oracle.atm_cells(oracle.params(reps[r]["box"], 2.5, NU),
                               np.ascontiguousarray(xs[:, sl]), "3c08", "pair", "fp32")
        assert res[r]["n_int3"] == ref["n_int3"] and res[r]["n_cand3"] == ref["n_cand3"], r
        assert res[r]["e3"] == pytest.approx(ref["e3"], rel=RTOL["fp32c"]), r
        assert close(fa[:, sl], ref["f"], RTOL["fp32c"]), r


def test_profiling_levels(atm3):
    """atm_set_profiling: level 1 times every launch group of a step, level 2
    the force evaluations only; both count the library's launches; the profile
    is folded in when it is read."""
    cfg = synth.homogeneous(4000, 0.8, 1.0, seed=1400)
    with atm3.AtmSystem(cfg["box"], cfg["n"], nu=NU, dt=0.002) as s:
        s.set_state(cfg["x"], cfg["v"])
        s.step(1, "3c08", "pair", "fp32c")
        out = {}
        for level in (1, 2):
            s.set_profiling(True, forces_only=(level == 2))
            for _ in range(3):
                s.step(1, "3c08", "pair", "fp32c", sync=False)
            out[level] = s.get_profile()
        s.set_profiling(False)
    full, forces = out[1], out[2]
    assert full["ms_atm"] > 0 and full["ms_cells"] > 0 and full["ms_md"] > 0
    assert forces["ms_atm"] > 0 and forces["ms_cells"] == 0 and forces["ms_md"] == 0
    assert full["n_atm_launches"] == forces["n_atm_launches"] == 3
    assert full["n_launches"] == forces["n_launches"] > 0
