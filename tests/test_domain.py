"""Domain decomposition (paper_2510_21230_gb300/domain.py) on the CPU: the
partition, halo exchange, force return and sums, with the oracle's linked-cell
ATM restricted to each rank's units as the compute backend.  The ranks' forces
must equal the single-domain oracle's (1e-10 relative per component, floor of
the same size times the RMS force) and the summed counts must be exact, for
two gloo ranks (torch.distributed) and for two or three ranks in one process.
"""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_2510_21230_gb300 import domain, synth

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

NU, RC = 0.073, 2.5


class OracleBackend:
    """ATM triplets of the units based or anchored in layers [z0, z1), by the
    oracle; cell layers from the oracle's cell build."""

    def _grid(self, box):
        prm = oracle.params(box, RC, NU)
        return prm, oracle.cell_grid(prm)[0]

    def layers(self, box, x):
        prm, nc = self._grid(box)
        return oracle.build_cells(prm, x)["cell_of"] // (int(nc[0]) * int(nc[1]))

    def forces(self, box, x, z0, z1, trav, trunc, prec):
        prm, nc = self._grid(box)
        per = int(nc[0]) * int(nc[1])
        units = np.arange(per * z0, per * z1, dtype=np.int64)
        r = oracle.atm_cells_units(prm, x, units, trav, trunc, prec)
        return r["f"], r, self.layers(box, x)


def _liquid():
    # 4000 molecules at rho 0.8: a 17.1-sigma box, 6 cells per axis
    return synth.homogeneous(4000, 0.8, 1.0, seed=3100)


def _close(got, ref, rtol=1e-10):
    scale = np.sqrt(np.mean(ref * ref))
    err = np.abs(got - ref)
    assert np.all(err <= rtol * np.abs(ref) + rtol * scale), float((err / (np.abs(ref) + scale)).max())


def _reference(cfg, trav, trunc):
    return oracle.atm_cells(oracle.params(cfg["box"], RC, NU), cfg["x"], trav, trunc, "fp64")


def test_slabs_partition_the_layers():
    assert domain.slabs(6, 2) == [(0, 3), (3, 6)]
    assert domain.slabs(13, 3) == [(0, 5), (5, 9), (9, 13)]
    assert domain.slabs(4, 2) == [(0, 2), (2, 4)]
    with pytest.raises(ValueError):
        domain.slabs(5, 3)  # two layers per rank at least


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("trav,trunc", [("3c01", "pair"), ("3c18", "pair"), ("3c08", "pair"),
                                        ("3c08a", "pair"), ("3c08", "product")])
def test_local_ranks_equal_the_single_domain_oracle(world, trav, trunc):
    cfg = _liquid()
    be = OracleBackend()
    nz = int(oracle.cell_grid(oracle.params(cfg["box"], RC, NU))[0][2])
    states = domain.distribute(cfg["x"], be.layers(cfg["box"], cfg["x"]), cfg["box"], nz, world)
    assert sorted(np.concatenate([s.ids for s in states]).tolist()) == list(range(cfg["n"]))
    ranks = domain.LocalRanks(states, [be] * world)
    res = ranks.evaluate(trav, trunc, "fp64")
    ref = _reference(cfg, trav, trunc)
    assert res["n_cand3"] == ref["n_cand3"] and res["n_int3"] == ref["n_int3"]
    assert res["e3"] == pytest.approx(ref["e3"], rel=1e-12)
    assert res["w3"] == pytest.approx(ref["w3"], rel=1e-12)
    _close(ranks.gather(cfg["n"]), ref["f"])


def test_migration_keeps_every_molecule_and_the_forces():
    """Molecules moved by up to half a cell along z change ranks; after the
    migration every molecule is on the rank of its layer and the forces still
    equal the oracle's on the moved system."""
    cfg = _liquid()
    be = OracleBackend()
    prm = oracle.params(cfg["box"], RC, NU)
    nc, w = oracle.cell_grid(prm)
    nz = int(nc[2])
    states = domain.distribute(cfg["x"], be.layers(cfg["box"], cfg["x"]), cfg["box"], nz, 2)
    ranks = domain.LocalRanks(states, [be, be])
    rng = np.random.default_rng(5)
    for st in states:
        st.x = st.x.copy()
        st.x[2] += rng.uniform(-0.5, 0.5, size=st.x.shape[1]) * w[2]
        st.layers = be.layers(st.box, st.x)
    moved = np.zeros_like(cfg["x"])
    for st in states:
        moved[:, st.ids] = st.x
    ranks.migrate()
    lay = be.layers(cfg["box"], moved)
    for st in states:
        z0, z1 = st.z0, st.z1
        assert np.all((lay[st.ids] >= z0) & (lay[st.ids] < z1))
    assert sorted(np.concatenate([s.ids for s in states]).tolist()) == list(range(cfg["n"]))
    res = ranks.evaluate("3c08", "pair", "fp64")
    ref = oracle.atm_cells(prm, moved, "3c08", "pair", "fp64")
    assert res["n_int3"] == ref["n_int3"]
    _close(ranks.gather(cfg["n"]), ref["f"])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cfg = _liquid()
    be = OracleBackend()
    nz = int(oracle.cell_grid(oracle.params(cfg["box"], RC, NU))[0][2])
    st = domain.distribute(cfg["x"], be.layers(cfg["box"], cfg["x"]), cfg["box"], nz, world)[rank]
    tr = domain.DistTransport("cpu")
    results = {}
    for trav, trunc in (("3c08", "pair"), ("3c18", "product"), ("3c01", "pair")):
        res = domain.evaluate_dist(st, be, tr, trav, trunc, "fp64")
        results[(trav, trunc)] = (res, st.ids.copy(), st.f.copy())
    out.put((rank, results))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_equal_the_single_domain_oracle():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=600) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    cfg = _liquid()
    for key in got[0]:
        ref = _reference(cfg, *key)
        res0, res1 = got[0][key][0], got[1][key][0]
        assert res0 == res1                       # every rank has the global sums
        assert res0["n_cand3"] == ref["n_cand3"] and res0["n_int3"] == ref["n_int3"], key
        assert res0["e3"] == pytest.approx(ref["e3"], rel=1e-12), key
        f = np.zeros((3, cfg["n"]))
        for r in (0, 1):
            _, ids, fr = got[r][key]
            f[:, ids] = fr
        _close(f, ref["f"])
