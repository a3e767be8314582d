"""Domain decomposition on the GPU: two or three ranks, each with its own
context of the CUDA library restricted to its slab of cell layers
(atm_set_owned_layers), exchanging halos in one process (domain.LocalRanks).
Total forces (LJ + ATM), energies, virials and counts must equal the
single-domain evaluation of the whole system by the same library (counts
exact; FP64 1e-10, FP32C 2e-5 relative per component, floor of the same size
times the RMS force), and the ATM part the oracle's.
"""
import numpy as np
import pytest

import oracle
from paper_2510_21230_gb300 import domain, synth

pytestmark = pytest.mark.gpu

NU, RC = 0.073, 2.5
RTOL = {"fp64": 1e-10, "fp32c": 2e-5}


@pytest.fixture(scope="module")
def atm3():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_21230_gb300 import atm3 as m, build
    build.build()
    return m


def _close(got, ref, rtol):
    scale = np.sqrt(np.mean(ref * ref))
    err = np.abs(got - ref)
    assert np.all(err <= rtol * np.abs(ref) + rtol * scale), float((err / (np.abs(ref) + scale)).max())


@pytest.fixture(scope="module")
def liquid():
    return synth.homogeneous(32000, 0.8, 1.0, seed=2000)  # 13 cell layers


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
@pytest.mark.parametrize("trav,trunc", [("3c01", "pair"), ("3c18", "pair"), ("3c08", "pair"),
                                        ("3c08a", "pair"), ("3c08", "product"),
                                        ("3c18", "product")])
def test_ranks_equal_the_single_domain_library(atm3, liquid, world, prec, trav, trunc):
    cfg = liquid
    n = cfg["n"]
    with atm3.AtmSystem(cfg["box"], n, rc=RC, nu=NU) as s:
        s.set_state(cfg["x"])
        s.build_cells()
        ref = s.compute_forces(trav, trunc, prec)
        f_ref = s.get_forces("total")
    backends = [domain.LibraryBackend(rc=RC, nu=NU) for _ in range(world)]
    try:
        nz = backends[0].nz(cfg["box"])
        states = domain.distribute(cfg["x"], backends[0].layers(cfg["box"], cfg["x"]), cfg["box"],
                                   nz, world)
        ranks = domain.LocalRanks(states, backends)
        res = ranks.evaluate(trav, trunc, prec)
        f = ranks.gather(n)
    finally:
        for b in backends:
            b.close()
    for k in ("n_cand3", "n_int3", "n_cand2", "n_int2"):
        assert res[k] == ref[k], k
    for k in ("e2", "e3", "w2", "w3"):
        assert res[k] == pytest.approx(ref[k], rel=RTOL[prec]), k
    _close(f, f_ref, RTOL[prec])


def test_ranks_atm_equal_the_oracle(atm3, liquid):
    """The ATM part of a two-rank FP64 3c08 evaluation -- its total minus the
    total of the same ranks with nu = 0 (LJ only) -- equals the oracle's ATM
    forces."""
    cfg = liquid
    ref = oracle.atm_cells(oracle.params(cfg["box"], RC, NU), cfg["x"], "3c08", "pair", "fp64")
    tot, lj = [], []
    for nu in (NU, 0.0):
        backends = [domain.LibraryBackend(rc=RC, nu=nu) for _ in range(2)]
        try:
            nz = backends[0].nz(cfg["box"])
            states = domain.distribute(cfg["x"], backends[0].layers(cfg["box"], cfg["x"]),
                                       cfg["box"], nz, 2)
            ranks = domain.LocalRanks(states, backends)
            res = ranks.evaluate("3c08", "pair", "fp64")
            (tot if nu else lj).append((res, ranks.gather(cfg["n"])))
        finally:
            for b in backends:
                b.close()
    assert tot[0][0]["n_int3"] == ref["n_int3"]
    _close(tot[0][1] - lj[0][1], ref["f"], 1e-10)
