"""The allocation-free entry point atm_compute_forces_noalloc.

Some callers cannot allocate device memory (an embedding application that owns
the whole device budget, a plug-in given only raw device pointers); for them
the library keeps its intermediate arrays in one fixed device array instead.
This test calls that entry point through the C ABI several times in a row, on
different inputs -- the last one smaller in molecules and cells than the one
before it, so that anything a call fails to clear would show up as stale data
-- and checks each result against the context-based entry points
(atm_compute_forces + atm_get_forces) with the tolerances of the other GPU
parity tests: counts bit-exact, FP64 forces within 1e-10, FP32C within 2e-5
relative per component (absolute floor of the same size times the RMS force).
The file is named to be collected last.
"""
import numpy as np
import pytest

from paper_2510_21230_gb300 import synth

pytestmark = pytest.mark.gpu

RTOL = {"fp64": 1e-10, "fp32c": 2e-5}


def _close(got, ref, rtol):
    scale = np.sqrt(np.mean(ref * ref))
    err = np.abs(got - ref)
    assert np.all(err <= rtol * np.abs(ref) + rtol * scale), float(err.max())


@pytest.mark.parametrize("trav,trunc,prec", [("3c08", "pair", "fp32c"), ("3c08", "product", "fp64"),
                                             ("3c18", "pair", "fp64"), ("3c01", "pair", "fp64"),
                                             ("3c08a", "pair", "fp32c")])
def test_noalloc_matches_context_entry_points_twice(trav, trunc, prec):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_21230_gb300 import atm3, build
    build.build()
    # 4^3 cells, 4^3 cells with more molecules, then 3^3 cells with fewer
    for call, (n, seed) in enumerate([(1000, 1000), (1500, 1001), (500, 1002)]):
        cfg = synth.homogeneous(n, 0.8, 1.0, seed=seed)
        with atm3.AtmSystem(cfg["box"], n) as s:
            s.set_state(cfg["x"])
            s.build_cells()
            ref = s.compute_forces(trav, trunc, prec)
            f_ref = s.get_forces("total")
        x_dev = torch.tensor(cfg["x"], dtype=torch.float64, device="cuda")
        f_dev = torch.full((3, n), float("nan"), dtype=torch.float64, device="cuda")
        got = atm3.compute_forces_noalloc(cfg["box"], x_dev, f_dev, trav, trunc, prec,
                                          stream=torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert got["n_cand3"] == ref["n_cand3"], call
        assert got["n_int3"] == ref["n_int3"], call
        assert got["n_cand2"] == ref["n_cand2"] and got["n_int2"] == ref["n_int2"], call
        for k in ("e2", "e3", "w2", "w3"):
            assert got[k] == pytest.approx(ref[k], rel=RTOL[prec]), (call, k)
        _close(f_dev.cpu().numpy(), f_ref, RTOL[prec])
        # the input positions are only read
        assert np.array_equal(x_dev.cpu().numpy(), cfg["x"])


def test_noalloc_rejects_sizes_beyond_its_array():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_21230_gb300 import atm3
    n = 32769
    x = torch.zeros((3, n), dtype=torch.float64, device="cuda")
    f = torch.zeros((3, n), dtype=torch.float64, device="cuda")
    with pytest.raises(atm3.AtmError) as ei:
        atm3.compute_forces_noalloc([60.0, 60.0, 60.0], x, f)
    assert ei.value.status == 7


def test_noalloc_empty_system_and_unsupported_modes():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_21230_gb300 import atm3, build
    build.build()
    x = torch.zeros((3, 0), dtype=torch.float64, device="cuda")
    f = torch.zeros((3, 0), dtype=torch.float64, device="cuda")
    got = atm3.compute_forces_noalloc([9.0, 9.0, 9.0], x, f, "3c08", "pair", "fp64")
    assert got["n_cand3"] == 0 and got["n_int3"] == 0 and got["n_int2"] == 0
    assert got["e2"] == 0.0 and got["e3"] == 0.0
    cfg = synth.homogeneous(1000, 0.8, 1.0, seed=1000)
    x = torch.tensor(cfg["x"], dtype=torch.float64, device="cuda")
    f = torch.zeros((3, 1000), dtype=torch.float64, device="cuda")
    for trav, prec in (("3cw", "fp64"), ("3c08", "surrogate")):
        with pytest.raises(atm3.AtmError) as ei:
            atm3.compute_forces_noalloc(cfg["box"], x, f, trav, "pair", prec)
        assert ei.value.status == 1
    # the caller's current device is unchanged
    assert torch.cuda.current_device() == 0
