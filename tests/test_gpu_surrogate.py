"""Learned ATM force surrogate through the C ABI against the FP64 oracle
(oracle/sur_oracle.c): descriptors, tensor-core inference, FP32 training
gradient, Adam, data-set statistics, stepping with interleaved exact steps.

Tolerances follow from the arithmetic:
 - descriptors are FP32 sums of ~50 neighbour terms from FP32 cell-local
   coordinates (~3e-7 absolute); the Gaussians amplify a position error by
   2 eta |r - mu| <= ~10, and the moment invariants cancel by up to the
   square root of the neighbour count: 1e-4 of each column's scale;
 - inference rounds its inputs, weights and hidden layers to bfloat16 as the
   oracle's bfloat16 mode does; a value within FP32 error of a bfloat16
   rounding boundary may round the other way (a 2^-8 step in one input):
   RMS 1e-3, max 1e-2 of the output scale;
 - the training gradient is FP32 on the same FP32 inputs: 1e-5 relative (norm).
"""
import os

import numpy as np
import pytest

import oracle
from paper_2510_21230_gb300 import synth

pytestmark = pytest.mark.gpu

NU, RC = 0.073, 2.5


@pytest.fixture(scope="module")
def atm3():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_21230_gb300 import atm3 as m, build
    build.build()
    return m


@pytest.fixture(scope="module")
def liquid():
    return synth.config("liquid_n1000")


@pytest.fixture(scope="module")
def liquid_desc(liquid):
    prm = oracle.params(liquid["box"], RC, NU)
    return oracle.sur_descriptors(prm, liquid["x"])


def _colscale(a):
    return np.maximum(np.abs(a).max(axis=0), 1e-30)


def _model_for(D, seed=7):
    """Random weights with the oracle's statistics of the given descriptors."""
    mean, scale, _ = oracle.sur_stats(D, np.zeros((len(D), 3)))
    return synth.sur_params(seed), mean.astype(np.float32), scale.astype(np.float32)


# ---------------------------------------------------------------- descriptors

def test_descriptors_match_oracle(atm3, liquid, liquid_desc):
    Do, Vo = liquid_desc
    with atm3.AtmSystem(liquid["box"], 1000, rc=RC, nu=NU) as s:
        s.set_state(liquid["x"])
        s.build_cells()
        D, V = s.surrogate_descriptors()
    assert np.all(np.abs(D - Do) <= 1e-4 * _colscale(Do)), np.abs(D - Do).max(axis=0) / _colscale(Do)
    assert np.all(np.abs(V - Vo) <= 1e-4 * _colscale(Vo))


@pytest.mark.parametrize("workload", ["liquid_n32k", "liquid_n256k"])
def test_descriptors_sampled_rows(atm3, workload):
    """400 sampled rows of the 32,000- and the 256,000-molecule liquids (the
    size the benchmark's surrogate runs) against the oracle's descriptors."""
    cfg = synth.config(workload)
    prm = oracle.params(cfg["box"], RC, NU)
    rows = np.random.default_rng(5).choice(cfg["n"], 400, replace=False)
    Do, Vo = oracle.sur_descriptors(prm, cfg["x"], rows)
    with atm3.AtmSystem(cfg["box"], cfg["n"], rc=RC, nu=NU) as s:
        s.set_state(cfg["x"])
        s.build_cells()
        D, V = s.surrogate_descriptors()
    assert np.all(np.abs(D[rows] - Do) <= 1e-4 * _colscale(Do))
    assert np.all(np.abs(V[rows] - Vo) <= 1e-4 * _colscale(Vo))


def test_descriptors_isolated_pair_and_empty(atm3):
    box = 9.0
    x = np.array([[1.0, 2.3], [1.0, 1.0], [1.0, 1.0]])  # distance 1.3 along x
    prm = oracle.params(box, RC, NU)
    Do, Vo = oracle.sur_descriptors(prm, x)
    with atm3.AtmSystem(box, 2, rc=RC, nu=NU) as s:
        s.set_state(x)
        s.build_cells()
        D, V = s.surrogate_descriptors()
    assert np.allclose(D, Do, rtol=2e-5, atol=1e-12)
    assert np.allclose(V, Vo, rtol=2e-5, atol=1e-12)
    with atm3.AtmSystem(box, 0, rc=RC, nu=NU) as s:
        s.set_state(np.zeros((3, 0)))
        s.build_cells()
        D, V = s.surrogate_descriptors()
        assert D.shape == (0, 32)


# ------------------------------------------------------------------ inference

@pytest.mark.parametrize("rows", [1, 127, 1000, 4099])
def test_mlp_rows_match_oracle_bf16(atm3, rows):
    P = synth.sur_params(11)
    mean = np.linspace(-1, 1, 32).astype(np.float32)
    scale = np.linspace(0.5, 2.0, 32).astype(np.float32)
    D, V, _ = synth.sur_rows(rows, 12, mean, scale)
    with atm3.AtmSystem(10.0, 1, rc=RC, nu=NU) as s:
        s.surrogate_set_model(P, mean, scale)
        w, F = s.surrogate_mlp(D, V)
    wo, Fo = oracle.sur_mlp(P.astype(np.float64), mean, scale, D, V, bf16_=True)
    sw = np.sqrt(np.mean(wo ** 2))
    assert np.sqrt(np.mean((w - wo) ** 2)) <= 1e-3 * sw
    assert np.max(np.abs(w - wo)) <= 1e-2 * max(sw, np.abs(wo).max())
    sf = np.sqrt(np.mean(Fo ** 2))
    assert np.sqrt(np.mean((F - Fo) ** 2)) <= 1e-3 * sf
    # and within the bfloat16 error of the exact FP64 model
    w64, _ = oracle.sur_mlp(P.astype(np.float64), mean, scale, D, V)
    assert np.sqrt(np.mean((w - w64) ** 2)) <= 3e-2 * np.sqrt(np.mean(w64 ** 2))


def test_surrogate_forces_match_oracle(atm3, liquid, liquid_desc):
    Do, Vo = liquid_desc
    P, mean, scale = _model_for(Do)
    _, Fo = oracle.sur_mlp(P.astype(np.float64), mean, scale, Do, Vo, bf16_=True)
    with atm3.AtmSystem(liquid["box"], 1000, rc=RC, nu=NU) as s:
        s.set_state(liquid["x"])
        s.surrogate_set_model(P, mean, scale)
        s.build_cells()
        s.compute_forces("3c08", "pair", "surrogate")
        res = s.results()[0]
        F = s.get_forces("atm").T
        lj = s.get_forces("lj")
    sf = np.sqrt(np.mean(Fo ** 2))
    assert np.sqrt(np.mean((F - Fo) ** 2)) <= 3e-3 * sf
    assert np.max(np.abs(F - Fo)) <= 3e-2 * max(sf, np.abs(Fo).max())
    assert res["e3"] == 0.0 and res["w3"] == 0.0 and res["n_int3"] == 0 and res["n_cand3"] == 0
    # LJ still runs (FP32 path)
    ref = oracle.lj_cells(oracle.params(liquid["box"], RC, NU), liquid["x"], "fp32")
    assert np.allclose(lj, ref["f"], rtol=2e-5, atol=2e-5 * np.sqrt(np.mean(ref["f"] ** 2)))


def test_surrogate_needs_model(atm3, liquid):
    with atm3.AtmSystem(liquid["box"], 1000, rc=RC, nu=NU) as s:
        s.set_state(liquid["x"])
        s.build_cells()
        with pytest.raises(atm3.AtmError) as e:
            s.compute_forces("3c08", "pair", "surrogate")
        assert e.value.status == 6


def test_batch_surrogate_equals_separate(atm3):
    reps = synth.replicas(count=3, n_lo=600, n_hi=2000)
    x = np.ascontiguousarray(np.concatenate([r["x"] for r in reps], axis=1))
    prm0 = oracle.params(reps[0]["box"], RC, NU)
    D0, _ = oracle.sur_descriptors(prm0, reps[0]["x"])
    P, mean, scale = _model_for(D0)
    with atm3.AtmSystem([r["box"] for r in reps], [r["n"] for r in reps], rc=RC, nu=NU) as b:
        b.set_state(x)
        b.surrogate_set_model(P, mean, scale)
        b.build_cells()
        b.compute_forces("3c08", "pair", "surrogate")
        fb = b.get_forces("atm")
    off = 0
    for r in reps:
        with atm3.AtmSystem(r["box"], r["n"], rc=RC, nu=NU) as s:
            s.set_state(r["x"])
            s.surrogate_set_model(P, mean, scale)
            s.build_cells()
            s.compute_forces("3c08", "pair", "surrogate")
            f = s.get_forces("atm")
        assert np.array_equal(fb[:, off:off + r["n"]], f)
        off += r["n"]


# ------------------------------------------------------------------- training

# parameter blocks of the flat parameter vector: W1, b1, W2, b2, W3, b3
BLOCKS = [(0, 2048), (2048, 2112), (2112, 6208), (6208, 6272), (6272, 7296), (7296, 7312)]


@pytest.mark.parametrize("rows", [64, 300, 2049])
def test_loss_grad_matches_oracle_fp32(atm3, rows):
    """FP32 gradients on the CUDA cores against the FP64 oracle (1e-5)."""
    P = synth.sur_params(21)
    mean = np.linspace(-0.5, 0.5, 32).astype(np.float32)
    scale = np.linspace(0.7, 1.5, 32).astype(np.float32)
    D, V, T = synth.sur_rows(rows, 22, mean, scale)
    s2 = 0.37
    with atm3.AtmSystem(10.0, 1, rc=RC, nu=NU) as s:
        s.surrogate_set_model(P, mean, scale)
        s.surrogate_training_arithmetic(tensor_cores=False)
        L, g = s.surrogate_loss_grad(D, V, T, s2)
    Lo, go = oracle.sur_loss_grad(P.astype(np.float64), mean, scale, D, V, T, s2)
    assert abs(L - Lo) <= 1e-5 * Lo
    assert np.linalg.norm(g - go) <= 1e-5 * np.linalg.norm(go)
    assert np.max(np.abs(g - go)) <= 1e-5 * np.abs(go).max()


@pytest.mark.parametrize("rows", [64, 300, 2049, 8192])
def test_loss_grad_tensor_cores_matches_oracle(atm3, rows):
    """Gradients on the tensor cores (bfloat16 operands, FP32 sums; ragged last
    tile for 300 and 2049 rows) against the FP64 oracle's backward pass.
    bfloat16 keeps 8 significant bits (unit roundoff 2^-9 = 3.9e-3); every
    gradient term is a product of two rounded operands whose own inputs were
    rounded in the forward pass, a few times 2^-9 per term, and the sums over
    the samples average the roundings, so each parameter block must agree to
    1e-2 of its norm (elementwise to 3e-2 of the block's largest entry).  The
    loss follows the same bfloat16 forward pass as the inference kernel, so it
    is checked against the oracle's bfloat16 emulation of that pass (1e-3)."""
    P = synth.sur_params(21)
    mean = np.linspace(-0.5, 0.5, 32).astype(np.float32)
    scale = np.linspace(0.7, 1.5, 32).astype(np.float32)
    D, V, T = synth.sur_rows(rows, 22, mean, scale)
    s2 = 0.37
    with atm3.AtmSystem(10.0, 1, rc=RC, nu=NU) as s:
        s.surrogate_set_model(P, mean, scale)
        L, g = s.surrogate_loss_grad(D, V, T, s2)
    _, go = oracle.sur_loss_grad(P.astype(np.float64), mean, scale, D, V, T, s2)
    _, Fb = oracle.sur_mlp(P.astype(np.float64), mean, scale, D, V, bf16_=True)
    Lb = float(np.sum((Fb - T.astype(np.float64).reshape(-1, 3)) ** 2) / (3 * rows * s2))
    assert abs(L - Lb) <= 1e-3 * Lb, (L, Lb)
    for a, b in BLOCKS:
        d = g[a:b] - go[a:b]
        assert np.linalg.norm(d) <= 1e-2 * np.linalg.norm(go[a:b]), (a, b, np.linalg.norm(d) / np.linalg.norm(go[a:b]))
        assert np.abs(d).max() <= 3e-2 * np.abs(go[a:b]).max(), (a, b)


def test_tensor_core_and_fp32_training_agree(atm3):
    """Fifty Adam steps from the same start with either gradient arithmetic
    reach losses within 2 % of each other on teacher targets."""
    mean = np.zeros(32, dtype=np.float32)
    scale = np.ones(32, dtype=np.float32)
    D, V, _ = synth.sur_rows(4096, 51, mean, scale)
    teacher = synth.sur_params(52, wscale=0.2)
    _, T = oracle.sur_mlp(teacher.astype(np.float64), mean, scale, D, V)
    out = {}
    for tc in (True, False):
        with atm3.AtmSystem(10.0, 1, rc=RC, nu=NU) as s:
            s.surrogate_set_model(synth.sur_params(53, wscale=0.05), mean, scale)
            s.surrogate_training_arithmetic(tensor_cores=tc)
            s.surrogate_add_rows(D, V, T.astype(np.float32))
            out[tc] = s.surrogate_train(50, batch=1024, lr=2e-3, seed=3)
    assert np.all(np.isfinite(out[True]))
    assert out[True][-1] < 0.9 * out[True][0]
    assert abs(out[True][-1] - out[False][-1]) <= 2e-2 * out[False][-1]


def test_adam_step_matches_oracle(atm3):
    P = synth.sur_params(31)
    mean = np.zeros(32, dtype=np.float32)
    scale = np.ones(32, dtype=np.float32)
    D, V, T = synth.sur_rows(500, 32, mean, scale)
    lr = 1e-3
    with atm3.AtmSystem(10.0, 1, rc=RC, nu=NU) as s:
        s.surrogate_set_model(P, mean, scale)
        s.surrogate_training_arithmetic(tensor_cores=False)  # pins Adam on the exact gradient
        s.surrogate_add_rows(D, V, T)
        rows, s2 = s.surrogate_dataset()
        loss = s.surrogate_train(1, batch=0, lr=lr)
        P1, _, _ = s.surrogate_get_model()
    assert rows == 500
    _, _, s2o = oracle.sur_stats(D, T)
    assert abs(s2 - s2o) <= 1e-12 * s2o
    Lo, go = oracle.sur_loss_grad(P.astype(np.float64), mean, scale, D, V, T, s2o)
    assert abs(loss[0] - Lo) <= 1e-5 * Lo
    Po = P.astype(np.float64)
    oracle.sur_adam(Po, np.zeros_like(Po), np.zeros_like(Po), go, 1, lr)
    # step 1 moves each weight by lr sign(g): compare where g is not at FP32 noise
    big = np.abs(go) > 1e-4 * np.abs(go).max()
    assert big.mean() > 0.9
    assert np.all(np.abs(P1[big] - Po[big]) <= 1e-3 * lr + 1e-7 * np.abs(Po[big]))


def test_training_reduces_loss_on_teacher_targets(atm3):
    # targets from a teacher model of the same form: the student can fit them
    mean = np.zeros(32, dtype=np.float32)
    scale = np.ones(32, dtype=np.float32)
    D, V, _ = synth.sur_rows(4096, 41, mean, scale)
    teacher = synth.sur_params(42, wscale=0.2)
    _, T = oracle.sur_mlp(teacher.astype(np.float64), mean, scale, D, V)
    with atm3.AtmSystem(10.0, 1, rc=RC, nu=NU) as s:
        s.surrogate_set_model(synth.sur_params(43, wscale=0.05), mean, scale)
        s.surrogate_add_rows(D, V, T.astype(np.float32))
        loss = s.surrogate_train(300, batch=512, lr=3e-3, seed=1)
    assert np.all(np.isfinite(loss))
    assert loss[-20:].mean() < 0.5 * loss[:5].mean()


def test_frames_init_stats_match_oracle(atm3, liquid, liquid_desc):
    Do, _ = liquid_desc
    prm = oracle.params(liquid["box"], RC, NU)
    Fo = oracle.atm_cells(prm, liquid["x"], "3c18", "pair", "fp64")["f"].T
    mean_o, scale_o, s2o = oracle.sur_stats(Do, Fo)
    with atm3.AtmSystem(liquid["box"], 1000, rc=RC, nu=NU) as s:
        s.set_state(liquid["x"])
        s.build_cells()
        s.surrogate_add_frame("3c18", "pair", "fp64")
        rows, s2 = s.surrogate_dataset()
        s.surrogate_init(seed=3)
        P, mean, scale = s.surrogate_get_model()
    assert rows == 1000
    assert abs(s2 - s2o) <= 1e-6 * s2o
    assert np.all(np.abs(mean - mean_o) <= 1e-4 * _colscale(Do))
    assert np.allclose(scale, scale_o, rtol=1e-3)
    assert np.all(np.isfinite(P)) and np.abs(P).max() <= np.sqrt(6.0 / 96.0) + 1e-6


def test_save_load_roundtrip(atm3, tmp_path):
    P = synth.sur_params(51)
    mean = np.arange(32, dtype=np.float32)
    scale = np.full(32, 2.0, dtype=np.float32)
    path = os.path.join(str(tmp_path), "model.bin")
    with atm3.AtmSystem(10.0, 1, rc=RC, nu=NU) as s:
        s.surrogate_set_model(P, mean, scale)
        s.surrogate_save(path)
    with atm3.AtmSystem(10.0, 1, rc=RC, nu=NU) as s:
        s.surrogate_load(path)
        P2, m2, s2 = s.surrogate_get_model()
        assert np.array_equal(P2, P) and np.array_equal(m2, mean) and np.array_equal(s2, scale)
        bad = os.path.join(str(tmp_path), "bad.bin")
        with open(bad, "wb") as f:
            f.write(b"not a model")
        with pytest.raises(atm3.AtmError):
            s.surrogate_load(bad)
        with pytest.raises(atm3.AtmError):
            s.surrogate_set_model(P, mean, np.zeros(32, dtype=np.float32))


# -------------------------------------------------------------------- stepping

def test_surrogate_steps_with_exact_checks(atm3, liquid, liquid_desc):
    Do, _ = liquid_desc
    P, mean, scale = _model_for(Do)
    with atm3.AtmSystem(liquid["box"], 1000, rc=RC, nu=NU, dt=0.002) as s:
        s.set_state(liquid["x"], liquid["v"])
        s.surrogate_set_model(P, mean, scale)
        s.surrogate_options(exact_every=5)
        res = s.step(10, "3c08", "pair", "surrogate")
        d, e, k = s.surrogate_error()
        x1, v1 = s.get_state()
    assert k == 2
    assert e > 0 and np.isfinite(d)
    assert np.all(np.isfinite(x1)) and np.isfinite(res["ekin"])


def test_surrogate_graph_steps_equal_plain(atm3, liquid, liquid_desc):
    Do, _ = liquid_desc
    P, mean, scale = _model_for(Do)
    out = []
    for graph in (False, True):
        with atm3.AtmSystem(liquid["box"], 1000, rc=RC, nu=NU, dt=0.002) as s:
            s.set_state(liquid["x"], liquid["v"])
            s.surrogate_set_model(P, mean, scale)
            s.surrogate_options(exact_every=0)
            s.set_options(graph=graph)
            s.step(6, "3c08", "pair", "surrogate")
            out.append(s.get_state())
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_surrogate_lj_equals_fp32_lj_kernel(atm3, liquid, liquid_desc):
    # the surrogate's neighbour pass computes LJ with the FP32 LJ kernel's
    # decisions and arithmetic: same counts, same forces up to FMA contraction
    Do, _ = liquid_desc
    P, mean, scale = _model_for(Do)
    with atm3.AtmSystem(liquid["box"], 1000, rc=RC, nu=NU) as s:
        s.set_state(liquid["x"])
        s.surrogate_set_model(P, mean, scale)
        s.build_cells()
        s.compute_forces("3c08", "pair", "fp32c")
        r1 = s.results()[0]
        f1 = s.get_forces("lj")
        s.compute_forces("3c08", "pair", "surrogate")
        r2 = s.results()[0]
        f2 = s.get_forces("lj")
    assert r2["n_int2"] == r1["n_int2"] and r2["n_cand2"] == r1["n_cand2"]
    assert abs(r2["e2"] - r1["e2"]) <= 1e-6 * abs(r1["e2"])
    assert abs(r2["w2"] - r1["w2"]) <= 1e-6 * abs(r1["w2"])
    sc = np.sqrt(np.mean(f1 ** 2))
    assert np.max(np.abs(f2 - f1)) <= 1e-6 * sc


def test_trained_surrogate_gains_over_the_method_without_it(atm3):
    """What the learned part adds: trained on the GPU (forward and backward
    kernels, Adam) on exact FP32C ATM forces of 60 frames of the N = 1000
    liquid, the surrogate reproduces the exact FP64 ATM force of a state it
    never saw far better than leaving the three-body force out (relative RMS
    error 1) and than the untrained network, and the surrogate evaluation runs
    faster than the exact FP64 traversal of the same state."""
    import torch
    cfg = synth.config("liquid_n1000")
    stream = torch.cuda.current_stream()
    with atm3.AtmSystem(cfg["box"], cfg["n"], rc=RC, nu=NU, dt=0.002,
                        stream=stream.cuda_stream) as s:
        s.set_state(cfg["x"], cfg["v"])
        for _ in range(60):
            s.step(10, "3c08", "pair", "fp32c")
            s.surrogate_add_frame("3c08", "pair", "fp32c")
        s.surrogate_init(seed=1)
        s.step(100, "3c08", "pair", "fp32c")   # a state outside the training frames
        s.build_cells()
        s.compute_forces("3c08", "pair", "fp64")
        f_exact = s.get_forces("atm")
        s.compute_forces("3c08", "pair", "surrogate")
        f_untrained = s.get_forces("atm")
        s.surrogate_train(1500, batch=4096, lr=2e-3, seed=2)
        s.surrogate_train(1500, batch=4096, lr=5e-4, seed=3)
        s.compute_forces("3c08", "pair", "surrogate")
        f_trained = s.get_forces("atm")

        def ms_per_eval(prec, reps=5):
            s.compute_forces("3c08", "pair", prec)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                s.compute_forces("3c08", "pair", prec, sync=False)
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / reps

        t_exact = ms_per_eval("fp64")
        t_sur = ms_per_eval("surrogate")

    def err(f):
        return np.sqrt(np.mean((f - f_exact) ** 2)) / np.sqrt(np.mean(f_exact ** 2))

    e_tr, e_un = err(f_trained), err(f_untrained)
    assert e_tr < 0.25, e_tr                # without the surrogate (no ATM force): error 1.0; measured 0.158
    assert e_tr < 0.7 * e_un, (e_tr, e_un)  # training is what brings it there
    assert t_sur < t_exact, (t_sur, t_exact)
