"""Pins of the FP64 surrogate oracle (oracle/sur_oracle.c) against closed
forms, symmetries, library routines and finite differences -- no GPU.

The surrogate is defined in the oracle's header comment: 16 radial Gaussian
channels and 16 angular invariants of the neighbourhood r < r_c with a cosine
cutoff, 16 equivariant vectors (the four vector channels
p_a = sum_j phi_a(r) rhat and the products T_a p_b of the three quadrupole
channels with them), an MLP 32 -> 64 -> 64 -> 16 (SiLU) and
F_i = sum_m w_m v_m.
"""
import math

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")

RC = 2.5


def _prm(L):
    return oracle.params(L, RC, 0.073)


def _random_model(rng, scale=0.3):
    P = rng.normal(0.0, scale, oracle.SUR_NP)
    mean = rng.normal(0.0, 1.0, 32)
    sd = rng.uniform(0.5, 2.0, 32)
    return P, mean, sd


def _phi(r, mu, eta):
    return math.exp(-eta * (r - mu) ** 2) * 0.5 * (math.cos(math.pi * r / RC) + 1.0)


# ------------------------------------------------------------- descriptors

def test_fcut_values():
    assert oracle.sur_fcut(0.0, RC) == 1.0
    assert abs(oracle.sur_fcut(RC / 2, RC) - 0.5) < 1e-15
    assert oracle.sur_fcut(RC, RC) == 0.0
    # continuous with zero slope at the cutoff
    h = 1e-4
    assert oracle.sur_fcut(RC - h, RC) < 1e-7


def test_basis_spacing():
    mu_g, eta_g, mu_v, eta_v = oracle.sur_basis(RC)
    assert mu_g[0] == 0.8 and abs(mu_g[-1] - RC) < 1e-15
    d = np.diff(mu_g)
    assert np.allclose(d, d[0], rtol=0, atol=1e-15)
    # Gaussians of neighbouring channels cross at exp(-1/8): width = spacing
    assert abs(math.exp(-eta_g * (d[0] / 2) ** 2) - math.exp(-1.0 / 8.0)) < 1e-14
    dv = np.diff(mu_v)
    assert np.allclose(dv, (RC - 0.8) / 4, atol=1e-15)
    assert abs(math.exp(-eta_v * (dv[0] / 2) ** 2) - math.exp(-1.0 / 8.0)) < 1e-14


def test_single_neighbour_closed_form():
    # two molecules at distance r along an arbitrary unit direction
    L = 12.0
    r = 1.3
    u = np.array([1.0, 2.0, -2.0]) / 3.0
    x = np.zeros((3, 2))
    x[:, 0] = [5.0, 5.0, 5.0]
    x[:, 1] = x[:, 0] + r * u
    D, V = oracle.sur_descriptors(_prm(L), x)
    mu_g, eta_g, mu_v, eta_v = oracle.sur_basis(RC)
    G = [_phi(r, m, eta_g) for m in mu_g]
    ph = [_phi(r, m, eta_v) for m in mu_v]
    for row, sgn in ((0, 1.0), (1, -1.0)):
        assert np.allclose(D[row, :16], G, rtol=1e-13, atol=0)
        pairs = [(0, 0), (0, 1), (0, 2), (0, 3), (1, 1), (1, 2), (1, 3), (2, 2), (2, 3), (3, 3)]
        assert np.allclose(D[row, 16:26], [ph[a] * ph[b] for a, b in pairs], rtol=1e-13)
        # tr((uu^T - I/3)^2) = 1 - 2/3 + 1/3 = 2/3
        tpairs = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
        assert np.allclose(D[row, 26:], [2.0 / 3.0 * ph[a] * ph[b] for a, b in tpairs],
                           rtol=1e-13)
        for m in range(4):
            assert np.allclose(V[row, 3 * m:3 * m + 3], sgn * ph[m] * u, rtol=1e-13, atol=1e-16)
        # (uu^T - I/3) u = 2/3 u: T_a p_b = 2/3 phi_a phi_b u
        for a in range(3):
            for b in range(4):
                m = 4 + 4 * a + b
                assert np.allclose(V[row, 3 * m:3 * m + 3], sgn * 2.0 / 3.0 * ph[a] * ph[b] * u,
                                   rtol=1e-13, atol=1e-16)


def test_two_orthogonal_neighbours_quadrupole_products():
    # neighbours at r1 along u1 and r2 along u2 (u1 . u2 = 0): with
    # P_k = uk uk^T - I/3, P_1 u1 = 2/3 u1 and P_1 u2 = -u2/3, so
    # T_a p_b = phi_a(r1) (2/3 phi_b(r1) u1 - 1/3 phi_b(r2) u2)
    #         + phi_a(r2) (2/3 phi_b(r2) u2 - 1/3 phi_b(r1) u1)
    L = 12.0
    r1, r2 = 1.05, 1.9
    u1 = np.array([2.0, 1.0, 2.0]) / 3.0
    u2 = np.array([1.0, 2.0, -2.0]) / 3.0
    assert abs(u1 @ u2) < 1e-15
    x = np.zeros((3, 3))
    x[:, 0] = [5.0, 5.0, 5.0]
    x[:, 1] = x[:, 0] + r1 * u1
    x[:, 2] = x[:, 0] + r2 * u2
    _, V = oracle.sur_descriptors(_prm(L), x, rows=[0])
    _, _, mu_v, eta_v = oracle.sur_basis(RC)
    f1 = [_phi(r1, m, eta_v) for m in mu_v]
    f2 = [_phi(r2, m, eta_v) for m in mu_v]
    for b in range(4):
        assert np.allclose(V[0, 3 * b:3 * b + 3], f1[b] * u1 + f2[b] * u2, rtol=1e-13)
    for a in range(3):
        for b in range(4):
            m = 4 + 4 * a + b
            expect = (f1[a] * (2.0 / 3.0 * f1[b] * u1 - f2[b] / 3.0 * u2)
                      + f2[a] * (2.0 / 3.0 * f2[b] * u2 - f1[b] / 3.0 * u1))
            assert np.allclose(V[0, 3 * m:3 * m + 3], expect, rtol=1e-12, atol=1e-16), (a, b)


def test_beyond_cutoff_and_periodic_image():
    L = 9.0
    x = np.zeros((3, 3))
    x[:, 0] = [0.2, 4.0, 4.0]
    x[:, 1] = [L - 0.9, 4.0, 4.0]   # image distance 1.1 across the boundary
    x[:, 2] = [0.2, 4.0, 4.0 + RC]  # exactly at the cutoff: excluded
    D, V = oracle.sur_descriptors(_prm(L), x, rows=[0])
    mu_g, eta_g, mu_v, eta_v = oracle.sur_basis(RC)
    assert np.allclose(D[0, :16], [_phi(1.1, m, eta_g) for m in mu_g], rtol=1e-12)
    assert np.allclose(V[0, 0:3], [-_phi(1.1, mu_v[0], eta_v), 0, 0], rtol=1e-12, atol=1e-16)


def test_octahedral_environment_cancels_moments():
    # six neighbours on +-x, +-y, +-z: p_a = 0 and T_a = 0
    L = 12.0
    r = 1.1
    x = np.full((3, 7), 6.0)
    k = 1
    for ax in range(3):
        for s in (1.0, -1.0):
            x[ax, k] += s * r
            k += 1
    D, V = oracle.sur_descriptors(_prm(L), x, rows=[0])
    mu_g, eta_g, _, _ = oracle.sur_basis(RC)
    assert np.allclose(D[0, :16], [6 * _phi(r, m, eta_g) for m in mu_g], rtol=1e-13)
    assert np.all(np.abs(D[0, 16:]) < 1e-28)
    assert np.all(np.abs(V[0]) < 1e-15)


def test_cube_corners_cancel_quadrupole():
    # eight neighbours on the corners of a cube: sum u u^T = 8/3 I, so T_a = 0
    L = 12.0
    h = 0.7
    x = [[6.0, 6.0, 6.0]]
    for sx in (-1, 1):
        for sy in (-1, 1):
            for sz in (-1, 1):
                x.append([6 + sx * h, 6 + sy * h, 6 + sz * h])
    D, V = oracle.sur_descriptors(_prm(L), np.array(x).T, rows=[0])
    assert np.all(np.abs(D[0, 26:]) < 1e-28)
    assert np.all(np.abs(V[0]) < 1e-15)


def _cluster(rng, m=40, L=24.0):
    c = np.full(3, L / 2)
    pts = [c]
    while len(pts) < m:
        p = c + rng.uniform(-3.5, 3.5, 3)
        if np.linalg.norm(p - c) < 3.5 and min(np.linalg.norm(p - q) for q in pts) > 0.8:
            pts.append(p)
    return np.array(pts).T, c


def test_rotation_invariance_and_equivariance():
    rng = np.random.default_rng(11)
    L = 24.0
    x, c = _cluster(rng, L=L)
    D0, V0 = oracle.sur_descriptors(_prm(L), x, rows=[0])
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    xr = (q @ (x - c[:, None])) + c[:, None]
    D1, V1 = oracle.sur_descriptors(_prm(L), xr, rows=[0])
    assert np.allclose(D1, D0, rtol=1e-11, atol=1e-13)
    for m in range(16):
        assert np.allclose(V1[0, 3 * m:3 * m + 3], q @ V0[0, 3 * m:3 * m + 3], atol=1e-12)


def test_translation_and_permutation_invariance():
    rng = np.random.default_rng(12)
    L = 10.0
    x = rng.uniform(0, L, (3, 300))
    D0, V0 = oracle.sur_descriptors(_prm(L), x)
    shift = rng.uniform(-20, 20, 3)
    D1, V1 = oracle.sur_descriptors(_prm(L), x + shift[:, None])
    assert np.allclose(D1, D0, rtol=1e-9, atol=1e-11)
    assert np.allclose(V1, V0, rtol=1e-9, atol=1e-11)
    perm = rng.permutation(300)
    D2, V2 = oracle.sur_descriptors(_prm(L), x[:, perm])
    assert np.allclose(D2, D0[perm], rtol=1e-12, atol=1e-14)
    assert np.allclose(V2, V0[perm], rtol=1e-12, atol=1e-14)


def test_box_too_small_rejected():
    with pytest.raises(oracle.OracleError):
        oracle.sur_descriptors(_prm(4.0), np.zeros((3, 2)))


# --------------------------------------------------------------- bfloat16

def test_bf16_ties_and_library():
    assert oracle.bf16(1.0 + 2.0 ** -8) == 1.0            # tie -> even
    assert oracle.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2 * 2.0 ** -7  # tie -> even (up)
    assert oracle.bf16(1.0 + 3 * 2.0 ** -9) == 1.0 + 2.0 ** -7
    assert oracle.bf16(-0.0) == 0.0 and oracle.bf16(0.0) == 0.0
    rng = np.random.default_rng(3)
    v = (rng.normal(size=4000) * np.exp(rng.uniform(-20, 20, 4000))).astype(np.float32)
    ref = torch.from_numpy(v).to(torch.bfloat16).to(torch.float64).numpy()
    got = np.array([oracle.bf16(float(a)) for a in v])
    assert np.array_equal(got, ref)


# --------------------------------------------------------------------- MLP

def _torch_mlp(P, mean, sd, D, V, bf16=False):
    """The MLP written with torch layers (float64), an independent check."""
    P = torch.from_numpy(P)
    W1 = P[0:2048].reshape(32, 64)
    b1 = P[2048:2112]
    W2 = P[2112:6208].reshape(64, 64)
    b2 = P[6208:6272]
    W3 = P[6272:7296].reshape(64, 16)
    b3 = P[7296:7312]
    q = (lambda t: t.to(torch.bfloat16).to(torch.float64)) if bf16 else (lambda t: t)
    xn = q((torch.from_numpy(D) - torch.from_numpy(mean)) / torch.from_numpy(sd))
    h1 = q(torch.nn.functional.silu(xn @ q(W1) + b1))
    h2 = q(torch.nn.functional.silu(h1 @ q(W2) + b2))
    w = h2 @ q(W3) + b3
    F = torch.einsum("nm,nmc->nc", w, torch.from_numpy(V).reshape(-1, 16, 3))
    return w.numpy(), F.numpy()


def test_mlp_zero_weights_gives_bias_combination():
    rng = np.random.default_rng(4)
    P = np.zeros(oracle.SUR_NP)
    b3 = np.linspace(-1.5, 2.0, 16)
    P[7296:7312] = b3
    D = rng.normal(size=(5, 32))
    V = rng.normal(size=(5, 48))
    w, F = oracle.sur_mlp(P, np.zeros(32), np.ones(32), D, V)
    assert np.allclose(w, [b3] * 5, atol=0)
    expect = sum(b3[m] * V[:, 3 * m:3 * m + 3] for m in range(16))
    assert np.allclose(F, expect, rtol=1e-15, atol=1e-15)


def test_mlp_single_path_closed_form():
    # xn_0 = 1 -> z1_0 = 1 -> h1_0 = silu(1) = e/(1+e); W2[0][0] = 1/silu(1)
    # -> z2_0 = 1 -> h2_0 = silu(1); w = W3[0] silu(1) + b3
    s1 = math.e / (1.0 + math.e)
    P = np.zeros(oracle.SUR_NP)
    P[0 * 64 + 0] = 1.0                 # W1[0][0]
    P[2112 + 0 * 64 + 0] = 1.0 / s1     # W2[0][0]
    P[6272 + 0 * 16 + 0] = 2.0          # W3[0][0]
    P[6272 + 0 * 16 + 2] = -3.0         # W3[0][2]
    P[7296 + 1] = 0.25                  # b3[1]
    mean = np.full(32, 0.5)
    sd = np.full(32, 2.0)
    D = np.full((1, 32), 0.5)
    D[0, 0] = 2.5                       # xn_0 = (2.5 - 0.5) / 2 = 1
    V = np.arange(48, dtype=np.float64).reshape(1, 48)
    w, F = oracle.sur_mlp(P, mean, sd, D, V)
    assert np.allclose(w[0], [2.0 * s1, 0.25, -3.0 * s1] + [0.0] * 13, rtol=1e-15, atol=1e-16)


def test_mlp_matches_torch_layers():
    rng = np.random.default_rng(5)
    P, mean, sd = _random_model(rng)
    D = rng.normal(size=(64, 32)) * sd + mean
    V = rng.normal(size=(64, 48))
    w, F = oracle.sur_mlp(P, mean, sd, D, V)
    wt, Ft = _torch_mlp(P, mean, sd, D, V)
    assert np.allclose(w, wt, rtol=1e-12, atol=1e-12)
    assert np.allclose(F, Ft, rtol=1e-12, atol=1e-12)


def test_mlp_bf16_matches_torch_rounding():
    rng = np.random.default_rng(6)
    P, mean, sd = _random_model(rng)
    D = rng.normal(size=(256, 32)) * sd + mean
    V = rng.normal(size=(256, 48))
    w, F = oracle.sur_mlp(P, mean, sd, D, V, bf16_=True)
    wt, Ft = _torch_mlp(P, mean, sd, D, V, bf16=True)
    # torch rounds float64 -> bfloat16 directly as the oracle does; rows agree
    # up to summation order (a rounding flip moves one input by 2^-8 relative)
    scale = np.sqrt(np.mean(Ft ** 2))
    assert np.median(np.abs(F - Ft)) < 1e-12 * scale
    assert np.max(np.abs(F - Ft)) < 2e-2 * scale
    # and bfloat16 changes the result by about its unit roundoff, not more
    w64, F64 = oracle.sur_mlp(P, mean, sd, D, V)
    err = np.sqrt(np.mean((F - F64) ** 2)) / np.sqrt(np.mean(F64 ** 2))
    assert 1e-4 < err < 3e-2


def test_mlp_equivariance():
    rng = np.random.default_rng(7)
    P, mean, sd = _random_model(rng)
    D = rng.normal(size=(16, 32))
    V = rng.normal(size=(16, 48))
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    Vr = np.einsum("ij,nmj->nmi", q, V.reshape(16, 16, 3)).reshape(16, 48)
    _, F = oracle.sur_mlp(P, mean, sd, D, V)
    _, Fr = oracle.sur_mlp(P, mean, sd, D, Vr)
    assert np.allclose(Fr, F @ q.T, atol=1e-12)


# ------------------------------------------------------------ loss, grad

def _problem(rng, n=24):
    P, mean, sd = _random_model(rng)
    D = rng.normal(size=(n, 32)) * sd + mean
    V = rng.normal(size=(n, 48))
    Fref = rng.normal(size=(n, 3))
    return P, mean, sd, D, V, Fref


def test_loss_value_and_zero_model():
    rng = np.random.default_rng(8)
    P, mean, sd, D, V, Fref = _problem(rng)
    s2 = 0.7
    L, _ = oracle.sur_loss_grad(P, mean, sd, D, V, Fref, s2)
    _, F = oracle.sur_mlp(P, mean, sd, D, V)
    assert abs(L - np.sum((F - Fref) ** 2) / (3 * len(D) * s2)) < 1e-12 * L
    # the zero model scores exactly 1 with sigma2 = mean squared component
    _, _, sig2 = oracle.sur_stats(D, Fref)
    L0, _ = oracle.sur_loss_grad(np.zeros(oracle.SUR_NP), mean, sd, D, V, Fref, sig2)
    assert abs(L0 - 1.0) < 1e-14


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(9)
    P, mean, sd, D, V, Fref = _problem(rng)
    L, g = oracle.sur_loss_grad(P, mean, sd, D, V, Fref, 1.3)
    idx = np.concatenate([rng.choice(2048, 12, replace=False), 2048 + np.arange(4),
                          2112 + rng.choice(4096, 12, replace=False), 6208 + np.arange(4),
                          6272 + rng.choice(1024, 8, replace=False), [7296, 7301, 7311]])
    h = 1e-5
    # truncation error O(h^2), rounding error about eps L / h
    round_tol = 8 * np.finfo(float).eps * L / h
    for k in idx:
        Pp = P.copy()
        Pm = P.copy()
        Pp[k] += h
        Pm[k] -= h
        lp, _ = oracle.sur_loss_grad(Pp, mean, sd, D, V, Fref, 1.3)
        lm, _ = oracle.sur_loss_grad(Pm, mean, sd, D, V, Fref, 1.3)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * abs(g[k]) + round_tol, (k, fd, g[k])


def test_gradient_matches_torch_autograd():
    rng = np.random.default_rng(10)
    P, mean, sd, D, V, Fref = _problem(rng, n=40)
    L, g = oracle.sur_loss_grad(P, mean, sd, D, V, Fref, 0.9)
    Pt = torch.from_numpy(P.copy()).requires_grad_(True)
    W1 = Pt[0:2048].reshape(32, 64)
    W2 = Pt[2112:6208].reshape(64, 64)
    W3 = Pt[6272:7296].reshape(64, 16)
    xn = (torch.from_numpy(D) - torch.from_numpy(mean)) / torch.from_numpy(sd)
    h1 = torch.nn.functional.silu(xn @ W1 + Pt[2048:2112])
    h2 = torch.nn.functional.silu(h1 @ W2 + Pt[6208:6272])
    w = h2 @ W3 + Pt[7296:7312]
    F = torch.einsum("nm,nmc->nc", w, torch.from_numpy(V).reshape(-1, 16, 3))
    Lt = ((F - torch.from_numpy(Fref)) ** 2).sum() / (3 * len(D) * 0.9)
    Lt.backward()
    assert abs(Lt.item() - L) < 1e-12 * L
    assert np.allclose(g, Pt.grad.numpy(), rtol=1e-10, atol=1e-13)


# -------------------------------------------------------------------- Adam

def test_adam_first_step_is_signed_lr():
    rng = np.random.default_rng(13)
    P = rng.normal(size=50)
    g = rng.normal(size=50)
    m = np.zeros(50)
    v = np.zeros(50)
    P0 = P.copy()
    oracle.sur_adam(P, m, v, g, 1, 1e-3, eps=0.0)
    # m_hat = g, v_hat = g^2 after the bias correction of step 1
    assert np.allclose(P, P0 - 1e-3 * np.sign(g), rtol=0, atol=1e-15)


def test_adam_matches_torch_optimizer():
    rng = np.random.default_rng(14)
    P = rng.normal(size=40)
    m = np.zeros(40)
    v = np.zeros(40)
    pt = torch.from_numpy(P.copy()).requires_grad_(True)
    opt = torch.optim.Adam([pt], lr=2e-3, betas=(0.9, 0.999), eps=1e-8)
    for t in range(1, 6):
        g = rng.normal(size=40)
        oracle.sur_adam(P, m, v, g, t, 2e-3)
        pt.grad = torch.from_numpy(g.copy())
        opt.step()
    assert np.allclose(P, pt.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_stats_match_numpy():
    rng = np.random.default_rng(15)
    D = rng.normal(size=(500, 32)) * 3 + 1
    D[:, 5] = 2.0  # constant column
    F = rng.normal(size=(500, 3))
    mean, sd, s2 = oracle.sur_stats(D, F)
    assert np.allclose(mean, D.mean(axis=0), rtol=1e-13, atol=1e-13)
    ref = D.std(axis=0)
    ref[5] = 1.0
    assert np.allclose(sd, ref, rtol=1e-12)
    assert abs(s2 - np.mean(F ** 2)) < 1e-14
