"""Pins of the CPU oracle against facts the paper and mathematics fix.

Each test checks the oracle against something other than itself: closed-form
energies of Eq. atm, the paper's separately printed gradient (Eq. ATMGradient),
finite differences, the Euler identity of a degree -9 homogeneous potential,
Newton's third law (Eq. newton3rdlaw), the counting identities of section 3,
invariances, and brute force against linked cells.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
from paper_2510_21230_gb300 import synth

NU = 0.073
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append([float(t) for t in line.split()])
    return np.array(rows)


# ---------------------------------------------------------------- potential

def test_equilateral_and_collinear_closed_forms():
    """Eq. atm: equilateral side r gives 11 nu / (8 r^9); collinear r, r, 2r gives -nu / (4 r^9)."""
    g = _read_golden("atm_closed_forms.txt")
    for nu, r, e_eq, e_col in g:
        u_eq = oracle.atm_u(r * r, r * r, r * r, nu)
        u_col = oracle.atm_u(r * r, 4 * r * r, r * r, nu)  # i--j = r, i--k = 2r, j--k = r
        assert u_eq == pytest.approx(e_eq, rel=4e-16 * 8)
        assert u_col == pytest.approx(e_col, rel=4e-16 * 64)
        assert u_eq == pytest.approx(11 * nu / (8 * r ** 9), rel=1e-14)
        assert u_col == pytest.approx(-nu / (4 * r ** 9), rel=1e-13)


def test_energy_symmetric_in_sides():
    rng = np.random.default_rng(1)
    for _ in range(200):
        p = rng.normal(size=(3, 3))
        a = np.sum((p[0] - p[1]) ** 2)
        b = np.sum((p[0] - p[2]) ** 2)
        c = np.sum((p[1] - p[2]) ** 2)
        vals = [oracle.atm_u(*perm, NU) for perm in itertools.permutations((a, b, c))]
        assert np.allclose(vals, vals[0], rtol=1e-13, atol=0)


def test_gradient_matches_paper_eleven_term_form():
    """2 r_ij du/da equals du/dr_ij of Eq. ATMGradient; the other sides by cycling i, j, k."""
    rng = np.random.default_rng(2)
    for _ in range(300):
        p = rng.uniform(0, 2.5, size=(3, 3))
        rij = np.linalg.norm(p[0] - p[1])
        rik = np.linalg.norm(p[0] - p[2])
        rjk = np.linalg.norm(p[1] - p[2])
        if min(rij, rik, rjk) < 0.7:
            continue
        du = oracle.atm_du_dsq(rij * rij, rik * rik, rjk * rjk, NU)
        assert 2 * rij * du[0] == pytest.approx(oracle.atm_dudr_paper(rij, rik, rjk, NU), rel=1e-11)
        # du/dr_ik: r_ik plays the role of r_ij, with (r_ij, r_jk) as the other two
        assert 2 * rik * du[1] == pytest.approx(oracle.atm_dudr_paper(rik, rij, rjk, NU), rel=1e-11)
        assert 2 * rjk * du[2] == pytest.approx(oracle.atm_dudr_paper(rjk, rij, rik, NU), rel=1e-11)


def test_gradient_by_finite_differences_of_side_squares():
    a, b, c = 1.21, 1.69, 2.89
    du = oracle.atm_du_dsq(a, b, c, NU)
    h = 1e-6
    fd = [(oracle.atm_u(a + h, b, c, NU) - oracle.atm_u(a - h, b, c, NU)) / (2 * h),
          (oracle.atm_u(a, b + h, c, NU) - oracle.atm_u(a, b - h, c, NU)) / (2 * h),
          (oracle.atm_u(a, b, c + h, NU) - oracle.atm_u(a, b, c - h, NU)) / (2 * h)]
    assert np.allclose(du, fd, rtol=1e-7)


# ---------------------------------------------------------------- small systems

def _small_fluid(n=60, rho=0.5, seed=7, rc=2.5):
    rng = np.random.default_rng(seed)
    box = (n / rho) ** (1 / 3)
    box = max(box, 3 * rc + 0.1)
    x = synth.random_sequential(n, [0, 0, 0], [box] * 3, 0.9, rng, box=np.array([box] * 3))
    return np.ascontiguousarray(x.T), box


def _prm(box, rc=2.5, nu=NU, shift=False):
    return oracle.params(box, rc, nu, lj_shift=shift)


@pytest.mark.parametrize("trunc", ["pair", "product"])
def test_forces_are_minus_energy_gradient(trunc):
    """Central finite differences of the brute-force E3 reproduce its forces (F = -grad u)."""
    x, box = _small_fluid(n=40, rho=0.3, seed=11)
    prm = _prm(box)
    ref = oracle.atm_brute(prm, x, trunc)
    assert ref["n_int3"] > 20
    h = 1e-6
    rng = np.random.default_rng(3)
    for _ in range(12):
        d, i = rng.integers(3), rng.integers(x.shape[1])
        xp = x.copy(); xp[d, i] += h
        xm = x.copy(); xm[d, i] -= h
        ep = oracle.atm_brute(prm, xp, trunc)["e3"]
        em = oracle.atm_brute(prm, xm, trunc)["e3"]
        fd = -(ep - em) / (2 * h)
        scale = np.abs(ref["f"]).max()
        assert abs(fd - ref["f"][d, i]) < 1e-6 * scale + 1e-7 * abs(fd)


def test_lj_forces_are_minus_energy_gradient():
    x, box = _small_fluid(n=40, rho=0.3, seed=12)
    prm = _prm(box)
    ref = oracle.lj_brute(prm, x)
    h = 1e-6
    for d, i in [(0, 3), (1, 17), (2, 29)]:
        xp = x.copy(); xp[d, i] += h
        xm = x.copy(); xm[d, i] -= h
        fd = -(oracle.lj_brute(prm, xp)["e2"] - oracle.lj_brute(prm, xm)["e2"]) / (2 * h)
        assert fd == pytest.approx(ref["f"][d, i], rel=1e-6, abs=1e-7)


def test_lj_closed_form_minimum():
    """At r = 2^(1/6) sigma the LJ pair energy is -eps and the force vanishes."""
    r = 2 ** (1 / 6)
    box = 10.0
    x = np.array([[1.0, 1.0 + r], [2.0, 2.0], [3.0, 3.0]])
    out = oracle.lj_brute(_prm(box), x)
    assert out["e2"] == pytest.approx(-1.0, rel=1e-14)
    assert np.abs(out["f"]).max() < 1e-13
    x1 = np.array([[1.0, 2.0], [2.0, 2.0], [3.0, 3.0]])
    assert oracle.lj_brute(_prm(box), x1)["e2"] == pytest.approx(0.0, abs=1e-14)


@pytest.mark.parametrize("trunc", ["pair", "product"])
def test_virial_is_nine_times_energy(trunc):
    """u is homogeneous of degree -9 in lengths, so r . grad u = -9 u and W3 = 9 E3."""
    x, box = _small_fluid(n=80, rho=0.5, seed=13)
    prm = _prm(box)
    for trav in ["3c01", "3c18", "3c08"]:
        out = oracle.atm_cells(prm, x, trav, trunc)
        assert out["w3"] == pytest.approx(9 * out["e3"], rel=1e-12)
    bf = oracle.atm_brute(prm, x, trunc)
    assert bf["w3"] == pytest.approx(9 * bf["e3"], rel=1e-12)


@pytest.mark.parametrize("trav", ["3c18", "3c08"])
@pytest.mark.parametrize("trunc", ["pair", "product"])
def test_net_force_vanishes_with_newton3(trav, trunc):
    x, box = _small_fluid(n=80, rho=0.5, seed=14)
    out = oracle.atm_cells(_prm(box), x, trav, trunc)
    scale = np.abs(out["f"]).max()
    assert np.abs(out["f"].sum(axis=1)).max() < 1e-12 * scale * x.shape[1]


def test_permutation_invariance():
    x, box = _small_fluid(n=70, rho=0.5, seed=15)
    prm = _prm(box)
    rng = np.random.default_rng(4)
    p = rng.permutation(x.shape[1])
    for trav in ["3c01", "3c18", "3c08"]:
        a = oracle.atm_cells(prm, x, trav, "pair")
        b = oracle.atm_cells(prm, x[:, p], trav, "pair")
        assert a["n_int3"] == b["n_int3"] and a["n_cand3"] == b["n_cand3"]
        assert b["e3"] == pytest.approx(a["e3"], rel=1e-12)
        assert np.allclose(b["f"], a["f"][:, p], rtol=1e-10, atol=1e-13)


def test_translation_invariance_pair_rule():
    x, box = _small_fluid(n=70, rho=0.5, seed=16)
    prm = _prm(box)
    shift = np.array([[0.37], [-1.91], [4.4]])
    for trav in ["3c01", "3c18", "3c08"]:
        a = oracle.atm_cells(prm, x, trav, "pair")
        b = oracle.atm_cells(prm, x + shift, trav, "pair")
        assert a["n_int3"] == b["n_int3"]
        assert b["e3"] == pytest.approx(a["e3"], rel=1e-10)
        assert np.allclose(b["f"], a["f"], rtol=1e-8, atol=1e-11)


def test_periodic_image_shift_changes_nothing():
    x, box = _small_fluid(n=70, rho=0.5, seed=17)
    prm = _prm(box)
    img = x.copy()
    img[:, ::3] += box * np.array([[1.0], [-2.0], [3.0]])
    a = oracle.atm_brute(prm, x, "pair")
    b = oracle.atm_brute(prm, img, "pair")
    assert a["n_int3"] == b["n_int3"]
    assert b["e3"] == pytest.approx(a["e3"], rel=1e-12)


# ---------------------------------------------------------------- brute force vs cells

@pytest.mark.parametrize("ncell_target", [3, 4, 5])
@pytest.mark.parametrize("seed", [21, 22])
def test_brute_force_equals_every_traversal_pair_rule(ncell_target, seed):
    """Pair rule: every traversal finds exactly the interacting triplets of the
    O(N^3) minimum-image brute force (cell edge >= r_c, >= 3 cells per axis)."""
    rc = 2.5
    box = ncell_target * rc + 0.3
    rng = np.random.default_rng(seed)
    n = int(0.35 * box ** 3)
    x = synth.random_sequential(n, [0, 0, 0], [box] * 3, 0.85, rng, box=np.array([box] * 3)).T
    x = np.ascontiguousarray(x)
    prm = _prm(box, rc)
    bf = oracle.atm_brute(prm, x, "pair")
    assert bf["n_int3"] > 100
    for trav in ["3c18", "3c08"]:
        lc = oracle.atm_cells(prm, x, trav, "pair")
        assert lc["n_int3"] == bf["n_int3"], trav
        assert lc["e3"] == pytest.approx(bf["e3"], rel=1e-11)
        assert np.allclose(lc["f"], bf["f"], rtol=1e-9, atol=1e-12)
    # 3c01 visits each triplet once per owner and adds u/3 per visit
    lc = oracle.atm_cells(prm, x, "3c01", "pair")
    assert lc["n_int3"] == 3 * bf["n_int3"]
    assert lc["e3"] == pytest.approx(bf["e3"], rel=1e-11)
    assert np.allclose(lc["f"], bf["f"], rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("trav", ["3c01", "3c18", "3c08", "3c08a"])
def test_brute_force_with_membership_equals_cells_product_rule(trav):
    """Product rule: the brute force restricted to the cell triples a traversal
    visits equals the linked-cell traversal (box of 6 cells per axis, so the
    base-frame displacement of every visited pair is its minimum image)."""
    rc = 1.0
    box = 6.4
    rng = np.random.default_rng(31)
    x = np.ascontiguousarray(
        synth.random_sequential(240, [0, 0, 0], [box] * 3, 0.45, rng, box=np.array([box] * 3)).T)
    prm = _prm(box, rc)
    bf = oracle.atm_brute(prm, x, "product", member=trav)
    lc = oracle.atm_cells(prm, x, trav, "product")
    assert lc["n_int3"] == bf["n_int3"]
    assert lc["e3"] == pytest.approx(bf["e3"], rel=1e-11)
    assert np.allclose(lc["f"], bf["f"], rtol=1e-9, atol=1e-12)


def test_pair_cutoff_is_subset_of_product_and_traversal_order():
    """Pair-rule triplets are product-rule triplets; product triplets found:
    3c01 >= 3c18 >= 3c08 (section 4)."""
    x, box = _small_fluid(n=300, rho=0.6, seed=18, rc=2.5)
    prm = _prm(box)
    full = oracle.atm_brute(prm, x, "product")
    got = {}
    for trav in ["3c01", "3c18", "3c08"]:
        pr = oracle.atm_cells(prm, x, trav, "pair")
        pd = oracle.atm_cells(prm, x, trav, "product")
        assert pr["n_int3"] <= pd["n_int3"]
        got[trav] = pd["n_int3"]
    assert got["3c18"] >= got["3c08"]
    assert got["3c01"] >= got["3c18"]
    assert full["n_int3"] >= got["3c18"]


# ---------------------------------------------------------------- counting identities

def _counts_per_cell(cells):
    st = cells["cell_start"]
    return np.diff(st).astype(np.int64)


def _comb2(n):
    return n * (n - 1) // 2


def _comb3(n):
    return n * (n - 1) * (n - 2) // 6


def test_candidate_counts_follow_cell_identities():
    """Candidate triplets of each traversal equal the sums of Eq. celltriplet,
    Eq. twoonetriplets and Eq. carttriplets over the tasks it visits."""
    x, box = _small_fluid(n=200, rho=0.5, seed=19)
    prm = _prm(box)
    cells = oracle.build_cells(prm, x)
    nc = cells["ncell"]
    cnt = _counts_per_cell(cells).reshape(nc[2], nc[1], nc[0])

    def N(z, y, xx):
        return int(cnt[z % nc[2], y % nc[1], xx % nc[0]])

    fwd = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
           if (dz, dy, dx) > (0, 0, 0)]
    t18 = t08 = t01 = t08a = 0
    for z in range(nc[2]):
        for y in range(nc[1]):
            for xx in range(nc[0]):
                nb = N(z, y, xx)
                t18 += _comb3(nb)
                for (dx, dy, dz) in fwd:
                    nn = N(z + dz, y + dy, xx + dx)
                    t18 += nn * _comb2(nb) + nb * _comb2(nn)
                for p, q in itertools.combinations(fwd, 2):
                    t18 += nb * N(z + p[2], y + p[1], xx + p[0]) * N(z + q[2], y + q[1], xx + q[0])
                # 3c08 block
                sl = [N(z + (s >> 2 & 1), y + (s >> 1 & 1), xx + (s & 1)) for s in range(8)]
                t08 += _comb3(sl[0])
                for s, t in itertools.combinations(range(8), 2):
                    if s & t == 0:
                        t08 += sl[t] * _comb2(sl[s]) + sl[s] * _comb2(sl[t])
                for s, t, u in itertools.combinations(range(8), 3):
                    if s & t & u == 0:
                        t08 += sl[s] * sl[t] * sl[u]
                # corner-anchored 3c08: the tasks that hold the corner cell
                t08a += _comb3(sl[0])
                for t in range(1, 8):
                    t08a += sl[t] * _comb2(sl[0]) + sl[0] * _comb2(sl[t])
                for t, u in itertools.combinations(range(1, 8), 2):
                    t08a += sl[0] * sl[t] * sl[u]
                # 3c01: each molecule of the base cell against all pairs of the other
                # molecules in its 27-cell neighbourhood
                m = sum(N(z + dz, y + dy, xx + dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1)
                        for dx in (-1, 0, 1))
                t01 += nb * _comb2(m - 1)
    assert oracle.atm_cells(prm, x, "3c18", "pair")["n_cand3"] == t18
    assert oracle.atm_cells(prm, x, "3c08", "product")["n_cand3"] == t08
    assert oracle.atm_cells(prm, x, "3c01", "pair")["n_cand3"] == t01
    assert oracle.atm_cells(prm, x, "3c08a", "pair")["n_cand3"] == t08a


@pytest.mark.parametrize("trav", ["3c18", "3c08"])
def test_three_cell_toy_visits_every_triple_once(trav):
    """Eq. totalInteractions: molecules in three mutually adjacent cells are
    split into one-, two- and three-cell triplets adding up to C(N,3)."""
    rc = 2.5
    box = 3 * rc + 0.03
    w = box / 3
    rng = np.random.default_rng(5)
    pts = []
    for cx, cy, cz, m in [(0, 0, 0, 5), (1, 0, 0, 4), (0, 1, 1, 6)]:
        for _ in range(m):
            pts.append([(cx + 0.1 + 0.8 * rng.random()) * w, (cy + 0.1 + 0.8 * rng.random()) * w,
                        (cz + 0.1 + 0.8 * rng.random()) * w])
    x = np.ascontiguousarray(np.array(pts).T)
    n = x.shape[1]
    out = oracle.atm_cells(_prm(box, rc), x, trav, "pair")
    assert out["n_cand3"] == _comb3(n)


# ---------------------------------------------------------------- cells

def test_cells_bin_and_stable_sort():
    x, box = _small_fluid(n=150, rho=0.5, seed=20)
    x = x + np.array([[box], [-box], [2.5 * box]])  # outside the box: must wrap
    prm = _prm(box)
    c = oracle.build_cells(prm, x)
    nc, w = oracle.cell_grid(prm)
    n = x.shape[1]
    assert c["cell_start"][0] == 0 and c["cell_start"][-1] == n
    assert np.all(np.diff(c["cell_start"]) >= 0)
    assert sorted(c["perm"]) == list(range(n))
    for cid in range(len(c["cell_start"]) - 1):
        seg = c["perm"][c["cell_start"][cid]:c["cell_start"][cid + 1]]
        assert np.all(np.diff(seg) > 0)  # stable: original order inside a cell
        assert np.all(c["cell_of"][seg] == cid)
    xw = c["xw"]
    assert np.all(xw >= 0) and np.all(xw < box)
    cz, rem = np.divmod(c["cell_of"], nc[0] * nc[1])
    cy, cx = np.divmod(rem, nc[0])
    for d, cd in enumerate([cx, cy, cz]):
        assert np.all(xw[d] >= cd * w[d] - 1e-12) and np.all(xw[d] <= (cd + 1) * w[d] + 1e-12)
        xl = c["xl"][d]
        assert np.all(xl >= 0) and np.all(xl <= w[d])
        assert np.allclose(xl, xw[d][c["perm"]] - cd[c["perm"]] * w[d], atol=1e-12)
    assert np.array_equal(c["xl32"], c["xl"].astype(np.float32))


def test_cell_grid_rule():
    """n_d is the largest k with L/k >= r_c; fewer than three cells is an error."""
    nc, w = oracle.cell_grid(oracle.params([37.5, 10.0, 7.6], 2.5, NU))
    assert list(nc) == [15, 4, 3]
    assert w[0] == 2.5
    with pytest.raises(oracle.OracleError):
        oracle.cell_grid(oracle.params([7.4, 10.0, 10.0], 2.5, NU))


# ---------------------------------------------------------------- FP32 decisions, LJ, MD

def test_fp32_decisions_close_to_fp64():
    x, box = _small_fluid(n=300, rho=0.6, seed=23)
    prm = _prm(box)
    for trunc in ["pair", "product"]:
        a = oracle.atm_cells(prm, x, "3c18", trunc, "fp64")
        b = oracle.atm_cells(prm, x, "3c18", trunc, "fp32")
        assert a["n_cand3"] == b["n_cand3"]
        assert abs(a["n_int3"] - b["n_int3"]) <= max(2, 1e-4 * a["n_int3"])


# An independent float32 statement of the FP32 decision sequence: positions
# wrapped into [0, L), cell c = min(n - 1, floor(x / w)), cell-local
# coordinate x - c w in FP64 rounded once to float32; per pair
# d = (l_q - l_p) + float32(dc) * float32(w) in float32 with dc the wrapped
# cell offset, |d|^2 = (dx dx + dy dy) + dz dz in float32; r_c^2 and r_c^6
# as float32 products of float32(r_c); pair rule: every side below r_c^2;
# product rule: (lo * mid) * hi of the sorted sides below r_c^6.  numpy's
# float32 operations round each result once and never contract.

def _grid(L, rc):
    n = []
    for Ld in L:
        k = 1
        while Ld / (k + 1) >= rc:
            k += 1
        n.append(k)
    return np.array(n)


def _f32_decisions(x, box, rc, trunc, tri, variant=None):
    """Decisions of the triangles tri[:, 0..2] (molecule indices)."""
    L = np.asarray(box, dtype=np.float64)
    n = _grid(L, rc)
    w = L / n
    c = np.minimum(n[:, None] - 1, np.floor(x / w[:, None])).astype(np.int64)
    loc = np.clip(x - c * w[:, None], 0.0, w[:, None])
    l32 = loc.astype(np.float32)
    if variant == "local_from_rounded":  # planted: float32(x) - c float32(w)
        l32 = x.astype(np.float32) - c.astype(np.float32) * w.astype(np.float32)[:, None]
    wf = w.astype(np.float32)

    def d2(p, q):
        dc = (c[:, q] - c[:, p] + 1) % n[:, None] - 1  # wrapped offset of adjacent cells
        d = (l32[:, q] - l32[:, p]) + dc.astype(np.float32) * wf[:, None]
        if variant == "fp64":  # planted: the decision taken in FP64
            d = (loc[:, q] - loc[:, p]) + dc * w[:, None]
        if variant == "sum_order":  # planted: dx dx + (dy dy + dz dz)
            return d[0] * d[0] + (d[1] * d[1] + d[2] * d[2])
        return (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]

    rcf = np.float32(rc)
    rc2f = rcf * rcf
    if variant == "rc2_from_fp64":  # planted: r_c^2 rounded from FP64
        rc2f = np.float32(rc * rc)
    rc6f = (rc2f * rc2f) * rc2f
    a, b, cc = d2(tri[:, 0], tri[:, 1]), d2(tri[:, 0], tri[:, 2]), d2(tri[:, 1], tri[:, 2])
    if variant == "fp64":
        rc2f = rc * rc
        rc6f = (rc2f * rc2f) * rc2f
    if trunc == "pair":
        return (a < rc2f) & (b < rc2f) & (cc < rc2f)
    srt = np.sort(np.stack([a, b, cc]), axis=0)
    if variant == "product_order":  # planted: (hi * mid) * lo
        return (srt[2] * srt[1]) * srt[0] < rc6f
    return (srt[0] * srt[1]) * srt[2] < rc6f


def _near_cutoff_triangles(rc, trunc, seed, k=5, L_over_rc=14.5):
    """k^3 isolated triangles (no molecule of another triangle within 1.4 r_c)
    whose pair-rule sides, or whose product of sides, lie within a few float32
    ulps of the cutoff; rotated at random, shifted by a random vector and
    wrapped (some straddle cell faces and the periodic boundary)."""
    rng = np.random.default_rng(seed)
    L = L_over_rc * rc
    sp = L / k
    pts = []
    for ix, iy, iz in itertools.product(range(k), repeat=3):
        if trunc == "pair":
            a, b, c = rc * (1.0 + rng.uniform(-1.5e-7, 1.5e-7, 3))
        else:
            f1, f2 = rng.uniform(0.99, 1.01, 2)
            a, b, c = rc * f1, rc * f2, rc / (f1 * f2) * (1.0 + rng.uniform(-1.5e-7, 1.5e-7))
        xx = (a * a + b * b - c * c) / (2 * a)
        t = np.array([[0.0, 0.0, 0.0], [a, 0.0, 0.0], [xx, math.sqrt(b * b - xx * xx), 0.0]])
        q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        t = (t - t.mean(axis=0)) @ q.T
        pts.append(t + (np.array([ix, iy, iz]) + 0.5) * sp + rng.uniform(-0.3, 0.3, 3))
    x = np.concatenate(pts).T + rng.uniform(0.0, L, size=(3, 1))
    x = x - np.floor(x / L) * L
    x[x >= L] = 0.0
    assert np.all((x >= 0.0) & (x < L))
    tri = np.arange(3 * k ** 3).reshape(-1, 3)
    return np.ascontiguousarray(x), np.array([L, L, L]), tri


@pytest.mark.parametrize("rc", [2.5, 2.314])
@pytest.mark.parametrize("trunc", ["pair", "product"])
def test_fp32_decision_mode_equals_an_independent_float32_statement(rc, trunc):
    """The oracle's FP32-decision mode (the triplet set the FP32C kernels are
    compared with bit for bit) decides every near-cutoff triangle as the
    float32 statement above does, for every traversal; and the fixture is
    sharp enough that the FP64 decision and each planted variant of the
    statement (another summation or product order, local coordinates from
    rounded positions, r_c^2 rounded from FP64) decide some triangle
    differently."""
    for seed in range(5):
        x, box, tri = _near_cutoff_triangles(rc, trunc, 7100 + seed)
        keep = _f32_decisions(x, box, rc, trunc, tri)
        assert 0 < keep.sum() < len(keep)
        prm = oracle.params(box, rc, NU)
        for trav, visits in (("3c01", 3), ("3c18", 1), ("3c08", 1)):
            r = oracle.atm_cells(prm, x, trav, trunc, "fp32")
            assert r["n_int3"] == visits * int(keep.sum()), (trav, seed)
            hit = np.any(r["f"][:, tri[:, 0]] != 0.0, axis=0)
            assert np.array_equal(hit, keep), (trav, seed)
    # sensitivity over the five fixtures together
    for variant in ("fp64", "sum_order", "local_from_rounded", "product_order",
                    "rc2_from_fp64"):
        if variant == "product_order" and trunc == "pair":
            continue
        if variant == "rc2_from_fp64" and np.float32(rc * rc) == np.float32(rc) * np.float32(rc):
            continue
        differs = False
        for seed in range(5):
            x, box, tri = _near_cutoff_triangles(rc, trunc, 7100 + seed)
            differs |= not np.array_equal(_f32_decisions(x, box, rc, trunc, tri),
                                          _f32_decisions(x, box, rc, trunc, tri, variant))
        assert differs, variant


def test_lj_cells_equal_brute_force():
    x, box = _small_fluid(n=200, rho=0.5, seed=24)
    prm = _prm(box)
    a = oracle.lj_brute(prm, x)
    b = oracle.lj_cells(prm, x)
    assert a["n_int2"] == b["n_int2"]
    assert b["e2"] == pytest.approx(a["e2"], rel=1e-12)
    assert b["w2"] == pytest.approx(a["w2"], rel=1e-12)
    assert np.allclose(a["f"], b["f"], rtol=1e-10, atol=1e-12)


def test_velocity_verlet_is_time_reversible_and_conserves_energy():
    cfg = synth.homogeneous(256, 0.8, 1.0, seed=99)
    prm = oracle.params(cfg["box"], 2.5, NU, lj_shift=True)
    # the fcc box for 256 at rho 0.8 is 6.84 < 3 r_c: shrink the cutoff
    prm[3] = 2.2
    out = oracle.md_run(prm, cfg["x"], cfg["v"], 40, 0.002, "3c18", "pair")
    en = out["energies"]
    etot = en[:, 0] + en[:, 1] + en[:, 2]
    assert np.max(np.abs(etot - etot[0])) < 2e-3 * abs(etot[0]) + 0.05
    back = oracle.md_run(prm, out["x"], -out["v"], 40, 0.002, "3c18", "pair")
    d = back["x"] - np.mod(cfg["x"], cfg["box"][:, None])
    d -= np.rint(d / cfg["box"][:, None]) * cfg["box"][:, None]
    assert np.abs(d).max() < 1e-8


# ---------------------------------------------------- wide owner traversal

def _wide_system(n=1000, rho=0.5, seed=77):
    cfg = synth.homogeneous(n, rho, 1.0, seed)
    return cfg, oracle.params(cfg["box"], 2.5, 0.073)


def test_wide_traversal_equals_brute_force_with_member_filter():
    cfg, prm = _wide_system()
    nc, w = oracle.cell_grid(prm)
    assert nc.min() >= 5
    bf = oracle.atm_brute(prm, cfg["x"], "product", member="3cw")
    lc = oracle.atm_cells(prm, cfg["x"], "3cw", "product", "fp64")
    # owner traversal: each triplet visited by its three members
    assert lc["n_int3"] == 3 * bf["n_int3"]
    assert abs(lc["e3"] - bf["e3"]) <= 1e-10 * abs(bf["e3"])
    assert abs(lc["w3"] - bf["w3"]) <= 1e-10 * abs(bf["w3"])
    scale = np.sqrt(np.mean(bf["f"] ** 2))
    assert np.max(np.abs(lc["f"] - bf["f"])) <= 1e-10 * scale


def test_wide_traversal_is_complete_for_the_product_rule():
    # closest pair r_min: every product-rule triplet has its longest side below
    # (r_min + sqrt(r_min^2 + 4 rc^3 / r_min)) / 2, here below R_w = 2 min(w)
    cfg, prm = _wide_system()
    x = cfg["x"]
    L = cfg["box"][0]
    d = x[:, :, None] - x[:, None, :]
    d -= L * np.rint(d / L)
    r = np.sqrt((d ** 2).sum(0))
    np.fill_diagonal(r, np.inf)
    rmin = r.min()
    lmax = (rmin + np.sqrt(rmin ** 2 + 4 * 2.5 ** 3 / rmin)) / 2
    _, w = oracle.cell_grid(prm)
    assert lmax < 2 * w.min()
    full = oracle.atm_brute(prm, x, "product")
    wide = oracle.atm_brute(prm, x, "product", member="3cw")
    assert full["n_int3"] == wide["n_int3"]
    assert abs(full["e3"] - wide["e3"]) <= 1e-12 * abs(full["e3"])
    # and the paper's traversals find a subset
    for trav in ("3c01", "3c18", "3c08"):
        t = oracle.atm_cells(prm, x, trav, "product", "fp64")
        n_unique = t["n_int3"] // 3 if trav == "3c01" else t["n_int3"]
        assert n_unique <= full["n_int3"]


def test_wide_traversal_pair_rule_and_candidates():
    cfg, prm = _wide_system(n=600, rho=0.3, seed=78)
    x = cfg["x"]
    lc = oracle.atm_cells(prm, x, "3cw", "pair", "fp64")
    bf = oracle.atm_brute(prm, x, "pair")
    assert lc["n_int3"] == 3 * bf["n_int3"]
    assert abs(lc["e3"] - bf["e3"]) <= 1e-10 * abs(bf["e3"])
    # candidates: the partner pairs of every owner (pair rule: partners within r_c)
    rw2 = 2.5 ** 2
    L = cfg["box"][0]
    d = x[:, :, None] - x[:, None, :]
    d -= L * np.rint(d / L)
    d2 = (d ** 2).sum(0)
    np.fill_diagonal(d2, np.inf)
    npart = (d2 < rw2).sum(1)
    assert lc["n_cand3"] == int((npart * (npart - 1) // 2).sum())


def test_wide_traversal_needs_five_cells():
    cfg = synth.config("liquid_n1000")  # 4 cells per axis
    prm = oracle.params(cfg["box"], 2.5, 0.073)
    with pytest.raises(oracle.OracleError):
        oracle.atm_cells(prm, cfg["x"], "3cw", "product", "fp64")


# ---------------------------------------------------------------- observables

def _minimum_image_histogram(box, x, r_max, nbins):
    """All pairs, minimum image, numpy distances: an independent histogram."""
    L = np.asarray(box, dtype=np.float64)[:, None, None]
    d = x[:, None, :] - x[:, :, None]
    d -= L * np.round(d / L)
    r = np.sqrt((d * d).sum(axis=0))
    iu = np.triu_indices(x.shape[1], 1)
    r = r[iu]
    r = r[r < r_max]
    return np.bincount(np.minimum((r / (r_max / nbins)).astype(np.int64), nbins - 1),
                       minlength=nbins)


@pytest.mark.parametrize("box,n,seed", [((9.0, 10.0, 11.5), 700, 61), ((7.6, 7.6, 15.2), 450, 62)])
def test_rdf_histogram_equals_all_pairs_minimum_image(box, n, seed):
    """Section 5.1 RDFs: the linked-cell pair histogram holds every pair within
    r_max exactly once (against an all-pairs minimum-image count)."""
    rng = np.random.default_rng(seed)
    x = synth.uniform_positions(n, box, rng)
    prm = oracle.params(box, 2.5, NU)
    _, w = oracle.cell_grid(prm)
    r_max = float(min(w))
    got = oracle.rdf_counts(prm, x, r_max, 40)
    ref = _minimum_image_histogram(box, x, r_max, 40)
    assert np.array_equal(got.astype(np.int64), ref)


def test_rdf_of_a_simple_cubic_lattice_counts_its_coordination_shells():
    """Simple cubic lattice of spacing 1: shells at 1, sqrt2, sqrt3, 2, sqrt5,
    sqrt6 hold 6, 12, 8, 6, 24, 24 neighbours per site, each pair counted once."""
    m = 8
    g = np.arange(m, dtype=np.float64) + 0.25
    cx, cy, cz = np.meshgrid(g, g, g, indexing="ij")
    x = np.ascontiguousarray(np.stack([cx.ravel(), cy.ravel(), cz.ravel()]))
    prm = oracle.params(float(m), 2.5, NU)
    r_max, nbins = 2.55, 17
    got = oracle.rdf_counts(prm, x, r_max, nbins).astype(np.int64)
    ref = np.zeros(nbins, dtype=np.int64)
    for r2, z in ((1, 6), (2, 12), (3, 8), (4, 6), (5, 24), (6, 24)):
        ref[int(math.sqrt(r2) / (r_max / nbins))] += m ** 3 * z // 2
    assert np.array_equal(got, ref)


def test_rdf_of_an_ideal_gas_is_one():
    """Uniform random positions: g(r) = 1 within counting noise."""
    rng = np.random.default_rng(63)
    box = 20.0
    n = 4000
    x = synth.uniform_positions(n, box, rng)
    prm = oracle.params(box, 2.5, NU)
    counts = oracle.rdf_counts(prm, x, 2.5, 10)
    r, g = oracle.rdf_normalise(counts, 1, n, box ** 3, 2.5)
    assert r[0] == pytest.approx(0.125)
    sigma = 1.0 / np.sqrt(np.maximum(counts, 1))
    assert np.all(np.abs(g[2:] - 1.0) < 5 * sigma[2:])


def test_rdf_rejects_a_range_beyond_the_cell_edge():
    prm = oracle.params(10.0, 2.5, NU)
    x = synth.uniform_positions(50, 10.0, np.random.default_rng(64))
    with pytest.raises(oracle.OracleError):
        oracle.rdf_counts(prm, x, 3.4, 10)


@pytest.mark.parametrize("rc,rho", [(2.5, 0.8), (3.0, 0.65), (2.0, 0.3)])
def test_lj_tail_corrections_equal_the_closed_forms(rc, rho):
    """Tail integrals of the LJ 12-6 pair potential (homogeneous fluid, g = 1
    beyond r_c): E_tail / N = 8/3 pi rho [(1/3) rc^-9 - rc^-3] and
    P_tail = 16/3 pi rho^2 [(2/3) rc^-9 - rc^-3] in reduced units."""
    n = 1000
    box = (n / rho) ** (1.0 / 3.0)
    e, p = oracle.lj_tail(oracle.params(box, rc, NU), n)
    assert e / n == pytest.approx(8 / 3 * math.pi * rho * (rc ** -9 / 3 - rc ** -3), rel=1e-11)
    assert p == pytest.approx(16 / 3 * math.pi * rho ** 2 * (2 / 3 * rc ** -9 - rc ** -3), rel=1e-11)


def test_lj_tail_scales_with_epsilon_and_sigma():
    """u = 4 eps [(s/r)^12 - (s/r)^6]: E_tail is linear in eps and, at fixed
    r_c / sigma and rho sigma^3, scales as eps (dimensionless form)."""
    base = oracle.lj_tail(oracle.params(10.0, 2.5, NU), 800)
    scaled = oracle.lj_tail(oracle.params(20.0, 5.0, NU, lj_eps=3.0, lj_sigma=2.0), 800)
    assert scaled[0] == pytest.approx(3.0 * base[0], rel=1e-12)
    assert scaled[1] == pytest.approx(3.0 / 8.0 * base[1], rel=1e-12)


def test_velocity_rescaling_sets_the_kinetic_temperature():
    """NVT by velocity rescaling: afterwards 2K / (3n - 3) equals the target,
    every velocity keeps its direction, the total momentum stays zero, and a
    resting system (K = 0) is left alone."""
    rng = np.random.default_rng(65)
    n = 500
    v = synth.maxwell_boltzmann(n, 1.7, rng)
    w = oracle.rescale(v, 0.746)
    k = 0.5 * (w * w).sum()
    assert 2.0 * k / (3 * n - 3) == pytest.approx(0.746, rel=1e-13)
    ratio = w / v
    assert np.allclose(ratio, ratio.flat[0], rtol=1e-14)
    assert ratio.flat[0] == pytest.approx(math.sqrt(0.746 / 1.7), rel=1e-12)
    assert np.abs(w.sum(axis=1)).max() < 1e-10
    z = np.zeros((3, n))
    assert np.array_equal(oracle.rescale(z, 1.0), z)


# ---------------------------------------------------------------- corner-anchored 3c08

def test_corner_anchored_3c08_omits_exactly_the_cornerless_block_triples():
    """The 3c08 of the text (every task holds the block's corner cell) finds
    the pair-rule triplets whose cell triple contains its own bounding-box
    corner, and misses the rest (section 4 says some are omitted): brute force
    with that membership filter = the traversal; the complete 3c08 = all."""
    rc = 2.5
    box = 4 * rc + 0.3
    rng = np.random.default_rng(41)
    n = int(0.35 * box ** 3)
    x = np.ascontiguousarray(
        synth.random_sequential(n, [0, 0, 0], [box] * 3, 0.85, rng, box=np.array([box] * 3)).T)
    prm = _prm(box, rc)
    full = oracle.atm_brute(prm, x, "pair")
    anch_bf = oracle.atm_brute(prm, x, "pair", member="3c08a")
    anch = oracle.atm_cells(prm, x, "3c08a", "pair")
    assert anch["n_int3"] == anch_bf["n_int3"]
    assert anch["e3"] == pytest.approx(anch_bf["e3"], rel=1e-11)
    assert np.allclose(anch["f"], anch_bf["f"], rtol=1e-9, atol=1e-12)
    assert 0.5 * full["n_int3"] < anch["n_int3"] < full["n_int3"]
    assert oracle.atm_cells(prm, x, "3c08", "pair")["n_int3"] == full["n_int3"]
    # fewer candidates than the complete 3c08 and a higher hit rate
    c08 = oracle.atm_cells(prm, x, "3c08", "pair")
    assert anch["n_cand3"] < c08["n_cand3"]
    assert anch["n_int3"] / anch["n_cand3"] > c08["n_int3"] / c08["n_cand3"]


def test_corner_anchored_3c08_on_three_cells_skips_the_cornerless_triple():
    """Three molecules, one in each face neighbour of a corner cell (cells
    (1,0,0), (0,1,0), (0,0,1) of a 4^3 grid) and mutually within r_c: the
    complete 3c08 finds the triplet, the corner-anchored one does not; moving
    one molecule into the corner cell makes both find it."""
    rc = 2.5
    box = 4 * rc
    w = rc
    x = np.array([[w + 0.2, w - 0.4, w - 0.4],
                  [w - 0.4, w + 0.2, w - 0.4],
                  [w - 0.4, w - 0.4, w + 0.2]]).T.copy()
    # cells (1,0,0), (0,1,0), (0,0,1) relative to the corner (0,0,0)
    prm = _prm(box, rc)
    assert oracle.atm_cells(prm, x, "3c08", "pair")["n_int3"] == 1
    assert oracle.atm_cells(prm, x, "3c08a", "pair")["n_int3"] == 0
    x2 = x.copy()
    x2[0, 0] = w - 0.1
    assert oracle.atm_cells(prm, x2, "3c08", "pair")["n_int3"] == 1
    assert oracle.atm_cells(prm, x2, "3c08a", "pair")["n_int3"] == 1
