"""Pins for the FP64 oracle: values the paper prints, closed forms, library
routines and invariants, none of which reuse the oracle's own formulas.

Each check is chosen so that a plausible slip in the oracle (a dropped
symmetrization term, a sign error, a rank off by one, a transposed pair index,
a missing factor d or 1/2) fails at least one of them.
"""
import itertools
import json
import os

import numpy as np
import pytest
from scipy.stats import rankdata

from oracle import gini_oracle as orc
from paper_2605_25124_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# ---------------------------------------------------------------- ranks ----

def test_midranks_match_scipy_average_ranks():
    # Midranks are scipy's "average" ranks (a library routine).
    rng = np.random.default_rng(0)
    for m in (1, 2, 3, 7, 31, 100):
        for v in (rng.standard_normal(m), rng.integers(0, 3, m).astype(float)):
            np.testing.assert_array_equal(orc.midrank2(v), (2 * rankdata(v)).astype(np.int32))


def test_midranks_golden_all_ties():
    for case in _load("rank_ties.json")["cases"]:
        np.testing.assert_array_equal(orc.midrank2(case["v"]) / 2.0, case["midranks"])


def test_midrank_invariants():
    rng = np.random.default_rng(1)
    for m in (5, 17, 64):
        v = rng.integers(-3, 4, m).astype(float)
        r = orc.midrank2(v) / 2.0
        assert r.sum() == m * (m + 1) / 2                      # sum of ranks
        np.testing.assert_array_equal(orc.midrank2(-v) / 2.0, m + 1 - r)  # R(-x) = d+1-R(x)


# --------------------------------------------------------- worked example --

def test_worked_example_594():
    g = _load("worked_example.json")
    assert orc.gini_dg(g["u"], g["v"]) == g["D_G"]
    # The generalized, symmetrized distance at nu = 2 equals D_G.
    assert orc.pd(g["u"], g["v"], 2.0) == pytest.approx(g["D_G"], rel=1e-15)


@pytest.mark.parametrize("nu", [1.1, 1.5, 2.0, 2.7, 3.0, 5.0])
def test_two_component_closed_form(nu):
    # d = 2: W(1) = -(1/2)^(nu-1), W(2) = +(1/2)^(nu-1) so
    # Dbar = 2^(1-nu) |z1 - z2|; the worked example gives 1188 * 2^(1-nu).
    assert orc.pd([10, 1200], [10, 12], nu) == pytest.approx(1188 * 2.0 ** (1 - nu), rel=1e-14)
    rng = np.random.default_rng(int(nu * 10))
    for _ in range(20):
        x, y = rng.standard_normal(2), rng.standard_normal(2)
        z = x - y
        assert orc.pd(x, y, nu) == pytest.approx(2.0 ** (1 - nu) * abs(z[0] - z[1]), rel=1e-12)


@pytest.mark.parametrize("nu", [1.3, 2.0, 4.0])
def test_three_component_closed_form(nu):
    # d = 3, distinct components: W(2) = 0 and W(3) = -W(1) = (2/3)^(nu-1),
    # so Dbar = (3/2) (2/3)^(nu-1) (max z - min z).
    rng = np.random.default_rng(3)
    for _ in range(20):
        x, y = rng.standard_normal(3), rng.standard_normal(3)
        z = x - y
        want = 1.5 * (2.0 / 3.0) ** (nu - 1) * (z.max() - z.min())
        assert orc.pd(x, y, nu) == pytest.approx(want, rel=1e-12)


def test_nu2_equals_half_pairwise_l1():
    # sum_k (2k - d - 1) z_(k) = sum_{a<b} |z_a - z_b|  (Gini mean difference),
    # and tied values cancel in the same way, so at nu = 2
    # Dbar = D_G = 1/2 sum_{a<b} |z_a - z_b|, ties or not.
    rng = np.random.default_rng(4)
    for d in (1, 2, 5, 13, 50):
        for gen in ("cont", "ties"):
            if gen == "cont":
                x, y = rng.standard_normal(d), rng.standard_normal(d)
            else:
                x, y = rng.integers(0, 3, d).astype(float), rng.integers(0, 3, d).astype(float)
            z = x - y
            want = 0.5 * np.abs(z[:, None] - z[None, :]).sum() / 2.0
            assert orc.pd(x, y, 2.0) == pytest.approx(want, rel=1e-12, abs=1e-12)
            assert orc.gini_dg(x, y) == pytest.approx(want, rel=1e-12, abs=1e-12)


def test_nu3_is_the_nu2_distance_times_d_minus_1_over_d():
    # W_{d,3}(R) = ((R-1)/d)^2 - ((d-R)/d)^2 = (2R - d - 1)(d - 1)/d^2 is
    # affine in R, (d-1)/d times W_{d,2}: so at nu = 3
    # Dbar = ((d-1)/d) * 1/2 sum_{a<b} |z_a - z_b|, ties or not.
    rng = np.random.default_rng(5)
    for d in (1, 2, 5, 13, 50):
        for gen in ("cont", "ties"):
            if gen == "cont":
                x, y = rng.standard_normal(d), rng.standard_normal(d)
            else:
                x, y = rng.integers(0, 3, d).astype(float), rng.integers(0, 3, d).astype(float)
            z = x - y
            want = (d - 1) / d * 0.5 * np.abs(z[:, None] - z[None, :]).sum() / 2.0
            assert orc.pd(x, y, 3.0) == pytest.approx(want, rel=1e-12, abs=1e-12)


def test_general_nu_against_rank_weight_identity_with_ties():
    # With Fbar = 1 - R/d and R_{-z}(-z_j) = d + 1 - R_z(z_j) the two terms of
    # the symmetrization combine into (d/2) sum_j z_j W(R_j),
    # W(R) = ((R-1)/d)^(nu-1) - ((d-R)/d)^(nu-1); ranks from scipy here.
    rng = np.random.default_rng(5)
    for d in (4, 9, 30):
        for nu in (1.2, 1.5, 3.0, 4.5):
            for ints in (False, True):
                if ints:
                    x, y = rng.integers(0, 4, d).astype(float), rng.integers(0, 4, d).astype(float)
                else:
                    x, y = rng.standard_normal(d), rng.standard_normal(d)
                z = x - y
                R = rankdata(z)
                W = ((R - 1) / d) ** (nu - 1) - ((d - R) / d) ** (nu - 1)
                assert orc.pd(x, y, nu) == pytest.approx(d / 2 * np.sum(z * W), rel=1e-12, abs=1e-12)


def test_sorted_positional_form_nu2():
    # Without ties, D_G = sum_k z_(k) (k - (d+1)/2) on the sorted vector.
    rng = np.random.default_rng(6)
    for d in (3, 8, 40):
        x, y = rng.standard_normal(d), rng.standard_normal(d)
        zs = np.sort(x - y)
        k = np.arange(1, d + 1)
        assert orc.gini_dg(x, y) == pytest.approx(np.sum(zs * (k - (d + 1) / 2)), rel=1e-12)


# ------------------------------------------------------------- properties --

def _tie_free(rng, d):
    return rng.standard_normal(d), rng.standard_normal(d), rng.standard_normal(d)


@pytest.mark.parametrize("nu", [1.2, 2.0, 3.5])
def test_pseudo_distance_properties_tie_free(nu):
    # Propositions 2 and 3: null, symmetry, non-negativity, triangle inequality;
    # plus absolute homogeneity (Prop. 1 (i)), translation by c 1_d and a common
    # permutation of the features.  Tie-free inputs (Prop. 3 relies on distinct
    # ranks through the rearrangement inequality).
    rng = np.random.default_rng(7)
    for d in (2, 3, 6, 20):
        for _ in range(30):
            x, y, w = _tie_free(rng, d)
            dxy = orc.pd(x, y, nu)
            assert orc.pd(x, x, nu) == 0.0
            assert dxy >= 0.0
            assert dxy == pytest.approx(orc.pd(y, x, nu), rel=1e-12)
            assert dxy <= orc.pd(x, w, nu) + orc.pd(w, y, nu) + 1e-12
            lam = rng.uniform(-3, 3)
            assert orc.pd(lam * x, lam * y, nu) == pytest.approx(abs(lam) * dxy, rel=1e-10)
            c = rng.uniform(-2, 2)
            assert orc.pd(x + c, y, nu) == pytest.approx(dxy, rel=1e-9, abs=1e-12)
            perm = rng.permutation(d)
            assert orc.pd(x[perm], y[perm], nu) == pytest.approx(dxy, rel=1e-12)


def test_properties_with_ties_at_nu2():
    rng = np.random.default_rng(8)
    for d in (3, 7, 16):
        for _ in range(40):
            x, y, w = (rng.integers(0, 3, d).astype(float) for _ in range(3))
            dxy = orc.pd(x, y, 2.0)
            assert dxy >= 0.0
            assert dxy == pytest.approx(orc.pd(y, x, 2.0), abs=1e-12)
            assert dxy <= orc.pd(x, w, 2.0) + orc.pd(w, y, 2.0) + 1e-12
            assert orc.pd(x + 1.5, y, 2.0) == pytest.approx(dxy, abs=1e-12)


def test_egalitarian_and_null_cases():
    # Prop. 2 (ii): x = c 1_d = lambda y gives 0; seminorm null cases of
    # Section III-A: ||0||_G = 0 and ||c 1_d||_G = 0.
    for d in (2, 5, 11):
        for nu in (1.5, 2.0, 3.0):
            assert orc.pd(np.full(d, 3.0), np.full(d, 1.5), nu) == 0.0
        assert orc.gini_norm(np.zeros(d)) == 0.0
        assert orc.gini_norm(np.full(d, -2.0)) == 0.0


def test_seminorm_proposition_1():
    rng = np.random.default_rng(9)
    for d in (2, 5, 12):
        for _ in range(30):
            x, y = rng.standard_normal(d), rng.standard_normal(d)
            lam = rng.uniform(-4, 4)
            assert orc.gini_norm(lam * x) == pytest.approx(abs(lam) * orc.gini_norm(x), rel=1e-10)
            assert orc.gini_norm(x + y) <= orc.gini_norm(x) + orc.gini_norm(y) + 1e-12
            assert orc.gini_norm(x) >= 0.0


def test_brute_force_tiny_against_permutation_definition():
    # Brute force of Definition 1 on tiny vectors: the rank of u_a is 1 plus the
    # number of strictly smaller components, averaged over all orderings of tied
    # components (each ordering of a tie group is equally likely) -> midrank.
    rng = np.random.default_rng(10)
    for _ in range(50):
        d = int(rng.integers(1, 6))
        v = rng.integers(0, 3, d).astype(float)
        acc = np.zeros(d)
        perms = list(itertools.permutations(range(d)))
        for perm in perms:
            # break ties by the position in perm
            key = [(v[a], perm.index(a)) for a in range(d)]
            acc += [1 + sum(key[b] < key[a] for b in range(d)) for a in range(d)]
        np.testing.assert_allclose(orc.midrank2(v) / 2.0, acc / len(perms))


# ------------------------------------------------------------------ Delta --

def test_delta_matrix_structure_and_pairs():
    X = wl.gaussian_outliers(23, 7, seed=11)
    nus = [1.5, 2.0, 3.0]
    D, s = orc.delta(X, nus)
    for q, nu in enumerate(nus):
        assert np.all(np.diag(D[q]) == 0.0)
        np.testing.assert_array_equal(D[q], D[q].T)
        assert np.all(D[q] >= 0)
        iu = np.triu_indices(23, 1)
        assert s[q] == pytest.approx(np.sum(D[q][iu] ** 2), rel=1e-13)
        for (i, j) in [(0, 1), (3, 17), (22, 5)]:
            assert D[q, i, j] == pytest.approx(orc.pd(X[i].astype(float), X[j].astype(float), nu),
                                               rel=1e-15)
    I = np.array([0, 4, 9, 22]); J = np.array([1, 8, 2, 21])
    np.testing.assert_array_equal(orc.delta_pairs(X, nus, I, J), D[:, I, J].T)


def test_delta_nu2_against_pairwise_l1_on_image_rows():
    X = wl.image_like(6, seed=12)
    D, _ = orc.delta(X, [2.0])
    for i in range(6):
        for j in range(6):
            z = X[i].astype(float) - X[j].astype(float)
            # sum over a<b of |z_a - z_b| via the sorted form (O(d log d))
            zs = np.sort(z)
            k = np.arange(1, z.size + 1)
            want = np.sum(zs * (2 * k - z.size - 1)) / 2.0
            assert D[0, i, j] == pytest.approx(want, rel=1e-12, abs=1e-9)


# -------------------------------------------------------- stress, gradient --

def _planted(n, k, nu, seed):
    Ystar = wl.y_init(n, k, seed, sd=1.0).astype(np.float64)
    I, J = np.triu_indices(n, 1)
    d = orc.embed_dist_pairs(Ystar, nu, I, J)
    D = np.zeros((n, n)); D[I, J] = d; D[J, I] = d
    return Ystar, D, float(np.sum(d ** 2))


def test_two_point_hand_case():
    # n = 2, k = 2: d = 2^(1-nu)|u1 - u2|, u = y_1 - y_2 (per point),
    # S = (d - delta)^2 / delta^2,
    # dS/dy_1 = 2 (d - delta)/delta^2 * 2^(1-nu) sign(u1 - u2) * (1, -1), dS/dy_2 = -dS/dy_1.
    nu, delta = 1.7, 0.9
    Y = np.array([[0.3, -0.2], [0.1, 0.4]])
    u = Y[:, 0] - Y[:, 1]
    c = 2.0 ** (1 - nu)
    d = c * abs(u[0] - u[1])
    D = np.array([[0.0, delta], [delta, 0.0]])
    S, g = orc.stress_grad(Y, nu, D, delta ** 2)
    assert S == pytest.approx((d - delta) ** 2 / delta ** 2, rel=1e-14)
    g1 = 2 * (d - delta) / delta ** 2 * c * np.sign(u[0] - u[1]) * np.array([1.0, -1.0])
    np.testing.assert_allclose(g[0], g1, rtol=1e-13)
    np.testing.assert_allclose(g[1], -g1, rtol=1e-13)


@pytest.mark.parametrize("k,nu", [(2, 2.0), (2, 1.5), (3, 2.0), (3, 3.0), (4, 1.8)])
def test_gradient_central_differences(k, nu):
    n = 14
    Y = wl.y_init(n, k, seed=13 + k, sd=1.0).astype(np.float64)
    Delta = orc.delta(wl.gaussian_outliers(n, 5, seed=14), [nu])[0][0]
    sd2 = float(np.sum(np.triu(Delta, 1) ** 2))
    S, g = orc.stress_grad(Y, nu, Delta, sd2)
    h = 1e-6
    # stay away from kinks: every pairwise component gap must exceed 100 h
    gaps = np.abs((Y[:, None, :, None] - Y[None, :, :, None])
                  - (Y[:, None, None, :] - Y[None, :, None, :]))
    off = ~np.eye(k, dtype=bool)[None, None]
    assert np.min(np.where(off & ~np.eye(n, dtype=bool)[:, :, None, None], gaps, np.inf)) > 100 * h
    for i in range(n):
        for c in range(k):
            Yp, Ym = Y.copy(), Y.copy()
            Yp[i, c] += h
            Ym[i, c] -= h
            fd = (orc.stress_grad(Yp, nu, Delta, sd2, grad=False)[0]
                  - orc.stress_grad(Ym, nu, Delta, sd2, grad=False)[0]) / (2 * h)
            assert g[i, c] == pytest.approx(fd, rel=1e-6, abs=1e-7 * np.abs(g).max())


def test_gradient_invariants():
    # Tie-free embedding: adding c 1_k to one point leaves every distance
    # unchanged (sum_c W(R_c) = 0), so each gradient row sums to 0; moving all
    # points together changes nothing, so the rows sum to 0 too.
    for k in (2, 3, 5):
        n = 17
        Y = wl.y_init(n, k, seed=20 + k).astype(np.float64)
        Delta = orc.delta(wl.gaussian_mixture(n, 6, seed=21), [2.0])[0][0]
        sd2 = float(np.sum(np.triu(Delta, 1) ** 2))
        _, g = orc.stress_grad(Y, 2.0, Delta, sd2)
        np.testing.assert_allclose(g.sum(axis=1), 0.0, atol=1e-12 * np.abs(g).max())
        np.testing.assert_allclose(g.sum(axis=0), 0.0, atol=1e-12 * np.abs(g).max())


@pytest.mark.parametrize("k,nu", [(2, 2.0), (3, 1.5)])
def test_planted_configuration_has_zero_stress_and_gradient(k, nu):
    Ystar, D, sd2 = _planted(12, k, nu, seed=30)
    S, g = orc.stress_grad(Ystar, nu, D, sd2)
    assert S == 0.0
    assert np.all(g == 0.0)
    # and a perturbed configuration has positive stress
    S2, _ = orc.stress_grad(Ystar + 0.05 * wl.y_init(12, k, seed=31), nu, D, sd2)
    assert S2 > 0


def test_grad_rows_matches_full_gradient():
    n, k, nu = 19, 2, 2.5
    Y = wl.y_init(n, k, seed=40).astype(np.float64)
    Delta = orc.delta(wl.gaussian_outliers(n, 4, seed=41), [nu])[0][0]
    sd2 = float(np.sum(np.triu(Delta, 1) ** 2))
    _, g = orc.stress_grad(Y, nu, Delta, sd2)
    rows = np.array([0, 7, 18])
    np.testing.assert_allclose(orc.grad_rows(Y, nu, Delta[rows], rows, sd2), g[rows], rtol=1e-14)


def test_fit_is_gradient_descent_and_decreases_stress():
    n, k, nu = 25, 2, 2.0
    X = wl.gaussian_outliers(n, 10, seed=50)
    D, s = orc.delta(X, [nu])
    Y0 = wl.y_init(n, k, seed=51).astype(np.float64)
    c = 2.0 ** (1 - nu)
    eta = 0.5 * s[0] / (4 * (n - 1) * c * c)
    YT, hist = orc.fit(D[0], nu, s[0], Y0, eta, 30)
    # manual steps
    Y = Y0.copy()
    for t in range(30):
        S, g = orc.stress_grad(Y, nu, D[0], s[0])
        assert S == pytest.approx(hist[t], rel=1e-14)
        Y -= eta * g
    np.testing.assert_allclose(YT, Y, rtol=1e-14, atol=0)
    assert hist[-1] < hist[0]
    assert np.all(np.diff(hist) <= 1e-15)
