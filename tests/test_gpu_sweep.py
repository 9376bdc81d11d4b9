"""A seeded sweep of awkward sizes against the oracle: Delta for p across the
sort's segment boundaries and ragged n, several nu from one sort, every
layout/storage; stress and gradient for every k and storage form."""
import numpy as np
import pytest
import torch

from oracle import gini_oracle as orc
from paper_2605_25124_gb300 import workloads as wl
from util import ENTRY_TOL, host_col_scale, quantize, tile_pack, untile

pytestmark = pytest.mark.gpu

P_EDGES = [1, 2, 3, 4, 5, 7, 8, 9, 15, 16, 17, 31, 32, 33, 63, 64, 65, 127, 128, 129, 255, 256,
           257, 511, 512, 513, 700, 1023, 1024]


def _dist_cases():
    rng = np.random.default_rng(4040)
    cases = []
    for i, p in enumerate(P_EDGES):
        n = int(rng.choice([2, 3, 5, 17, 64, 129, 200, 257]))
        n_nu = int(rng.integers(1, 9))
        nus = sorted(set(np.round(rng.uniform(1.05, 5.0, n_nu), 3)))
        if i % 5 == 0:
            nus = [2.0]  # the positional-weight path
        cases.append((n, p, [float(v) for v in nus], ["gauss", "ties"][i % 2], i))
    return cases


def _X(data, n, p, seed):
    if data == "ties":
        return wl.integer_valued(n, p, seed=seed, levels=3)
    return wl.gaussian_outliers(n, p, seed=seed)


@pytest.mark.parametrize("n,p,nus,data,i", _dist_cases())
def test_delta_sweep(G, n, p, nus, data, i):
    X = _X(data, n, p, 4100 + i)
    Dref, sref = orc.delta(X, nus)
    Xd = torch.from_numpy(X).cuda()
    mats, sd2 = G.gini_dist(Xd, nus, layout="full")
    for v in range(len(nus)):
        got = mats[v].data.cpu().numpy().astype(np.float64)
        scale = max(np.abs(Dref[v]).max(), 1e-30)
        assert np.max(np.abs(got - Dref[v])) <= 1e-5 * scale, (v, nus[v])
        assert sd2[v].item() == pytest.approx(sref[v], rel=1e-5, abs=1e-30)
    # tiled storage of the same matrices
    tmats, _ = G.gini_dist(Xd, nus, layout="tiled", dtype="bf16x2")
    for v in range(len(nus)):
        t = tmats[v].data.view(torch.int16).cpu().numpy().view(np.uint16).astype(np.uint32)
        vals = (t << 16).view(np.float32).astype(np.float64)
        got = untile(vals, n, planes=2)
        want = np.triu(Dref[v], 1)
        assert np.max(np.abs(got - want)) <= ENTRY_TOL["bf16x2"] * max(np.abs(want).max(), 1e-30)


# nu = 2 or 3 alone: the alternating-layout network, at every boundary of its
# dispatch (segment sizes, and the register counts of 32-lane segments).
P_AFFINE = [1, 2, 3, 4, 5, 8, 9, 16, 17, 32, 33, 64, 65, 128, 129, 256, 257, 512, 513, 600, 640,
            641, 700, 767, 768, 769, 770, 784, 785, 792, 799, 800, 801, 896, 897, 1000, 1023, 1024]


@pytest.mark.parametrize("p", P_AFFINE)
@pytest.mark.parametrize("data", ["gauss", "ties"])
@pytest.mark.parametrize("nu", [2.0, 3.0])
def test_delta_affine_sweep(G, p, data, nu):
    n = 37 if p > 256 else 130
    X = _X(data, n, p, 4500 + p)
    Dref, sref = orc.delta(X, [nu])
    mats, sd2 = G.gini_dist(torch.from_numpy(X).cuda(), [nu], layout="full")
    got = mats[0].data.cpu().numpy().astype(np.float64)
    scale = max(np.abs(Dref[0]).max(), 1e-30)
    assert np.max(np.abs(got - Dref[0])) <= 1e-5 * scale
    np.testing.assert_array_equal(got, got.T)
    assert sd2[0].item() == pytest.approx(sref[0], rel=1e-5, abs=1e-30)


# Any other nu (the cell-key kernel) at the edges of the 32-lane shapes (20,
# 24, 25, 28 and 32 registers per lane): one nu (merge levels as a loop), four
# and eight nu slots.
@pytest.mark.parametrize("p", [512, 513, 640, 641, 767, 768, 769, 784, 800, 801, 896, 897])
@pytest.mark.parametrize("nus", [[1.5], [1.3, 2.0, 3.5], [1.1, 1.4, 1.8, 2.2, 2.6, 3.0, 3.9, 4.8]])
@pytest.mark.parametrize("data", ["gauss", "ties"])
def test_delta_keyed_sweep_at_the_32_lane_shapes(G, p, nus, data):
    n = 37
    X = _X(data, n, p, 4700 + p)
    Dref, sref = orc.delta(X, nus)
    mats, sd2 = G.gini_dist(torch.from_numpy(X).cuda(), nus, layout="full")
    for v in range(len(nus)):
        got = mats[v].data.cpu().numpy().astype(np.float64)
        scale = max(np.abs(Dref[v]).max(), 1e-30)
        assert np.max(np.abs(got - Dref[v])) <= 1e-5 * scale, (v, nus[v])
        np.testing.assert_array_equal(got, got.T)
        assert sd2[v].item() == pytest.approx(sref[v], rel=1e-5, abs=1e-30)


def _stress_cases():
    rng = np.random.default_rng(4200)
    cases = []
    for i in range(20):
        n = int(rng.choice([2, 3, 4, 127, 128, 129, 255, 256, 300]))
        k = int(rng.integers(2, 9))
        nu = float(np.round(rng.uniform(1.1, 4.5), 2))
        form = ["full", "f32", "bf16", "bf16x2", "fp8"][i % 5]
        cases.append((n, k, nu, form, i))
    return cases


@pytest.mark.parametrize("n,k,nu,form,i", _stress_cases())
def test_stress_grad_sweep(G, n, k, nu, form, i):
    X = wl.gaussian_outliers(n, 6, seed=4300 + i)
    D, sd2 = orc.delta(X, [nu])
    D, sd2 = D[0], float(sd2[0])
    if sd2 == 0.0:
        pytest.skip("degenerate")
    if form == "full":
        Dd = G.Dissimilarity(torch.from_numpy(D.astype(np.float32)).cuda(), n, "full", "f32", sd2)
        Dq = quantize(D, "f32")
    else:
        sc = host_col_scale(D) if form == "fp8" else None
        Dd = G.Dissimilarity(torch.from_numpy(tile_pack(D, n, form, sc)).cuda(), n, "tiled", form,
                             sd2, torch.from_numpy(sc).cuda() if sc is not None else None)
        Dq = quantize(D, form, sc)
    Dq = np.triu(Dq, 1) + np.triu(Dq, 1).T
    Y = wl.y_init(n, k, seed=4400 + i, sd=1.0)
    Sref, gref = orc.stress_grad(Y.astype(np.float64), nu, Dq, sd2)
    S, g = G.gini_stress_grad(torch.from_numpy(Y).cuda(), nu, Dd)
    assert float(S) == pytest.approx(Sref, rel=1e-5, abs=1e-12)
    assert np.max(np.abs(g.cpu().numpy() - gref)) <= 1e-5 * max(np.abs(gref).max(), 1e-30)


@pytest.mark.parametrize("n", [2, 3, 4, 127, 128, 129, 255, 256, 257])
@pytest.mark.parametrize("nu,form", [(1.7, "f32"), (2.0, "bf16x2"), (2.0, "fp8"), (3.3, "bf16")])
def test_stress_grad_k3_every_tile_shape(G, n, nu, form):
    """k = 3 with the Gini metric and Kruskal loss (the bulk-copy kernel, both
    its general and its affine body) from one point pair to several tiles with
    ragged edges, against the oracle on the same stored values."""
    X = wl.gaussian_outliers(n, 5, seed=4500 + n)
    D, sd2 = orc.delta(X, [nu])
    D, sd2 = D[0], float(sd2[0])
    if sd2 == 0.0:
        pytest.skip("degenerate")
    sc = host_col_scale(D) if form == "fp8" else None
    Dd = G.Dissimilarity(torch.from_numpy(tile_pack(D, n, form, sc)).cuda(), n, "tiled", form,
                         sd2, torch.from_numpy(sc).cuda() if sc is not None else None)
    Dq = quantize(D, form, sc)
    Dq = np.triu(Dq, 1) + np.triu(Dq, 1).T
    Y = wl.y_init(n, 3, seed=4600 + n, sd=1.0)
    Sref, gref = orc.stress_grad(Y.astype(np.float64), nu, Dq, sd2)
    S, g = G.gini_stress_grad(torch.from_numpy(Y).cuda(), nu, Dd)
    assert float(S) == pytest.approx(Sref, rel=1e-5, abs=1e-12)
    assert np.max(np.abs(g.cpu().numpy() - gref)) <= 1e-5 * np.abs(gref).max() + 1e-12
