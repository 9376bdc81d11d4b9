"""gini_dist (Delta build) on the GPU against the FP64 oracle.

Tolerances (per entry relative, with a floor of 1e-6 x the largest entry for
near-zero dissimilarities, and norm-wise): FP32 1e-5 / 1e-5; BF16 2^-8 (the
round-to-nearest bound of an 8-bit significand) / 2e-3; BF16 hi+lo 2^-16 /
1e-5; FP8 e4m3 against its rounding bound.
"""
import numpy as np
import pytest
import torch

from oracle import gini_oracle as orc
from paper_2605_25124_gb300 import workloads as wl
from util import ENTRY_TOL, NORM_TOL, fro_rel, rel_err, tiled_flat_index, untile

pytestmark = pytest.mark.gpu


def _gpu_full(G, X, nus):
    mats, sd2 = G.gini_dist(torch.from_numpy(X).cuda(), nus, layout="full")
    return [m.data.cpu().numpy().astype(np.float64) for m in mats], sd2.cpu().numpy()


def _check_full(got, ref, tol=1e-5):
    floor = 1e-6 * np.abs(ref).max()
    assert rel_err(got, ref, floor) <= tol
    np.testing.assert_array_equal(got, got.T)
    assert np.all(np.diag(got) == 0)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 7, 10, 16, 33, 50, 64, 100, 129, 300, 784, 1024])
def test_delta_full_f32_all_vector_lengths(G, p):
    n = 41 if p < 300 else 23
    X = wl.gaussian_outliers(n, p, seed=100 + p)
    nus = [1.5, 2.0, 3.0]
    ref, sref = orc.delta(X, nus)
    got, sd2 = _gpu_full(G, X, nus)
    for q in range(3):
        _check_full(got[q], ref[q])
        assert sd2[q] == pytest.approx(sref[q], rel=1e-5)


@pytest.mark.parametrize("nu", [2.0, 3.0, 1.1, 4.5])
def test_delta_single_nu_paths(G, nu):
    # nu = 2 or 3 alone takes the positional-weight path; other nu the tie-run path.
    X = wl.image_like(30, seed=7)
    ref, sref = orc.delta(X, [nu])
    got, sd2 = _gpu_full(G, X, [nu])
    _check_full(got[0], ref[0])
    assert sd2[0] == pytest.approx(sref[0], rel=1e-5)


def test_delta_ties_integer_and_image_data(G):
    for X in (wl.integer_valued(60, 50, seed=8), wl.image_like(40, seed=9),
              wl.uci_like_batch(4, seed=10)[3][:50]):
        nus = [1.5, 2.0, 3.0]
        ref, _ = orc.delta(X, nus)
        got, _ = _gpu_full(G, X, nus)
        for q in range(3):
            _check_full(got[q], ref[q])


def test_delta_affine_path_equals_table_path(G):
    X = wl.image_like(50, seed=11)
    a, _ = _gpu_full(G, X, [2.0])
    b, _ = _gpu_full(G, X, [2.0, 2.0])
    assert rel_err(a[0], b[0], 1e-6 * np.abs(a[0]).max()) <= 2e-6


@pytest.mark.parametrize("dtype", ["f32", "bf16", "bf16x2"])
def test_delta_tiled_layouts(G, dtype):
    n = 300  # 3 tiles per edge, ragged tail of 44
    X = wl.gaussian_mixture(n, 20, seed=12)
    nus = [1.5, 2.0]
    ref, sref = orc.delta(X, nus)
    mats, sd2 = G.gini_dist(torch.from_numpy(X).cuda(), nus, layout="tiled", dtype=dtype)
    planes = 2 if dtype == "bf16x2" else 1
    for q in range(2):
        flat = mats[q].data.float().cpu().numpy()
        got = untile(flat, n, planes)
        iu = np.triu_indices(n, 1)
        floor = 1e-6 * np.abs(ref[q]).max()
        assert rel_err(got[iu], ref[q][iu], floor) <= ENTRY_TOL[dtype]
        assert fro_rel(got[iu], ref[q][iu]) <= NORM_TOL[dtype]
        assert sd2.cpu().numpy()[q] == pytest.approx(sref[q], rel=1e-5)


def test_pack_from_full(G):
    n = 260
    X = wl.gaussian_outliers(n, 9, seed=13)
    ref, _ = orc.delta(X, [1.8])
    mats, _ = G.gini_dist(torch.from_numpy(X).cuda(), [1.8], layout="full")
    iu = np.triu_indices(n, 1)
    floor = 1e-6 * np.abs(ref[0]).max()
    for dtype in ("f32", "bf16", "bf16x2"):
        P = G.gini_pack(mats[0], dtype)
        got = untile(P.data.float().cpu().numpy(), n, 2 if dtype == "bf16x2" else 1)
        assert rel_err(got[iu], ref[0][iu], floor) <= ENTRY_TOL[dtype], dtype
        assert fro_rel(got[iu], ref[0][iu]) <= NORM_TOL[dtype], dtype
    P = G.gini_pack(mats[0], "fp8")
    q = P.data.cpu().numpy().view(np.uint8)
    sc = P.col_scale.cpu().numpy()
    # decode e4m3 on the host (sign, 4-bit exponent with bias 7, 3-bit mantissa)
    s = np.where(q & 0x80, -1.0, 1.0)
    e = (q >> 3) & 0xF
    mant = (q & 7).astype(np.float64)
    val = s * np.where(e == 0, mant / 8 * 2.0 ** -6, (1 + mant / 8) * 2.0 ** (e.astype(np.float64) - 7))
    T = -(-n // 128)
    full = untile(val, n) * sc[None, :]
    err = np.abs(full[iu] - ref[0][iu])
    # normal e4m3: half an ulp of a 3-bit mantissa (2^-4 relative); subnormal: 2^-10 absolute
    bound = 2.0 ** -4 * np.abs(ref[0][iu]) + 2.0 ** -10 * sc[iu[1]]
    assert np.all(err <= bound + 1e-6)
    colmax = np.max(np.triu(ref[0], 1), axis=0)
    np.testing.assert_allclose(sc[1:], np.where(colmax[1:] > 0, colmax[1:] / 448, 1), rtol=1e-5)
    assert T >= 3


def test_delta_full_size_image_workload_sampled(G):
    """n = 2000, p = 784, nu in {1.5, 2, 3}: the whole matrix on the GPU,
    300 sampled pairs (and one full row) from the oracle."""
    w = wl.WORKLOADS["image-n2000-p784"]
    X = wl.make_X("image-n2000-p784")
    mats, sd2 = G.gini_dist(torch.from_numpy(X).cuda(), w["nu"], layout="full")
    rng = np.random.default_rng(14)
    I = rng.integers(0, w["n"], 300)
    J = rng.integers(0, w["n"], 300)
    I = np.concatenate([I, np.full(w["n"], 1234)])
    J = np.concatenate([J, np.arange(w["n"])])
    ref = orc.delta_pairs(X, w["nu"], I, J)
    for q in range(3):
        got = mats[q].data[torch.from_numpy(I).cuda(), torch.from_numpy(J).cuda()].cpu().numpy()
        assert rel_err(got, ref[:, q], 1e-6 * np.abs(ref[:, q]).max()) <= 1e-5
    # sum of squares by symmetry of the stored square
    for q in range(3):
        d = mats[q].data.double()
        assert sd2[q].item() == pytest.approx(0.5 * float((d * d).sum()), rel=1e-9)


def _e4m3_decode(q):
    """e4m3 bytes -> float64 (sign, 4-bit exponent with bias 7, 3-bit mantissa)."""
    q = np.asarray(q, dtype=np.uint8)
    s = np.where(q & 0x80, -1.0, 1.0)
    e = ((q >> 3) & 0xF).astype(np.float64)
    m = (q & 7).astype(np.float64)
    return s * np.where(e == 0, m / 8 * 2.0 ** -6, (1 + m / 8) * 2.0 ** (e - 7))


def test_delta_storage_forms_at_the_image_configuration(G):
    """n = 2000, p = 784, nu in {1.5, 2, 3}: the tiled BF16, BF16 hi+lo and
    FP8 e4m3 (per-column scale) outputs of gini_dist against the FP64 oracle on
    2,000 sampled pairs and one whole row, each within its storage bound:
    bf16 round-to-nearest 2^-8 relative, hi+lo 2^-16, e4m3 half an ulp of a
    3-bit mantissa (2^-4 relative) or 2^-10 of the column scale near zero; plus
    the FP32 build's own 1e-5.  The worst errors are printed for the record."""
    w = wl.WORKLOADS["image-n2000-p784"]
    n, nus = w["n"], [float(v) for v in w["nu"]]
    X = wl.make_X("image-n2000-p784")
    rng = np.random.default_rng(2024)
    I = rng.integers(0, n, 2000)
    J = rng.integers(0, n, 2000)
    keep = I != J
    I, J = np.minimum(I[keep], J[keep]), np.maximum(I[keep], J[keep])
    row = 777
    I = np.concatenate([I, np.full(n - 1 - row, row), np.arange(row)])
    J = np.concatenate([J, np.arange(row + 1, n), np.full(row, row)])
    ref = orc.delta_pairs(X, nus, I, J)  # (pairs, nu)
    idx = tiled_flat_index(I, J, n)
    plane = -(-n // 128) * (-(-n // 128) + 1) // 2 * 128 * 128
    Xd = torch.from_numpy(X).cuda()
    worst = {}
    for dtype in ("bf16", "bf16x2", "fp8"):
        mats, _ = G.gini_dist(Xd, nus, layout="tiled", dtype=dtype)
        for q in range(len(nus)):
            r = ref[:, q]
            if dtype == "fp8":
                got = _e4m3_decode(mats[q].data.cpu().numpy()[idx])
                sc = mats[q].col_scale.cpu().numpy().astype(np.float64)[J]
                got = got * sc
                err = np.abs(got - r)
                bound = (2.0 ** -4 + 1e-5) * np.abs(r) + 2.0 ** -10 * sc + 1e-7
                assert np.all(err <= bound), (q, float(np.max(err / bound)))
                worst[(dtype, nus[q])] = float(np.max(err / np.abs(r).max()))
            else:
                bits = mats[q].data.view(torch.int16).cpu().numpy().astype(np.uint16)
                hi = (bits[idx].astype(np.uint32) << 16).view(np.float32).astype(np.float64)
                got = hi
                if dtype == "bf16x2":
                    lo = (bits[plane + idx].astype(np.uint32) << 16).view(np.float32)
                    got = hi + lo.astype(np.float64)
                tol = (2.0 ** -8 if dtype == "bf16" else 2.0 ** -16) + 1e-5
                e = rel_err(got, r, 1e-6 * np.abs(r).max())
                assert e <= tol, (dtype, q, e)
                worst[(dtype, nus[q])] = e
    print("worst entry errors against the FP64 oracle:",
          {f"{k[0]} nu={k[1]}": f"{v:.2e}" for k, v in worst.items()})


def test_delta_nonfinite_reported(G):
    from paper_2605_25124_gb300._lib import GiniError
    X = wl.gaussian_outliers(20, 6, seed=15)
    X[3, 2] = np.inf
    with pytest.raises(GiniError, match="ENONFINITE"):
        G.gini_dist(torch.from_numpy(X).cuda(), [2.0])


def test_delta_two_points_worked_example(G):
    X = np.array([[10, 1200], [10, 12]], dtype=np.float32)
    mats, sd2 = G.gini_dist(torch.from_numpy(X).cuda(), [2.0, 1.5, 3.0])
    for q, nu in enumerate([2.0, 1.5, 3.0]):
        assert mats[q].data[0, 1].item() == pytest.approx(1188 * 2.0 ** (1 - nu), rel=1e-6)


@pytest.mark.parametrize("p", [40, 784])
@pytest.mark.parametrize("nus", [[1.3], [1.3, 2.0, 3.7]])
def test_delta_exact_order_of_colliding_differences(G, nus, p):
    # 1 - 2^-25 rounds to 1.0f: in the pair (0, 1) it meets an exact 1.0 at the
    # top of the order, where W is steepest for nu < 2.  The two differences are
    # distinct, so their ranks must differ as in the exact (oracle) order.
    # (p = 784: 25 registers per lane, the colliding pair in lanes 0 and 1.)
    rng = np.random.default_rng(5000)
    n = 24
    X = rng.standard_normal((n, p)).astype(np.float32)
    X[0, :2] = [1.0, 1.0]
    X[1, :2] = [2.0 ** -25, 0.0]
    X[0, 2:] = rng.uniform(-0.5, 0.5, p - 2).astype(np.float32)
    X[1, 2:] = rng.uniform(-0.5, 0.5, p - 2).astype(np.float32)
    z = X[0].astype(np.float32) - X[1].astype(np.float32)
    assert z[0] == z[1] == 1.0  # the collision really happens in FP32
    D, sd2 = orc.delta(X, nus)
    mats, s2 = G.gini_dist(torch.from_numpy(X).cuda(), nus, layout="full")
    for v in range(len(nus)):
        got = mats[v].data.cpu().numpy().astype(np.float64)
        assert abs(got[0, 1] - D[v][0, 1]) <= 1e-6 * abs(D[v][0, 1]), (nus[v], got[0, 1], D[v][0, 1])
        assert np.max(np.abs(got - D[v])) <= 1e-5 * np.abs(D[v]).max()
        assert s2[v].item() == pytest.approx(sd2[v], rel=1e-6)
    tm, _ = G.gini_dist(torch.from_numpy(X).cuda(), nus, layout="tiled", dtype="f32")
    for v in range(len(nus)):
        got = untile(tm[v].data.cpu().numpy(), n)
        assert abs(got[0, 1] - D[v][0, 1]) <= 1e-6 * abs(D[v][0, 1])


@pytest.mark.parametrize("p", [5, 33, 784])
@pytest.mark.parametrize("nus", [[2.0], [1.5, 3.0]])
def test_delta_rows_differing_by_a_constant_vector_are_zero(G, p, nus):
    # x_i - x_j = (c_i - c_j) * 1: every component ties, the midrank is (m+1)/2
    # where W vanishes, so delta = 0 exactly (translation invariance); integer
    # data keep the differences exact in FP32.  A fit on it is degenerate.
    from paper_2605_25124_gb300._lib import GiniError
    rng = np.random.default_rng(900 + p)
    n = 70
    base = rng.integers(-20, 20, p).astype(np.float32)
    c = rng.integers(-50, 50, n).astype(np.float32)
    X = base[None, :] + c[:, None]
    mats, sd2 = G.gini_dist(torch.from_numpy(X).cuda(), nus, layout="full")
    for v in range(len(nus)):
        assert float(mats[v].data.abs().max()) == 0.0
        assert float(sd2[v]) == 0.0
    D = mats[0]
    Y0 = torch.from_numpy(wl.y_init(n, 2, seed=901)).cuda()
    with pytest.raises(GiniError, match="EDEGENERATE"):
        G.gini_mds_fit(Y0, nus[0], D, 1.0, 3, history=False)


@pytest.mark.parametrize("p", [47, 784])
@pytest.mark.parametrize("nus", [[1.3], [1.3, 2.0, 3.7, 5.0]])
def test_delta_exact_order_within_one_fp32_cell(G, nus, p):
    # Three differences strictly between 1 and the next float up, two of them
    # equal: 1 + 2^-26 (twice) and 1 + 2^-25.  Their cell keys tie; the exact
    # order (and the tie of the equal two) must still give the oracle's ranks.
    rng = np.random.default_rng(5100)
    n = 20
    X = rng.uniform(-0.5, 0.5, (n, p)).astype(np.float32)
    X[0, :3] = [1.0, 1.0, 1.0]
    X[1, :3] = [-2.0 ** -26, -2.0 ** -25, -2.0 ** -26]
    z = X[0].astype(np.float32) - X[1].astype(np.float32)
    assert z[0] == z[1] == z[2] == 1.0  # all three round to 1.0f
    D, sd2 = orc.delta(X, nus)
    for layout in ("full", "tiled"):
        mats, s2 = G.gini_dist(torch.from_numpy(X).cuda(), nus, layout=layout, dtype="f32")
        for v in range(len(nus)):
            got = mats[v].data.cpu().numpy().astype(np.float64)
            if layout == "tiled":
                got = untile(got, n)
                got = got + got.T
            assert abs(got[0, 1] - D[v][0, 1]) <= 2e-6 * abs(D[v][0, 1]), (nus[v], layout)
            assert np.max(np.abs(got - D[v])) <= 1e-5 * np.abs(D[v]).max()
            assert s2[v].item() == pytest.approx(sd2[v], rel=1e-6)


@pytest.mark.parametrize("p", [6, 100, 784])
def test_delta_wide_range_data_take_the_64bit_network(G, p):
    # A range of 1e4 with nonzero values near 1e-38: scaling the cell keys by
    # 2^-14 would push those below the normal range, so the pre-pass sends the
    # build to the 64-bit TwoSum network.  Results must match the oracle.
    rng = np.random.default_rng(5200 + p)
    n = 33
    X = (rng.standard_normal((n, p)) * 3000).astype(np.float32)
    X[rng.integers(0, n, 8), rng.integers(0, p, 8)] = np.float32(3e-38)
    nus = [1.7, 2.5]
    D, sd2 = orc.delta(X, nus)
    mats, s2 = G.gini_dist(torch.from_numpy(X).cuda(), nus, layout="full")
    for v in range(2):
        got = mats[v].data.cpu().numpy().astype(np.float64)
        _check_full(got, D[v])
        assert s2[v].item() == pytest.approx(sd2[v], rel=1e-5)


def test_delta_sum_of_squares_is_run_to_run_identical(G):
    # Sum delta^2 is accumulated exactly (128-bit integer units), so repeated
    # builds return the same bits whatever order the CTAs finish in.
    X = torch.from_numpy(wl.make_X("image-n2000-p784")[:1500]).cuda()
    for nus in ([2.0], [1.5, 3.0]):
        a = [G.gini_dist(X, nus, layout="tiled", dtype="f32")[1].cpu().numpy() for _ in range(3)]
        for b in a[1:]:
            np.testing.assert_array_equal(a[0], b)


def _e4m3_decode(q):
    q = np.asarray(q).view(np.uint8)
    s = np.where(q & 0x80, -1.0, 1.0)
    e = (q >> 3) & 0xF
    mant = (q & 7).astype(np.float64)
    return s * np.where(e == 0, mant / 8 * 2.0 ** -6, (1 + mant / 8) * 2.0 ** (e.astype(np.float64) - 7))


@pytest.mark.parametrize("strips", ["one", "many"])
def test_delta_fp8_output_direct(G, strips):
    # gini_dist writing e4m3 tiles with per-column scales itself: against the
    # oracle at the e4m3 bound, and bit for bit against packing the FULL FP32
    # build (same values, same scale rule).  "many": a workspace with room for
    # one tile column of FP32 scratch, so the build runs strip by strip.
    import ctypes
    from paper_2605_25124_gb300._lib import DTYPES, LAYOUTS, OPS, lib
    n, nus = 300, [1.6, 2.0]
    X = wl.gaussian_outliers(n, 11, seed=5300)
    ref, sref = orc.delta(X, nus)
    Xd = torch.from_numpy(X).cuda()
    L = lib()
    plane = G.tiled_elems(n)
    out = torch.zeros(2 * plane, dtype=torch.uint8, device="cuda")
    scale = torch.empty(2 * n, dtype=torch.float32, device="cuda")
    sd2 = torch.zeros(2, dtype=torch.float64, device="cuda")
    base = L.gini_workspace_size(OPS["dist"], n, 11, 0, 0)
    full = L.gini_workspace_size(OPS["dist_fp8"], n, 11, 0, 0)
    nbytes = base + 4 * n * 128 * 2 if strips == "many" else full
    assert nbytes <= full
    ws = torch.zeros(nbytes, dtype=torch.uint8, device="cuda")
    nu_arr = (ctypes.c_double * 2)(*nus)
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    st = L.gini_dist(p(Xd), n, 11, 11, nu_arr, 2, LAYOUTS["tiled"], DTYPES["fp8"], p(out), 0,
                     plane, p(scale), p(sd2), p(ws), nbytes,
                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    torch.cuda.synchronize()
    iu = np.triu_indices(n, 1)
    mats, _ = G.gini_dist(Xd, nus, layout="full")
    for q in range(2):
        sc = scale[q * n:(q + 1) * n].cpu().numpy()
        got = untile(_e4m3_decode(out[q * plane:(q + 1) * plane].cpu().numpy()), n) * sc[None, :]
        err = np.abs(got[iu] - ref[q][iu])
        bound = 2.0 ** -4 * np.abs(ref[q][iu]) + 2.0 ** -10 * sc[iu[1]]
        assert np.all(err <= bound + 1e-6)
        colmax = np.max(np.triu(ref[q], 1), axis=0)
        np.testing.assert_allclose(sc[1:], np.where(colmax[1:] > 0, colmax[1:] / 448, 1),
                                   rtol=1e-5)
        assert sd2[q].item() == pytest.approx(sref[q], rel=1e-6)
        P = G.gini_pack(mats[q], "fp8")
        assert torch.equal(P.col_scale, scale[q * n:(q + 1) * n])
        assert torch.equal(P.data, out[q * plane:(q + 1) * plane])
    # the Python binding's FP8 path and a stress evaluation on it
    m8, _ = G.gini_dist(Xd, nus, layout="tiled", dtype="fp8")
    assert torch.equal(m8[0].data, out[:plane]) and torch.equal(m8[0].col_scale, scale[:n])


@pytest.mark.parametrize("p", [1025, 2048, 3072])
@pytest.mark.parametrize("nus", [[2.0], [1.5, 2.0, 3.0]])
def test_delta_vectors_longer_than_a_warp(G, p, nus):
    # 1024 < p: the pair's differences are sorted in 1024-slot chunks and
    # ranked by search; exact (hi, lo) order for every nu, ties included.
    n = 19
    rng = np.random.default_rng(5400 + p)
    X = rng.standard_normal((n, p)).astype(np.float32)
    X[:, ::7] = np.round(X[:, ::7])  # ties within and across chunks
    X[5] = np.round(X[5] * 8) / 8     # multiples of 1/8: adding 1/4 is exact,
    X[3] = X[5] + np.float32(0.25)   # so this pair's differences all tie
    ref, sref = orc.delta(X, nus)
    got, sd2 = _gpu_full(G, X, nus)
    for q in range(len(nus)):
        _check_full(got[q], ref[q])
        assert sd2[q] == pytest.approx(sref[q], rel=1e-5)
    assert np.all(got[0][3, 5] == 0.0)
    mats, _ = G.gini_dist(torch.from_numpy(X).cuda(), nus, layout="tiled", dtype="bf16x2")
    iu = np.triu_indices(n, 1)
    for q in range(len(nus)):
        t = untile(mats[q].data.float().cpu().numpy(), n, 2)
        assert rel_err(t[iu], ref[q][iu], 1e-6 * np.abs(ref[q]).max()) <= ENTRY_TOL["bf16x2"]
