"""ctypes binding of the FP64 CPU oracle (gini_oracle.c).

TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and the CPU-baseline
/ reference arm of bench.py are the only users.  The product path never imports
this module.  The per-pair and per-iteration functions forward to the C oracle,
whose header lists the paper passages each routine follows; classical_mds is
the textbook definition in numpy (its eigensolver a library step); nu_search
composes delta and fit in the loops of Algorithm 1 and alternating_nu those of
Algorithm 2; default_step is the step rule's formula; the evaluation measures
of Section V (trustworthiness, NN(k), silhouette, distance correlations) are
their definitions in numpy.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gini_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liborcgini.so")
_lib = None

_F64P = ctypes.POINTER(ctypes.c_double)
_F32P = ctypes.POINTER(ctypes.c_float)
_I64P = ctypes.POINTER(ctypes.c_int64)
_I32P = ctypes.POINTER(ctypes.c_int32)
_I64 = ctypes.c_int64


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (IEEE double, no contraction, OpenMP)."""
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_OUT), exist_ok=True)
        tmp = _OUT + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp",
                               "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_OUT)
        L.orc_midrank2.argtypes = [_F64P, _I64, _I32P]
        L.orc_gini_norm.argtypes = [_F64P, _I64]
        L.orc_gini_norm.restype = ctypes.c_double
        L.orc_gini_dg.argtypes = [_F64P, _F64P, _I64]
        L.orc_gini_dg.restype = ctypes.c_double
        L.orc_pd.argtypes = [_F64P, _F64P, _I64, ctypes.c_double]
        L.orc_pd.restype = ctypes.c_double
        L.orc_pd_grad.argtypes = [_F64P, _F64P, _I64, ctypes.c_double, _F64P]
        L.orc_pd_grad.restype = ctypes.c_double
        L.orc_delta.argtypes = [_F32P, _I64, _I64, _I64, _F64P, ctypes.c_int, _F64P, _F64P]
        L.orc_delta_pairs.argtypes = [_F32P, _I64, _I64, _I64, _F64P, ctypes.c_int,
                                      _I64P, _I64P, _I64, _F64P]
        L.orc_embed_dist_pairs.argtypes = [_F64P, _I64, ctypes.c_int, ctypes.c_double,
                                           _I64P, _I64P, _I64, _F64P]
        L.orc_stress_grad.argtypes = [_F64P, _I64, ctypes.c_int, ctypes.c_double, _F64P,
                                      _I64, ctypes.c_double, _F64P]
        L.orc_stress_grad.restype = ctypes.c_double
        L.orc_grad_rows.argtypes = [_F64P, _I64, ctypes.c_int, ctypes.c_double, _F64P,
                                    _I64P, _I64, ctypes.c_double, _F64P]
        L.orc_fit.argtypes = [_F64P, _I64, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                              ctypes.c_double, ctypes.c_int, _F64P, _F64P]
        L.orc_stress_grad_ex.argtypes = [_F64P, _I64, ctypes.c_int, ctypes.c_double, _F64P,
                                         _I64, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                         _F64P]
        L.orc_stress_grad_ex.restype = ctypes.c_double
        L.orc_set_threads.argtypes = [ctypes.c_int]
        L.orc_get_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def set_threads(t: int) -> None:
    lib().orc_set_threads(int(t))


def get_threads() -> int:
    return int(lib().orc_get_threads())


def midrank2(v) -> np.ndarray:
    """Twice the midrank of each element of one vector."""
    v = _f64(v)
    out = np.empty(v.shape[0], dtype=np.int32)
    lib().orc_midrank2(_p(v, _F64P), v.shape[0], _p(out, _I32P))
    return out


def gini_norm(x) -> float:
    x = _f64(x)
    return float(lib().orc_gini_norm(_p(x, _F64P), x.shape[0]))


def gini_dg(x, y) -> float:
    x, y = _f64(x), _f64(y)
    return float(lib().orc_gini_dg(_p(x, _F64P), _p(y, _F64P), x.shape[0]))


def pd(x, y, nu: float) -> float:
    """Symmetrized generalized Gini pseudo-distance of two vectors."""
    x, y = _f64(x), _f64(y)
    return float(lib().orc_pd(_p(x, _F64P), _p(y, _F64P), x.shape[0], float(nu)))


def pd_grad(x, y, nu: float):
    """(Dbar(x, y), dDbar/dz) with z = x - y, ranks held fixed."""
    x, y = _f64(x), _f64(y)
    dz = np.empty(x.shape[0], dtype=np.float64)
    v = lib().orc_pd_grad(_p(x, _F64P), _p(y, _F64P), x.shape[0], float(nu), _p(dz, _F64P))
    return float(v), dz


def delta(X, nus):
    """Full Delta (len(nus), n, n) and sum_{i<j} delta^2 per nu."""
    X = _f32(X)
    nus = _f64(np.atleast_1d(nus))
    n, p = X.shape
    D = np.empty((nus.shape[0], n, n), dtype=np.float64)
    s = np.empty(nus.shape[0], dtype=np.float64)
    lib().orc_delta(_p(X, _F32P), n, p, p, _p(nus, _F64P), nus.shape[0], _p(D, _F64P),
                    _p(s, _F64P))
    return D, s


def delta_pairs(X, nus, I, J) -> np.ndarray:
    """delta for listed pairs, shape (npairs, len(nus))."""
    X = _f32(X)
    nus = _f64(np.atleast_1d(nus))
    I = np.ascontiguousarray(I, dtype=np.int64)
    J = np.ascontiguousarray(J, dtype=np.int64)
    n, p = X.shape
    out = np.empty((I.shape[0], nus.shape[0]), dtype=np.float64)
    lib().orc_delta_pairs(_p(X, _F32P), n, p, p, _p(nus, _F64P), nus.shape[0],
                          _p(I, _I64P), _p(J, _I64P), I.shape[0], _p(out, _F64P))
    return out


def embed_dist_pairs(Y, nu, I, J) -> np.ndarray:
    Y = _f64(Y)
    I = np.ascontiguousarray(I, dtype=np.int64)
    J = np.ascontiguousarray(J, dtype=np.int64)
    out = np.empty(I.shape[0], dtype=np.float64)
    lib().orc_embed_dist_pairs(_p(Y, _F64P), Y.shape[0], Y.shape[1], float(nu),
                               _p(I, _I64P), _p(J, _I64P), I.shape[0], _p(out, _F64P))
    return out


def stress_grad(Y, nu, Delta, sum_delta2, grad: bool = True):
    """(S, dS/dY or None) with S = sum_{i<j} r_ij^2 / sum_delta2."""
    Y = _f64(Y)
    Delta = _f64(Delta)
    n, k = Y.shape
    g = np.empty((n, k), dtype=np.float64) if grad else None
    S = lib().orc_stress_grad(_p(Y, _F64P), n, k, float(nu), _p(Delta, _F64P),
                              Delta.shape[1], float(sum_delta2),
                              _p(g, _F64P) if grad else None)
    return float(S), g


def grad_rows(Y, nu, Delta_rows, rows, sum_delta2) -> np.ndarray:
    Y = _f64(Y)
    Delta_rows = _f64(Delta_rows)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    n, k = Y.shape
    g = np.empty((rows.shape[0], k), dtype=np.float64)
    lib().orc_grad_rows(_p(Y, _F64P), n, k, float(nu), _p(Delta_rows, _F64P),
                        _p(rows, _I64P), rows.shape[0], float(sum_delta2), _p(g, _F64P))
    return g


def fit(Delta, nu, sum_delta2, Y0, eta, T):
    """T fixed-step GD iterations; returns (Y_T, history[T+1])."""
    Delta = _f64(Delta)
    Y = _f64(Y0).copy()
    n, k = Y.shape
    h = np.empty(T + 1, dtype=np.float64)
    lib().orc_fit(_p(Delta, _F64P), n, k, float(nu), float(sum_delta2), float(eta), int(T),
                  _p(Y, _F64P), _p(h, _F64P))
    return Y, h


METRICS = {"gini": 0, "euclid": 1}
LOSSES = {"kruskal": 0, "sammon": 1}


def stress_grad_ex(Y, nu, Delta, norm, metric="gini", loss="kruskal", grad: bool = True):
    """(S, dS/dY or None) for metric "gini"/"euclid" and loss "kruskal"/"sammon";
    norm = sum delta^2 (Kruskal) or sum delta (Sammon) over i<j."""
    Y = _f64(Y)
    Delta = _f64(Delta)
    n, k = Y.shape
    g = np.empty((n, k), dtype=np.float64) if grad else None
    S = lib().orc_stress_grad_ex(_p(Y, _F64P), n, k, float(nu), _p(Delta, _F64P),
                                 Delta.shape[1], METRICS[metric], LOSSES[loss], float(norm),
                                 _p(g, _F64P) if grad else None)
    return float(S), g


def classical_mds(Delta, k: int):
    """Classical MDS (Section IV-A) written as its definition: B = -1/2 H D2 H,
    eigenpairs by numpy's symmetric eigensolver (a library step), the top k by
    value, Y = V_k Lambda_k^{1/2} (negative eigenvalues give zero columns).
    Returns (Y, eigenvalues descending)."""
    D = np.asarray(Delta, dtype=np.float64)
    n = D.shape[0]
    H = np.eye(n) - np.full((n, n), 1.0 / n)
    B = -0.5 * H @ (D * D) @ H
    w, V = np.linalg.eigh(B)
    idx = np.argsort(w)[::-1][:k]
    lam = w[idx]
    return V[:, idx] * np.sqrt(np.maximum(lam, 0.0)), lam


def default_step(n, k, nu, sum_delta2, eta0=1.0):
    """The fixed step the fits use (the paper gives none): eta0 over a
    Gershgorin bound on the Gauss-Newton curvature of S,
    eta0 * sum_delta2 / (2 (n-1) k ((k/2) w_max)^2), w_max = ((k-1)/k)^(nu-1)."""
    if n < 2:
        return 0.0
    w = ((k - 1) / k) ** (nu - 1.0)
    return eta0 * sum_delta2 / (2.0 * (n - 1) * k * (0.5 * k * w) ** 2)


def nu_search(X, folds, nus, Y0, iters, eta0=1.0):
    """Algorithm 1 as written: for each nu, for each fold, the fold's Delta,
    `iters` fixed-step GD iterations from each start (Y0: restarts x n x 2, in
    point order), KS = sqrt(S(Y_T)) of the best start; nu* = argmin of the mean
    KS over folds (the first minimiser).  Returns (ks (n_nu, K), mean_ks, best,
    Y (n, 2) of nu*'s fits)."""
    X = np.asarray(X, dtype=np.float32)
    folds = np.asarray(folds)
    Y0 = np.asarray(Y0, dtype=np.float64)
    K = int(folds.max()) + 1
    n = X.shape[0]
    ks = np.empty((len(nus), K))
    Ys = np.empty((len(nus), n, 2))
    for q in range(K):
        idx = np.flatnonzero(folds == q)  # increasing point order
        D, sd2 = delta(X[idx], nus)
        for v, nu in enumerate(nus):
            eta = default_step(len(idx), 2, nu, sd2[v], eta0)
            best = np.inf
            for r in range(Y0.shape[0]):
                Yr, h = fit(D[v], nu, sd2[v], Y0[r][idx], eta, iters)
                if h[-1] < best:
                    best = h[-1]
                    Ys[v][idx] = Yr
            ks[v, q] = np.sqrt(best)
    mean_ks = ks.mean(axis=1)
    b = int(np.argmin(mean_ks))
    return ks, mean_ks, b, Ys[b]


def _curv(metric, k, nu):
    if metric == "euclid":
        return 1.0
    w = ((k - 1) / k) ** (nu - 1.0)
    return k * (0.5 * k * w) ** 2


def alternating_nu(X, nus, nu_start, rounds, iters, Y0, eta0=1.0, metric="gini",
                   loss="sammon"):
    """Algorithm 2's alternation as written: fit at the current nu (fixed-step
    GD on the loss, warm-started), then nu <- the first grid value minimising
    the Kruskal stress KS(nu) of the fixed embedding.  The step is eta0 over a
    Gershgorin bound on the Gauss-Newton curvature (Kruskal:
    sum delta^2 / (2 (n-1) c), Sammon: sum delta / (2 c max_i sum_j 1/delta_ij)).
    Returns (Y, nu path, KS table (rounds, n_nu))."""
    allnus = list(nus) + [nu_start]
    D, s2 = delta(X, allnus)
    n = D.shape[1]
    iu = np.triu_indices(n, 1)
    s1 = np.array([D[v][iu].sum() for v in range(len(allnus))])
    Y = np.array(Y0, dtype=np.float64)
    k = Y.shape[1]
    cur = len(nus)
    path, table = [nu_start], []
    for _ in range(rounds):
        nu = allnus[cur]
        c = _curv(metric, k, nu)
        if loss == "kruskal":
            norm = s2[cur]
            eta = eta0 * norm / (2.0 * (n - 1) * c)
        else:
            norm = s1[cur]
            Dc = D[cur].copy()
            np.fill_diagonal(Dc, 0.0)
            inv = np.where(Dc > 0, 1.0 / np.where(Dc > 0, Dc, 1.0), 0.0)
            eta = eta0 * norm / (2.0 * c * inv.sum(axis=1).max())
        for _ in range(iters):
            _, g = stress_grad_ex(Y, nu, D[cur], norm, metric, loss)
            Y = Y - eta * g
        row = [np.sqrt(stress_grad_ex(Y, nus[v], D[v], s2[v], metric, "kruskal",
                                      grad=False)[0]) for v in range(len(nus))]
        table.append(row)
        cur = int(np.argmin(row))
        path.append(nus[cur])
    return Y, path, np.array(table)


# --- Evaluation measures of Section V (plain definitions, FP64) -------------

def sq_dists(A):
    """Squared Euclidean distances of the rows of A, in float64."""
    A = np.asarray(A, dtype=np.float64)
    return ((A[:, None, :] - A[None, :, :]) ** 2).sum(-1)


def _order(d_row, i):
    """Indices of the other points by increasing (distance, index)."""
    n = d_row.shape[0]
    idx = np.array([l for l in range(n) if l != i])
    return idx[np.lexsort((idx, d_row[idx]))]


def trustworthiness(X, Y, k):
    """T(k) = 1 - 2/(n k (2n - 3k - 1)) sum_i sum_{j in N_i} max(0, r(i, j) - k):
    N_i the k nearest neighbours of i in the embedding, r(i, j) the rank of j
    among the original-space distances from i (1 = nearest); Euclidean in both
    spaces, ties broken by the smaller index."""
    dX, dY = sq_dists(X), sq_dists(Y)
    n = dX.shape[0]
    total = 0
    for i in range(n):
        rank = np.empty(n, dtype=np.int64)
        rank[_order(dX[i], i)] = np.arange(1, n)
        for j in _order(dY[i], i)[:k]:
            total += max(0, rank[j] - k)
    return 1.0 - 2.0 * total / (n * k * (2.0 * n - 3.0 * k - 1.0))


def nn_agreement(Y, labels, k):
    """NN(k) = (1/(n k)) sum_i sum_{j in N_i} [label_j = label_i], N_i the k
    nearest neighbours of i in the embedding (Euclidean, ties by index)."""
    dY = sq_dists(Y)
    labels = np.asarray(labels)
    n = dY.shape[0]
    hits = sum(int(np.sum(labels[_order(dY[i], i)[:k]] == labels[i])) for i in range(n))
    return hits / (n * k)


def silhouette(Y, labels):
    """Mean of s_i = (b_i - a_i) / max(a_i, b_i): a_i the mean distance to the
    other points of i's label, b_i the smallest mean distance to another
    label's points; s_i = 0 when i's label has no other point."""
    D = np.sqrt(sq_dists(Y))
    labels = np.asarray(labels)
    n = D.shape[0]
    s = np.zeros(n)
    classes = np.unique(labels)
    for i in range(n):
        own = labels == labels[i]
        if own.sum() <= 1:
            continue
        a = D[i][own].sum() / (own.sum() - 1)
        b = min(D[i][labels == c].mean() for c in classes if c != labels[i])
        s[i] = (b - a) / max(a, b)
    return float(s.mean())


def _pearson(u, v):
    u = np.asarray(u, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    du, dv = u - u.mean(), v - v.mean()
    return float((du * dv).sum() / np.sqrt((du * du).sum() * (dv * dv).sum()))


def midranks(v):
    """1-based ranks of v with ties given the mean of their positions."""
    v = np.asarray(v)
    order = np.argsort(v, kind="stable")
    r = np.empty(len(v))
    sv = v[order]
    s = 0
    while s < len(v):
        e = s
        while e + 1 < len(v) and sv[e + 1] == sv[s]:
            e += 1
        r[order[s:e + 1]] = (s + e) / 2.0 + 1.0
        s = e + 1
    return r


def distance_correlations(X, Y):
    """(Pearson, Spearman) correlation between the n(n-1)/2 pairwise Euclidean
    distances of X and those of Y (pairs i < j; Spearman = Pearson of midranks)."""
    iu = np.triu_indices(np.asarray(X).shape[0], 1)
    dx = np.sqrt(sq_dists(X)[iu])
    dy = np.sqrt(sq_dists(Y)[iu])
    return _pearson(dx, dy), _pearson(midranks(dx), midranks(dy))
