"""Torch-facing wrappers of the C ABI (same names as include/gini_mds.h).

PyTorch supplies device memory and the current stream; every step of the
computation runs in libginimds.so.  Nothing here computes the method.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np
import torch

from . import _lib
from ._lib import DTYPES, LAYOUTS, LOSSES, METRICS, OPS, check, lib


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _require_cuda(*ts):
    for t in ts:
        if t is not None and not t.is_cuda:
            raise ValueError("libginimds works on CUDA tensors only")


class Workspace:
    """Caller-owned scratch memory for the library (zero-initialised once)."""

    def __init__(self, device=None):
        self.device = torch.device(device or "cuda")
        self.buf = torch.zeros(256, dtype=torch.uint8, device=self.device)

    def ensure(self, nbytes: int) -> torch.Tensor:
        if self.buf.numel() < nbytes:
            torch.cuda.current_stream(self.device).synchronize()
            self.buf = torch.zeros(int(nbytes), dtype=torch.uint8, device=self.device)
        return self.buf

    def check(self, stream=None) -> None:
        check(lib().gini_check(_ptr(self.buf), _stream(stream)), "gini_check")


_ws_cache = {}


def workspace(device=None) -> Workspace:
    d = torch.device(device or "cuda")
    key = (d.type, d.index if d.index is not None else torch.cuda.current_device())
    if key not in _ws_cache:
        _ws_cache[key] = Workspace(d)
    return _ws_cache[key]


def tile_size() -> int:
    return int(lib().gini_tile_size())


def tiled_elems(n: int) -> int:
    return int(lib().gini_tiled_elems(int(n)))


def workspace_size(op: str, n: int, m: int = 0, k: int = 0, iters: int = 0) -> int:
    return int(lib().gini_workspace_size(OPS[op], int(n), int(m), int(k), int(iters)))


class deterministic:
    """Deterministic mode of the library for the calling thread
    (gini_set_deterministic), as a context manager or a plain call:

        with G.deterministic():        # fixed-order reductions inside
            Y, hist, S = G.gini_mds_fit(...)
        G.deterministic(True).apply()  # stays on
    """

    def __init__(self, on: bool = True):
        self.on = bool(on)
        self.prev = None

    def apply(self):
        lib().gini_set_deterministic(int(self.on))
        return self

    def __enter__(self):
        self.prev = bool(lib().gini_get_deterministic())
        return self.apply()

    def __exit__(self, *exc):
        lib().gini_set_deterministic(int(self.prev))


def is_deterministic() -> bool:
    return bool(lib().gini_get_deterministic())


def default_step(n: int, k: int, nu: float, sum_delta2: float, eta0: float = 1.0) -> float:
    return float(lib().gini_default_step(int(n), int(k), float(nu), float(sum_delta2),
                                         float(eta0)))


def gini_rank(v: torch.Tensor, ws: Optional[Workspace] = None, check_errors: bool = True):
    """Twice the midrank of every element of each row of v (nseg, m): int32."""
    _require_cuda(v)
    assert v.dtype == torch.float32 and v.dim() == 2 and v.stride(1) == 1
    nseg, m = v.shape
    out = torch.empty((nseg, m), dtype=torch.int32, device=v.device)
    ws = ws or workspace(v.device)
    buf = ws.ensure(workspace_size("rank", nseg, m))
    st = lib().gini_rank(_ptr(v), nseg, m, v.stride(0), _ptr(out), _ptr(buf), buf.numel(),
                         _stream())
    check(st, "gini_rank")
    if check_errors:
        ws.check()
    return out


@dataclass
class Dissimilarity:
    """A dissimilarity matrix as stored on the device."""
    data: torch.Tensor             # FULL: (n, n) f32; TILED: flat storage of one matrix
    n: int
    layout: str                    # "full" | "tiled"
    dtype: str                     # "f32" | "bf16" | "bf16x2" | "fp8"
    sum_delta2: float
    col_scale: Optional[torch.Tensor] = None

    @property
    def ldd(self) -> int:
        return self.data.stride(0) if self.layout == "full" else 0


_TORCH_DT = {"f32": torch.float32, "bf16": torch.bfloat16, "bf16x2": torch.bfloat16,
             "fp8": torch.uint8}


def gini_dist(X: torch.Tensor, nus: Sequence[float], layout: str = "full", dtype: str = "f32",
              ws: Optional[Workspace] = None, check_errors: bool = True):
    """Dissimilarity matrices for every nu: returns (list of Dissimilarity,
    sum_delta2 tensor (n_nu,) float64 on the device).  dtype "fp8" (tiled):
    e4m3 with per-column scales, built strip by strip without an n x n
    intermediate."""
    _require_cuda(X)
    assert X.dtype == torch.float32 and X.dim() == 2 and X.stride(1) == 1
    n, p = X.shape
    nus = [float(v) for v in nus]
    n_nu = len(nus)
    if layout == "full":
        out = torch.empty((n_nu, n, n), dtype=torch.float32, device=X.device)
        stride = n * n
    else:
        planes = 2 if dtype == "bf16x2" else 1
        stride = planes * tiled_elems(n)
        out = torch.empty((n_nu, stride), dtype=_TORCH_DT[dtype], device=X.device)
    sd2 = torch.zeros(n_nu, dtype=torch.float64, device=X.device)
    fp8 = dtype == "fp8"
    scale = torch.empty((n_nu, n), dtype=torch.float32, device=X.device) if fp8 else None
    ws = ws or workspace(X.device)
    buf = ws.ensure(workspace_size("dist_fp8" if fp8 else "dist", n, p))
    nu_arr = (ctypes.c_double * n_nu)(*nus)
    st = lib().gini_dist(_ptr(X), n, p, X.stride(0), nu_arr, n_nu, LAYOUTS[layout],
                         DTYPES[dtype], _ptr(out), n, stride, _ptr(scale), _ptr(sd2), _ptr(buf),
                         buf.numel(), _stream())
    check(st, "gini_dist")
    if check_errors:
        ws.check()
    sums = sd2.cpu().tolist()
    mats = [Dissimilarity(out[q], n, layout, dtype, sums[q], scale[q] if fp8 else None)
            for q in range(n_nu)]
    return mats, sd2


def gini_pack(D: Dissimilarity, dtype: str) -> Dissimilarity:
    """FULL f32 -> TILED of the given dtype (FP8 with per-column scales)."""
    assert D.layout == "full" and D.dtype == "f32"
    n = D.n
    planes = 2 if dtype == "bf16x2" else 1
    out = torch.empty(planes * tiled_elems(n), dtype=_TORCH_DT[dtype], device=D.data.device)
    scale = torch.empty(n, dtype=torch.float32, device=D.data.device) if dtype == "fp8" else None
    st = lib().gini_pack(_ptr(D.data), n, D.data.stride(0), DTYPES[dtype], _ptr(out),
                         _ptr(scale), _stream())
    check(st, "gini_pack")
    return Dissimilarity(out, n, "tiled", dtype, D.sum_delta2, scale)


def gini_delta_sums(D: Dissimilarity):
    """(sum_{i<j} delta, sum_{i<j} delta^2) of a stored matrix, as a float64
    tensor of 2 on the device."""
    out = torch.empty(2, dtype=torch.float64, device=D.data.device)
    st = lib().gini_delta_sums(_ptr(D.data), D.n, LAYOUTS[D.layout], DTYPES[D.dtype], D.ldd,
                               _ptr(D.col_scale), _ptr(out), _stream())
    check(st, "gini_delta_sums")
    return out


def gini_stress_grad(Y: torch.Tensor, nu: float, D: Dissimilarity, grad: bool = True,
                     ws: Optional[Workspace] = None, check_errors: bool = True,
                     metric: str = "gini", loss: str = "kruskal", norm: Optional[float] = None):
    """(S as a float64 0-d tensor, dS/dY or None).  norm defaults to
    D.sum_delta2 (the Kruskal normaliser); Sammon needs sum_{i<j} delta."""
    _require_cuda(Y)
    assert Y.dtype == torch.float32 and Y.is_contiguous()
    n, k = Y.shape
    stress = torch.empty((), dtype=torch.float64, device=Y.device)
    g = torch.empty_like(Y) if grad else None
    ws = ws or workspace(Y.device)
    buf = ws.ensure(workspace_size("stress_det" if is_deterministic() else "stress", n, 0, k))
    nrm = D.sum_delta2 if norm is None else float(norm)
    st = lib().gini_stress_grad_ex(_ptr(Y), n, k, float(nu), _ptr(D.data), LAYOUTS[D.layout],
                                   DTYPES[D.dtype], D.ldd, _ptr(D.col_scale), METRICS[metric],
                                   LOSSES[loss], nrm, _ptr(stress), _ptr(g), _ptr(buf),
                                   buf.numel(), _stream())
    check(st, "gini_stress_grad")
    if check_errors:
        ws.check()
    return stress, g


def gini_mds_fit(Y0: torch.Tensor, nu: float, D: Dissimilarity, eta: float, iters: int,
                 polish_iters: int = 0, history: bool = True, ws: Optional[Workspace] = None,
                 check_errors: bool = True, out: Optional[torch.Tensor] = None,
                 metric: str = "gini", loss: str = "kruskal", norm: Optional[float] = None,
                 deterministic: bool = False):
    """Fixed-step GD on the normalized stress; returns (Y_T, history or None, S(Y_T)).
    deterministic: fixed-order gradient reductions for this call (also on when
    the thread's mode is)."""
    _require_cuda(Y0)
    n, k = Y0.shape
    Y = out if out is not None else Y0.clone()
    if out is not None:
        out.copy_(Y0)
    hist = torch.empty(iters + 1, dtype=torch.float64, device=Y0.device) if history else None
    final = torch.empty((), dtype=torch.float64, device=Y0.device)
    ws = ws or workspace(Y0.device)
    det = bool(deterministic) or is_deterministic()
    buf = ws.ensure(workspace_size("fit_det" if det else "fit", n, 0, k, iters))
    a = _lib.FitArgs(deterministic=int(det), n=n, k=k, nu=float(nu), delta_dev=D.data.data_ptr(),
                     layout=LAYOUTS[D.layout], dtype=DTYPES[D.dtype], ldd=D.ldd,
                     col_scale_dev=(D.col_scale.data_ptr() if D.col_scale is not None else None),
                     sum_delta2=(D.sum_delta2 if norm is None else float(norm)),
                     eta=float(eta), iters=int(iters), metric=METRICS[metric],
                     loss=LOSSES[loss],
                     polish_iters=int(polish_iters), Y_dev=Y.data_ptr(),
                     history_dev=(hist.data_ptr() if hist is not None else None),
                     final_stress_dev=final.data_ptr())
    st = lib().gini_mds_fit(ctypes.byref(a), _ptr(buf), buf.numel(), _stream())
    check(st, "gini_mds_fit")
    if check_errors:
        ws.check()
    return Y, hist, final


def gini_fit_batched(Xs, nus, restarts: int, iters: int, Y0: torch.Tensor, eta0: float = 1.0,
                     history: bool = False, ws: Optional[Workspace] = None,
                     check_errors: bool = True, deterministic: bool = False,
                     delta_dtype: str = "f32", tile=None):
    """Batched k = 2 fits of every problem x nu x restart.

    delta_dtype: storage of the Delta pool, "f32" or "bf16".  tile: None (the
    autotuner chooses) or (rows per warp 8 | 16, CTAs per SM 1..3).

    Xs: list of (n_q, p_q) float32 CUDA tensors.  Y0: flat float32 tensor,
    problem-major, restarts x n_q x 2 per problem.  Returns a dict with
    "Y" (flat, (problem, nu, restart)-major), "final" ((nprob, n_nu,
    restarts) float64), "history" ((iters+1, nprob, n_nu, restarts) or None)
    and "tuned" (100 x rows per warp + CTAs per SM chosen by the autotuner).
    """
    nus = [float(v) for v in nus]
    nprob, n_nu = len(Xs), len(nus)
    probs = (_lib.Problem * nprob)()
    keep = []
    for q, X in enumerate(Xs):
        _require_cuda(X)
        assert X.dtype == torch.float32 and X.dim() == 2 and X.stride(1) == 1
        keep.append(X)
        probs[q] = _lib.Problem(X.data_ptr(), X.shape[0], X.shape[1], X.stride(0))
    ns = [X.shape[0] for X in Xs]
    assert Y0.numel() == sum(restarts * n * 2 for n in ns)
    dev = Xs[0].device
    Y = torch.empty(sum(n_nu * restarts * n * 2 for n in ns), dtype=torch.float32, device=dev)
    nfits = nprob * n_nu * restarts
    final = torch.empty(nfits, dtype=torch.float64, device=dev)
    hist = torch.empty((iters + 1) * nfits, dtype=torch.float64, device=dev) if history else None
    opts = _lib.BatchOpts(deterministic=int(bool(deterministic) or is_deterministic()),
                          delta_dtype=DTYPES[delta_dtype],
                          tile_rows=int(tile[0]) if tile else 0,
                          ctas_per_sm=int(tile[1]) if tile else 0)
    nbytes = int(lib().gini_batch_workspace_size(probs, nprob, n_nu, restarts, iters,
                                                 ctypes.byref(opts)))
    ws = ws or workspace(dev)
    buf = ws.ensure(nbytes)
    nu_arr = (ctypes.c_double * n_nu)(*nus)
    tuned = ctypes.c_int(0)
    st = lib().gini_fit_batched(probs, nprob, nu_arr, n_nu, restarts, iters, float(eta0),
                                _ptr(Y0.contiguous()), _ptr(Y), _ptr(hist), _ptr(final),
                                ctypes.byref(tuned), ctypes.byref(opts), _ptr(buf), buf.numel(),
                                _stream())
    check(st, "gini_fit_batched")
    if check_errors:
        ws.check()
    return {"Y": Y, "final": final.view(nprob, n_nu, restarts),
            "history": hist.view(iters + 1, nprob, n_nu, restarts) if hist is not None else None,
            "tuned": tuned.value}


def gini_nu_search(X: torch.Tensor, folds, nus, restarts: int, iters: int, Y0: torch.Tensor,
                   eta0: float = 1.0, ws: Optional[Workspace] = None, check_errors: bool = True):
    """Algorithm 1's search over a nu grid with K folds.  folds: n ints in [0, K)
    (host sequence or array); Y0: (restarts, n, 2) float32 CUDA tensor.  Returns a
    dict with "ks" ((n_nu, K) float64), "mean_ks" ((n_nu,)), "best" (index of
    nu*, a 0-d int32 tensor) and "Y" ((n, 2): the fold embeddings at nu*)."""
    _require_cuda(X)
    assert X.dtype == torch.float32 and X.dim() == 2 and X.stride(1) == 1
    n, p = X.shape
    fold = np.ascontiguousarray(np.asarray(folds, dtype=np.int32))
    assert fold.shape == (n,)
    K = int(fold.max()) + 1 if n else 0
    nus = [float(v) for v in nus]
    n_nu = len(nus)
    assert Y0.shape == (restarts, n, 2) and Y0.dtype == torch.float32
    dev = X.device
    fptr = fold.ctypes.data_as(ctypes.c_void_p)
    nbytes = int(lib().gini_nu_search_workspace_size(n, p, fptr, K, n_nu, restarts, iters))
    if nbytes == 0:
        raise _lib.GiniError(_lib.GINI_EINVAL, "gini_nu_search_workspace_size")
    ws = ws or workspace(dev)
    buf = ws.ensure(nbytes)
    ks = torch.empty((n_nu, K), dtype=torch.float64, device=dev)
    mean_ks = torch.empty(n_nu, dtype=torch.float64, device=dev)
    best = torch.empty((), dtype=torch.int32, device=dev)
    Y = torch.empty((n, 2), dtype=torch.float32, device=dev)
    nu_arr = (ctypes.c_double * n_nu)(*nus)
    st = lib().gini_nu_search(_ptr(X), n, p, X.stride(0), fptr, K, nu_arr, n_nu, restarts, iters,
                              float(eta0), _ptr(Y0.contiguous()), _ptr(ks), _ptr(mean_ks),
                              _ptr(best), _ptr(Y), _ptr(buf), buf.numel(), _stream())
    check(st, "gini_nu_search")
    if check_errors:
        ws.check()
    return {"ks": ks, "mean_ks": mean_ks, "best": best, "Y": Y}


def gini_alternating_nu(X: torch.Tensor, nus, nu_start: float, rounds: int, iters: int,
                        Y0: torch.Tensor, eta0: float = 1.0, metric: str = "gini",
                        loss: str = "sammon", ws: Optional[Workspace] = None):
    """Algorithm 2's alternating nu update.  Returns (Y (n, k) float32 CUDA tensor,
    nu path (rounds + 1 floats), KS table ((rounds, n_nu) float64 numpy array))."""
    _require_cuda(X)
    assert X.dtype == torch.float32 and X.dim() == 2 and X.stride(1) == 1
    n, p = X.shape
    k = Y0.shape[1]
    assert Y0.shape == (n, k) and Y0.dtype == torch.float32
    nus = [float(v) for v in nus]
    n_nu = len(nus)
    Y = Y0.clone().contiguous()
    nbytes = int(lib().gini_alternating_nu_workspace_size(n, p, k, n_nu, iters))
    ws = ws or workspace(X.device)
    buf = ws.ensure(nbytes)
    nu_arr = (ctypes.c_double * n_nu)(*nus)
    path = (ctypes.c_double * (rounds + 1))()
    ks = np.zeros((rounds, n_nu), dtype=np.float64)
    st = lib().gini_alternating_nu(_ptr(X), n, p, X.stride(0), k, nu_arr, n_nu, float(nu_start),
                                   int(rounds), int(iters), float(eta0), METRICS[metric],
                                   LOSSES[loss], _ptr(Y), path,
                                   ks.ctypes.data_as(ctypes.c_void_p), _ptr(buf), buf.numel(),
                                   _stream())
    check(st, "gini_alternating_nu")
    return Y, list(path), ks


def _xy(X, Y):
    _require_cuda(X)
    assert X.dtype == torch.float32 and X.dim() == 2 and X.stride(1) == 1
    assert Y.dtype == torch.float32 and Y.is_contiguous() and Y.shape[0] == X.shape[0]
    return X.shape[0], X.shape[1], Y.shape[1]


def gini_neighbour_scores(X: torch.Tensor, Y: torch.Tensor, labels: Optional[torch.Tensor] = None,
                          k_trust: int = 5, k_nn: int = 10, ws: Optional[Workspace] = None):
    """(T(k_trust), NN(k_nn)) as a float64 CUDA tensor of 2 (NaN where not asked)."""
    n, p, k = _xy(X, Y)
    if labels is None:
        k_nn = 0
    else:
        assert labels.dtype == torch.int32 and labels.is_contiguous() and labels.numel() == n
    out = torch.empty(2, dtype=torch.float64, device=X.device)
    ws = ws or workspace(X.device)
    buf = ws.ensure(int(lib().gini_eval_workspace_size(n, 1, 0)))
    st = lib().gini_neighbour_scores(_ptr(X), n, p, X.stride(0), _ptr(Y), k, _ptr(labels),
                                     int(k_trust), int(k_nn), _ptr(out), _ptr(buf), buf.numel(),
                                     _stream())
    check(st, "gini_neighbour_scores")
    return out


def gini_silhouette(Y: torch.Tensor, labels: torch.Tensor, n_labels: Optional[int] = None,
                    ws: Optional[Workspace] = None, check_errors: bool = True):
    """Silhouette score of the embedding under integer labels in [0, n_labels)."""
    _require_cuda(Y)
    assert Y.dtype == torch.float32 and Y.is_contiguous()
    assert labels.dtype == torch.int32 and labels.is_contiguous()
    n, k = Y.shape
    if n_labels is None:
        n_labels = int(labels.max().item()) + 1
    out = torch.empty(1, dtype=torch.float64, device=Y.device)
    ws = ws or workspace(Y.device)
    buf = ws.ensure(int(lib().gini_eval_workspace_size(n, n_labels, 0)))
    st = lib().gini_silhouette(_ptr(Y), n, k, _ptr(labels), int(n_labels), _ptr(out), _ptr(buf),
                               buf.numel(), _stream())
    check(st, "gini_silhouette")
    if check_errors:
        ws.check()
    return out[0]


def gini_distance_correlations(X: torch.Tensor, Y: torch.Tensor, spearman: bool = True,
                               ws: Optional[Workspace] = None):
    """(Pearson, Spearman) between pairwise distances of X and of Y (float64 tensor of 2)."""
    n, p, k = _xy(X, Y)
    out = torch.empty(2, dtype=torch.float64, device=X.device)
    ws = ws or workspace(X.device)
    buf = ws.ensure(int(lib().gini_eval_workspace_size(n, 1, int(spearman))))
    st = lib().gini_distance_correlations(_ptr(X), n, p, X.stride(0), _ptr(Y), k, int(spearman),
                                          _ptr(out), _ptr(buf), buf.numel(), _stream())
    check(st, "gini_distance_correlations")
    return out


def gini_classical_mds(D: Dissimilarity, k: int, iters: int = 20, seed: int = 0,
                       ws: Optional[Workspace] = None, check_errors: bool = True):
    """Classical MDS of D: (Y (n, k) float32, eigenvalues (k,) float64, descending)."""
    n = D.n
    dev = D.data.device
    Y = torch.empty((n, k), dtype=torch.float32, device=dev)
    lam = torch.empty(k, dtype=torch.float64, device=dev)
    ws = ws or workspace(dev)
    buf = ws.ensure(int(lib().gini_cmds_workspace_size(n, k)))
    st = lib().gini_classical_mds(_ptr(D.data), n, LAYOUTS[D.layout], DTYPES[D.dtype], D.ldd,
                                  _ptr(D.col_scale), int(k), int(iters),
                                  int(seed) & 0xFFFFFFFFFFFFFFFF, _ptr(Y), _ptr(lam), _ptr(buf),
                                  buf.numel(), _stream())
    check(st, "gini_classical_mds")
    if check_errors:
        ws.check()
    return Y, lam


class GiniStress(torch.autograd.Function):
    """S(Y) = sum_{i<j} (Dbar(y_i, y_j) - delta_ij)^2 / sum_delta2 as an autograd op.

    The forward pass runs the fused stress+adjoint kernel when Y needs a
    gradient and keeps only dS/dY (n x k); nothing n x n is stored.  The
    backward pass scales it by the incoming gradient.
    """

    @staticmethod
    def forward(ctx, Y, nu, D):
        S, g = gini_stress_grad(Y.detach().contiguous(), nu, D, grad=Y.requires_grad)
        ctx.save_for_backward(g if g is not None else torch.empty(0, device=Y.device))
        return S

    @staticmethod
    def backward(ctx, gS):
        (g,) = ctx.saved_tensors
        return (gS.to(g.dtype) * g), None, None


def gini_stress(Y: torch.Tensor, nu: float, D: Dissimilarity) -> torch.Tensor:
    return GiniStress.apply(Y, nu, D)


def fit_host(X: np.ndarray, nu: float, k: int, iters: int, Y0: np.ndarray, eta0: float = 1.0,
             dtype: str = "bf16x2", polish_iters: int = 20, device="cuda"):
    """End-to-end from host arrays: copy X and Y0 in, build Delta, fit, copy
    Y_T and S(Y_T) out.  Returns (Y_T as numpy, S(Y_T), sum_delta2)."""
    dev = torch.device(device)
    Xh = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).pin_memory()
    Yh = torch.from_numpy(np.ascontiguousarray(Y0, dtype=np.float32)).pin_memory()
    Xd = Xh.to(dev, non_blocking=True)
    Yd = Yh.to(dev, non_blocking=True)
    layout = "full" if dtype == "full" else "tiled"
    mats, _ = gini_dist(Xd, [nu], layout=layout, dtype=("f32" if dtype == "full" else dtype),
                        check_errors=False)
    D = mats[0]
    eta = default_step(X.shape[0], k, nu, D.sum_delta2, eta0)
    Y, _, final = gini_mds_fit(Yd, nu, D, eta, iters, polish_iters=polish_iters, history=False,
                               check_errors=False)
    Yout = torch.empty(Y.shape, dtype=torch.float32, pin_memory=True)
    Yout.copy_(Y, non_blocking=True)
    fin = final.to("cpu", non_blocking=True)
    torch.cuda.current_stream().synchronize()
    return Yout.numpy(), float(fin), D.sum_delta2
