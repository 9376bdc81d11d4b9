"""Test helpers: unpacking the documented tiled layout, tolerances."""
import numpy as np

B = 128


def untile(flat, n, planes=1):
    """Tiled upper triangle (one matrix, `planes` planes summed) -> dense upper
    triangle (n, n) float64 with zeros on and below the diagonal."""
    flat = np.asarray(flat, dtype=np.float64)
    T = -(-n // B)
    plane = T * (T + 1) // 2 * B * B
    v = flat[:plane].copy()
    for q in range(1, planes):
        v += flat[q * plane:(q + 1) * plane]
    out = np.zeros((T * B, T * B))
    t = 0
    for I in range(T):
        for J in range(I, T):
            out[I * B:(I + 1) * B, J * B:(J + 1) * B] = v[t * B * B:(t + 1) * B * B].reshape(B, B)
            t += 1
    out = out[:n, :n]
    return np.triu(out, 1)


def tiled_flat_index(i, j, n):
    """Flat index of entry (i, j), i < j, in the tiled upper-triangle layout:
    tiles (I, J), I <= J, in row-major order of (I, J), each B x B row-major."""
    i = np.asarray(i, dtype=np.int64)
    j = np.asarray(j, dtype=np.int64)
    T = -(-n // B)
    I, J = i // B, j // B
    t = I * T - I * (I - 1) // 2 + (J - I)
    return t * B * B + (i % B) * B + (j % B)


def rel_err(got, ref, floor=0.0):
    """max |got - ref| / max(|ref|, floor); entries equal on both sides count 0."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if not ref.size:
        return 0.0
    den = np.maximum(np.abs(ref), floor)
    err = np.abs(got - ref)
    return float(np.max(np.where(err == 0, 0.0, err / np.where(den == 0, 1.0, den))))


def fro_rel(got, ref):
    """Norm-wise relative error ||got - ref||_F / ||ref||_F."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.linalg.norm(got - ref) / np.linalg.norm(ref))


# Storage tolerances of a dissimilarity matrix against the FP64 oracle:
# per entry, round-to-nearest of an 8-bit significand (bf16) is within 2^-8;
# hi + lo within 2^-16; plus 1e-6 for the FP32 build.  Norm-wise (Frobenius),
# BF16 within 2e-3 and hi + lo within 1e-5.
ENTRY_TOL = {"f32": 1e-5, "bf16": 2.0 ** -8 + 1e-6, "bf16x2": 2.0 ** -16 + 1e-6}
NORM_TOL = {"f32": 1e-5, "bf16": 2e-3, "bf16x2": 1e-5}


def quantize(full, dtype, col_scale=None):
    """Host round-to-nearest of a dense float matrix to the storage dtype,
    returned as float64 values (plain PyTorch CPU conversions)."""
    import torch
    t = torch.from_numpy(np.asarray(full, dtype=np.float32))
    if dtype == "f32":
        return t.double().numpy()
    if dtype == "bf16":
        return t.to(torch.bfloat16).double().numpy()
    if dtype == "bf16x2":
        hi = t.to(torch.bfloat16).float()
        lo = (t - hi).to(torch.bfloat16).float()
        return (hi + lo).double().numpy()
    if dtype == "fp8":
        sc = torch.from_numpy(np.asarray(col_scale, dtype=np.float32))
        q = (t / sc[None, :]).to(torch.float8_e4m3fn).float() * sc[None, :]
        return q.double().numpy()
    raise ValueError(dtype)


def host_col_scale(full):
    """max_{i<j} |delta_ij| / 448 per column in float32 (1 for an empty column)."""
    f = np.triu(np.abs(np.asarray(full, dtype=np.float32)), 1)
    mx = f.max(axis=0)
    return np.where(mx > 0, mx / np.float32(448), np.float32(1)).astype(np.float32)


def tile_pack(full, n, dtype, col_scale=None):
    """Dense (n, n) -> flat tiled storage (numpy) in the documented layout.
    Returns an array of uint16 (bf16 bits), uint8 (e4m3 bits) or float32."""
    import torch
    T = -(-n // B)
    pad = np.zeros((T * B, T * B), dtype=np.float32)
    pad[:n, :n] = np.triu(np.asarray(full, dtype=np.float32), 1)
    tiles = [pad[I * B:(I + 1) * B, J * B:(J + 1) * B].reshape(-1)
             for I in range(T) for J in range(I, T)]
    flat = torch.from_numpy(np.concatenate(tiles))
    if dtype == "f32":
        return flat.numpy()
    if dtype in ("bf16", "bf16x2"):
        hi = flat.to(torch.bfloat16)
        if dtype == "bf16":
            return hi.view(torch.int16).numpy().view(np.uint16)
        lo = (flat - hi.float()).to(torch.bfloat16)
        return np.concatenate([hi.view(torch.int16).numpy().view(np.uint16),
                               lo.view(torch.int16).numpy().view(np.uint16)])
    if dtype == "fp8":
        sc = np.asarray(col_scale, dtype=np.float32)
        scpad = np.ones(T * B, dtype=np.float32)
        scpad[:n] = sc
        cols = np.concatenate([np.tile(np.arange(J * B, (J + 1) * B), B)
                               for I in range(T) for J in range(I, T)])
        q = (flat / torch.from_numpy(scpad[cols])).to(torch.float8_e4m3fn)
        return q.view(torch.uint8).numpy()
    raise ValueError(dtype)
