"""Device tile arrays for the tiled Cholesky tasks (torch for memory only).

A packed lower-tile array is a tensor of shape (T(T+1)/2, b, b); tile
(i, j), i >= j, is entry j*T - j(j-1)/2 + (i - j), and element (r, c) of a
tile is ``tiles[t, c, r]`` (each tile is column-major, like the task bodies
expect).  These helpers only move data and collect pointers.
"""
import torch


def ntiles(T):
    return T * (T + 1) // 2


def tile_index(i, j, T):
    return j * T - j * (j - 1) // 2 + (i - j)


def tile_ptrs(t):
    """Device addresses of every tile of a (nt, ...) tensor."""
    base = t.data_ptr()
    step = t.stride(0) * t.element_size()
    return [base + k * step for k in range(t.shape[0])]


def to_tiles(A, b):
    """Dense (N, N) tensor -> packed lower tiles (copy, same device/dtype)."""
    N = A.shape[0]
    T = N // b
    assert T * b == N
    out = torch.empty((ntiles(T), b, b), dtype=A.dtype, device=A.device)
    for j in range(T):
        for i in range(j, T):
            out[tile_index(i, j, T)] = A[i * b:(i + 1) * b, j * b:(j + 1) * b].T
    return out


def from_tiles(tl, N, b):
    """Packed lower tiles -> dense (N, N) with zero upper blocks."""
    T = N // b
    A = torch.zeros((N, N), dtype=tl.dtype, device=tl.device)
    for j in range(T):
        for i in range(j, T):
            A[i * b:(i + 1) * b, j * b:(j + 1) * b] = tl[tile_index(i, j, T)].T
    return A


def q_tiles(T, b, fmt, device):
    """Byte buffer for the quantised panel tiles: (nt, q_bytes) uint8."""
    from ._lib import q_bytes
    return torch.empty((ntiles(T), q_bytes(b, fmt)), dtype=torch.uint8, device=device)


_gather_cache = {}


def packed_index(T, device):
    """(rows, cols) index tensors of the packed lower tiles in column order."""
    key = (T, str(device))
    if key not in _gather_cache:
        ii, jj = [], []
        for j in range(T):
            for i in range(j, T):
                ii.append(i)
                jj.append(j)
        _gather_cache[key] = (torch.tensor(ii, device=device), torch.tensor(jj, device=device))
    return _gather_cache[key]


def pack_lower(C, b):
    """Dense (N, N) tensor -> packed lower tiles in one gather (N % b == 0):
    out[t, c, r] = C[i*b + r, j*b + c] for tile t = (i, j)."""
    N = C.shape[0]
    T = N // b
    v = C.view(T, b, T, b).permute(0, 2, 3, 1)       # [I, J, c, r]
    ii, jj = packed_index(T, C.device)
    return v[ii, jj].contiguous()


def pad_size(N, b):
    return (N + b - 1) // b * b
