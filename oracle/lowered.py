"""The SPIDER transform written out step by step -- TEST INFRASTRUCTURE ONLY.

Plain numpy / Python, following the order of Sec. 3.1 and Sec. 3.2:

1. ``kernel_matrix``: a kernel row of radius r becomes the banded matrix
   K in R^{L x (2r+L)} by repeating it L times along the diagonal, so that
   ``Y = K X`` updates L consecutive points (Sec. 3.1.1).
2. ``pad_kernel_matrix``: two zero columns bring K to L x 2L, the shape
   the sparse MMA wants (Sec. 3.1.2, stage 1; the r = 3 example goes from
   8 x 14 to 8 x 16).
3. ``strided_swap_permutation``: column j is exchanged with column j + L for
   every j of one parity below L (Sec. 3.1.2 says odd j; Sec. 3.2 says
   j = 0, 2, ..., L-1.  Both are provided; even is the default because the
   row-offset equation of Sec. 3.2 adds its extra term for even element
   indices).
4. ``compress_2_4`` / ``decompress_2_4``: the value matrix keeps the (at
   most two) non-zeros of every group of four in their original order, and
   2-bit indices, increasing and packed from the least significant bit,
   record their positions; a group with a single non-zero keeps a zero
   placeholder (Sec. 3.1.2, stage 3, with the E0G0 and 0G00 examples).
   ``compress_1_2`` is the same idea for pairs (one value per pair), the
   pattern TF32 sparse MMAs accept.
5. ``lowered_step``: one stencil step computed as the sum over kernel rows
   of K X products on x-tiles of L points (Sec. 3.1.1), either with the
   plain banded K or with the swapped-and-compressed K' = K P applied to the
   row-swapped input P^T X (Sec. 3.2).  With integer inputs every product
   is exact, so this must equal the direct sweep bit for bit.

Nothing here is shared with the CUDA path.
"""
from __future__ import annotations

import itertools

import numpy as np


def default_L(r: int) -> int:
    """Eq. 1: the non-zero fraction (2r+1)/(2r+L) is at most 1/2 iff L >= 2r+2;
    the paper takes L = 2r+2 (Sec. 3.1.1)."""
    return 2 * r + 2


def nonzero_fraction(r: int, L: int) -> float:
    """Eq. 1 (labelled "Sparsity" in the paper; it is the fraction of non-zeros)."""
    return (L * (2 * r + 1)) / (L * (2 * r + L))


def kernel_matrix(w_row, L: int | None = None) -> np.ndarray:
    """Banded K with K[m][n] = w_row[n - m] for 0 <= n - m <= 2r (Sec. 3.1.1).

    ``w_row`` holds the 2r+1 coefficients of one kernel row for offsets
    -r..r.  Row m of ``K @ X`` is output point m of the tile, and row n of X
    is input point n - r of the tile (so X spans the tile plus r on each side).
    """
    w_row = np.asarray(w_row)
    r = (len(w_row) - 1) // 2
    if L is None:
        L = default_L(r)
    K = np.zeros((L, 2 * r + L), dtype=w_row.dtype)
    for m in range(L):
        for j in range(2 * r + 1):
            K[m, m + j] = w_row[j]
    return K


def pad_kernel_matrix(K: np.ndarray) -> np.ndarray:
    """Append zero columns so that K is L x 2L (Sec. 3.1.2, stage 1)."""
    L, ncols = K.shape
    if ncols > 2 * L:
        raise ValueError("kernel matrix wider than 2L: L is below 2r+2")
    out = np.zeros((L, 2 * L), dtype=K.dtype)
    out[:, :ncols] = K
    return out


def strided_swap_permutation(L: int, parity: str = "even") -> np.ndarray:
    """Index map pi of the strided column swap: column j <-> j + L for every
    j < L of the given parity (Sec. 3.1.2, Sec. 3.2).  ``K @ P`` has column
    ``K[:, pi[j]]`` in position j; pi is an involution."""
    if parity not in ("even", "odd"):
        raise ValueError("parity must be 'even' or 'odd'")
    start = 0 if parity == "even" else 1
    pi = np.arange(2 * L)
    for j in range(start, L, 2):
        pi[j], pi[j + L] = j + L, j
    return pi


def permutation_matrix(pi: np.ndarray) -> np.ndarray:
    """P with (K P)[:, j] = K[:, pi[j]]."""
    n = len(pi)
    P = np.zeros((n, n), dtype=np.int64)
    for j in range(n):
        P[pi[j], j] = 1
    return P


def swap_columns(K: np.ndarray, pi: np.ndarray) -> np.ndarray:
    """K' = K P (Sec. 3.1.2, stage 2)."""
    return K[:, pi]


def swap_rows(X: np.ndarray, pi: np.ndarray) -> np.ndarray:
    """X' = P^T X: row j of X' is row pi[j] of X (Sec. 3.2)."""
    return X[pi, :]


def _group_indices(nz_positions, group: int):
    """Positions kept for one group (increasing), with the placeholder rule."""
    nz = list(nz_positions)
    if group == 4:
        if len(nz) > 2:
            raise ValueError("group of four with more than two non-zeros: not 2:4")
        if len(nz) == 2:
            return nz
        if len(nz) == 1:
            a = nz[0]
            # Sec. 3.1.2 example 0G00 -> values G0, indices 01 10: the zero
            # placeholder takes the next position; at the last position the
            # pair becomes (2, 3).
            return [a, a + 1] if a < 3 else [2, 3]
        return [0, 1]
    if group == 2:
        if len(nz) > 1:
            raise ValueError("pair with two non-zeros: not 1:2")
        return nz if nz else [0]
    raise ValueError("group must be 2 or 4")


def compress_2_4(Kp: np.ndarray):
    """Value matrix (rows x cols/2) and index matrix (rows x cols/4 x 2).

    Zeros are decided on the structural pattern given by ``Kp != 0``.
    """
    rows, cols = Kp.shape
    if cols % 4:
        raise ValueError("column count must be a multiple of 4")
    vals = np.zeros((rows, cols // 2), dtype=Kp.dtype)
    idx = np.zeros((rows, cols // 4, 2), dtype=np.int64)
    for m in range(rows):
        for g in range(cols // 4):
            seg = Kp[m, 4 * g:4 * g + 4]
            keep = _group_indices([i for i in range(4) if seg[i] != 0], 4)
            idx[m, g] = keep
            vals[m, 2 * g] = seg[keep[0]]
            vals[m, 2 * g + 1] = seg[keep[1]]
    return vals, idx


def metadata_bits(idx: np.ndarray) -> list[str]:
    """Per group, the two 2-bit indices written as in the paper ('00 10'):
    first kept index, then second."""
    return [f"{int(a):02b} {int(b):02b}" for a, b in idx]


def metadata_word(idx_row: np.ndarray) -> int:
    """Pack one row's indices LSB first: group g occupies bits 4g..4g+3,
    its first index in the low two bits (Sec. 3.1.2, "increasing order,
    starting from the least significant bit")."""
    word = 0
    for g, (a, b) in enumerate(idx_row):
        word |= (int(a) | (int(b) << 2)) << (4 * g)
    return word


def decompress_2_4(vals: np.ndarray, idx: np.ndarray) -> np.ndarray:
    rows, half = vals.shape
    out = np.zeros((rows, 2 * half), dtype=vals.dtype)
    for m in range(rows):
        for g in range(half // 2):
            a, b = idx[m, g]
            out[m, 4 * g + a] += vals[m, 2 * g]
            out[m, 4 * g + b] += vals[m, 2 * g + 1]
    return out


def compress_1_2(Kp: np.ndarray):
    """One value per pair of columns and its 1-bit index (pattern for TF32)."""
    rows, cols = Kp.shape
    if cols % 2:
        raise ValueError("column count must be even")
    vals = np.zeros((rows, cols // 2), dtype=Kp.dtype)
    idx = np.zeros((rows, cols // 2), dtype=np.int64)
    for m in range(rows):
        for p in range(cols // 2):
            seg = Kp[m, 2 * p:2 * p + 2]
            keep = _group_indices([i for i in range(2) if seg[i] != 0], 2)
            idx[m, p] = keep[0]
            vals[m, p] = seg[keep[0]]
    return vals, idx


def decompress_1_2(vals: np.ndarray, idx: np.ndarray) -> np.ndarray:
    rows, half = vals.shape
    out = np.zeros((rows, 2 * half), dtype=vals.dtype)
    for m in range(rows):
        for p in range(half):
            out[m, 2 * p + idx[m, p]] = vals[m, p]
    return out


def is_2_4(mask: np.ndarray) -> bool:
    rows, cols = mask.shape
    return all(np.count_nonzero(mask[m, 4 * g:4 * g + 4]) <= 2
               for m in range(rows) for g in range(cols // 4))


def is_1_2(mask: np.ndarray) -> bool:
    rows, cols = mask.shape
    return all(np.count_nonzero(mask[m, 2 * p:2 * p + 2]) <= 1
               for m in range(rows) for p in range(cols // 2))


def swapped_kernel_matrix(w_row, parity: str = "even", L: int | None = None) -> np.ndarray:
    """Stages 1-2 of Sec. 3.1.2 for one kernel row: pad then swap."""
    K = pad_kernel_matrix(kernel_matrix(w_row, L))
    return swap_columns(K, strided_swap_permutation(K.shape[0], parity))


def _kernel_rows(w: np.ndarray):
    """Kernel-row decomposition (Sec. 3.1.1): one 1-D row along x for every
    offset of the slower axes.  Yields (offsets of slower axes, row)."""
    d = w.ndim
    r = (w.shape[0] - 1) // 2
    for outer in itertools.product(range(-r, r + 1), repeat=d - 1):
        sl = tuple(o + r for o in outer)
        yield outer, w[sl]


def lowered_step(u: np.ndarray, w: np.ndarray, mode: str = "dense", parity: str = "even") -> np.ndarray:
    """One zero-Dirichlet stencil step as a sum of K X products (Sec. 3.1.1).

    mode = "dense"   : Y += K_rho X_rho with the padded banded K (L = 2r+2);
    mode = "swapped" : Y += decompress(compress(K_rho P)) (P^T X_rho), i.e. the
                       strided-swapped 2:4 form and the row-swapped input.
    The result has the dtype of ``u`` (use int64 for exact checks).
    """
    r = (w.shape[0] - 1) // 2
    L = default_L(r)
    d = u.ndim
    shape = u.shape
    nx = shape[-1]
    ntiles = -(-nx // L)
    # zero padding: r on every side of the slower axes; r on the left of x and
    # enough on the right for full tiles plus r, plus the 2 padding rows of X.
    pad = [(r, r)] * (d - 1) + [(r, ntiles * L - nx + r + (2 * L - (2 * r + L)))]
    up = np.pad(u, pad)
    outer_shape = shape[:-1]
    ncol = int(np.prod(outer_shape)) if d > 1 else 1
    Y = np.zeros(outer_shape + (ntiles * L,), dtype=u.dtype)
    pi = strided_swap_permutation(L, parity)
    for outer, w_row in _kernel_rows(w):
        K = pad_kernel_matrix(kernel_matrix(np.asarray(w_row, dtype=u.dtype), L))
        if mode == "swapped":
            vals, idx = compress_2_4(swap_columns(K, pi))
            A = decompress_2_4(vals, idx)
        elif mode == "dense":
            A = K
        else:
            raise ValueError("mode must be 'dense' or 'swapped'")
        # input rows shifted by the outer offsets: column c of X is output row c
        sl = tuple(slice(r + o, r + o + n) for o, n in zip(outer, outer_shape))
        rows = up[sl].reshape(ncol, -1)
        for t in range(ntiles):
            x0 = t * L
            X = rows[:, x0:x0 + 2 * L].T          # (2L) x C, row n = input x0 - r + n
            if mode == "swapped":
                X = swap_rows(X, pi)
            Yt = A @ X                             # L x C
            Y.reshape(ncol, -1)[:, x0:x0 + L] += Yt.T
    return Y[..., :nx]


def lowered_stencil(u0: np.ndarray, w: np.ndarray, steps: int, mode: str = "dense",
                    parity: str = "even") -> np.ndarray:
    u = np.array(u0)
    for _ in range(steps):
        u = lowered_step(u, w, mode, parity)
    return u
