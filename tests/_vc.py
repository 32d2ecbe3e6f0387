"""Test helper: the variable-coefficient oracle operator as a sparse matrix,
for exact discrete solutions by sparse LU (independent of any iteration)."""

import numpy as np
import scipy.sparse as sp

from oracle import vc_operator as V


def sparse_operator(a, Ls):
    """The oracle's A as a sparse matrix: 27 probes, one per colour
    (x%3, y%3, z%3); same-coloured cells share no stencil neighbour."""
    shape = a.shape
    N = a.size
    idx = np.arange(N).reshape(shape)
    zz, yy, xx = np.meshgrid(*[np.arange(s) for s in shape], indexing="ij")
    rows, cols, vals = [], [], []
    for c in range(27):
        cz, cy, cx = c // 9, (c // 3) % 3, c % 3
        mask = (zz % 3 == cz) & (yy % 3 == cy) & (xx % 3 == cx)
        Av = V.apply_operator(mask.astype(np.float64), a, Ls)
        # each row i gets its value from the unique probed cell j in its stencil
        owner = np.full(shape, -1, dtype=np.int64)
        for dz, dy, dx in [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]:
            src = np.roll(np.where(mask, idx, -1), (dz, dy, dx), axis=(0, 1, 2))
            # np.roll wraps: drop wrapped entries
            valid = np.ones(shape, bool)
            for ax, d in zip(range(3), (dz, dy, dx)):
                if d == 1:
                    sl = [slice(None)] * 3
                    sl[ax] = 0
                    valid[tuple(sl)] = False
                elif d == -1:
                    sl = [slice(None)] * 3
                    sl[ax] = -1
                    valid[tuple(sl)] = False
            take = valid & (src >= 0)
            owner[take] = src[take]
        has = owner >= 0
        rows.append(idx[has])
        cols.append(owner[has])
        vals.append(Av[has])
    return sp.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))
