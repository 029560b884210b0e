"""Archive code-stream layout restated in numpy for the tests.

Codec blocks: 1-D 4096, 2-D 64x64, 3-D 16^3; Lorenzo chunks: 1-D 256, 2-D 16x16,
3-D 8^3.  The code of element (z,y,x) sits at slot 4096*b + j, with b the block's
row-major index and j the element's row-major index among the block's in-field
elements.
"""
import numpy as np

BLOCK = {1: (1, 1, 4096), 2: (1, 64, 64), 3: (16, 16, 16)}
CHUNK = {1: (1, 1, 256), 2: (1, 16, 16), 3: (8, 8, 8)}


def dims3(dims):
    d = [1, 1, 1]
    d[3 - len(dims):] = list(dims)
    return tuple(d)


def slot_index(dims):
    """slot of every element, as an array of the field's shape (z,y,x order)."""
    nd = len(dims)
    n = dims3(dims)
    B = BLOCK[nd]
    g = [(n[d] + B[d] - 1) // B[d] for d in range(3)]
    z, y, x = np.meshgrid(*[np.arange(s, dtype=np.int64) for s in n], indexing="ij")
    bz, by, bx = z // B[0], y // B[1], x // B[2]
    rz, ry, rx = z % B[0], y % B[1], x % B[2]
    wz = np.minimum(B[0], n[0] - bz * B[0])
    wy = np.minimum(B[1], n[1] - by * B[1])
    wx = np.minimum(B[2], n[2] - bx * B[2])
    b = (bz * g[1] + by) * g[2] + bx
    j = (rz * wy + ry) * wx + rx
    return (b * 4096 + j).reshape(dims)


def chunk_cumsum(q, dims):
    """Inclusive prefix sums along x, then y, then z, restarted at every chunk
    edge (the N-D partial sum of the reconstruction, per chunk)."""
    nd = len(dims)
    n = dims3(dims)
    C = CHUNK[nd]
    a = q.reshape(n).astype(np.int64)
    for ax in (2, 1, 0):
        if C[ax] == 1:
            continue
        out = np.empty_like(a)
        for s in range(0, n[ax], C[ax]):
            sl = [slice(None)] * 3
            sl[ax] = slice(s, min(s + C[ax], n[ax]))
            out[tuple(sl)] = np.cumsum(a[tuple(sl)], axis=ax)
        a = out
    return a.reshape(dims)


def chunk_start_mask(dims):
    """boolean per axis: element is the first of its chunk along that axis."""
    nd = len(dims)
    n = dims3(dims)
    C = CHUNK[nd]
    idx = np.meshgrid(*[np.arange(s) for s in n], indexing="ij")
    return [(idx[d] % C[d] == 0).reshape(dims) if C[d] > 1 else np.zeros(dims, bool) for d in range(3)]


def block_counts(dims):
    nd = len(dims)
    n = dims3(dims)
    B = BLOCK[nd]
    g = [(n[d] + B[d] - 1) // B[d] for d in range(3)]
    out = []
    for bz in range(g[0]):
        for by in range(g[1]):
            for bx in range(g[2]):
                w = [min(B[0], n[0] - bz * B[0]), min(B[1], n[1] - by * B[1]), min(B[2], n[2] - bx * B[2])]
                out.append(w[0] * w[1] * w[2])
    return np.array(out, dtype=np.int64)
