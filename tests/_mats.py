"""Independent sparse operators for the oracle pins, built entry by entry from the
definitions of Sec. 2.2 (forward differences, zero at the last column/row)."""
import numpy as np
import scipy.sparse as sp


def grad_matrix(H, W):
    """Returns (Dx, Dy) as N x N sparse matrices, N = H*W, row-major pixels."""
    N = H * W
    rx, cx, vx, ry, cy, vy = [], [], [], [], [], []
    for i in range(H):
        for j in range(W):
            k = i * W + j
            if j < W - 1:
                rx += [k, k]; cx += [k + 1, k]; vx += [1.0, -1.0]
            if i < H - 1:
                ry += [k, k]; cy += [k + W, k]; vy += [1.0, -1.0]
    Dx = sp.csr_matrix((vx, (rx, cx)), shape=(N, N))
    Dy = sp.csr_matrix((vy, (ry, cy)), shape=(N, N))
    return Dx, Dy


def neumann_laplacian(H, W):
    """(Delta f)_ij = sum over in-domain 4-neighbours of (f_n - f_ij)."""
    N = H * W
    rows, cols, vals = [], [], []
    for i in range(H):
        for j in range(W):
            k = i * W + j
            for di, dj in ((0, 1), (0, -1), (1, 0), (-1, 0)):
                ii, jj = i + di, j + dj
                if 0 <= ii < H and 0 <= jj < W:
                    rows += [k, k]; cols += [ii * W + jj, k]; vals += [1.0, -1.0]
    return sp.csr_matrix((vals, (rows, cols)), shape=(N, N))
