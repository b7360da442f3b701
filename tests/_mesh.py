"""Test helpers: node coordinates of the hex mesh and small dense utilities.

Pure geometry (no method arithmetic), used to build exact solutions."""
import numpy as np


def hex_nodes(n: int) -> np.ndarray:
    """Coordinates (N, 3) of every DOF: DOF 8e + a sits at node a of element e."""
    h = 1.0 / n
    e = np.repeat(np.arange(n ** 3), 8)
    a = np.tile(np.arange(8), n ** 3)
    ix, iy, iz = e % n, (e // n) % n, e // (n * n)
    return np.stack([(ix + (a & 1)) * h, (iy + ((a >> 1) & 1)) * h, (iz + ((a >> 2) & 1)) * h], axis=1)


def csr_dense(rowptr, col, val, n, m=None):
    A = np.zeros((n, n if m is None else m))
    for i in range(n):
        for p in range(rowptr[i], rowptr[i + 1]):
            A[i, col[p]] += val[p]
    return A


def q1_l2_error(n, x, exact, nq=4):
    """L2 norm of (u_h - exact) over the unit cube with an nq^3 Gauss rule per element."""
    gp, gw = np.polynomial.legendre.leggauss(nq)
    gp = (gp + 1) / 2
    gw = gw / 2
    h = 1.0 / n
    P = np.stack(np.meshgrid(gp, gp, gp, indexing="ij"), -1).reshape(-1, 3)
    W = np.einsum("i,j,k->ijk", gw, gw, gw).reshape(-1)
    # basis values at the Gauss points (nq^3, 8)
    B = np.ones((P.shape[0], 8))
    for a in range(8):
        for d in range(3):
            bit = (a >> d) & 1
            B[:, a] *= P[:, d] if bit else 1 - P[:, d]
    err = 0.0
    E = n ** 3
    for e in range(E):
        ix, iy, iz = e % n, (e // n) % n, e // (n * n)
        uh = B @ x[8 * e: 8 * e + 8]
        X = (np.array([ix, iy, iz]) + P) * h
        err += np.sum(W * (uh - exact(X)) ** 2) * h ** 3
    return np.sqrt(err)
