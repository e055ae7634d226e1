"""Dense textbook routines used to pin the oracle (tests only).

These restate the mathematics with dense numpy/scipy primitives (matrix
products, triangular solves, direct solves) rather than the oracle's loops,
so that an index, sign or ordering slip in the oracle shows up as a mismatch.
"""
import numpy as np
import scipy.linalg as sla


def tridiag_ones(m):
    """m x m matrix with ones on the diagonal and both off-diagonals."""
    return np.eye(m) + np.eye(m, k=1) + np.eye(m, k=-1)


def kron_operator(nx, ny, nz, kappa=None):
    """27-point operator as 27 I - Tz (x) Ty (x) Tx (+ diag(kappa)).

    The box of ones over |dx|,|dy|,|dz| <= 1 is the Kronecker product of three
    1D 'tridiagonal ones' matrices (x fastest); the HPCG operator has 26 on the
    diagonal and -1 on the other 26 entries, i.e. 27 I minus that box."""
    B = np.kron(tridiag_ones(nz), np.kron(tridiag_ones(ny), tridiag_ones(nx)))
    A = 27.0 * np.eye(nx * ny * nz) - B
    if kappa is not None:
        A = A + np.diag(kappa)
    return A


def kron_eigenvalues(nx, ny, nz):
    """Closed-form spectrum: 27 - prod_d (1 + 2 cos(k_d pi / (n_d + 1)))."""
    lx = 1 + 2 * np.cos(np.arange(1, nx + 1) * np.pi / (nx + 1))
    ly = 1 + 2 * np.cos(np.arange(1, ny + 1) * np.pi / (ny + 1))
    lz = 1 + 2 * np.cos(np.arange(1, nz + 1) * np.pi / (nz + 1))
    prod = (lz[:, None, None] * ly[None, :, None] * lx[None, None, :]).ravel()
    return np.sort(27.0 - prod)


def parity_colors(nx, ny, nz):
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return ((x & 1) + 2 * (y & 1) + 4 * (z & 1)).ravel()


def gs_forward_sorted(A, colors, r, z):
    """One forward Gauss-Seidel sweep in colour-sorted order (P^T A P):
    z_new = (D + L)^{-1} (r - U z) in the permuted numbering."""
    perm = np.argsort(colors, kind="stable")
    Ap = A[np.ix_(perm, perm)]
    rp, zp = r[perm], z[perm]
    DL = np.tril(Ap)
    U = np.triu(Ap, 1)
    zn = sla.solve_triangular(DL, rp - U @ zp, lower=True)
    out = np.empty_like(z)
    out[perm] = zn
    return out


def gs_backward_sorted(A, colors, r, z):
    """One backward sweep, colours in reverse: z_new = (D + U)^{-1} (r - L z)."""
    perm = np.argsort(colors, kind="stable")
    Ap = A[np.ix_(perm, perm)]
    rp, zp = r[perm], z[perm]
    DU = np.triu(Ap)
    L = np.tril(Ap, -1)
    zn = sla.solve_triangular(DU, rp - L @ zp, lower=False)
    out = np.empty_like(z)
    out[perm] = zn
    return out


def injection_matrix(nf, f2c):
    R = np.zeros((len(f2c), nf))
    R[np.arange(len(f2c)), f2c] = 1.0
    return R


def dense_vcycle(As, colors, Rs, r, level=0, symmetric=True):
    """Listing 1 with dense pieces: smoother = textbook GS sweeps on the
    colour-sorted matrix, restriction = R, refinement = R^T."""
    A = As[level]
    z = np.zeros_like(r)

    def smooth(zv):
        zv = gs_forward_sorted(A, colors[level], r, zv)
        if symmetric:
            zv = gs_backward_sorted(A, colors[level], r, zv)
        return zv

    z = smooth(z)
    if level == len(As) - 1:
        return z
    rc = Rs[level] @ (r - A @ z)
    zc = dense_vcycle(As, colors, Rs, rc, level + 1, symmetric)
    z = z + Rs[level].T @ zc
    return smooth(z)
