"""Textbook 1D finite-element matrices and tensor-product assembly, written independently of
both the oracle and the CUDA path; the tests use them to pin the oracle on uniform meshes.

1D Lagrange elements on an interval of length h (standard tables, e.g. Hughes, The Finite
Element Method, Sec. 3):
  Q1: stiffness (1/h)[[1,-1],[-1,1]],             consistent mass (h/6)[[2,1],[1,2]]
  Q2: stiffness (1/(3h))[[7,-8,1],[-8,16,-8],[1,-8,7]], mass (h/30)[[4,2,-1],[2,16,2],[-1,2,4]]
On a tensor-product brick, the Laplacian stiffness is K = Kz(x)My(x)Mx + Mz(x)Ky(x)Mx +
Mz(x)My(x)Kx and the consistent mass is Mz(x)My(x)Mx, with (x) the Kronecker product and x
the fastest index.
"""
import numpy as np

ELEM = {
    1: (np.array([[1.0, -1.0], [-1.0, 1.0]]), np.array([[2.0, 1.0], [1.0, 2.0]]) / 6.0),
    2: (np.array([[7.0, -8.0, 1.0], [-8.0, 16.0, -8.0], [1.0, -8.0, 7.0]]) / 3.0,
        np.array([[4.0, 2.0, -1.0], [2.0, 16.0, 2.0], [-1.0, 2.0, 4.0]]) / 30.0),
}


def assemble_1d(p, ncell, h):
    n = p * ncell + 1
    K = np.zeros((n, n))
    M = np.zeros((n, n))
    ke, me = ELEM[p]
    for e in range(ncell):
        idx = slice(p * e, p * e + p + 1)
        K[idx, idx] += ke / h
        M[idx, idx] += me * h
    return K, M


def brick_matrices(p, ncell, h):
    """3D stiffness (unit conductivity) and consistent mass in lexicographic node order."""
    Kx, Mx = assemble_1d(p, ncell[0], h[0])
    Ky, My = assemble_1d(p, ncell[1], h[1])
    Kz, Mz = assemble_1d(p, ncell[2], h[2])
    K = np.kron(Kz, np.kron(My, Mx)) + np.kron(Mz, np.kron(Ky, Mx)) + np.kron(Mz, np.kron(My, Kx))
    M = np.kron(Mz, np.kron(My, Mx))
    return K, M


def lex_index(dof_coord, p, ncell):
    """Map node-lattice coordinates (in units of h/p) to lexicographic indices."""
    n = [p * c + 1 for c in ncell]
    c = np.asarray(dof_coord)
    return c[:, 0] + n[0] * (c[:, 1] + n[1] * c[:, 2])
