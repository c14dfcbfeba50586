"""Brute-force assembly for the oracle's pins: explicit constraint matrices P_e and textbook
element matrices (tests/textbook.py) summed into dense global matrices sum_e P_e^T A_e P_e,
written independently of the oracle and of the CUDA path."""
import numpy as np

from paper_2302_05164_gb300 import inputs as I
from tests import textbook as TB


def small_amr(p, L=2, dirichlet=I.DIRICHLET_BOTTOM, top=1e30):
    regions = [(I.BALL, (0.3, 0.4, 0.9), (0, 0, 0), 0.35, L), (I.BOX, (1.2, 0.2, 0.3), (1.3, 0.3, 0.5), 0.05, L)]
    return I.mesh_desc((2, 1, 1), (1.0, 1.0, 1.0), p, L, regions, dirichlet_faces=dirichlet, active_top_z=top)


def cells(m, desc):
    """Active cells in the oracle's cell order: lower corner, size (from the leaf table) and
    material of each."""
    t = m.tables()
    act = t["leaves"][:, 4] == 1
    lv = t["leaves"][act]
    mat = t["material"][act]
    L = desc["max_level"]
    th = np.array(desc["tree_h"])
    lo = np.array(desc["origin"]) + lv[:, :3] * th / 2.0 ** L
    h = th[None, :] / 2.0 ** lv[:, 3:4]
    return lo, h, mat, t


def element_matrices(p, h):
    """Textbook Q_p stiffness (unit conductivity) and consistent mass of one brick cell."""
    K1 = [TB.ELEM[p][0] / h[d] for d in range(3)]
    M1 = [TB.ELEM[p][1] * h[d] for d in range(3)]
    K = np.kron(K1[2], np.kron(M1[1], M1[0])) + np.kron(M1[2], np.kron(K1[1], M1[0])) + \
        np.kron(M1[2], np.kron(M1[1], K1[0]))
    M = np.kron(M1[2], np.kron(M1[1], M1[0]))
    return K, M


def prolongation(t, c, n_dofs):
    """P_e: cell node values = P_e T, from the cell's dof list and the constraint rows."""
    cd = t["cell_dofs"][c]
    P = np.zeros((len(cd), n_dofs))
    for a, v in enumerate(cd):
        if v >= 0:
            P[a, v] = 1.0
        else:
            r = -1 - v
            for e in range(t["con_ptr"][r], t["con_ptr"][r + 1]):
                P[a, t["con_idx"][e]] += t["con_w"][e]
    return P


def assemble(m, desc, coef_k, coef_m):
    """sum_e P_e^T (coef_k(mat) K_e + coef_m M_e) P_e over the active cells."""
    lo, h, mat, t = cells(m, desc)
    n = m.n_dofs
    A = np.zeros((n, n))
    for c in range(m.n_active):
        K, M = element_matrices(desc["degree"], h[c])
        P = prolongation(t, c, n)
        A += P.T @ (coef_k(mat[c]) * K + coef_m * M) @ P
    return A, t
