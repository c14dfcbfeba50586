"""Pins of the oracle's octree mesh, numbering and hanging-node constraints (Sec. 4.1 of the
paper: octree forest, 2:1 balance, Z-curve order, inactive cells; hanging-node constraints).
Each check is a property fixed by the definition, verified by brute force on small meshes."""
import itertools

import numpy as np
import pytest

from paper_2302_05164_gb300 import inputs as I


def small_amr(p, active_top_z=1e30, regions=None):
    regions = regions or [(I.BALL, (0.3, 0.45, 2.0), (0, 0, 0), 0.6, 3),
                          (I.BOX, (1.2, 0.2, 0.0), (1.3, 0.3, 0.4), 0.05, 2)]
    return I.mesh_desc((2, 2, 2), (1.0, 1.0, 1.0), p, 3, regions, active_top_z=active_top_z)


@pytest.mark.parametrize("p", [1, 2])
def test_uniform_counts(oracle_mod, p):
    d = I.mesh_desc((3, 2, 2), (1.0, 1.0, 0.5), p, 1, [I.uniform_region(1)])
    m = oracle_mod.Mesh(d)
    assert m.n_active == 3 * 2 * 2 * 8
    assert m.n_dofs == (p * 6 + 1) * (p * 4 + 1) * (p * 4 + 1)
    assert m.n_hanging == 0
    assert m.n_colours == 8  # vertex-sharing cells of a structured brick need 2^3 colours
    t = m.tables()
    # the Dirichlet (bottom) dofs are exactly those with z = 0
    assert np.array_equal(t["dirichlet"].astype(bool), t["dof_coord"][:, 2] == 0)
    assert m.n_top == 6 * 4


def test_c1_workload_sizes(oracle_mod):
    m = oracle_mod.Mesh(I.c1_mesh())
    assert (m.n_active, m.n_dofs, m.n_hanging, m.n_top) == (32768, 65 * 33 * 17, 0, 64 * 32)


def leaf_boxes(t, L):
    lv = t["leaves"]
    s = (1 << (L - lv[:, 3]))
    lo = lv[:, :3]
    return lo, lo + s[:, None], lv[:, 3], lv[:, 4].astype(bool)


@pytest.mark.parametrize("p", [1, 2])
def test_forest_partition_balance_order(oracle_mod, p):
    d = small_amr(p)
    m = oracle_mod.Mesh(d)
    t = m.tables()
    L = d["max_level"]
    lo, hi, lev, act = leaf_boxes(t, L)
    # leaves tile the lattice box exactly (volumes add up, no overlaps)
    N = np.array(d["ntree"]) << L
    assert ((hi - lo).prod(axis=1)).sum() == N.prod()
    n = len(lev)
    for i in range(n):
        ov = np.all((np.maximum(lo[i], lo) < np.minimum(hi[i], hi)), axis=1)
        assert ov.sum() == 1
    # 2:1 balance across faces, edges and vertices
    for i in range(n):
        touch = np.all((lo <= hi[i]) & (lo[i] <= hi), axis=1)
        assert np.all(np.abs(lev[touch] - lev[i]) <= 1)
    # refinement targets are met: leaves near the ball centre reach level 3
    assert lev.max() == 3
    # canonical order: tree index, then Morton key of the anchor inside the tree
    def key(row):
        x, y, z = (int(v) for v in row[:3])
        tx, ty, tz = x >> L, y >> L, z >> L
        tree = tx + d["ntree"][0] * (ty + d["ntree"][1] * tz)
        mk = 0
        for b in range(L):
            mk |= ((x >> b) & 1) << (3 * b) | ((y >> b) & 1) << (3 * b + 1) | ((z >> b) & 1) << (3 * b + 2)
        return (tree, mk)
    keys = [key(r) for r in t["leaves"]]
    assert keys == sorted(keys) and len(set(keys)) == len(keys)


def node_sets(t, p, L):
    """Brute force: nodal points of every active cell, on the node lattice (h_min / p)."""
    lo, hi, lev, act = leaf_boxes(t, L)
    cells = []
    for i in np.nonzero(act)[0]:
        s = hi[i][0] - lo[i][0]
        pts = {tuple(p * lo[i] + np.array(ijk) * s) for ijk in itertools.product(range(p + 1), repeat=3)}
        cells.append((p * lo[i], p * hi[i], pts))
    return cells


@pytest.mark.parametrize("p", [1, 2])
@pytest.mark.parametrize("top", [1e30, 1.375])
def test_hanging_nodes_and_constraints(oracle_mod, p, top):
    d = small_amr(p, active_top_z=top)
    m = oracle_mod.Mesh(d)
    t = m.tables()
    L = d["max_level"]
    cells = node_sets(t, p, L)
    assert len(cells) == m.n_active
    dofs = {tuple(c) for c in t["dof_coord"]}
    hang = {tuple(c) for c in t["hang_coord"]}
    allnodes = set().union(*[c[2] for c in cells])
    assert dofs | hang == allnodes and not (dofs & hang)
    # a node hangs iff an active cell holds it in its closure without it being a nodal point
    for node in allnodes:
        x = np.array(node)
        is_h = any(np.all(lo <= x) and np.all(x <= hi) and node not in pts for lo, hi, pts in cells)
        assert is_h == (node in hang)
    # rows sum to one, masters are sorted dofs, weights are dyadic (exact)
    ptr, idx, w = t["con_ptr"], t["con_idx"], t["con_w"]
    for r in range(m.n_hanging):
        seg = slice(ptr[r], ptr[r + 1])
        assert np.sum(w[seg]) == 1.0
        assert np.all(np.diff(idx[seg]) > 0)
        assert np.all(w[seg] != 0)
        assert np.all(w[seg] * 1024 == np.round(w[seg] * 1024))
    # a global Q_p polynomial is reproduced at hanging nodes by its constraint
    rng = np.random.default_rng(3)
    coef = rng.normal(size=(p + 1, p + 1, p + 1))

    def u(c):
        x, y, z = (np.asarray(c, float) / (p * (1 << L))).T
        return sum(coef[a, b, g] * x ** a * y ** b * z ** g
                   for a in range(p + 1) for b in range(p + 1) for g in range(p + 1))
    ud = u(t["dof_coord"])
    uh = u(t["hang_coord"])
    for r in range(m.n_hanging):
        seg = slice(ptr[r], ptr[r + 1])
        assert abs(np.dot(w[seg], ud[idx[seg]]) - uh[r]) < 1e-12 * max(1.0, abs(uh[r]))


@pytest.mark.parametrize("p", [1, 2])
def test_numbering_colouring(oracle_mod, p):
    d = small_amr(p)
    m = oracle_mod.Mesh(d)
    t = m.tables()
    cd = t["cell_dofs"]
    # first-touch numbering: dof ids appear in increasing order of first use
    seen = []
    s = set()
    for v in cd.ravel():
        if v >= 0 and v not in s:
            s.add(v)
            seen.append(v)
    assert seen == list(range(m.n_dofs))
    ptr, idx = t["con_ptr"], t["con_idx"]

    def touched(c):
        out = set()
        for v in cd[c]:
            out |= {int(v)} if v >= 0 else set(idx[ptr[-1 - v]:ptr[-v]].tolist())
        return out
    tsets = [touched(c) for c in range(m.n_active)]
    col = t["colour"]
    for c in range(m.n_active):
        clash = {col[e] for e in range(c) if tsets[e] & tsets[c]}
        assert col[c] not in clash  # valid
        assert all(k in clash for k in range(col[c]))  # greedy: smallest free colour
    assert m.n_colours == col.max() + 1


def test_activation_inactive_cells(oracle_mod):
    d = small_amr(1, active_top_z=1.375)
    m = oracle_mod.Mesh(d)
    t = m.tables()
    L = d["max_level"]
    lo, hi, lev, act = leaf_boxes(t, L)
    zlo = lo[:, 2] / (1 << L)
    assert np.array_equal(act, zlo < 1.375)
    # the top faces are those of active cells whose upper neighbours are inactive or absent
    zhi = hi[act][:, 2] / (1 << L)
    assert np.array_equal(t["top"].astype(bool), (zhi >= 1.375) | (hi[act][:, 2] == 2 << L))
