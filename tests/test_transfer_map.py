"""The library's transfer map of a mesh change, on the host (no GPU): the rows that
`pbf_mesh_transfer` applies on the device, read back through `pbf_mesh_transfer_map` and
applied here with numpy.
- Re-adaptation (prolongation and injection of the old FE field, Q1 and Q2 with hanging
  nodes): the map reproduces every polynomial of the element space, its rows are partitions
  of unity over ascending old dofs, and a smooth field moves as the oracle moves it.
- Layer activation: shared nodes copy their old value exactly, the new ones take T_init, as in
  the oracle.
Also: the sizes-only call and the error cases."""
import numpy as np
import pytest

from paper_2302_05164_gb300 import inputs as I
from paper_2302_05164_gb300 import pbf


def apply_map(t, T_old):
    out = np.full(t["n_new"], t["fill"])
    ptr = t["ptr"]
    contrib = t["w"] * T_old[t["idx"]]
    row = np.repeat(np.arange(t["n_new"]), np.diff(ptr))
    filled = np.diff(ptr) > 0
    out[filled] = 0.0
    np.add.at(out, row, contrib)
    return out


def desc(p, x, top=1e30):
    return I.mesh_desc((8, 4, 2), (125e-6,) * 3, p, 3, I.c2_spot_regions(x, 0.25e-3, 0.25e-3, 150e-6),
                       active_top_z=top)


def coords(d, tables):
    return np.array(d["origin"]) + np.array(d["tree_h"]) * tables["dof_coord"] / (d["degree"] * 2.0 ** d["max_level"])


@pytest.mark.parametrize("p", [1, 2])
def test_adapt_map_reproduces_the_element_space_and_matches_the_oracle(oracle_mod, p):
    d0, d1 = desc(p, 0.3e-3), desc(p, 0.5e-3)
    m = pbf.Mesh(d0)
    x0 = coords(d0, m.tables())
    pbf.pbf_mesh_adapt(m.h, d1["regions"])
    t = pbf.pbf_mesh_transfer_map(m.h)
    x1 = coords(d0, m.tables())
    assert t["n_old"] == len(x0) and t["n_new"] == len(x1) and t["n_new"] != t["n_old"]
    ptr, idx, w = t["ptr"], t["idx"], t["w"]
    lens = np.diff(ptr)
    assert lens.min() >= 1  # same activation: every new dof lies in the old domain
    assert lens.max() > 1 and np.any(lens == 1)  # prolongation and injection both occur
    for i in range(t["n_new"]):
        r = slice(ptr[i], ptr[i + 1])
        assert np.all(np.diff(idx[r]) > 0)
        assert abs(w[r].sum() - 1.0) < 1e-14 * lens[i]
    # every polynomial of degree p in each coordinate (Q_p) is carried over exactly
    rng = np.random.default_rng(11)
    coef = rng.normal(size=(p + 1, p + 1, p + 1))
    s = 1.0 / 1e-3  # coordinates in mm: the monomials stay of order one

    def u(x):
        y = x * s
        return sum(coef[i, j, k] * y[:, 0] ** i * y[:, 1] ** j * y[:, 2] ** k
                   for i in range(p + 1) for j in range(p + 1) for k in range(p + 1))
    assert np.max(np.abs(apply_map(t, u(x0)) - u(x1))) < 1e-12 * np.abs(u(x1)).max()
    # a smooth field as the oracle moves it
    o0, o1 = oracle_mod.Mesh(d0), oracle_mod.Mesh(d1)
    T0 = I.smooth_field(o0.dof_xyz(), seed=6)
    ref = oracle_mod.transfer(o0, T0, o1, -1.0)
    got = apply_map(t, T0)
    assert np.max(np.abs(got - ref)) < 1e-13 * np.abs(ref).max()
    m.close()


def test_activation_map_copies_shared_nodes_and_fills_new_ones(oracle_mod):
    d0 = I.c3_mesh(active_top_z=0.25e-3)
    d1 = dict(d0, active_top_z=0.3e-3)
    m = pbf.Mesh(d0)
    pbf.pbf_mesh_activate_layer(m.h, d1["active_top_z"], 1, 353.0)
    t = pbf.pbf_mesh_transfer_map(m.h)
    assert t["fill"] == 353.0
    lens = np.diff(t["ptr"])
    assert set(np.unique(lens)) == {0, 1}  # a copy or the fill: the old nodes keep their place
    assert np.all(t["w"] == 1.0)
    o0, o1 = oracle_mod.Mesh(d0), oracle_mod.Mesh(d1)
    T0 = I.smooth_field(o0.dof_xyz(), seed=8)
    ref = oracle_mod.transfer(o0, T0, o1, 353.0)
    got = apply_map(t, T0)
    assert np.array_equal(got, ref)
    assert np.sum(lens == 0) == np.sum(ref == 353.0) > 0
    m.close()


def test_sizes_only_call_and_errors():
    m = pbf.Mesh(I.c1_mesh())
    L = pbf.lib()
    t = pbf.TransferMapC()
    assert L.pbf_mesh_transfer_map(m.h, pbf.C.byref(t)) == 8  # nothing pending
    pbf.pbf_mesh_adapt(m.h, [I.uniform_region(2), (I.BALL, (0.5e-3, 0.25e-3, 0.25e-3), (0, 0, 0), 100e-6, 3)])
    assert L.pbf_mesh_transfer_map(m.h, pbf.C.byref(t)) == 0
    assert t.n_old == 36465 and t.n_new == m.info()["n_dofs"] and t.n_entries >= t.n_new
    buf = np.zeros(8, np.int32)
    t.n_new, t.ptr = 7, buf.ctypes.data
    assert L.pbf_mesh_transfer_map(m.h, pbf.C.byref(t)) == 1 and (buf == 0).all()
    assert L.pbf_mesh_transfer_map(None, pbf.C.byref(t)) == 1
    assert L.pbf_mesh_transfer_map(m.h, None) == 1
    m.close()
