"""Bit-exact parity of the library's host mesh (a1: forest, balance, Z-order, activity,
first-touch dofs, hanging-node constraints, Dirichlet flags, colours, top faces) with the
oracle's independent implementation, on seeded random refinement patterns."""
import numpy as np
import pytest

from paper_2302_05164_gb300 import inputs as I
from paper_2302_05164_gb300 import pbf

KEYS = ("leaves", "cell_dofs", "con_ptr", "con_idx", "con_w", "hang_coord", "dof_coord", "dirichlet",
        "colour", "top")


def compare(o_tables, l_tables, keys=KEYS):
    for k in keys:
        a, b = o_tables[k], l_tables[k]
        assert a.shape == b.shape, (k, a.shape, b.shape)
        assert np.array_equal(a, b), k


def random_desc(seed, p):
    rng = np.random.default_rng(seed)
    nt = tuple(int(v) for v in rng.integers(1, 4, 3))
    th = tuple(float(v) for v in rng.uniform(0.5, 1.5, 3))
    L = int(rng.integers(1, 4))
    regions = []
    ext = np.array(nt) * np.array(th)
    for _ in range(int(rng.integers(1, 4))):
        kind = int(rng.integers(0, 2))
        a = rng.uniform(0, 1, 3) * ext
        b = a + rng.uniform(0, 0.3, 3) * ext
        regions.append((kind, tuple(a), tuple(b), float(rng.uniform(0.05, 0.5) * ext.min()), int(rng.integers(1, L + 1))))
    top = float(rng.uniform(0.4, 1.1) * ext[2])
    faces = int(rng.integers(0, 64))
    exists = None
    if seed % 3 == 0:
        exists = (rng.uniform(size=nt[::-1]) > 0.25).astype(np.uint8)
        exists.flat[0] = 1
    return I.mesh_desc(nt, th, p, L, regions, active_top_z=top, dirichlet_faces=faces, tree_exists=exists,
                       powder_z0=0.3 * ext[2], powder_z1=0.6 * ext[2])


@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("p", [1, 2])
def test_random_meshes_bit_exact(oracle_mod, seed, p):
    d = random_desc(seed, p)
    om = oracle_mod.Mesh(d)
    lm = pbf.Mesh(d)
    info = lm.info()
    assert (info["n_active"], info["n_dofs"], info["n_hanging"], info["n_colours"], info["n_top_faces"]) == \
        (om.n_active, om.n_dofs, om.n_hanging, om.n_colours, om.n_top)
    ot, lt = om.tables(), lm.tables()
    compare(ot, lt, KEYS + ("material",))


@pytest.mark.parametrize("name", ["c1", "c2", "c4", "c5"])
def test_workload_meshes_bit_exact(oracle_mod, name):
    # c5: the part-scale stand-in's first layer at level 4 (213,120 cells, 1.72 M dofs; rib
    # pillars as a tree mask, a powder layer, the heat-affected zone refined)
    d = {"c1": I.c1_mesh, "c2": I.c2_mesh, "c4": I.c4_mesh, "c5": lambda: I.c5_mesh(level=4)}[name]()
    om, lm = oracle_mod.Mesh(d), pbf.Mesh(d)
    compare(om.tables(), lm.tables())


def test_layer_activation_topology(oracle_mod):
    """After pbf_mesh_activate_layer the library mesh equals the canonical mesh of the new
    activation height; newly active cells carry the requested material."""
    d0 = I.c3_mesh()
    lm = pbf.Mesh(d0)
    old = lm.tables()
    pbf.pbf_mesh_activate_layer(lm.h, I.C3_LAYER_TOP, 1, I.T0)
    om = oracle_mod.Mesh(I.c3_mesh(active_top_z=I.C3_LAYER_TOP))
    new = lm.tables()
    compare(om.tables(), new)
    newly = (new["leaves"][:, 4] == 1) & (old["leaves"][:, 4] == 0)
    assert newly.sum() == 64 * 32 * 3
    assert np.all(new["material"][newly] == 1) and np.all(new["material"][~newly] == 0)
    assert lm.info()["generation"] == 2


def test_adapt_topology(oracle_mod):
    d0 = I.c2_mesh(spot=(0.5e-3, 0.55e-3))
    lm = pbf.Mesh(d0)
    regs = I.c2_spot_regions(0.6e-3, 0.55e-3)
    pbf.pbf_mesh_adapt(lm.h, regs)
    d1 = I.c2_mesh(spot=(0.6e-3, 0.55e-3))
    compare(oracle_mod.Mesh(d1).tables(), lm.tables())


@pytest.mark.parametrize("p", [1, 2])
def test_wide_lattice_mesh_bit_exact(oracle_mod, p):
    """A forest whose node lattice needs more than 64 bits together with the slot index (255 x 64
    trees at up to 12 levels: the library sorts its node entries as (key, slot) pairs instead of
    single words), refined to level 2 in a ball, with hanging nodes."""
    regions = [(I.BALL, (16e-3, 4e-3, 0.06e-3), (0, 0, 0), 0.4e-3, 2)]
    d = I.mesh_desc((255, 64, 1), (125e-6,) * 3, p, 12, regions)
    om, lm = oracle_mod.Mesh(d), pbf.Mesh(d)
    info = lm.info()
    ext = np.array([255, 64, 1]) << 12
    lattice_bits = int(np.ceil(np.log2(float(np.prod(p * ext + 1)))))
    slot_bits = int(np.ceil(np.log2(info["n_active"] * info["nodes_per_cell"])))
    assert lattice_bits + slot_bits > 64 and info["n_hanging"] > 0
    compare(om.tables(), lm.tables())
