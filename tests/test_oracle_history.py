"""Pins of the oracle's treatment of the material history across mesh changes (Sec. 4.1: the
coarsening restriction with r_coarsen = 0.9; Sec. 2: r_c is history data that moves with the
mesh): the transfer is the identity on an unchanged mesh, refining then coarsening back
returns every value exactly (copy on refinement, injection on coarsening), refined cells only
take values of the cell they came from, newly activated cells start at 0 (powder) or 1, and
the pins keep every family with a cell below r_coarsen from merging while the others merge."""
import numpy as np
import pytest

from paper_2302_05164_gb300 import inputs as I


def leaf_boxes(m, desc):
    t = m.tables()
    lv = t["leaves"]
    L = desc["max_level"]
    size = 2 ** (L - lv[:, 3])
    return lv[:, :3], size, lv[:, 4] == 1, lv[:, 3]


def meshes(oracle_mod, p):
    base = [I.uniform_region(1)]
    ball = (I.BALL, (0.3e-3, 0.25e-3, 0.25e-3), (0, 0, 0), 90e-6, 3)
    da = I.mesh_desc((4, 2, 2), (125e-6,) * 3, p, 3, base)
    db = I.mesh_desc((4, 2, 2), (125e-6,) * 3, p, 3, base + [ball])
    return da, db, oracle_mod.Mesh(da), oracle_mod.Mesh(db)


@pytest.mark.parametrize("p", [1, 2])
def test_history_transfer_identity_and_round_trip(oracle_mod, p):
    da, db, ma, mb = meshes(oracle_mod, p)
    assert mb.n_active > ma.n_active
    rng = np.random.default_rng(3)
    ha = rng.uniform(0.0, 1.0, size=(ma.n_active, (p + 1) ** 3))
    assert np.array_equal(oracle_mod.transfer_history(ma, ha, oracle_mod.Mesh(da)), ha)
    hb = oracle_mod.transfer_history(ma, ha, mb)
    # every refined cell holds only values of the coarse cell it lies in
    pa, sa, acta, _ = leaf_boxes(ma, da)
    pb, sb, actb, _ = leaf_boxes(mb, db)
    ia, ib = np.where(acta)[0], np.where(actb)[0]
    for c, leaf in enumerate(ib):
        inside = np.all((pa[ia] <= pb[leaf]) & (pb[leaf] + sb[leaf] <= pa[ia] + sa[ia][:, None]), axis=1)
        assert inside.sum() == 1
        assert set(hb[c]) <= set(ha[np.where(inside)[0][0]])
    # coarsening back injects the copied values: the round trip is exact
    assert np.array_equal(oracle_mod.transfer_history(mb, hb, ma), ha)


def test_history_of_newly_activated_cells(oracle_mod):
    d0 = I.c3_mesh()
    d1 = I.c3_mesh(active_top_z=I.C3_LAYER_TOP)
    m0, m1 = oracle_mod.Mesh(d0), oracle_mod.Mesh(d1)
    t0, t1 = m0.tables(), m1.tables()
    newly = (t1["leaves"][:, 4] == 1) & ~(t0["leaves"][:, 4] == 1)
    m1.set_material(newly[t1["leaves"][:, 4] == 1].astype(np.uint8))
    h0 = np.random.default_rng(1).uniform(0.2, 0.8, size=(m0.n_active, 8))
    h1 = oracle_mod.transfer_history(m0, h0, m1)
    new_cells = newly[t1["leaves"][:, 4] == 1]
    assert np.all(h1[new_cells] == 0.0)  # the new powder layer starts unconsolidated
    assert np.array_equal(h1[~new_cells], h0)  # the old cells keep theirs (same cells, same order)


@pytest.mark.parametrize("p", [1, 2])
def test_gated_coarsening_keeps_unconsolidated_families(oracle_mod, p):
    """Coarsen everything back to level 1 after a refined ball (level 3): the families that
    hold a cell with r_c below 0.9 keep their level, all other fine cells merge."""
    da, db, ma, mb = meshes(oracle_mod, p)
    pb, sb, actb, lvb = leaf_boxes(mb, db)
    ib = np.where(actb)[0]
    rng = np.random.default_rng(7)
    rc_min = np.where(rng.uniform(size=mb.n_active) < 0.05, 0.5, 0.95)
    rc_min[lvb[ib] <= 1] = 0.95
    low = ib[rc_min < 0.9]
    assert len(low) > 0
    pins = mb.gate_pins(rc_min, 0.9)
    dg = dict(da, regions=da["regions"] + pins)
    mg = oracle_mod.Mesh(dg)
    pg, sg, actg, lvg = leaf_boxes(mg, dg)
    for leaf in low:
        ps = 2 * sb[leaf]
        parent = pb[leaf] // ps * ps
        # no leaf of the new mesh coarser than the pinned level covers the parent's box
        over = np.all((pg < parent + ps) & (parent < pg + sg[:, None]), axis=1)
        assert np.all(lvg[over] >= lvb[leaf]), (leaf, lvg[over].min(), lvb[leaf])
    # a fine family without low cells (and not within reach of a pin or balance) merged
    fine = [leaf for leaf in ib if lvb[leaf] == 3]
    kept = sum(1 for leaf in fine if np.any(np.all(pg == pb[leaf], axis=1) & (lvg == 3)))
    assert kept < len(fine)
    assert mg.n_active < mb.n_active
