"""The library's history map of a mesh change, on the host (no GPU): the map that
`pbf_ctx_transfer_history` applies on the device, read back through `pbf_mesh_history_map`
and applied here with numpy to a history of the old mesh, equals the oracle's transfer of the
consolidated fraction r_c exactly:
- after a gated adaptation (the coarsening restriction of Sec. 4.1 with r_coarsen = 0.9),
  whose mesh is also the oracle's, bit for bit, with the oracle's pins;
- after a layer activation, where the new powder cells start at 0.
Also: a mesh that has not changed has no map."""
import numpy as np
import pytest

from paper_2302_05164_gb300 import inputs as I
from paper_2302_05164_gb300 import pbf


def apply_history_map(hmap, rc_old):
    out = np.where(hmap == -1, 0.0, 1.0)
    kept = hmap >= 0
    out[kept] = rc_old.reshape(-1)[hmap[kept]]
    return out


@pytest.mark.parametrize("p", [1, 2])
def test_gated_adaptation_history_map_matches_oracle(oracle_mod, p):
    top = 0.25e-3

    def regions(x):
        return [I.uniform_region(1), (I.BALL, (x, 0.25e-3, top), (0, 0, 0), 80e-6, 3)]

    d0 = I.mesh_desc((8, 4, 2), (125e-6,) * 3, p, 3, regions(0.30e-3), powder_z0=0.2e-3, powder_z1=0.3e-3)
    om = oracle_mod.Mesh(d0)
    nq = (p + 1) ** 3
    rng = np.random.default_rng(13)
    rc = rng.uniform(0.0, 1.0, size=(om.n_active, nq))
    rc[rng.uniform(size=om.n_active) < 0.7] = 1.0  # consolidated cells; the others gate coarsening
    r_min = rc.min(axis=1)
    pins = om.gate_pins(r_min, 0.9)
    assert len(pins) > 0
    om1 = oracle_mod.Mesh(dict(d0, regions=regions(0.55e-3) + pins))
    m = pbf.Mesh(d0)
    pbf.pbf_mesh_adapt_gated(m.h, regions(0.55e-3), r_min, 0.9)
    got_t, ref_t = m.tables(), om1.tables()
    for k in ("leaves", "cell_dofs", "con_ptr", "con_idx", "con_w", "dirichlet"):
        assert np.array_equal(got_t[k], ref_t[k]), k
    hmap, n_old = pbf.pbf_mesh_history_map(m.h)
    assert n_old == om.n_active and hmap.shape == (om1.n_active, nq)
    assert hmap.min() >= 0 and hmap.max() < n_old * nq  # same activation: every point has a source
    assert np.array_equal(apply_history_map(hmap, rc), oracle_mod.transfer_history(om, rc, om1))
    m.close()


def test_activation_history_map_matches_oracle(oracle_mod):
    d0 = I.c3_mesh(active_top_z=0.25e-3)
    d1 = dict(I.c3_mesh(active_top_z=I.C3_LAYER_TOP), powder_z0=0.25e-3, powder_z1=I.C3_LAYER_TOP)
    om, om1 = oracle_mod.Mesh(d0), oracle_mod.Mesh(d1)
    m = pbf.Mesh(d0)
    pbf.pbf_mesh_activate_layer(m.h, I.C3_LAYER_TOP, 1, I.T0)
    assert np.array_equal(m.tables()["cell_dofs"], om1.tables()["cell_dofs"])
    hmap, n_old = pbf.pbf_mesh_history_map(m.h)
    assert n_old == om.n_active and np.any(hmap == -1) and not np.any(hmap == -2)
    rc = np.random.default_rng(14).uniform(size=(om.n_active, 8))
    assert np.array_equal(apply_history_map(hmap, rc), oracle_mod.transfer_history(om, rc, om1))
    m.close()


def test_an_unchanged_mesh_has_no_history_map():
    m = pbf.Mesh(I.c1_mesh())
    with pytest.raises(pbf.PbfError) as e:
        pbf.pbf_mesh_history_map(m.h)
    assert e.value.status == 8
    m.close()
