"""Host logic of the benchmark's metadata record (no GPU): the bytes it reports are the sizes of
the arrays that the two forms of the explicit step read at least once per step (the fused
step's patch tables; the per-cell form's cell-to-dof table and hanging-node rows with FP32
weights; per cell its level, material and top flag, the FP32 corner of a top cell; per dof the
FP32 inverse lumped mass), recomputed here from the exported mesh, and batching divides them
over the instances."""
import numpy as np

import bench
from paper_2302_05164_gb300 import inputs as I
from paper_2302_05164_gb300 import pbf


def test_metadata_bytes_are_the_array_sizes():
    m = pbf.Mesh(I.c4_mesh())
    info, t, st = m.info(), m.tables(), pbf.pbf_mesh_step_tables(m.h)
    fused = bench.metadata_bytes(pbf, m, True)
    per_cell = bench.metadata_bytes(pbf, m, False, 64)
    m.close()
    common = 3 * info["n_active"] + 12 * int(t["top"].sum()) + 4 * info["n_dofs"]
    assert fused["cell_and_dof_bytes"] == per_cell["cell_and_dof_bytes"] == common
    n_p = len(st["ptr"])
    assert fused["tables_bytes"] == (4 * n_p + 16 * n_p + 4 * st["slot"].size + 4 * st["cell"].size
                                     + 2 * st["loc"].size + (2 + 4) * st["hloc"].size)
    assert per_cell["tables_bytes"] == (t["cell_dofs"].nbytes + t["con_ptr"].nbytes + t["con_idx"].nbytes
                                        + t["con_w"].size * 4)
    for rec, batch in ((fused, 1), (per_cell, 64)):
        assert rec["bytes_per_step"] == rec["tables_bytes"] + rec["cell_and_dof_bytes"]
        assert rec["instances"] == batch
        assert np.isclose(rec["bytes_per_dof_update"], rec["bytes_per_step"] / (batch * info["n_dofs"]))
    assert fused["form"] == "fused step" and per_cell["form"] == "per-cell"


def test_a_failure_is_reported_not_raised():
    class Broken:
        h = None

        def info(self):
            raise RuntimeError("no mesh")
    assert "no mesh" in bench.metadata_bytes(pbf, Broken(), True)["error"]
