"""The host mesh builder runs its independent work on all host cores (balance, node table,
numbering, constraint rows, holders, the fused step's patch tables, the transfer and history
maps); its tables must not depend on the number of threads.
Two processes, one with a single OpenMP thread and one with four, build a Q2 mesh with nested
refinement, hanging nodes and an inactive layer, adapt it twice (the spot moves), and export
the tables after each step: all arrays are equal. No GPU is needed."""
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys
import numpy as np
sys.path.insert(0, {root!r})
from paper_2302_05164_gb300 import inputs as I
from paper_2302_05164_gb300 import pbf

def regions(x):
    return [I.uniform_region(2), (I.BALL, (x, 0.25e-3, 0.25e-3), (0, 0, 0), 120e-6, 3),
            (I.BOX, (x - 40e-6, 0.2e-3, 0.2e-3), (x + 40e-6, 0.3e-3, 0.25e-3), 0.0, 4)]

desc = I.mesh_desc((8, 4, 2), (125e-6,) * 3, 2, 4, regions(0.3e-3), active_top_z=0.23e-3,
                   powder_z0=0.15e-3, powder_z1=0.2e-3)
m = pbf.Mesh(desc)
out = {{}}
for step, x in enumerate((None, 0.45e-3, 0.6e-3)):
    if x is not None:
        pbf.pbf_mesh_adapt(m.h, regions(x))
        for k, v in pbf.pbf_mesh_transfer_map(m.h).items():
            out[f"{{step}}_map_{{k}}"] = np.asarray(v)
        out[f"{{step}}_history_map"] = pbf.pbf_mesh_history_map(m.h)[0]
    for k, v in m.tables().items():
        out[f"{{step}}_{{k}}"] = np.asarray(v)
    for k, v in pbf.pbf_mesh_step_tables(m.h).items():
        out[f"{{step}}_step_{{k}}"] = np.asarray(v)
np.savez(sys.argv[1], **out)
"""


def run(threads, path):
    env = dict(os.environ, OMP_NUM_THREADS=str(threads))
    subprocess.run([sys.executable, "-c", SCRIPT.format(root=ROOT), path], env=env, check=True, timeout=600)
    return np.load(path)


def test_mesh_tables_do_not_depend_on_the_thread_count(tmp_path):
    one = run(1, str(tmp_path / "one.npz"))
    four = run(4, str(tmp_path / "four.npz"))
    assert sorted(one.files) == sorted(four.files)
    assert any(k.endswith("_con_idx") and one[k].size > 0 for k in one.files)  # hanging nodes exist
    assert one["0_cell_dofs"].size > 2 * 65536  # three or more chunks of the prefix sums over slots
    assert all(one[f"{s}_step_ptr"].size > 8 for s in range(3))  # patches for several threads
    # rows of every thread, with prolongation (several entries) among them
    assert all(one[f"{s}_map_ptr"].size > 10000 and one[f"{s}_map_idx"].size > one[f"{s}_map_ptr"].size for s in (1, 2))
    for k in one.files:
        assert one[k].shape == four[k].shape, k
        assert np.array_equal(one[k], four[k]), k
