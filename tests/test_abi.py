"""The C-ABI library loads without a GPU and exports every entry point include/pbf.h declares;
host-only entry points validate their arguments."""
import os
import re

import pytest

from paper_2302_05164_gb300 import inputs as I
from paper_2302_05164_gb300 import pbf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "pbf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pbf_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported():
    names = declared_symbols()
    assert len(names) >= 20
    lib = pbf.lib()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # the binding covers the same names
    assert set(names) <= set(pbf._SIGS)


def test_host_entry_points_validate_arguments():
    bad = I.c1_mesh()
    bad["degree"] = 3
    with pytest.raises(pbf.PbfError) as e:
        pbf.pbf_mesh_create(bad)
    assert e.value.status == 1 and "degree" in str(e.value)
    m = pbf.Mesh(I.c1_mesh())
    with pytest.raises(pbf.PbfError):
        pbf.pbf_mesh_activate_layer(m.h, -1.0, 0, 353.0)  # activation height may not decrease
    with pytest.raises(pbf.PbfError):
        pbf.pbf_mesh_transfer(m.h, None, None, stream=0)  # nothing pending / null pointers
    assert pbf.pbf_mesh_info(m.h)["generation"] == 1


def test_options_and_schedules_validate_arguments_without_a_gpu():
    """Host-side checks of the option entry points and the checkpoint schedule (no context,
    no device work)."""
    for call in (lambda: pbf.pbf_ctx_set_surface_loss(None, I.SURFACE_LOSS),
                 lambda: pbf.pbf_ctx_set_surface_loss(None, None),
                 lambda: pbf.pbf_ctx_set_phase(None, I.PHASE),
                 lambda: pbf.pbf_ctx_set_kernel_shape(None, 5),
                 lambda: pbf.pbf_revolve_cost(0, 3),
                 lambda: pbf.pbf_revolve_cost(10, 0)):
        with pytest.raises(pbf.PbfError) as e:
            call()
        assert e.value.status == 1
    # revolve: 2000 steps with 40 stored states cost 5097 forward steps (Griewank-Walther)
    assert pbf.pbf_revolve_cost(2000, 40) == 5097
