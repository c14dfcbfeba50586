"""The allocation-free critical-time-step entry point, for callers that cannot allocate
device memory during a call (pool-managed device memory, latency-bound loops). Called twice
in a row through the C ABI, it must give the eigenvalue estimate of the regular entry point
within the tolerance of the CFL parity test, and the device's free memory must not change
across either call. This file is collected last on purpose."""
import pytest

from paper_2302_05164_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_noalloc_estimate_matches_regular_entry_point():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_05164_gb300 import pbf
    regions = [(I.BALL, (0.3e-3, 0.25e-3, 0.25e-3), (0, 0, 0), 120e-6, 3)]
    desc = I.mesh_desc((8, 4, 2), (125e-6,) * 3, 2, 3, regions)
    mesh = pbf.Mesh(desc)
    ctx = pbf.Context(mesh, I.TI64_CONST, pbf.PBF_F64)
    n = mesh.info()["n_dofs"]
    x0 = torch.tensor(I.start_vector(n, seed=11), dtype=torch.float64, device="cuda")
    y = torch.empty(n, dtype=torch.float64, device="cuda")
    xs = [x0.clone() for _ in range(2)]
    torch.cuda.synchronize()
    # first the allocation-free calls (in a fresh process nothing else has run on this
    # context yet), each bracketed by the device's free memory
    results = []
    for x in xs:  # two calls in a row share the static scratch
        free0 = torch.cuda.mem_get_info()[0]
        alloc0 = torch.cuda.memory_allocated()
        lam, dtc, it = pbf.pbf_estimate_dt_noalloc(ctx.h, x, y, max_iter=60, rtol=0.0)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0, "the call changed the device's free memory"
        assert torch.cuda.memory_allocated() == alloc0
        results.append((lam, dtc, it))
    lam_ref, dt_ref, it_ref = pbf.pbf_estimate_dt(ctx.h, x0.clone(), max_iter=60, rtol=0.0)
    for (lam, dtc, it), x in zip(results, xs):
        assert it == it_ref == 60
        assert abs(lam - lam_ref) < 1e-9 * lam_ref
        assert abs(dtc - 2.0 / lam) < 1e-15
        assert torch.isfinite(x).all() and x.abs().max().item() > 0
    # overlapping vectors are refused before any work
    with pytest.raises(pbf.PbfError):
        pbf.pbf_estimate_dt_noalloc(ctx.h, xs[0], xs[0], max_iter=2, rtol=0.0)
    ctx.close()
    mesh.close()
