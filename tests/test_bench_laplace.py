"""Host logic of the benchmark's constant-coefficient entry (no GPU): with stand-ins for the
binding and for torch's device calls, the entry builds an FP32-operator context of the
constant material, keeps the headline's kernel shape, runs warm-up and timed calls without a
source, closes the context, and turns the event times into GDoF/s and the full-step ratio."""
import types

import numpy as np

import bench
from paper_2302_05164_gb300 import inputs as I


class FakeEvent:
    clock = 0.0

    def __init__(self, enable_timing=False):
        self.t = None

    def record(self, stream=None):
        self.t = FakeEvent.clock

    def elapsed_time(self, other):
        return other.t - self.t


def fake_modules(calls, ms_per_call):
    class Context:
        def __init__(self, mesh, mat, prec):
            calls.append(("ctx", dict(mat), prec))
            self.h = "ctx"

        def close(self):
            calls.append(("close",))

    def explicit_step(h, T, laser, t0, dt, n, stream=None):
        calls.append(("step", laser, t0, dt, n))
        FakeEvent.clock += ms_per_call

    pbf = types.SimpleNamespace(Context=Context, PBF_F32OP=1, pbf_explicit_step=explicit_step,
                                pbf_ctx_set_kernel_shape=lambda h, s: calls.append(("shape", s)))
    cuda = types.SimpleNamespace(Event=FakeEvent, synchronize=lambda: None)
    torch = types.SimpleNamespace(tensor=lambda x, dtype=None, device=None: np.array(x), float64=np.float64,
                                  cuda=cuda)
    return pbf, torch


def test_constant_coefficient_entry():
    calls = []
    pbf, torch = fake_modules(calls, ms_per_call=1.0)
    mesh = types.SimpleNamespace(info=lambda: {"n_dofs": 1_000_000})
    flush = types.SimpleNamespace(fill_=lambda v: None)
    K, dt = 4, 1e-7
    out = bench.bench_laplace(pbf, I, torch, None, flush, mesh, np.zeros(3), dt, 5, K, full_gdofs=25.0)
    kinds = [c[0] for c in calls]
    assert kinds == ["ctx", "shape"] + ["step"] * (3 + K) + ["close"]
    mat, prec = calls[0][1], calls[0][2]
    assert prec == 1 and mat["k0"] == mat["k1"] and mat["latent"] == 0.0 and mat["powder_k_scale"] == 1.0
    assert calls[1] == ("shape", 5)
    steps = [c for c in calls if c[0] == "step"]
    assert all(s[1] is None and s[3] == dt and s[4] == bench.CHUNK for s in steps)  # no source
    assert [s[2] for s in steps] == [k * bench.CHUNK * dt for k in range(3 + K)]  # times continue
    # 1 ms per call of CHUNK steps over 1e6 dofs
    assert np.isclose(out["ms_per_step"], 1.0)
    assert np.isclose(out["value"], 1e6 * bench.CHUNK / 1e-3 / 1e9)
    assert np.isclose(out["full_step_over_laplace"], 25.0 / out["value"])
    assert out["step_shape"] == bench.SHAPES[5] and out["paper_full_step_over_laplace"] == 0.44
