"""The integer-only IEEE-754 conversions of the FP32-operator form agree bit for bit with
CUDA's own conversions (torch .float() / .double() on the device) on normal-range values,
including exact ties, powers of two, signs and values that round up into the next binade."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_05164_gb300 import pbf
    return pbf


def test_round_to_f32_matches_cuda(P):
    rng = np.random.default_rng(0)
    x = rng.uniform(-1, 1, 200000) * 10.0 ** rng.uniform(-30, 30, 200000)
    f = rng.uniform(-3000, 3000, 50000).astype(np.float32).astype(np.float64)
    ulp = np.spacing(np.abs(f).astype(np.float32)).astype(np.float64)
    ties = np.concatenate([f + 0.5 * ulp * np.sign(f), f - 0.25 * ulp, f + 0.75 * ulp])
    special = np.array([0.0, -0.0, 1.0, -1.0, 2.0 ** 100, 3000.0, 353.0, 1.0 - 2 ** -30, 2.0 ** -120,
                        np.float64(np.float32(1.5)) + 2.0 ** -24, 2.0 ** 127 * 1.5])
    x = np.concatenate([x, ties, special])
    x = x[(np.abs(x) >= 2.0 ** -126) | (x == 0)]  # the flush range is tested separately
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    y = torch.empty(len(x), dtype=torch.float32, device="cuda")
    P.pbf_round_to_f32(xd, y, len(x))
    ref = xd.float()
    torch.cuda.synchronize()
    assert torch.equal(y.view(torch.int32), ref.view(torch.int32))


def test_round_to_f32_flushes_below_normal_range(P):
    x = torch.tensor([1e-39, -1e-39, 2.0 ** -127, 0.0], dtype=torch.float64, device="cuda")
    y = torch.empty(4, dtype=torch.float32, device="cuda")
    P.pbf_round_to_f32(x, y, 4)
    torch.cuda.synchronize()
    assert y.abs().max().item() == 0.0 and np.signbit(y[1].item())


def test_widen_to_f64_is_exact(P):
    rng = np.random.default_rng(1)
    f = (rng.uniform(-1, 1, 100000) * 10.0 ** rng.uniform(-37, 37, 100000)).astype(np.float32)
    f = f[(np.abs(f) >= np.float32(2.0 ** -126)) | (f == 0)]  # subnormals flush by design
    f = np.concatenate([f, np.array([0.0, -0.0, 1.0, np.inf, -np.inf], np.float32)])
    xf = torch.tensor(f, device="cuda")
    y = torch.empty(len(f), dtype=torch.float64, device="cuda")
    P.pbf_widen_to_f64(xf, y, len(f))
    ref = xf.double()
    torch.cuda.synchronize()
    assert torch.equal(y.view(torch.int64), ref.view(torch.int64))
