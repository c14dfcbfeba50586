"""Parity gates of the GPU tests against the oracle.

FP64 operator: 1e-10 relative max-norm, max |gpu - oracle| / max |oracle|.
FP32 operator, temperatures after explicit steps, three gates at once:
  - relative max-norm max |gpu - oracle| / max |oracle| <= 2e-4 (the stated FP32-operator gate);
  - relative to the change the steps made, max |gpu - oracle| / max |oracle - T_0| <= 1e-3,
    so that a small increment cannot hide a large error in it behind the size of T itself;
  - relative L2 error ||gpu - oracle||_2 / ||oracle||_2, reported (and held to 2e-4).
The FP32 operator's single residual evaluations are held to 2e-5 of max |f| (FP32 rounding
of sums of about 30 terms of comparable size), and an increment of n steps accumulates at
most n such errors relative to the increment itself; 1e-3 leaves room for that without
letting a wrong term through (a term of the operator that is off by 0.1% fails it).
"""
import numpy as np

TOL64 = 1e-10
TOL32_T = 2e-4
TOL32_INC = 1e-3
TOL32_F = 2e-5


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def rel_increment(got, ref, T0):
    return float(np.max(np.abs(got - ref)) / max(np.max(np.abs(ref - T0)), 1e-300))


def rel_l2(got, ref):
    return float(np.linalg.norm(np.ravel(got - ref)) / max(np.linalg.norm(np.ravel(ref)), 1e-300))


def check_f32_steps(got, ref, T0, min_change=1.0):
    """The FP32-operator gates for temperatures after explicit steps from T0; the steps must
    have changed the field by at least min_change kelvin. Returns the three measures."""
    got, ref = np.asarray(got), np.asarray(ref)
    T0 = np.broadcast_to(np.asarray(T0, dtype=np.float64), ref.shape)
    change = float(np.max(np.abs(ref - T0)))
    out = {"rel_max": rel(got, ref), "rel_increment": rel_increment(got, ref, T0), "rel_l2": rel_l2(got, ref),
           "max_change_K": change}
    assert change >= min_change, out
    assert out["rel_max"] < TOL32_T, out
    assert out["rel_increment"] < TOL32_INC, out
    assert out["rel_l2"] < TOL32_T, out
    return out


def check_f64_steps(got, ref, T0=None):
    out = {"rel_max": rel(got, ref), "rel_l2": rel_l2(got, ref)}
    if T0 is not None:
        out["rel_increment"] = rel_increment(np.asarray(got), np.asarray(ref),
                                             np.broadcast_to(np.asarray(T0, dtype=np.float64), np.shape(ref)))
        assert out["rel_increment"] < 1e-8, out
    assert out["rel_max"] < TOL64, out
    return out
