"""The temporal-convergence experiment of Appendix A (two powder layers, one track each, the
combined explicit / implicit scheme with the switch during the interlayer cool-down and the
activation of the second layer): the GPU run at the reference steps equals the oracle's run
of the same sequence (FP64, 1e-9 relative on the observation point's series and the final
field), and the temperature at the observation point converges at first order as the steps
shrink (dt_ref, dt_ref / 2, dt_ref / 4; Sec. 3.2: forward and backward Euler are first-order
schemes): the differences to the finest run, maximum and root mean square over the sample
times, shrink by about 3 when the steps halve. The paper shows the series as a figure and
prints no error value."""
import numpy as np
import pytest

from paper_2302_05164_gb300 import inputs as I
from paper_2302_05164_gb300 import temporal as TM

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_05164_gb300 import pbf
    return pbf


def oracle_run(O, newton_rtol=1e-10):
    """The same sequence at the reference steps in the oracle."""
    mat = I.APPA_MATERIAL
    dte, dti = I.APPA_DT_EXPLICIT, I.APPA_DT_IMPLICIT
    om = O.Mesh(I.appa_mesh(1))
    om.set_phase(I.APPA_PHASE)
    om.set_surface_loss(I.APPA_LOSS)
    obs = int(np.where(np.all(np.isclose(om.dof_xyz(), I.APPA_OBS, rtol=0.0, atol=1e-12), axis=1))[0][0])
    T = np.full(om.n_dofs, I.APPA_T0)
    times, temps, t = [0.0], [I.APPA_T0], 0.0

    def scan(m, T, t, obs):
        ls = I.appa_laser(t0=t)
        for _ in range(TM.SCAN_STEPS_REF):
            T = m.explicit(mat, T, ls, t, dte, 1)
            t += dte
            times.append(t)
            temps.append(T[obs])
        return T, t

    T, t = scan(om, T, t, obs)
    for _ in range(TM.COOL_EXPLICIT_REF // 50):
        T = om.explicit(mat, T, None, t, dte, 50)
        t += 50 * dte
        times.append(t)
        temps.append(T[obs])
    lmin, lmax = om.lanczos_bounds(mat, dti, I.start_vector(om.n_dofs, seed=3), 30)
    bounds = (lmin, 1.1 * lmax)
    for _ in range(TM.COOL_IMPLICIT_REF):
        T, nit, lit, st = om.implicit_newton(mat, T, dti, 1, newton_rtol, 30, 1e-4, 2000, 5, *bounds)
        assert st == 0
        t += dti
        times.append(t)
        temps.append(T[obs])
    om2 = O.Mesh(I.appa_mesh(2))
    T = O.transfer(om, T, om2, I.APPA_T0)
    h = O.transfer_history(om, om.history(), om2)
    om2.set_phase(I.APPA_PHASE)
    om2.set_history(h)
    om2.set_surface_loss(I.APPA_LOSS)
    obs2 = int(np.where(np.all(np.isclose(om2.dof_xyz(), I.APPA_OBS, rtol=0.0, atol=1e-12), axis=1))[0][0])
    T, t = scan(om2, T, t, obs2)
    return {"t": np.array(times), "T": np.array(temps), "T_final": T, "bounds": bounds}


@pytest.fixture(scope="module")
def runs(P, oracle_mod):
    ref = oracle_run(oracle_mod)
    out = {"oracle": ref}
    for k in (1, 2, 4):
        out[k] = TM.run(P, torch, dt_scale=1.0 / k, cheb_bounds=(ref["bounds"] if k == 1 else None, None))
    return out


def test_two_layer_sequence_matches_oracle(runs):
    ref, got = runs["oracle"], runs[1]
    assert np.allclose(got["t"], ref["t"], rtol=1e-12, atol=0.0)
    rise = np.max(ref["T"]) - I.APPA_T0
    assert rise > 1000.0  # the track melts the powder at the observation point
    err = np.max(np.abs(got["T"] - ref["T"])) / np.max(np.abs(ref["T"]))
    fin = np.max(np.abs(got["T_final"] - ref["T_final"])) / np.max(np.abs(ref["T_final"]))
    print(f"Appendix A at dt_ref: GPU vs oracle, observation series {err:.2e}, final field {fin:.2e}; "
          f"peak rise {rise:.0f} K; Newton (corrections, BiCGStab) {got['newton']}")
    assert err < 1e-9 and fin < 1e-9


def test_two_layer_sequence_converges_in_time(runs):
    finest = runs[4]
    errs = {}
    for k in (1, 2):
        samples = TM.common_samples(runs[1], runs[k], k)
        ref = TM.common_samples(runs[1], finest, 4)
        errs[k] = np.max(np.abs(samples - ref))
    rise = np.max(finest["T"]) - I.APPA_T0
    ratio = errs[1] / errs[2]
    rms = {k: float(np.sqrt(np.mean((TM.common_samples(runs[1], runs[k], k) - TM.common_samples(runs[1], finest, 4)) ** 2)))
           for k in (1, 2)}
    print(f"Appendix A: max |T_obs(dt) - T_obs(dt_ref/4)| over the reference sample times: dt_ref {errs[1]:.2f} K, "
          f"dt_ref/2 {errs[2]:.2f} K (ratio {ratio:.2f}, first order gives 3); rms {rms[1]:.2f} K, {rms[2]:.2f} K; "
          f"peak rise {rise:.0f} K")
    # first order: the differences to the finest run shrink by 3 when the steps halve
    assert 2.0 < ratio < 4.5
    assert 2.0 < rms[1] / rms[2] < 4.5
    # the paper prints no error value (a figure); the pointwise maximum sits on the heating front,
    # where the spot advances 19 um per reference step, so only a loose bound is checked on it
    assert errs[1] < 0.2 * rise
