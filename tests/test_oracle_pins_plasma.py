"""Pins of the oracle's plasma functions (Sec. 4: the analytic current J1 and
the fields of a plane wave in a linear cold plasma) against what the
mathematics fixes independently of the formulas:

- closed forms of the continuum plasma dispersion (omega^2 = omega_p^2 + k^2,
  v_phi v_g = c^2, B = (c k / omega) E);
- the textbook vacuum Yee relation as omega_p -> 0, and the continuum as
  dt, dz -> 0;
- exactness on the discrete scheme: a CW wave sampled from the oracle's E1,
  B1 and J1 is carried by the Yee line with a leapfrog cold-fluid current to
  rounding, and the split (analytic-current) line keeps E2 at rounding --
  this fixes k, B0/E0, zeta and the sign of J1 all at once;
- the finite-duration terms against quadrature: J1 against omega_p^2 times
  the time integral of E, B1 against the time integral of -dE/dz (Faraday),
  both converging as (omega T)^-3 with the pulse length T (a dropped or
  mis-signed term leaves (omega T)^-1 or ^-2);
- v_g as d omega/dk of the oracle's own dispersion relation;
- the envelope's logarithmic derivatives against finite differences."""
import math

import numpy as np
import pytest

import oracle

L = 2.0 * math.pi


def _yee_plasma(wp, ppl=20.0, cr=0.9, **kw):
    dz = L / ppl
    return dict(kind="plane", pol="x", a0=1.0, omega_p=wp, yee=True, yee_dx=dz, yee_dt=cr * dz, **kw)


def test_plasma_continuum_closed_forms():
    for wp in (0.05, 0.3, 0.7):
        st = oracle.state(dict(kind="plane", pol="x", env="cw", a0=1.0, omega_p=wp))
        k = math.sqrt(1.0 - wp * wp)
        assert st["k"] == pytest.approx(k, rel=1e-15)
        assert st["vphi"] * st["vg"] == pytest.approx(1.0, rel=1e-14)
        assert st["bratio"] == pytest.approx(k, rel=1e-15)
        assert st["zeta"] == 1.0 and st["jamp"] == pytest.approx(wp * wp, rel=1e-15)
    with pytest.raises(ValueError):  # omega below the cut-off
        oracle.state(dict(kind="plane", env="cw", omega_p=1.2))
    with pytest.raises(ValueError):  # only plane waves carry the analytic current
        oracle.state(dict(kind="gauss", env="cw", w0=5.0, omega_p=0.1))


def test_plasma_discrete_relation_limits():
    """omega_p -> 0: the textbook vacuum Yee relation sin(w dt/2) = (dt/dz)
    sin(k dz/2), v_g = cos(k dz/2)/cos(w dt/2), B0/E0 = cos(w dt/2) at whole
    steps.  dz, dt -> 0 at fixed omega_p: the continuum values, at second
    order."""
    dz = L / 20.0
    dt = 0.9 * dz
    st = oracle.state(dict(kind="plane", env="cw", omega_p=1e-7, yee=True, yee_dx=dz, yee_dt=dt))
    k = 2.0 / dz * math.asin(math.sin(0.5 * dt) / (dt / dz))
    assert st["k"] == pytest.approx(k, rel=1e-12)
    assert st["vg"] == pytest.approx(math.cos(0.5 * k * dz) / math.cos(0.5 * dt), rel=1e-12)
    assert st["bratio"] == pytest.approx(math.cos(0.5 * dt), rel=1e-12)
    wp = 0.3
    errs = []
    for ppl in (20.0, 40.0, 80.0, 160.0):
        st = oracle.state(_yee_plasma(wp, ppl=ppl, env="cw"))
        kc = math.sqrt(1.0 - wp * wp)
        errs.append([st["k"] - kc, st["vg"] - kc, st["bratio"] - kc, st["zeta"] - 1.0])
    errs = np.abs(np.array(errs))
    ratios = errs[:-1] / errs[1:]
    assert np.all(np.abs(ratios - 4.0) < 0.1), ratios


def test_plasma_group_velocity_is_domega_dk():
    for pulse in (_yee_plasma(0.3, env="cw"), dict(kind="plane", env="cw", omega_p=0.3)):
        d = 1e-5
        kp = oracle.state(dict(pulse, omega=1.0 + d))["k"]
        km = oracle.state(dict(pulse, omega=1.0 - d))["k"]
        assert oracle.state(pulse)["vg"] == pytest.approx(2.0 * d / (kp - km), rel=1e-8)


def _cw_line(pulse, nz, z0, dz, dt):
    z = z0 + dz * np.arange(nz)
    E = oracle.fields(pulse, 0.0, 0.0, z, 0.0)[0]
    B = oracle.fields(pulse, 0.0, 0.0, z + 0.5 * dz, 0.0)[4]
    J = oracle.current(pulse, 0.0, 0.0, z, -0.5 * dt)[0]
    return z, E, B, J


@pytest.mark.parametrize("wp,ppl,cr", [(0.3, 20.0, 0.9), (0.6, 16.0, 0.7), (0.1, 30.0, 0.99)])
def test_plasma_cw_is_carried_exactly_by_the_yee_fluid_line(wp, ppl, cr):
    pulse = _yee_plasma(wp, ppl=ppl, cr=cr, env="cw", phase0=0.3)
    dz, dt = pulse["yee_dx"], pulse["yee_dt"]
    nz, n = 400, 120
    z, E, B, J = _cw_line(pulse, nz, -37.0, dz, dt)
    E, B, J = oracle.plasma1d(E, B, J, wp * wp, dz, dt, n)
    T = n * dt
    inner = slice(n + 2, nz - n - 2)
    Ea = oracle.fields(pulse, 0.0, 0.0, z, T)[0]
    Ba = oracle.fields(pulse, 0.0, 0.0, z + 0.5 * dz, T)[4]
    Ja = oracle.current(pulse, 0.0, 0.0, z, T - 0.5 * dt)[0]
    assert np.max(np.abs(E - Ea)[inner]) < 1e-11
    assert np.max(np.abs(B - Ba)[inner]) < 1e-11
    assert np.max(np.abs(J - Ja)[inner]) < 1e-11
    assert np.max(np.abs(Ja)) > 0.5 * wp * wp


def test_plasma_cw_split_line_keeps_e2_at_rounding():
    """With E1 and J1 an exact discrete solution, the physical current driven
    by E1 + E2 follows J1 and the source J - J1 of E2 vanishes, on every node
    of the line, ends included (vacuum boundary conditions for E2)."""
    wp = 0.3
    pulse = _yee_plasma(wp, env="cw", phase0=-1.1)
    dz, dt = pulse["yee_dx"], pulse["yee_dt"]
    nz = 300
    z0 = -20.0
    z = z0 + dz * np.arange(nz)
    J = oracle.current(pulse, 0.0, 0.0, z, -0.5 * dt)[0]
    E2, B2, J = oracle.apt1d(pulse, np.zeros(nz), np.zeros(nz), J, wp * wp, z0, dz, 0.0, dt, 150)
    assert np.max(np.abs(E2)) < 1e-12 and np.max(np.abs(B2)) < 1e-12
    Ja = oracle.current(pulse, 0.0, 0.0, z, 150 * dt - 0.5 * dt)[0]
    assert np.max(np.abs(J - Ja)) < 1e-12


def test_plasma_split_line_in_vacuum_is_identically_zero():
    pulse = dict(kind="plane", pol="x", env="sgauss", sg_order=4, env_len=10.0, a0=1.0, yee=True,
                 yee_dx=L / 20, yee_dt=0.9 * L / 20)
    nz = 200
    E2, B2, J = oracle.apt1d(pulse, np.zeros(nz), np.zeros(nz), np.zeros(nz), 0.0, -30.0,
                             pulse["yee_dx"], 0.0, pulse["yee_dt"], 100)
    assert not np.any(E2) and not np.any(B2) and not np.any(J)
    with pytest.raises(ValueError):
        oracle.apt1d(dict(pulse, pol="y"), np.zeros(4), np.zeros(4), np.zeros(4), 0.0, 0.0, 1.0, 0.0, 0.5, 1)


def test_plasma_line_without_plasma_is_the_vacuum_yee_line():
    rng = np.random.default_rng(11)
    E, B = rng.standard_normal(64), rng.standard_normal(64)
    Ey, By = oracle.yee1d(E, B, 0.05, 0.045, 37)
    Ep, Bp, Jp = oracle.plasma1d(E, B, np.zeros(64), 0.0, 0.05, 0.045, 37)
    assert np.array_equal(Ey, Ep) and np.array_equal(By, Bp) and not np.any(Jp)


def _cumulative(f, h):
    """Cumulative integral of samples f spaced by h (composite Simpson on
    each pair of intervals, the odd points from Simpson's 3/8 on the last
    three intervals or the trapezoid-corrected midpoint), exact to h^4."""
    from scipy.integrate import cumulative_simpson
    return np.concatenate([[0.0], cumulative_simpson(f, dx=h)])


def _fd_errors(kind, T, wp=0.3):
    """Largest |exact - oracle| over |t| <= 1.5 T at z = 0 for J1 (exact:
    omega_p^2 times the integral of E) or B1 (exact: the integral of
    -dE/dz), Gaussian envelope of intensity FWHM T, continuum plasma."""
    pulse = dict(kind="plane", pol="x", env="gauss", env_len=T, a0=1.0, omega_p=wp, phase0=0.4)
    h = 0.01
    t = np.arange(-5.0 * T, 1.5 * T + h / 2, h)
    if kind == "J":
        f = wp * wp * oracle.fields(pulse, 0.0, 0.0, 0.0, t)[0]
        got = oracle.current(pulse, 0.0, 0.0, 0.0, t)[0]
    else:
        d = 1e-3
        Ex = [oracle.fields(pulse, 0.0, 0.0, s * d, t)[0] for s in (-2, -1, 1, 2)]
        dEdz = (Ex[0] - 8.0 * Ex[1] + 8.0 * Ex[2] - Ex[3]) / (12.0 * d)
        f = -dEdz
        got = oracle.fields(pulse, 0.0, 0.0, 0.0, t)[4]
    exact = _cumulative(f, h)
    win = np.abs(t) <= 1.5 * T
    return np.max(np.abs(exact - got)[win]), np.max(np.abs(exact)[win])


@pytest.mark.parametrize("kind", ["J", "B"])
def test_plasma_finite_duration_terms_against_quadrature(kind):
    Ts = (10.0, 20.0, 40.0)
    res = [_fd_errors(kind, T) for T in Ts]
    errs = np.array([e for e, _ in res])
    scale = res[-1][1]
    assert scale > 0.05
    ratios = errs[:-1] / errs[1:]
    assert np.all(ratios > 6.0), (errs, ratios)
    assert errs[-1] < 2e-4 * scale, errs


@pytest.mark.parametrize("env,g", [("gauss", 1), ("sgauss", 1), ("sgauss", 2), ("sgauss", 4)])
def test_envelope_log_derivatives_match_finite_differences(env, g):
    pulse = dict(kind="plane", env=env, sg_order=g, env_len=7.0)
    eta = np.array([-9.0, -4.3, -0.7, 0.0, 0.2, 3.1, 6.5])
    l1, l2 = oracle.envelope_logd(pulse, eta)
    h = 1e-3
    G = oracle.envelope(pulse, eta)
    Gp, Gm = oracle.envelope(pulse, eta + h), oracle.envelope(pulse, eta - h)
    assert np.allclose(l1, (Gp - Gm) / (2 * h) / G, rtol=1e-5, atol=1e-7)
    assert np.allclose(l2, (Gp - 2 * G + Gm) / (h * h) / G, rtol=1e-4, atol=1e-6)
    with pytest.raises(ValueError):
        oracle.envelope_logd(dict(pulse, env="sin2"), [0.0])
