"""Field parity: ap_eval_fields (the push's own field code at one time step)
against the oracle's textbook fields, element by element, for every pulse
kind, polarisation, envelope and the optional terms.

Tolerances (absolute, in units of a0): FP64 1e-10 (the oracle's
finite-difference longitudinal terms are accurate to ~1e-12); FP32 with a
double or float-float phase 4e-6 for single beams (float arithmetic of
~20 operations on O(1) quantities, MUFU sin/cos absolute error ~4e-7 and
exp2 relative error ~2e-7), 4e-5 for the 64-component flying focus (64
float terms summed)."""
import math
import zlib

import numpy as np
import pytest

import oracle
from paper_2307_04843_gb300 import workloads

L = 2 * math.pi

CASES = {
    "plane-x-sin2": dict(kind="plane", pol="x", env="sin2", env_len=10, a0=1.0, t_focus=10 * math.pi),
    "plane-y-sgauss": dict(kind="plane", pol="y", env="sgauss", env_len=25.0, sg_order=4, a0=2.0),
    "plane-cp-gauss": dict(kind="plane", pol="cp", env="gauss", env_len=30.0, a0=3.0, phase0=0.4),
    "gauss-x-lon": dict(kind="gauss", pol="x", env="gauss", env_len=30.0, a0=10.0, w0=3 * L,
                        longitudinal=True),
    "gauss-y-nolon": dict(kind="gauss", pol="y", env="cw", a0=2.0, w0=2 * L, z_focus=5.0, t_focus=3.0),
    "gauss-cm-lon-yee": dict(kind="gauss", pol="cm", env="gauss", env_len=20.0, a0=1.5, w0=4 * L,
                             longitudinal=True, yee=True, yee_dx=0.2, yee_dt=0.1),
    "lg12-cp-lon": dict(kind="lg", pol="cp", env="sin2", env_len=20, a0=20.0, w0=2 * L, lg_p=1, lg_l=2,
                        longitudinal=True, t_focus=30.0),
    "lg2m1-x-lon": dict(kind="lg", pol="x", env="cw", a0=1.0, w0=3 * L, lg_p=2, lg_l=-1, longitudinal=True),
    "lg03-y": dict(kind="lg", pol="y", env="gauss", env_len=40.0, a0=1.0, w0=3 * L, lg_p=0, lg_l=3),
    # |l| = 0 with p > 0 (no azimuthal power, the radial recurrence only) and LG_00
    "lg20-cm-lon": dict(kind="lg", pol="cm", env="cw", a0=1.5, w0=2.5 * L, lg_p=2, lg_l=0, longitudinal=True,
                        z_focus=-3.0),
    "lg00-x-lon": dict(kind="lg", pol="x", env="gauss", env_len=30.0, a0=3.0, w0=3 * L, lg_p=0, lg_l=0,
                       longitudinal=True),
    "flying-8-lon": dict(kind="flying", pol="x", a0=2.0, w0=2 * L, n_comp=8, bw_frac=0.05, beta_f=0.9,
                         ff_length=40 * L, longitudinal=True),
    # closed-form flying focus: counter-propagating (beta_f = -1) and subluminal focus
    "flyingcf-x-lon": dict(kind="flying_cf", pol="x", env="gauss", env_len=40.0, a0=2.0, w0=3 * L,
                           beta_f=-1.0, z_focus=2.0, t_focus=1.0, longitudinal=True),
    "flyingcf-cp-sub": dict(kind="flying_cf", pol="cp", env="cw", a0=1.0, w0=2 * L, beta_f=0.6,
                            z_focus=-3.0, phase0=0.7),
}


def _points(pulse, n, seed):
    rng = np.random.default_rng(seed)
    w0 = pulse.get("w0", 3 * L)
    zR = 0.5 * w0 * w0
    x = rng.uniform(-1.5, 1.5, n) * w0
    y = rng.uniform(-1.5, 1.5, n) * w0
    if pulse["kind"] == "flying":
        st = oracle.state(pulse)
        z = st["z_mid"] + rng.uniform(-60, 60, n)
        t = st["t_mid"] + rng.uniform(-60, 60, n)
    else:
        z = pulse.get("z_focus", 0.0) + rng.uniform(-1, 1, n) * min(zR, 100.0)
        t = pulse.get("t_focus", 0.0) + (z - pulse.get("z_focus", 0.0)) + rng.uniform(-40, 40, n)
    return x, y, z, t


def _tol(pulse, precision):
    a0 = pulse["a0"]
    if precision == "fp64":
        return 1e-10 * a0
    return (4e-5 if pulse["kind"] == "flying" else 4e-6) * a0


@pytest.mark.gpu
@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("precision", ["fp64", "fp32_phase64", "fp32"])
def test_fields_match_oracle(name, precision):
    from paper_2307_04843_gb300 import _lib
    pulse = CASES[name]
    n = 257  # several blocks and a ragged tail
    x, y, z, t = _points(pulse, n, seed=zlib.crc32(name.encode()) % 1000)
    ref = oracle.fields(pulse, x, y, z, t)
    with _lib.Handle(pulse) as h:
        got = h.eval_fields(x, y, z, t, precision=precision).cpu().numpy()
    err = np.abs(got - ref)
    assert np.max(err) <= _tol(pulse, precision), (name, precision, np.max(err), np.unravel_index(np.argmax(err), err.shape))


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_flying_focus_64_components(precision):
    from paper_2307_04843_gb300 import _lib
    pulse = dict(workloads.config(4)["pulse"])
    x, y, z, t = _points(pulse, 129, seed=11)
    ref = oracle.fields(pulse, x, y, z, t)
    with _lib.Handle(pulse) as h:
        got = h.eval_fields(x, y, z, t, precision=precision).cpu().numpy()
    assert np.max(np.abs(got - ref)) <= _tol(pulse, precision)


@pytest.mark.gpu
def test_fields_far_from_origin_phase_accuracy():
    """Large |z| and t (phase ~ 1e4 rad): the float-float phase keeps the
    field within the FP32 bound; a plain float phase would not (~1e-3)."""
    from paper_2307_04843_gb300 import _lib
    pulse = dict(kind="plane", pol="x", env="cw", a0=1.0)
    rng = np.random.default_rng(5)
    z = rng.uniform(5000, 6000, 200)
    t = z + rng.uniform(-3000, 3000, 200)
    x = y = np.zeros(200)
    ref = oracle.fields(pulse, x, y, z, t)
    with _lib.Handle(pulse) as h:
        got = h.eval_fields(x, y, z, t, precision="fp32").cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 4e-6


@pytest.mark.gpu
def test_eval_fields_empty_and_bad_set():
    import torch
    from paper_2307_04843_gb300 import _lib
    with _lib.Handle(CASES["plane-x-sin2"]) as h:
        xyzt = torch.zeros((4, 0), dtype=torch.float64, device="cuda")
        EB = torch.zeros((6, 0), dtype=torch.float64, device="cuda")
        _lib.ap_eval_fields(h.h, 0, xyzt, EB, "fp64")
        with pytest.raises(_lib.APError):
            _lib.ap_eval_fields(h.h, 1, xyzt, EB, "fp64")


@pytest.mark.gpu
@pytest.mark.parametrize("kind,extra", [("gauss", {}), ("lg", dict(lg_p=1, lg_l=2, pol="cp"))])
def test_gpu_fields_maxwell_residual_slopes(kind, extra):
    """The GPU FP64 fields (ap_eval_fields) give the same Maxwell-residual
    slopes as the oracle: O(eps^2) with the longitudinal terms, div E = O(eps)
    without, eps = 1/(k w0) over w0 in {4, 8, 16, 32} lambda."""
    from paper_2307_04843_gb300 import _lib
    from test_oracle_pins import _residuals
    C = np.random.default_rng(5).uniform(-1, 1, (6, 4))
    ws = np.array([4, 8, 16, 32])
    res = {True: [], False: []}
    for lon in (True, False):
        for w in ws:
            w0 = w * L
            zR = 0.5 * w0 * w0
            p = dict(kind=kind, pol="x", env="cw", a0=1.0, w0=w0, longitudinal=lon, z_focus=0.0)
            p.update(extra)
            pts = [(0.7 * w0 * c[0], 0.7 * w0 * c[1], zR * c[2], 3 * c[3]) for c in C]
            with _lib.Handle(p) as h:
                f = lambda x, y, z, t: h.eval_fields(x, y, z, t, precision="fp64").cpu().numpy()
                res[lon].append(_residuals(p, pts, fields=f))
    eps = 1.0 / (ws * L)
    on, off = np.array(res[True]), np.array(res[False])
    slope = lambda col: np.polyfit(np.log(eps), np.log(col), 1)[0]
    assert 1.75 < slope(on[:, 0]) < 2.3 and 1.75 < slope(on[:, 1]) < 2.3
    assert slope(on[:, 2]) > 1.75 and slope(on[:, 3]) > 1.75
    assert 0.7 < slope(off[:, 2]) < 1.35
    assert np.all(on[:, 2] < 0.1 * off[:, 2])


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_maximum_table_sizes(precision):
    """The largest descriptions the ABI accepts: a flying focus of
    AP_MAX_COMP = 128 components and LG_pl with p = |l| = 8 (the Laguerre
    table limit) out to 3.75 w0, where the monomial form of L_8^8 cancels
    terms 1e4 times its value (the kernels use the three-term recurrence).
    Bounds: FP32 128 summed float terms 8e-5 a0, LG 4e-6 a0; FP64 LG 1e-9 a0,
    the accuracy of the oracle's finite-difference longitudinal terms for a
    mode with this much transverse structure."""
    from paper_2307_04843_gb300 import _lib
    ff = dict(kind="flying", pol="x", a0=1.0, w0=2 * L, n_comp=_lib.AP_MAX_COMP, bw_frac=0.05, beta_f=0.95,
              ff_length=60 * L, longitudinal=True)
    lg = dict(kind="lg", pol="cp", env="cw", a0=1.0, w0=4 * L, lg_p=8, lg_l=-8, longitudinal=True)
    for pulse, tol in ((ff, 8e-5 if precision == "fp32" else 1e-10), (lg, 4e-6 if precision == "fp32" else 1e-9)):
        x, y, z, t = _points(pulse, 193, seed=17)
        if pulse["kind"] == "lg":  # the outer rings of LG_88 lie near 4 w0
            x, y = 2.5 * x, 2.5 * y
        ref = oracle.fields(pulse, x, y, z, t)
        with _lib.Handle(pulse) as h:
            got = h.eval_fields(x, y, z, t, precision=precision).cpu().numpy()
        assert np.max(np.abs(got - ref)) <= tol * pulse["a0"], (pulse["kind"], np.max(np.abs(got - ref)))
        assert np.max(np.abs(ref)) > 0.05


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_lg00_equals_gaussian_through_both_device_paths(precision):
    """LG_00 is the Gaussian (Sec. 3.1): the device's LG evaluation (Laguerre
    recurrence, azimuthal and q powers) and its Gaussian evaluation give the
    same fields, longitudinal terms included."""
    from paper_2307_04843_gb300 import _lib
    common = dict(pol="cp", env="gauss", env_len=30.0, a0=3.0, w0=2.5 * L, z_focus=4.0, t_focus=1.0,
                  longitudinal=True)
    x, y, z, t = _points(dict(kind="gauss", **common), 300, seed=17)
    with _lib.Handle(dict(kind="lg", lg_p=0, lg_l=0, **common)) as h:
        lg = h.eval_fields(x, y, z, t, precision=precision).cpu().numpy()
    with _lib.Handle(dict(kind="gauss", **common)) as h:
        ga = h.eval_fields(x, y, z, t, precision=precision).cpu().numpy()
    tol = 1e-12 if precision == "fp64" else 2e-6
    assert np.max(np.abs(lg - ga)) <= tol * common["a0"]
    assert np.max(np.abs(ga)) > 0.5
