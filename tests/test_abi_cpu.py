"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a, loads, exports every entry point declared in include/ap.h, and its
argument validation rejects bad pulse descriptions before touching CUDA."""
import ctypes
import os
import re

import pytest

from paper_2307_04843_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ap.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ap_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return _lib.lib()


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n
    # the binding declares exactly the header's entry points
    assert sorted(_lib.SIGNATURES) == names


def test_version_and_status_strings(L):
    assert _lib.ap_version() == _lib.AP_ABI_VERSION == 3
    for code in (0, -1, -2, -3, -4, -5, -6, -7):
        s = _lib.ap_status_string(code)
        assert s and s != "unknown status"
    assert _lib.ap_status_string(12345) == "unknown status"


def _init_rc(L, d, n=1):
    arr = (_lib.ApPulseDesc * n)(*([_lib.pulse_desc(d)] * n))
    h = ctypes.c_void_p()
    return L.ap_init_pulse(arr, n, ctypes.byref(h)), h


@pytest.mark.parametrize("bad", [
    dict(kind="gauss", w0=0.0, env="cw"),                       # beam without a waist
    dict(kind="plane", omega=0.0),                               # no frequency
    dict(kind="plane", env="sin2", env_len=0.0),                 # empty envelope
    dict(kind="plane", env="sgauss", env_len=1.0, sg_order=0),   # bad super-Gaussian order
    dict(kind="lg", w0=1.0, lg_p=9),                             # p beyond the table
    dict(kind="lg", w0=1.0, lg_l=-9),
    dict(kind="flying", w0=1.0, n_comp=1, beta_f=0.99, ff_length=10.0),
    dict(kind="flying", w0=1.0, n_comp=500, beta_f=0.99, ff_length=10.0),
    dict(kind="flying", w0=1.0, n_comp=129, beta_f=0.99, ff_length=10.0),  # AP_MAX_COMP + 1
    dict(kind="flying_cf", w0=1.0, beta_f=1.0),                  # focus at the speed of light
    dict(kind="flying_cf", w0=1.0, beta_f=float("inf")),
    dict(kind="flying", w0=1.0, n_comp=8, beta_f=0.0, ff_length=10.0),
    dict(kind="plane", yee=True, yee_dx=0.1, yee_dt=0.2),       # Courant number > 1
    dict(kind="plane", a0=float("nan")),
    dict(kind="plane", env="cw", omega_p=1.5),                  # plasma: omega below the cut-off
    dict(kind="plane", env="cw", omega_p=-0.1),
    dict(kind="plane", env="cw", omega_p=float("nan")),
    dict(kind="gauss", w0=5.0, env="cw", omega_p=0.1),           # J1 only for plane waves
    dict(kind="plane", env="sin2", env_len=4.0, omega_p=0.1),    # envelope without Gamma''
    dict(kind="plane", env="cw", omega_p=0.05, yee=True, yee_dx=3.1, yee_dt=3.05),  # k beyond the grid
])
def test_invalid_descriptions_rejected_on_host(L, bad):
    rc, h = _init_rc(L, bad)
    assert rc == _lib.AP_ERR_ARG
    assert not h.value


def test_flying_focus_with_yee_dispersion_unsupported(L):
    rc, _ = _init_rc(L, dict(kind="flying", w0=1.0, n_comp=8, beta_f=0.99, ff_length=10.0, yee=True,
                             yee_dx=0.1, yee_dt=0.05))
    assert rc == _lib.AP_ERR_UNSUPPORTED


def test_null_and_count_arguments(L):
    h = ctypes.c_void_p()
    assert L.ap_init_pulse(None, 1, ctypes.byref(h)) == _lib.AP_ERR_ARG
    arr = (_lib.ApPulseDesc * 1)(_lib.pulse_desc(dict(kind="plane")))
    assert L.ap_init_pulse(arr, 0, ctypes.byref(h)) == _lib.AP_ERR_ARG
    assert L.ap_init_pulse(arr, _lib.AP_MAX_SETS + 1, ctypes.byref(h)) == _lib.AP_ERR_ARG
    assert L.ap_init_pulse(arr, 1, None) == _lib.AP_ERR_ARG
    assert L.ap_set_launch(None, None) == _lib.AP_ERR_ARG
    assert L.ap_num_sets(None) == _lib.AP_ERR_ARG
    assert L.ap_gather_push(None, None, None, 0.0, 0.1, 1, 0, None, None) == _lib.AP_ERR_ARG
    assert L.ap_batch_workspace_bytes(None) == 0
    L.ap_destroy(None)
    L.ap_graph_destroy(None)


def test_node_and_yee_arguments_rejected_on_host(L):
    """Argument checks of ap_eval_nodes and ap_yee1d_run run before any CUDA
    call (no GPU needed)."""
    g = _lib.ApYeeGrid()
    g.nx = g.ny = g.nz = 4
    assert L.ap_eval_nodes(None, 0, ctypes.byref(g), 0.0, 0, 0, None) == _lib.AP_ERR_ARG
    y = _lib.ApYee1d()
    y.nz, y.n_lines, y.dz, y.dt = 100, 1, 0.1, 0.05
    assert L.ap_yee1d_run(None, 10, 0, None) == _lib.AP_ERR_ARG
    assert L.ap_yee1d_run(ctypes.byref(y), -1, 0, None) == _lib.AP_ERR_ARG
    assert L.ap_yee1d_run(ctypes.byref(y), 10, 1, None) == _lib.AP_ERR_ARG  # FP32 with double phase: no
    for nz in (1, _lib.AP_YEE1D_MAX_NODES + 1):
        y.nz = nz
        assert L.ap_yee1d_run(ctypes.byref(y), 10, 0, None) == _lib.AP_ERR_ARG
    y.nz, y.dz = 100, 0.0
    assert L.ap_yee1d_run(ctypes.byref(y), 10, 0, None) == _lib.AP_ERR_ARG
    y.dz, y.n_lines = 0.1, 0
    assert L.ap_yee1d_run(ctypes.byref(y), 10, 0, None) == _lib.AP_OK  # nothing to do
    y.n_lines = 1
    assert L.ap_yee1d_run(ctypes.byref(y), 10, 0, None) == _lib.AP_ERR_ARG  # NULL arrays
    y.E, y.B = 8, 20  # misaligned for double (never dereferenced: rejected first)
    assert L.ap_yee1d_run(ctypes.byref(y), 10, 0, None) == _lib.AP_ERR_ALIGN


def test_build_is_up_to_date_after_build(L):
    assert build.up_to_date()
    assert os.path.exists(build.LIB)


def _line(nz=16, n_lines=1, E=16, B=16, J=16, wp2=None, dz=0.1, dt=0.05, omega_p=0.1, z0=0.0):
    y = _lib.ApLine1d()
    y.E, y.B, y.J, y.wp2 = E, B, J, wp2
    y.nz, y.n_lines, y.dz, y.dt, y.omega_p, y.z0 = nz, n_lines, dz, dt, omega_p, z0
    return y


@pytest.mark.parametrize("prec,max_nodes", [(0, 6144), (2, 12288)])
def test_plasma_line_arguments_checked_on_host(L, prec, max_nodes):
    """Validation before any launch: nothing is dereferenced (the pointers
    here are fake addresses) and no-work calls return before CUDA."""
    run = lambda y, n=1, p=prec: L.ap_plasma1d_run(ctypes.byref(y), n, p, None)  # noqa: E731
    assert L.ap_plasma1d_run(None, 1, prec, None) == _lib.AP_ERR_ARG
    assert run(_line(nz=1)) == _lib.AP_ERR_ARG
    assert run(_line(nz=max_nodes + 1)) == _lib.AP_ERR_ARG
    assert run(_line(dz=0.0)) == _lib.AP_ERR_ARG
    assert run(_line(dt=float("inf"))) == _lib.AP_ERR_ARG
    assert run(_line(omega_p=-1.0)) == _lib.AP_ERR_ARG
    assert run(_line(z0=float("nan"))) == _lib.AP_ERR_ARG
    assert run(_line(E=None)) == _lib.AP_ERR_ARG
    assert run(_line(), n=-1) == _lib.AP_ERR_ARG
    assert run(_line(), p=1) == _lib.AP_ERR_ARG        # AP_FP32_PHASE64: no line variant
    assert run(_line(J=18)) == _lib.AP_ERR_ALIGN
    assert run(_line(wp2=20 if prec == 0 else 22)) == _lib.AP_ERR_ALIGN
    assert run(_line(n_lines=0, nz=max_nodes)) == _lib.AP_OK  # no work, no launch
    assert run(_line(), n=0) == _lib.AP_OK
    y = _line()
    assert L.ap_apt1d_run(None, 0, ctypes.byref(y), 0.0, 1, prec, None) == _lib.AP_ERR_ARG

