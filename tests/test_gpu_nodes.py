"""Grid-node form of the technique: ap_eval_nodes (analytic E1/B1 on the
Yee-staggered nodes, Sec. 2.1 and Fig. 1) and ap_yee1d_run (the 1-D vacuum
Yee update of Sec. 2.1) against the oracle, element by element.

Tolerances: node values FP64 into double arrays 1e-10 a0 (the oracle's
finite-difference longitudinal terms), into float arrays that plus one
float rounding (6e-8 |value|); FP32 arithmetic 4e-6 a0 (as for the field
parity tests).  The double Yee update rounds every product and difference
separately in the oracle's order, so it is compared bit for bit; the float
one within 1e-5 after 400 steps (float rounding of O(1) values, ~1e-7 per
substep, accumulating)."""
import math

import numpy as np
import pytest

import oracle

L = 2 * math.pi

NODE_CASES = {
    "plane-sgauss-yee": dict(kind="plane", pol="x", env="sgauss", sg_order=4, env_len=30.0, a0=1.0,
                             yee=True, yee_dx=L / 30, yee_dt=0.95 * L / 30 / math.sqrt(3)),
    "gauss-cp-lon": dict(kind="gauss", pol="cp", env="gauss", env_len=30.0, a0=3.0, w0=1.5 * L,
                         longitudinal=True, z_focus=0.5, t_focus=0.3),
    "lg12-x-lon": dict(kind="lg", pol="x", env="cw", a0=2.0, w0=2 * L, lg_p=1, lg_l=2, longitudinal=True),
    "flyingcf-y": dict(kind="flying_cf", pol="y", env="gauss", env_len=40.0, a0=1.5, w0=2 * L, beta_f=-1.0,
                       longitudinal=True),
}


def _grid(shape, dtype, fill=None):
    import torch
    out = []
    for c in range(6):
        if fill is None:
            out.append(torch.zeros(shape, dtype=dtype, device="cuda"))
        else:
            out.append(torch.as_tensor(fill[c], dtype=dtype).cuda().contiguous())
    return out


@pytest.mark.gpu
@pytest.mark.parametrize("name", sorted(NODE_CASES))
@pytest.mark.parametrize("precision,f64", [("fp64", True), ("fp64", False), ("fp32", False),
                                           ("fp32_phase64", False)])
@pytest.mark.parametrize("shape", [(11, 6, 7), (4, 3, 70)], ids=["short-rows", "long-rows"])
def test_nodes_match_oracle(name, precision, f64, shape):
    """Every kind and precision on short rows (one thread per node) and on
    rows of 70 nodes (one warp per row, two full warps of nodes and a ragged
    third per lane group), ragged in every axis."""
    import torch
    from paper_2307_04843_gb300 import _lib
    pulse = NODE_CASES[name]
    d = (0.37 * L, 0.29 * L, 0.11 * L) if shape[2] < 32 else (0.05 * L, 0.29 * L, 0.11 * L)
    lo = (-1.1 * L, -0.8 * L, -0.6 * L) if shape[2] < 32 else (-1.75 * L, -0.8 * L, -0.6 * L)
    t = 0.9
    ref = oracle.yee_nodes(pulse, shape, lo, d, t)
    dtype = torch.float64 if f64 else torch.float32
    f = _grid(shape, dtype)
    with _lib.Handle(pulse) as h:
        h.eval_nodes(f, lo, d, t, precision=precision)
        assert h.status() == 0
    got = np.stack([x.double().cpu().numpy() for x in f])
    a0 = pulse["a0"]
    if precision == "fp64":
        tol = 1e-10 * a0 + (0.0 if f64 else 6e-8 * np.abs(ref))
    else:
        tol = 4e-6 * a0
    assert np.all(np.abs(got - ref) <= tol), (name, precision, f64, np.max(np.abs(got - ref)))
    assert np.max(np.abs(ref)) > 0.1 * a0  # the sample sees the pulse


@pytest.mark.gpu
def test_nodes_accumulate_skip_and_degenerate_axes():
    """accumulate adds E1 to what the arrays hold (E = E1 + E2); a NULL
    component is left alone; a 1-D grid puts Ex on whole and By on half nodes."""
    import torch
    from paper_2307_04843_gb300 import _lib
    pulse = NODE_CASES["gauss-cp-lon"]
    shape = (9, 4, 5)
    lo, d, t = (0.1, -0.2, -3.0), (0.8, 0.9, 0.7), 1.3
    rng = np.random.default_rng(3)
    prior = rng.standard_normal((6,) + shape)
    f = _grid(shape, torch.float64, fill=prior)
    f[2] = None
    with _lib.Handle(pulse) as h:
        h.eval_nodes(f, lo, d, t, accumulate=True, precision="fp64")
        got = np.stack([x.cpu().numpy() if x is not None else prior[2] for x in f])
        ref = prior + oracle.yee_nodes(pulse, shape, lo, d, t)
        ref[2] = prior[2]
        assert np.max(np.abs(got - ref)) <= 1e-10 * pulse["a0"]
    # 1-D grid along z
    plane = dict(kind="plane", pol="x", env="cw", a0=1.0)
    with _lib.Handle(plane) as h:
        ex = torch.zeros((64, 1, 1), dtype=torch.float64, device="cuda")
        by = torch.zeros_like(ex)
        h.eval_nodes([ex, None, None, None, by, None], (5.0, 5.0, 0.25), (0.0, 0.0, 0.5), 0.9)
        z = 0.25 + 0.5 * np.arange(64)
        assert np.max(np.abs(ex.cpu().numpy().ravel() - np.cos(0.9 - z))) < 1e-14
        assert np.max(np.abs(by.cpu().numpy().ravel() - np.cos(0.9 - z - 0.25))) < 1e-14
        # zero spacing on every axis: every node samples the same point
        bz = torch.full_like(by, 7.0)
        h.eval_nodes([None, None, None, None, by, bz], (0, 0, 0), (0, 0, 0), 0.0)
        assert np.all(by.cpu().numpy() == 1.0) and np.all(bz.cpu().numpy() == 0.0)


@pytest.mark.gpu
def test_nodes_bad_arguments():
    import ctypes
    import torch
    from paper_2307_04843_gb300 import _lib
    with _lib.Handle(dict(kind="plane")) as h:
        f = [torch.zeros((4, 4, 4), device="cuda") for _ in range(6)]
        with pytest.raises(_lib.APError):
            h.eval_nodes(f, (0, 0, 0), (-1.0, 1.0, 1.0), 0.0)
        with pytest.raises(_lib.APError):
            h.eval_nodes(f, (0, 0, 0), (1.0, 1.0, 1.0), 0.0, set_index=1)
        # a double array must be 8-byte aligned (checked before any launch)
        g = _lib.yee_grid_struct(f, (0, 0, 0), (1.0, 1.0, 1.0))
        g.f64 = 1
        g.f[0] = f[0].data_ptr() + 4
        rc = _lib.lib().ap_eval_nodes(h.h, 0, ctypes.byref(g), 0.0, 0, 0, _lib._stream(None))
        assert rc == _lib.AP_ERR_ALIGN
        g.f[0] = f[0].data_ptr()
        g.nz = 0
        rc = _lib.lib().ap_eval_nodes(h.h, 0, ctypes.byref(g), 0.0, 0, 0, _lib._stream(None))
        assert rc == _lib.AP_ERR_ARG
        assert h.status() == 0


@pytest.mark.gpu
@pytest.mark.parametrize("nz,n_lines,n_steps", [(2, 1, 3), (1000, 3, 400), (2048, 2, 100), (4099, 2, 150),
                                                (6000, 1, 60), (6145, 1, 50), (12288, 1, 40)])
def test_yee1d_double_bit_exact(nz, n_lines, n_steps):
    import torch
    from paper_2307_04843_gb300 import _lib
    rng = np.random.default_rng(nz)
    E0 = rng.standard_normal((n_lines, nz))
    B0 = rng.standard_normal((n_lines, nz))
    dz, dt = 0.05, 0.0475
    E = torch.as_tensor(E0).cuda()
    B = torch.as_tensor(B0).cuda()
    _lib.ap_yee1d_run(E, B, dz, dt, n_steps)
    for l in range(n_lines):
        Er, Br = oracle.yee1d(E0[l], B0[l], dz, dt, n_steps)
        assert np.array_equal(E[l].cpu().numpy(), Er), l
        assert np.array_equal(B[l].cpu().numpy(), Br), l


@pytest.mark.gpu
def test_yee1d_float_and_zero_steps():
    import torch
    from paper_2307_04843_gb300 import _lib
    rng = np.random.default_rng(1)
    nz = 3000
    z = np.arange(nz) * 0.05
    E0 = np.exp(-((z - 75) / 10) ** 2) * np.cos(z)
    B0 = np.exp(-((z + 0.025 - 75) / 10) ** 2) * np.cos(z + 0.025)
    E = torch.as_tensor(E0, dtype=torch.float32).cuda()
    B = torch.as_tensor(B0, dtype=torch.float32).cuda()
    _lib.ap_yee1d_run(E, B, 0.05, 0.0475, 400)
    Er, Br = oracle.yee1d(E0, B0, 0.05, 0.0475, 400)
    assert np.max(np.abs(E.double().cpu().numpy() - Er)) < 1e-5
    assert np.max(np.abs(B.double().cpu().numpy() - Br)) < 1e-5
    Ed = torch.as_tensor(rng.standard_normal(50)).cuda()
    Bd = torch.as_tensor(rng.standard_normal(50)).cuda()
    e0, b0 = Ed.clone(), Bd.clone()
    _lib.ap_yee1d_run(Ed, Bd, 0.05, 0.0475, 0)
    assert torch.equal(Ed, e0) and torch.equal(Bd, b0)


def _gpu_apt_vs_yee(ppl, g=4, tau=30.0, dist=40.0, cr=0.95):
    """Fig. 2e on the GPU: the analytic pulse on the 1-D nodes (ap_eval_nodes,
    FP64 into double arrays) as the initial condition of the Yee line
    (ap_yee1d_run), then against ap_eval_nodes at the final time."""
    import torch
    from paper_2307_04843_gb300 import _lib
    dz = L / ppl
    dt = cr * dz
    pulse = dict(kind="plane", pol="x", env="sgauss", sg_order=g, env_len=tau, a0=1.0,
                 z_focus=0.0, t_focus=0.0, yee=True, yee_dx=dz, yee_dt=dt)
    vg = oracle.state(pulse)["vg"]
    z0 = -2.5 * tau - 5 * L
    nz = int((5 * tau + dist * L + 10 * L) / dz)
    lo, d = (0.0, 0.0, z0), (0.0, 0.0, dz)
    ex = torch.zeros((nz, 1, 1), dtype=torch.float64, device="cuda")
    by = torch.zeros_like(ex)
    n = int(round(dist * L / dt))
    with _lib.Handle(pulse) as h:
        h.eval_nodes([ex, None, None, None, by, None], lo, d, 0.0)
        E, B = ex.view(-1).clone(), by.view(-1).clone()
        _lib.ap_yee1d_run(E, B, dz, dt, n)
        h.eval_nodes([ex, None, None, None, by, None], lo, d, n * dt)
    Ea = ex.view(-1).cpu().numpy()
    diff = np.abs(E.cpu().numpy() - Ea)
    z = z0 + dz * np.arange(nz)
    T = n * dt
    zp = vg * T
    ze = vg * (T + tau * math.log(2) ** (1 / (2 * g)))
    return diff[np.abs(z - zp) <= L].max(), diff[np.abs(z - ze) <= L].max()


@pytest.mark.gpu
def test_fig2e_fourth_order_peak_second_order_edge_on_gpu():
    ppls = np.array([20.0, 30.0, 40.0, 60.0])
    res = np.array([_gpu_apt_vs_yee(p) for p in ppls])
    x = np.log(L / ppls)
    assert abs(np.polyfit(x, np.log(res[:, 0]), 1)[0] - 4.0) < 0.2
    assert abs(np.polyfit(x, np.log(res[:, 1]), 1)[0] - 2.0) < 0.2
    # the same numbers as the oracle's run of the experiment
    from test_oracle_pins import _apt_vs_yee_errors
    for p, (ep, ee) in zip(ppls, res):
        op, oe = _apt_vs_yee_errors(p, True)
        assert abs(ep - op) <= 1e-6 * op + 1e-13 and abs(ee - oe) <= 1e-6 * oe + 1e-13, (p, ep, op, ee, oe)


@pytest.mark.gpu
@pytest.mark.parametrize("precision,f64", [("fp64", True), ("fp32", False)])
@pytest.mark.parametrize("pol", ["x", "cp"])
def test_plane_wave_rows_match_oracle(precision, f64, pol):
    """Plane waves depend on z and t only: for rows of >= 32 nodes one field
    evaluation per row is streamed along it.  Store and accumulate both
    match the oracle on every node (accumulating skips components that are
    identically zero, which leaves them as they were)."""
    import torch
    from paper_2307_04843_gb300 import _lib
    pulse = dict(kind="plane", pol=pol, env="sgauss", sg_order=4, env_len=20.0, a0=2.0, t_focus=5.0,
                 yee=True, yee_dx=L / 40, yee_dt=0.5 * L / 40)
    shape = (13, 5, 70)  # rows of 70 nodes: two full warps and a ragged third
    lo, d, t = (0.3, -0.7, -2.0 * L), (0.2, 0.3, 0.31 * L), 6.5
    ref = oracle.yee_nodes(pulse, shape, lo, d, t)
    dtype = torch.float64 if f64 else torch.float32
    tol = 1e-10 * pulse["a0"] if precision == "fp64" else 4e-6 * pulse["a0"]
    with _lib.Handle(pulse) as h:
        f = _grid(shape, dtype)
        h.eval_nodes(f, lo, d, t, precision=precision)
        got = np.stack([x.double().cpu().numpy() for x in f])
        assert np.max(np.abs(got - ref)) <= tol
        prior = np.random.default_rng(8).standard_normal((6,) + shape)
        f = _grid(shape, dtype, fill=prior)
        h.eval_nodes(f, lo, d, t, accumulate=True, precision=precision)
        got = np.stack([x.double().cpu().numpy() for x in f])
        assert np.max(np.abs(got - (prior.astype(dtype == torch.float32 and np.float32 or np.float64) + ref))) <= tol + 1e-6
        assert h.status() == 0
    assert np.max(np.abs(ref)) > 0.5


def _yee_float32_reference(E, B, dz, dt, n_steps):
    """The scheme with every product and difference rounded to float32 in
    the stated order (numpy float32 arithmetic, no fused multiply-add)."""
    E = np.array(E, dtype=np.float32)
    B = np.array(B, dtype=np.float32)
    r = np.float32(dt / dz)
    hr = np.float32(0.5 * (dt / dz))
    for _ in range(n_steps):
        B[:-1] = B[:-1] - hr * (E[1:] - E[:-1])
        E[1:] = E[1:] - r * (B[1:] - B[:-1])
        B[:-1] = B[:-1] - hr * (E[1:] - E[:-1])
    return E, B


@pytest.mark.gpu
@pytest.mark.parametrize("nz", [700, 3001, 6144, 12288])
def test_yee1d_float_bit_exact_all_blockings(nz):
    """Every register blocking (1, 4, 8 and 16 nodes per thread) gives the
    same float result as the plain per-node update."""
    import torch
    from paper_2307_04843_gb300 import _lib
    rng = np.random.default_rng(nz)
    E0 = rng.standard_normal(nz).astype(np.float32)
    B0 = rng.standard_normal(nz).astype(np.float32)
    E = torch.as_tensor(E0).cuda()
    B = torch.as_tensor(B0).cuda()
    _lib.ap_yee1d_run(E, B, 0.05, 0.0475, 37)
    Er, Br = _yee_float32_reference(E0, B0, 0.05, 0.0475, 37)
    assert np.array_equal(E.cpu().numpy(), Er) and np.array_equal(B.cpu().numpy(), Br)


@pytest.mark.gpu
@pytest.mark.parametrize("f64", [False, True])
def test_plane_wave_rows_at_unaligned_array_starts(f64):
    """The row path writes 16-byte vectors between a scalar head and tail:
    arrays that start 1..3 elements past a 16-byte boundary (allowed: the
    ABI asks for element alignment only), rows of a length that shifts the
    alignment from row to row, store and accumulate, all equal the oracle."""
    import torch
    from paper_2307_04843_gb300 import _lib
    pulse = dict(kind="plane", pol="cp", env="gauss", env_len=9.0, a0=1.5, t_focus=1.0, phase0=0.3)
    shape = (6, 3, 37)
    lo, d, t = (0.0, 0.2, -4.0), (0.1, 0.15, 0.9), 0.4
    ref = oracle.yee_nodes(pulse, shape, lo, d, t)
    dtype = torch.float64 if f64 else torch.float32
    size = int(np.prod(shape))
    tol = 1e-12 if f64 else 4e-6
    for off in ((1,) if f64 else (1, 2, 3)):
        bufs = [torch.zeros(size + 4, dtype=dtype, device="cuda") for _ in range(6)]
        f = [b[off:off + size].view(shape) for b in bufs]
        assert all(x.data_ptr() % 16 != 0 for x in f)
        with _lib.Handle(pulse) as h:
            h.eval_nodes(f, lo, d, t, precision="fp64" if f64 else "fp32")
            got = np.stack([x.double().cpu().numpy() for x in f])
            assert np.max(np.abs(got - ref)) <= tol, off
            h.eval_nodes(f, lo, d, t, accumulate=True, precision="fp64" if f64 else "fp32")
            got = np.stack([x.double().cpu().numpy() for x in f])
            assert np.max(np.abs(got - 2 * ref)) <= 2 * tol + 1e-6, off
            assert h.status() == 0
        for b in bufs:  # nothing written outside the arrays
            bb = b.cpu().numpy()
            assert not np.any(bb[:off]) and not np.any(bb[off + size:])
