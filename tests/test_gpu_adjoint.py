"""Discrete adjoint (ap_push_adjoint) and its torch.autograd.Function.

The gradient of the per-set mean final gamma with respect to (a0, w0,
z_focus) is checked against (i) the oracle's FP64 central finite
differences with Richardson extrapolation and (ii) GPU FP64 central finite
differences of the forward push, to relative error <= 1e-3 (the bound the
method's gradients are held to); the adjoint's objective equals the forward
push's mean gamma.  Segments: several checkpoints plus a ragged last one."""
import math

import numpy as np
import pytest

import oracle
from paper_2307_04843_gb300 import workloads
from support import THREADS

L = 2 * math.pi
NAMES = ("a0", "w0", "z_focus")


def _sets_case(n_sets=3, per=12, seed=3):
    cfg = workloads.config(5)
    sets, _ = workloads.batch_sets(cfg, seed=workloads.seed_for(5) + seed)
    sets = sets[:n_sets]
    counts = np.full(n_sets, per, dtype=np.int64)
    counts[-1] = per + 5
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    rng = np.random.default_rng(seed)
    n = int(off[-1])
    # particles near each set's focus region so the pulse does work
    parts = dict(x=rng.uniform(-1, 1, n) * 3 * L, y=rng.uniform(-1, 1, n) * 3 * L,
                 z=rng.uniform(-1, 1, n) * 2 * L, ux=np.zeros(n), uy=np.zeros(n), uz=np.zeros(n))
    for s in range(n_sets):
        parts["z"][off[s]:off[s + 1]] += sets[s]["z_focus"]
    return sets, off, parts


def _run_adjoint(sets, off, parts, t0, dt, n_steps, K, precision, grid=None):
    import torch
    from paper_2307_04843_gb300 import _lib
    from paper_2307_04843_gb300.autograd import adjoint
    dev = _lib.to_device(parts, precision)
    snap = {k: v.clone() for k, v in dev.items()}
    d_off = torch.as_tensor(off).cuda() if off is not None else None
    J, dJ = adjoint(sets, dev, d_off, t0, dt, n_steps, ckpt_every=K, precision=precision, grid=grid)
    for k in dev:  # the initial state is left unchanged
        assert torch.equal(dev[k], snap[k])
    return J.cpu().numpy(), dJ.cpu().numpy()


def _oracle_grads(sets, off, parts, t0, dt, n_steps, grid=None):
    out = []
    for s, pulse in enumerate(sets):
        sub = {k: v[off[s]:off[s + 1]] for k, v in parts.items()}
        g = oracle.grad_fd(pulse, sub, t0, dt, n_steps, names=NAMES, rel_h=1e-4, grid=grid,
                           scale=dict(z_focus=L))
        out.append([g[k] for k in NAMES])
    return np.array(out)


def _rel(a, b):
    return np.abs(a - b) / np.maximum(np.abs(b), 1e-3 * np.max(np.abs(b)))


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_adjoint_gauss_sets_vs_oracle_fd(precision):
    sets, off, parts = _sets_case()
    t0, dt, n_steps, K = -8.0, 0.02, 430, 100  # 5 segments, the last one of 30 steps
    J, dJ = _run_adjoint(sets, off, parts, t0, dt, n_steps, K, precision)
    ref = _oracle_grads(sets, off, parts, t0, dt, n_steps)
    err = _rel(dJ[:, :3], ref)
    assert np.max(err) <= 1e-3, (precision, err, dJ[:, :3], ref)
    assert np.all(dJ[:, 3] == 0.0)
    # objective equals the oracle's mean final gamma
    for s, pulse in enumerate(sets):
        sub = {k: v[off[s]:off[s + 1]] for k, v in parts.items()}
        mg = oracle.mean_gamma(pulse, sub, t0, dt, n_steps)
        assert J[s] == pytest.approx(mg, rel=1e-12 if precision == "fp64" else 1e-5)


@pytest.mark.gpu
def test_adjoint_vs_gpu_fp64_central_differences():
    """Against FP64 central differences of the GPU forward push itself."""
    import torch
    from paper_2307_04843_gb300 import _lib
    sets, off, parts = _sets_case(n_sets=2, per=16, seed=7)
    t0, dt, n_steps, K = -6.0, 0.02, 300, 64
    _, dJ = _run_adjoint(sets, off, parts, t0, dt, n_steps, K, "fp64")

    def J(pulse, sub):
        with _lib.Handle(pulse) as h:
            d = _lib.to_device(sub, "fp64")
            ss = torch.zeros(1, dtype=torch.float64, device="cuda")
            h.push(d, t0, dt, n_steps, precision="fp64", diag=dict(set_sum=ss))
            return float(ss.item()) / sub["x"].size

    for s, pulse in enumerate(sets):
        sub = {k: v[off[s]:off[s + 1]] for k, v in parts.items()}
        for k, name in enumerate(NAMES):
            h = 1e-5 * (abs(pulse[name]) if name != "z_focus" else L)
            fd = (J(dict(pulse, **{name: pulse[name] + h}), sub) - J(dict(pulse, **{name: pulse[name] - h}), sub)) / (2 * h)
            assert abs(dJ[s, k] - fd) <= 1e-3 * max(abs(fd), 1e-6), (s, name, dJ[s, k], fd)


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("kind", ["lg", "plane"])
def test_adjoint_other_kinds_vs_oracle_fd(kind, precision):
    if kind == "lg":
        pulse = dict(kind="lg", pol="cp", env="gauss", env_len=20.0, a0=4.0, w0=2.5 * L, lg_p=1, lg_l=2,
                     z_focus=3.0, t_focus=0.0, longitudinal=True)
    else:
        pulse = dict(kind="plane", pol="x", env="sin2", env_len=6, a0=2.0, z_focus=1.0, t_focus=6 * math.pi)
    rng = np.random.default_rng(11)
    n = 24
    parts = dict(x=rng.uniform(-1, 1, n) * L, y=rng.uniform(-1, 1, n) * L, z=rng.uniform(-1, 1, n) * L,
                 ux=np.zeros(n), uy=np.zeros(n), uz=np.zeros(n))
    off = np.array([0, n], dtype=np.int64)
    t0, dt, n_steps, K = -5.0 if kind == "lg" else 0.0, 0.02, 350, 128
    _, dJ = _run_adjoint([pulse], off, parts, t0, dt, n_steps, K, precision)
    names = NAMES if kind == "lg" else ("a0", "z_focus")
    g = oracle.grad_fd(pulse, parts, t0, dt, n_steps, names=names, rel_h=1e-4, scale=dict(z_focus=L))
    gmax = max(abs(g[k]) for k in names)
    for name in names:
        k = NAMES.index(name)
        floor = 1e-8 if precision == "fp64" else 1e-2 * gmax
        assert abs(dJ[0, k] - g[name]) <= 1e-3 * max(abs(g[name]), floor), (kind, precision, name, dJ[0, k], g[name])


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_adjoint_flying_focus_closed_form_vs_oracle_fd(precision):
    """All four rows, including d/dbeta_f, for the closed-form flying focus."""
    pulse = dict(kind="flying_cf", pol="x", env="gauss", env_len=20.0, a0=3.0, w0=2.5 * L, beta_f=-0.5,
                 z_focus=1.0, t_focus=0.0, longitudinal=True)
    rng = np.random.default_rng(19)
    n = 40
    parts = dict(x=rng.uniform(-1, 1, n) * 2 * L, y=rng.uniform(-1, 1, n) * 2 * L,
                 z=rng.uniform(-1, 1, n) * 2 * L, ux=np.zeros(n), uy=np.zeros(n), uz=np.zeros(n))
    off = np.array([0, n], dtype=np.int64)
    t0, dt, n_steps, K = -6.0, 0.02, 500, 96
    _, dJ = _run_adjoint([pulse], off, parts, t0, dt, n_steps, K, precision)
    names = NAMES + ("beta_f",)
    g = oracle.grad_fd(pulse, parts, t0, dt, n_steps, names=names, rel_h=1e-4,
                       scale=dict(z_focus=L, beta_f=0.1))
    gmax = max(abs(g[k]) for k in names)
    for k, name in enumerate(names):
        assert abs(dJ[0, k] - g[name]) <= 1e-3 * max(abs(g[name]), 1e-2 * gmax), (precision, name, dJ[0, k], g[name])
    assert abs(g["beta_f"]) > 1e-3 * gmax  # the focal velocity matters here


@pytest.mark.gpu
@pytest.mark.parametrize("kind,pol,env", [("gauss", "y", "sgauss"), ("gauss", "cp", "sin2"),
                                          ("gauss", "cm", "cw"), ("flying_cf", "cp", "sin2"),
                                          ("flying_cf", "y", "sgauss")])
def test_adjoint_beam_polarisations_envelopes_vs_oracle_fd(kind, pol, env):
    """The closed-form beam Jacobian for every polarisation and envelope
    (the other tests take linear x and a Gaussian envelope)."""
    pulse = dict(kind=kind, pol=pol, env=env, env_len=14.0, a0=3.0, w0=2.2 * L, z_focus=0.7, t_focus=0.0,
                 longitudinal=True)
    if env == "sgauss":
        pulse["sg_order"] = 2
    if env == "cw":
        pulse["a0"] = 0.5
    if kind == "flying_cf":
        pulse["beta_f"] = -0.4
    rng = np.random.default_rng(37)
    n = 24
    parts = dict(x=rng.uniform(-1, 1, n) * 2 * L, y=rng.uniform(-1, 1, n) * 2 * L,
                 z=rng.uniform(-1, 1, n) * L, ux=rng.normal(0, 0.05, n), uy=rng.normal(0, 0.05, n),
                 uz=np.zeros(n))
    off = np.array([0, n], dtype=np.int64)
    t0, dt, n_steps, K = -6.0, 0.02, 420, 100
    names = NAMES + (("beta_f",) if kind == "flying_cf" else ())
    g = oracle.grad_fd(pulse, parts, t0, dt, n_steps, names=names, rel_h=1e-4,
                       scale=dict(z_focus=L, beta_f=0.1))
    gmax = max(abs(g[k]) for k in names)
    for precision in ("fp64", "fp32"):
        _, dJ = _run_adjoint([pulse], off, parts, t0, dt, n_steps, K, precision)
        for k, name in enumerate(names):
            assert abs(dJ[0, k] - g[name]) <= 1e-3 * max(abs(g[name]), 1e-2 * gmax), \
                (precision, kind, pol, env, name, dJ[0, k], g[name])


@pytest.mark.gpu
@pytest.mark.parametrize("n,n_steps,K", [(1, 1, 1), (3, 257, 256), (257, 7, 2), (300, 64, 64)])
def test_adjoint_edge_sizes_vs_oracle_fd(n, n_steps, K):
    """Edge sizes of the adjoint (the two-particle kernel takes tiles of 256
    in FP32, the one-particle kernel tiles of 128 in FP64): a single electron
    and step, the largest segment with a last segment of one step, a ragged
    second tile with two-step segments, one whole segment."""
    pulse = dict(kind="gauss", pol="cp", env="gauss", env_len=10.0, a0=8.0, w0=2.0 * L, z_focus=0.3,
                 t_focus=0.0, longitudinal=True)
    rng = np.random.default_rng(41 + n)
    parts = dict(x=rng.uniform(-1, 1, n) * L, y=rng.uniform(-1, 1, n) * L, z=rng.uniform(-1, 1, n) * L,
                 ux=rng.normal(0, 0.1, n), uy=rng.normal(0, 0.1, n), uz=rng.normal(0, 0.1, n))
    off = np.array([0, n], dtype=np.int64)
    t0, dt = -2.0, 0.02
    g = oracle.grad_fd(pulse, parts, t0, dt, n_steps, names=NAMES, rel_h=1e-4, scale=dict(z_focus=L))
    gmax = max(abs(g[k]) for k in NAMES)
    for precision in ("fp64", "fp32"):
        J, dJ = _run_adjoint([pulse], off, parts, t0, dt, n_steps, K, precision)
        assert J[0] == pytest.approx(oracle.mean_gamma(pulse, parts, t0, dt, n_steps),
                                     rel=1e-12 if precision == "fp64" else 1e-5)
        tol = 1e-5 if precision == "fp64" else 1e-3
        for k, name in enumerate(NAMES):
            assert abs(dJ[0, k] - g[name]) <= tol * max(abs(g[name]), 1e-2 * gmax), \
                (precision, n, n_steps, K, name, dJ[0, k], g[name])


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_adjoint_single_set_without_offsets(precision):
    """One set given without offsets (the whole array is the set) gives the
    same objective and gradient, bit for bit, as the same set with offsets
    [0, n]; the FP32 call takes the two-particle kernel, with an odd count so
    the last thread carries one particle."""
    import torch
    from paper_2307_04843_gb300 import _lib
    from paper_2307_04843_gb300.autograd import adjoint
    sets, off, parts = _sets_case(n_sets=1, per=250, seed=13)  # 255: at most two tiles (sum order)
    t0, dt, n_steps, K = -8.0, 0.02, 230, 50
    dev = _lib.to_device(parts, precision)
    J0, d0 = adjoint(sets, dev, None, t0, dt, n_steps, ckpt_every=K, precision=precision)
    J1, d1 = adjoint(sets, dev, torch.as_tensor(off).cuda(), t0, dt, n_steps, ckpt_every=K, precision=precision)
    assert torch.equal(J0, J1) and torch.equal(d0, d1)
    assert torch.all(d0[0, :3] != 0)


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_adjoint_empty_sets(precision):
    """Empty sets before, between and after populated ones: their objective
    and gradient rows are zero, and a populated set's row equals that set run
    alone, bit for bit."""
    import torch
    from paper_2307_04843_gb300 import _lib
    from paper_2307_04843_gb300.autograd import adjoint
    sets, _, parts = _sets_case(n_sets=2, per=20, seed=23)
    n0 = 20
    four = [sets[0], sets[0], sets[1], sets[1]]
    off = np.array([0, 0, n0, n0, parts["x"].size], dtype=np.int64)  # sets 0 and 2 empty
    t0, dt, n_steps, K = -8.0, 0.02, 120, 40
    dev = _lib.to_device(parts, precision)
    J, dJ = adjoint(four, dev, torch.as_tensor(off).cuda(), t0, dt, n_steps, ckpt_every=K, precision=precision)
    J, dJ = J.cpu().numpy(), dJ.cpu().numpy()
    assert J[0] == 0.0 and J[2] == 0.0 and np.all(dJ[0] == 0.0) and np.all(dJ[2] == 0.0)
    for s, (lo, hi) in ((1, (0, n0)), (3, (n0, parts["x"].size))):
        sub = {k: v[lo:hi] for k, v in parts.items()}
        d1 = _lib.to_device(sub, precision)
        J1, dJ1 = adjoint([four[s]], d1, None, t0, dt, n_steps, ckpt_every=K, precision=precision)
        assert J[s] == float(J1[0]) and np.array_equal(dJ[s], dJ1[0].cpu().numpy()), s


@pytest.mark.gpu
def test_adjoint_one_d_lines_vs_oracle_fd():
    """1D-3V set (transverse position held): the position update and its
    reverse use dt only along z."""
    pulse = dict(kind="gauss", pol="x", env="gauss", env_len=12.0, a0=6.0, w0=2.0 * L, z_focus=0.5,
                 t_focus=0.0, longitudinal=True, one_d=True)
    rng = np.random.default_rng(29)
    n = 30
    parts = dict(x=rng.uniform(-1, 1, n) * L, y=rng.uniform(-1, 1, n) * L, z=rng.uniform(-1, 1, n) * L,
                 ux=rng.normal(0, 0.2, n), uy=rng.normal(0, 0.2, n), uz=rng.normal(0, 0.2, n))
    off = np.array([0, n], dtype=np.int64)
    t0, dt, n_steps, K = -8.0, 0.02, 600, 128
    _, dJ = _run_adjoint([pulse], off, parts, t0, dt, n_steps, K, "fp64")
    g = oracle.grad_fd(pulse, parts, t0, dt, n_steps, names=NAMES, rel_h=1e-4, scale=dict(z_focus=L))
    for k, name in enumerate(NAMES):
        assert abs(dJ[0, k] - g[name]) <= 1e-3 * max(abs(g[name]), 1e-8), (name, dJ[0, k], g[name])


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_adjoint_with_linear_grid_field(precision):
    """A grid holding linear fields (trilinear interpolation is then exact and
    smooth across cells) enters the trajectory and the position adjoint."""
    sets, off, parts = _sets_case(n_sets=1, per=20, seed=5)
    nx = ny = nz = 9
    lo, hi = (-25.0, -25.0, -60.0), (25.0, 25.0, 60.0)
    X = np.linspace(lo[0], hi[0], nx)[None, None, :]
    Y = np.linspace(lo[1], hi[1], ny)[:, None][None]
    Z = np.linspace(lo[2], hi[2], nz)[:, None, None]
    comps = [0.02 + 0.001 * X + 0 * Y + 0 * Z, 0.0005 * Y + 0 * X + 0 * Z, -0.0004 * Z + 0 * X + 0 * Y,
             0.0003 * X + 0.0002 * Y + 0 * Z, 0.01 + 0 * X + 0 * Y + 0 * Z, 0.0002 * Z + 0 * X + 0 * Y]
    grid = np.stack([np.broadcast_to(c, (nz, ny, nx)) for c in comps]).astype(np.float32)
    import torch
    g_dev = (torch.as_tensor(grid).cuda(), lo, hi)
    t0, dt, n_steps, K = -8.0, 0.02, 300, 100
    _, dJ = _run_adjoint(sets, off, parts, t0, dt, n_steps, K, precision, grid=g_dev)
    ref = _oracle_grads(sets, off, parts, t0, dt, n_steps, grid=(grid, lo, hi))
    assert np.max(_rel(dJ[:, :3], ref)) <= 1e-3, (dJ[:, :3], ref)


@pytest.mark.gpu
def test_adjoint_packed_grid_same_as_arrays():
    """A grid passed with its per-cell coefficient copy (the push's fast
    layout) gives the adjoint exactly the result of the plain arrays: the
    adjoint interpolates the raw corners either way."""
    import torch
    from paper_2307_04843_gb300 import _lib
    sets, off, parts = _sets_case(n_sets=2, per=40, seed=17)
    nx, ny, nz = 12, 10, 14
    lo, hi = (-25.0, -25.0, -60.0), (25.0, 25.0, 60.0)
    rng = np.random.default_rng(3)
    grid = (0.01 * rng.standard_normal((6, nz, ny, nx))).astype(np.float32)
    g = torch.as_tensor(grid).cuda()
    t0, dt, n_steps, K = -8.0, 0.02, 150, 50
    _, d_arr = _run_adjoint(sets, off, parts, t0, dt, n_steps, K, "fp32", grid=(g, lo, hi))
    packed = _lib.pack_grid((g, lo, hi), layout="cells")
    _, d_pk = _run_adjoint(sets, off, parts, t0, dt, n_steps, K, "fp32", grid=packed)
    assert np.array_equal(d_arr, d_pk)
    assert np.all(d_arr[:, :3] != 0)


@pytest.mark.gpu
def test_autograd_function_gradcheck_fp64():
    import torch
    from paper_2307_04843_gb300 import _lib
    from paper_2307_04843_gb300.autograd import mean_final_gamma
    sets, off, parts = _sets_case(n_sets=2, per=6, seed=9)
    dev = _lib.to_device(parts, "fp64")
    d_off = torch.as_tensor(off).cuda()
    params = torch.tensor([[s["a0"], s["w0"], s["z_focus"]] for s in sets], dtype=torch.float64,
                          requires_grad=True)

    def f(p):
        return mean_final_gamma(p, sets, dev, d_off, t0=-6.0, dt=0.02, n_steps=150, ckpt_every=40,
                                precision="fp64")

    assert torch.autograd.gradcheck(f, (params,), eps=1e-6, atol=1e-7, rtol=1e-4)
    J = f(params)
    J.sum().backward()
    assert params.grad is not None and torch.all(torch.isfinite(params.grad))


@pytest.mark.gpu
def test_adjoint_errors():
    import torch
    from paper_2307_04843_gb300 import _lib
    cfg = workloads.config(4)
    parts = workloads.particles(cfg, n=32)
    dev = _lib.to_device(parts, "fp32")
    with _lib.Handle(cfg["pulse"]) as h:
        dJ = torch.zeros((1, 4), dtype=torch.float64, device="cuda")
        ws = torch.zeros(1 << 20, dtype=torch.float32, device="cuda")
        with pytest.raises(_lib.APError) as e:
            _lib.ap_push_adjoint(h.h, dev, None, None, 0.0, 0.02, 10, 5, "fp32", dJ, None, ws)
        assert e.value.status == _lib.AP_ERR_UNSUPPORTED
    sets, off, p2 = _sets_case(n_sets=1, per=8)
    dev = _lib.to_device(p2, "fp32")
    with _lib.Handle(sets) as h:
        tiny = torch.zeros(64, dtype=torch.float32, device="cuda")
        with pytest.raises(_lib.APError) as e:
            _lib.ap_push_adjoint(h.h, dev, None, None, 0.0, 0.02, 10, 5, "fp32", dJ, None, tiny)
        assert e.value.status == _lib.AP_ERR_WORKSPACE
        assert _lib.ap_adjoint_workspace_bytes(h.h, 8, 10, 0) == 0
        assert _lib.ap_adjoint_workspace_bytes(h.h, 8, 10, 300) == 0
