"""The node and line kernels at the sizes and in the calls that bench.py
times (its secondary rates), checked on sampled outputs the oracle computes
one by one, or, for the lines, against a float32 replica of their
expressions (bit-exact) and by the identity of lines that carry the same
problem."""
import math

import numpy as np
import pytest

import oracle

L = 2.0 * math.pi


def _node_positions(lo, d, idx, comp):
    """Physical positions of nodes idx = (k, j, i) of component comp at its
    Yee offset (Ex (1/2,0,0), Ey (0,1/2,0), Ez (0,0,1/2), Bx (0,1/2,1/2),
    By (1/2,0,1/2), Bz (1/2,1/2,0))."""
    off = [(0.5, 0, 0), (0, 0.5, 0), (0, 0, 0.5), (0, 0.5, 0.5), (0.5, 0, 0.5), (0.5, 0.5, 0)][comp]
    k, j, i = idx
    return (lo[0] + (i + off[0]) * d[0], lo[1] + (j + off[1]) * d[1], lo[2] + (k + off[2]) * d[2])


@pytest.mark.gpu
@pytest.mark.parametrize("pulse_name", ["workload2", "plane"])
def test_eval_nodes_bench_grid_sampled(pulse_name):
    """256^3 float arrays, float-float phase, the bench's two pulses."""
    import torch
    import bench
    from paper_2307_04843_gb300 import _lib, workloads
    cfg = workloads.config(2)
    pulse = cfg["pulse"] if pulse_name == "workload2" else \
        dict(kind="plane", pol="x", env="sgauss", sg_order=4, env_len=30.0, a0=1.0)
    n = bench.NODE_N
    lo, hi = workloads.grid_box(cfg)
    d = tuple((hi[a] - lo[a]) / (n - 1) for a in range(3))
    f = [torch.empty((n, n, n), dtype=torch.float32, device="cuda") for _ in range(6)]
    with _lib.Handle(pulse) as h:
        h.eval_nodes(f, lo, d, 0.0, precision="fp32")
        assert h.status() == 0
    rng = np.random.default_rng(41)
    idx = rng.integers(0, n, size=(3, 150))
    # and nodes near the beam axis and the focus, where the field is largest
    near = np.stack([rng.integers(n // 2 - 20, n // 2 + 20, 50) for _ in range(3)])
    idx = np.concatenate([idx, near], axis=1)
    a0 = pulse["a0"]
    for c in range(6):
        x, y, z = _node_positions(lo, d, idx, c)
        ref = oracle.fields(pulse, x, y, z, np.zeros_like(x))[c]
        got = f[c][tuple(torch.as_tensor(v).cuda() for v in idx)].double().cpu().numpy()
        assert np.max(np.abs(got - ref)) <= 4e-6 * a0, (pulse_name, c, np.max(np.abs(got - ref)))
    if pulse_name == "workload2":
        assert np.max(np.abs(oracle.fields(pulse, *_node_positions(lo, d, near, 0), np.zeros(50))[0])) > 1.0


def _yee_f32(E, B, r, hr, n):
    for _ in range(n):
        B[:-1] = B[:-1] - hr * (E[1:] - E[:-1])
        E[1:] = E[1:] - r * (B[1:] - B[:-1])
        B[:-1] = B[:-1] - hr * (E[1:] - E[:-1])
    return E, B


@pytest.mark.gpu
def test_yee1d_bench_call_bit_exact():
    """152 float lines x 8192 nodes x 2000 steps from a unit pulse in the
    middle of every line (the bench's call)."""
    import torch
    import bench
    from paper_2307_04843_gb300 import _lib
    nl, nz, n = bench.YEE_LINES, bench.YEE_NZ, bench.YEE_STEPS
    E = torch.zeros((nl, nz), dtype=torch.float32, device="cuda")
    B = torch.zeros_like(E)
    E[:, nz // 2] = 1.0
    _lib.ap_yee1d_run(E, B, 0.05, 0.0475, n)
    assert torch.equal(E, E[0:1].expand_as(E)) and torch.equal(B, B[0:1].expand_as(B))
    f = np.float32
    e0 = np.zeros(nz, dtype=f)
    e0[nz // 2] = 1.0
    Er, Br = _yee_f32(e0, np.zeros(nz, dtype=f), f(0.0475 / 0.05), f(0.5 * (0.0475 / 0.05)), n)
    assert np.array_equal(E[0].cpu().numpy(), Er) and np.array_equal(B[0].cpu().numpy(), Br)
    assert np.max(np.abs(Er)) > 0.01


@pytest.mark.gpu
def test_plasma1d_bench_shape_bit_exact():
    """304 float lines x 4096 nodes x 20000 steps of the Yee + current line
    (the bench's shape and plasma) from a unit pulse on every line: all
    lines equal, line 0 equal to the float32 replica."""
    import torch
    import bench
    from paper_2307_04843_gb300 import _lib
    nl, nz, n = bench.LINE_LINES, bench.LINE_NZ, bench.PLASMA_STEPS
    wp = math.sqrt(1e-3)
    dz = L / 20.0
    dt = 0.9 * dz
    E = torch.zeros((nl, nz), dtype=torch.float32, device="cuda")
    B, J = torch.zeros_like(E), torch.zeros_like(E)
    E[:, nz // 3] = 1.0
    _lib.ap_plasma1d_run(E, B, J, dz, dt, n, omega_p=wp)
    for t in (E, B, J):
        assert torch.equal(t, t[0:1].expand_as(t))
    f = np.float32
    Er, Br, Jr = np.zeros(nz, dtype=f), np.zeros(nz, dtype=f), np.zeros(nz, dtype=f)
    Er[nz // 3] = 1.0
    r, hr, dtf = f(dt / dz), f(0.5 * (dt / dz)), f(dt)
    q = dtf * f(wp * wp)
    for _ in range(n):
        Br[:-1] = Br[:-1] - hr * (Er[1:] - Er[:-1])
        Jr = Jr + q * Er
        Er[1:] = (Er[1:] - r * (Br[1:] - Br[:-1])) - dtf * Jr[1:]
        Br[:-1] = Br[:-1] - hr * (Er[1:] - Er[:-1])
    assert np.array_equal(E[0].cpu().numpy(), Er) and np.array_equal(B[0].cpu().numpy(), Br)
    assert np.array_equal(J[0].cpu().numpy(), Jr)
