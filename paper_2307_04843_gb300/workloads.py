"""Seeded synthetic inputs for the analytic-pulse push.

This module holds no arithmetic of the method: it only describes the five
workloads (pulse parameters, particle counts, boxes, time steps) and draws
their seeded random inputs (particle ensembles, the static grid field, the
batched parameter sets) with numpy's PCG64.  Both the CUDA path (through the
binding) and the CPU oracle (in the tests and the benchmark's CPU leg)
consume these inputs unchanged.

Units: c = omega0 = k0 = 1, lambda = 2 pi.  Workloads, shaped after the
paper's inverse-Compton (Sec. 3.2, Fig. 6) and flying-focus (Sec. 3.3,
Fig. 7) examples:
  1 plane  -- 1e4 e- at rest in a 10 lambda cube, LP plane wave, a0 = 1,
              sin^2 envelope of 10 cycles, 2000 steps, FP64;
  2 gauss  -- 1e7 e- at rest in 20x20x40 lambda, Gaussian w0 = 3 lambda,
              a0 = 10, FWHM 30, longitudinal fields, 256^3 static grid,
              4000 steps;
  3 ics    -- 3.2e7 e- beam (gamma ~ N(1000, 10), 1 mrad), CP LG_{1,2},
              w0 = 2 lambda, a0 = 20, 20-cycle sin^2, 3000 steps, gamma histogram;
  4 ff     -- 1.6e7 e- at rest in a 10x10x200 lambda channel, flying focus of
              64 Gaussian components, v_f = 0.99, a0 = 5, 6000 steps;
  5 batch  -- 256 Gaussian sets, a0 ~ U[2, 20], w0 ~ U[2, 6] lambda,
              z_f ~ U[-10, 10] lambda, log-uniform counts in [1e4, 2e5],
              2000 steps, mean final gamma per set and its gradient;
  6 sweep  -- reduced-dimensionality inverse Compton (Sec. 3.2, Fig. 6):
              30 one-dimensional (1D-3V) electron lines at radii
              (s + 1/2) 0.1 lambda in a focused Gaussian, a0 = 50, 3-lambda
              intensity FWHM spot, 15-fs (4.5-cycle) intensity FWHM, and a
              2.6-GeV (gamma 5088) counter-propagating beam of 15-fs
              duration; 1e5 electrons per line, 4000 steps, one set per line.
"""
import math

import numpy as np

LAMBDA = 2.0 * math.pi
SEED_BASE = 2307048430
DT = 0.02


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def config(index):
    """Workload description (plain dict) for workload 1..5."""
    L = LAMBDA
    if index == 1:
        return dict(
            name="plane-fp64", index=1, n=10_000, n_steps=2000, dt=DT, t0=0.0,
            precision="fp64",
            pulse=dict(kind="plane", pol="x", env="sin2", env_len=10.0, a0=1.0, omega=1.0,
                       z_focus=0.0, t_focus=10.0 * math.pi, phase0=0.0),
            box=((0.0, 10 * L), (0.0, 10 * L), (0.0, 10 * L)), grid=None,
            diag=dict(lightfront=True))
    if index == 2:
        return dict(
            name="gauss-grid", index=2, n=10_000_000, n_steps=4000, dt=DT, t0=-40.0,
            precision="fp32",
            pulse=dict(kind="gauss", pol="x", env="gauss", env_len=30.0, a0=10.0, omega=1.0,
                       w0=3 * L, z_focus=0.0, t_focus=0.0, phase0=0.0, longitudinal=True),
            box=((-10 * L, 10 * L), (-10 * L, 10 * L), (-20 * L, 20 * L)),
            grid=dict(n=256, amplitude=0.1, n_terms=16, kmax=4), diag=dict())
    if index == 3:
        return dict(
            name="ics-lg12", index=3, n=32_000_000, n_steps=3000, dt=DT, t0=0.0,
            precision="fp32",
            pulse=dict(kind="lg", pol="cp", env="sin2", env_len=20.0, a0=20.0, omega=1.0,
                       w0=2 * L, lg_p=1, lg_l=2, z_focus=0.0, t_focus=30.0, phase0=0.0,
                       longitudinal=True),
            beam=dict(sigma_perp=0.5 * L, sigma_z=5 * L, z_center=30.0, gamma_mean=1000.0,
                      gamma_sigma=10.0, divergence=1e-3),
            box=None, grid=None,
            diag=dict(hist_bins=1024, hist_lo=940.0, hist_hi=1060.0))
    if index == 4:
        v_f = 0.99
        length = 200 * L
        t_mid = 0.5 * length / v_f
        return dict(
            name="flying-focus", index=4, n=16_000_000, n_steps=6000, dt=DT, t0=t_mid - 60.0,
            precision="fp32",
            pulse=dict(kind="flying", pol="x", env="cw", a0=5.0, omega=1.0,
                       w0=3 * L / math.sqrt(2 * math.log(2)), n_comp=64, bw_frac=0.05,
                       beta_f=v_f, ff_length=length, z_focus=0.0, t_focus=0.0, phase0=0.0,
                       longitudinal=True),
            box=((-5 * L, 5 * L), (-5 * L, 5 * L), (0.0, 200 * L)), grid=None, diag=dict())
    if index == 5:
        return dict(
            name="batched-gauss", index=5, n_sets=256, n_steps=2000, dt=DT, t0=-20.0,
            precision="fp32", ckpt_every=100,
            pulse=dict(kind="gauss", pol="x", env="gauss", env_len=30.0, omega=1.0,
                       t_focus=0.0, phase0=0.0, longitudinal=True),
            ranges=dict(a0=(2.0, 20.0), w0=(2 * L, 6 * L), z_focus=(-10 * L, 10 * L),
                        count=(1e4, 2e5)),
            box=((-10 * L, 10 * L), (-10 * L, 10 * L), (-20 * L, 20 * L)), grid=None,
            diag=dict(set_sums=True))
    if index == 6:
        cycle = 1.0 / 3.3356409519815204  # 1 fs in units of the laser period (lambda = 1 um)
        fwhm_t = 15.0 * cycle * L         # 15 fs in 1 / omega0
        return dict(
            name="ics-sweep-1d3v", index=6, n_sets=30, per_set=100_000, n_steps=4000, dt=DT,
            t0=-40.0, precision="fp32",
            pulse=dict(kind="gauss", pol="x", env="gauss", env_len=fwhm_t, a0=50.0, omega=1.0,
                       w0=3 * L / math.sqrt(2 * math.log(2)), z_focus=0.0, t_focus=0.0, phase0=0.0,
                       longitudinal=True, one_d=True),
            radius_step=0.1 * L,
            beam=dict(gamma=2600.0 / 0.51099895, sigma_z=fwhm_t / (2 * math.sqrt(2 * math.log(2))),
                      z_center=40.0),
            box=None, grid=None, diag=dict(set_sums=True))
    raise ValueError("workload index must be 1..6")


def seed_for(index):
    return SEED_BASE + index


def particles_uniform(box, n, seed):
    """n particles at rest, uniform in box ((x0,x1),(y0,y1),(z0,z1)).  The
    stream is drawn row by row, so the first m particles do not depend on n."""
    r = _rng(seed).random((n, 3))
    lo = np.array([b[0] for b in box])
    hi = np.array([b[1] for b in box])
    pos = lo + r * (hi - lo)
    zeros = np.zeros(n)
    return dict(x=pos[:, 0].copy(), y=pos[:, 1].copy(), z=pos[:, 2].copy(),
                ux=zeros.copy(), uy=zeros.copy(), uz=zeros.copy())


def particles_beam(beam, n, seed):
    """Counter-propagating electron beam (moving along -z): Gaussian position
    spread, Gaussian gamma spread, Gaussian angles in each transverse plane."""
    g = _rng(seed).standard_normal((n, 6))
    x = beam["sigma_perp"] * g[:, 0]
    y = beam["sigma_perp"] * g[:, 1]
    z = beam["z_center"] + beam["sigma_z"] * g[:, 2]
    gamma = beam["gamma_mean"] + beam["gamma_sigma"] * g[:, 3]
    thx = beam["divergence"] * g[:, 4]
    thy = beam["divergence"] * g[:, 5]
    p = np.sqrt(gamma * gamma - 1.0)
    ux = p * thx
    uy = p * thy
    uz = -p * np.sqrt(np.maximum(1.0 - thx * thx - thy * thy, 0.0))
    return dict(x=x, y=y, z=z, ux=ux, uy=uy, uz=uz)


def particles(cfg, n=None, seed=None):
    """Seeded particle ensemble of a workload (first n particles)."""
    n = cfg.get("n") if n is None else n
    seed = seed_for(cfg["index"]) if seed is None else seed
    if cfg["index"] == 3:
        return particles_beam(cfg["beam"], n, seed)
    return particles_uniform(cfg["box"], n, seed)


def batch_sets(cfg, seed=None):
    """Pulse-parameter sets and their particle counts (workload 5).
    Returns (list of pulse dicts, int64 counts)."""
    seed = seed_for(cfg["index"]) if seed is None else seed
    rng = _rng(seed)
    S = cfg["n_sets"]
    r = cfg["ranges"]
    u = rng.random((S, 4))
    a0 = r["a0"][0] + u[:, 0] * (r["a0"][1] - r["a0"][0])
    w0 = r["w0"][0] + u[:, 1] * (r["w0"][1] - r["w0"][0])
    zf = r["z_focus"][0] + u[:, 2] * (r["z_focus"][1] - r["z_focus"][0])
    lc = math.log(r["count"][0]) + u[:, 3] * (math.log(r["count"][1]) - math.log(r["count"][0]))
    counts = np.rint(np.exp(lc)).astype(np.int64)
    sets = []
    for s in range(S):
        d = dict(cfg["pulse"])
        d.update(a0=float(a0[s]), w0=float(w0[s]), z_focus=float(zf[s]))
        sets.append(d)
    return sets, counts


def sweep_lines(cfg, per_set=None, seed=None):
    """Pulse sets and particles of the radial sweep (workload 6): set s holds
    `per_set` electrons on the line x = (s + 1/2) dr, y = 0, with z drawn
    from N(z_center, sigma_z) and u = (0, 0, -sqrt(gamma^2 - 1)).  Returns
    (list of pulse dicts, particle dict, int64 offsets [n_sets + 1])."""
    seed = seed_for(cfg["index"]) if seed is None else seed
    m = cfg["per_set"] if per_set is None else int(per_set)
    S = cfg["n_sets"]
    b = cfg["beam"]
    g = _rng(seed).standard_normal((S, m))
    r = (np.arange(S) + 0.5) * cfg["radius_step"]
    n = S * m
    x = np.repeat(r, m)
    z = (b["z_center"] + b["sigma_z"] * g).reshape(n)
    uz = -math.sqrt(b["gamma"] ** 2 - 1.0)
    parts = dict(x=x, y=np.zeros(n), z=z, ux=np.zeros(n), uy=np.zeros(n), uz=np.full(n, uz))
    off = (np.arange(S + 1) * m).astype(np.int64)
    return [dict(cfg["pulse"]) for _ in range(S)], parts, off


def scaled_counts(counts, total):
    """Counts scaled down proportionally (each >= 1) so they sum to about
    `total`; used for small parity cases of the batched workload."""
    c = np.maximum(1, np.rint(counts * (total / counts.sum()))).astype(np.int64)
    return c


def grid_modes(seed, n_terms=16, kmax=4):
    """Random Fourier modes of the static grid: for each of the 6 components,
    n_terms integer wave-vectors drawn from {-kmax..kmax}^3 minus 0 and
    uniform phases.  Returns (int array [6, n_terms, 3], phases [6, n_terms])."""
    rng = _rng(seed)
    nvec = np.zeros((6, n_terms, 3), dtype=np.int64)
    phases = np.zeros((6, n_terms))
    for c in range(6):
        m = 0
        while m < n_terms:
            v = rng.integers(-kmax, kmax + 1, size=3)
            if np.all(v == 0):
                continue
            nvec[c, m] = v
            m += 1
        phases[c] = rng.random(n_terms) * 2.0 * math.pi
    return nvec, phases


def grid_field(box, n, amplitude=0.1, n_terms=16, kmax=4, seed=SEED_BASE + 2, torch_device=None):
    """Static node-centred grid E2/B2: component c is
        F_c = amplitude * S_c / max|S_c|,  S_c = sum_m cos(k_m . x + phi_m),
    k_m = 2 pi (n_x / L_x, n_y / L_y, n_z / L_z), on n^3 nodes spanning box.
    Returns float32 [6, n, n, n] (z, y, x order) as a numpy array, or a torch
    tensor on torch_device when given (same values; built there for speed)."""
    nvec, phases = grid_modes(seed, n_terms, kmax)
    lo = np.array([b[0] for b in box])
    hi = np.array([b[1] for b in box])
    ext = hi - lo
    if torch_device is not None:
        import torch
        dev = torch.device(torch_device)
        coords = [torch.linspace(lo[a], hi[a], n, dtype=torch.float64, device=dev) for a in range(3)]
        out = torch.empty((6, n, n, n), dtype=torch.float32, device=dev)
        for c in range(6):
            S = torch.zeros((n, n, n), dtype=torch.float64, device=dev)
            for m in range(n_terms):
                k = 2.0 * math.pi * nvec[c, m] / ext
                ax = torch.exp(1j * (k[0] * coords[0]))
                ay = torch.exp(1j * (k[1] * coords[1]))
                az = torch.exp(1j * (k[2] * coords[2] + phases[c, m]))
                S += (az[:, None, None] * ay[None, :, None] * ax[None, None, :]).real
            out[c] = (amplitude * S / S.abs().max()).to(torch.float32)
        return out
    coords = [np.linspace(lo[a], hi[a], n) for a in range(3)]
    out = np.empty((6, n, n, n), dtype=np.float32)
    for c in range(6):
        S = np.zeros((n, n, n))
        for m in range(n_terms):
            k = 2.0 * math.pi * nvec[c, m] / ext
            ax = np.exp(1j * (k[0] * coords[0]))
            ay = np.exp(1j * (k[1] * coords[1]))
            az = np.exp(1j * (k[2] * coords[2] + phases[c, m]))
            S += (az[:, None, None] * ay[None, :, None] * ax[None, None, :]).real
        out[c] = (amplitude * S / np.abs(S).max()).astype(np.float32)
    return out


def grid_box(cfg):
    return tuple(b[0] for b in cfg["box"]), tuple(b[1] for b in cfg["box"])
