"""ctypes wrapper of the C oracle (test infrastructure only; see __init__)."""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

KINDS = {"plane": 0, "gauss": 1, "lg": 2, "flying": 3, "flying_cf": 4}
POLS = {"x": 0, "y": 1, "cp": 2, "cm": 3}
ENVS = {"sin2": 0, "gauss": 1, "sgauss": 2, "cw": 3}
MAX_COMP = 256


class _Pulse(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int), ("pol", ctypes.c_int), ("env", ctypes.c_int),
        ("sg_order", ctypes.c_int), ("lg_p", ctypes.c_int), ("lg_l", ctypes.c_int),
        ("n_comp", ctypes.c_int), ("longitudinal", ctypes.c_int), ("yee", ctypes.c_int),
        ("one_d", ctypes.c_int),
        ("a0", ctypes.c_double), ("omega", ctypes.c_double), ("w0", ctypes.c_double),
        ("z_focus", ctypes.c_double), ("t_focus", ctypes.c_double),
        ("env_len", ctypes.c_double), ("phase0", ctypes.c_double),
        ("beta_f", ctypes.c_double), ("bw_frac", ctypes.c_double),
        ("ff_length", ctypes.c_double), ("yee_dx", ctypes.c_double),
        ("yee_dt", ctypes.c_double), ("omega_p", ctypes.c_double),
    ]


_DA = ctypes.c_double * MAX_COMP


class _State(ctypes.Structure):
    _fields_ = [
        ("p", _Pulse),
        ("k", ctypes.c_double), ("vphi", ctypes.c_double), ("vg", ctypes.c_double),
        ("bratio", ctypes.c_double), ("zR", ctypes.c_double), ("amp", ctypes.c_double),
        ("n", ctypes.c_int),
        ("fw", _DA), ("fk", _DA), ("fz", _DA), ("ft", _DA), ("fphi", _DA), ("fzR", _DA),
        ("z_mid", ctypes.c_double), ("t_mid", ctypes.c_double),
        ("zeta", ctypes.c_double), ("jamp", ctypes.c_double), ("fdc", ctypes.c_double),
    ]


def build(force=False):
    """Compile oracle.c into liboracle.so with plain gcc (no fast-math, no FMA
    contraction).  Rebuilds when the source is newer than the library."""
    with _lock:
        newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
        if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= newest:
            return _SO
        tmp = _SO + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
        return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        dp = ctypes.POINTER(ctypes.c_double)
        fp = ctypes.POINTER(ctypes.c_float)
        L.or_prepare.argtypes = [ctypes.POINTER(_Pulse), ctypes.POINTER(_State)]
        L.or_prepare.restype = ctypes.c_int
        L.or_envelope.argtypes = [ctypes.POINTER(_State), ctypes.c_double]
        L.or_envelope.restype = ctypes.c_double
        L.or_profile.argtypes = [ctypes.POINTER(_State), ctypes.c_int] + [ctypes.c_double] * 4 + [dp, dp]
        L.or_profile.restype = None
        L.or_fields.argtypes = [ctypes.POINTER(_State)] + [ctypes.c_double] * 4 + [dp]
        L.or_fields.restype = None
        L.or_grid_sample.argtypes = [fp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_double, dp]
        L.or_grid_sample.restype = None
        L.or_boris.argtypes = [dp, dp, dp, ctypes.c_double]
        L.or_boris.restype = None
        L.or_push.argtypes = [ctypes.POINTER(_State), fp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                              dp, dp, ctypes.c_int64, dp, dp, dp, dp, dp, dp,
                              ctypes.c_double, ctypes.c_double, ctypes.c_int64, dp]
        L.or_push.restype = ctypes.c_int
        L.or_gamma_hist.argtypes = [ctypes.c_int64, dp, dp, dp, ctypes.c_int, ctypes.c_double,
                                    ctypes.c_double, ctypes.POINTER(ctypes.c_uint32)]
        L.or_gamma_hist.restype = None
        L.or_set_gamma_sums.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int64), dp, dp, dp, dp]
        L.or_set_gamma_sums.restype = None
        L.or_yee_nodes.argtypes = [ctypes.POINTER(_State), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   dp, dp, ctypes.c_double, dp]
        L.or_yee_nodes.restype = None
        L.or_yee1d.argtypes = [ctypes.c_int64, dp, dp, ctypes.c_double, ctypes.c_double, ctypes.c_int64]
        L.or_yee1d.restype = None
        L.or_envelope_logd.argtypes = [ctypes.POINTER(_State), ctypes.c_double, dp, dp]
        L.or_envelope_logd.restype = ctypes.c_int
        L.or_current.argtypes = [ctypes.POINTER(_State)] + [ctypes.c_double] * 4 + [dp]
        L.or_current.restype = None
        L.or_plasma1d.argtypes = [ctypes.c_int64, dp, dp, dp, dp, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_int64]
        L.or_plasma1d.restype = None
        L.or_apt1d.argtypes = [ctypes.POINTER(_State), ctypes.c_int64, dp, dp, dp, dp] + \
            [ctypes.c_double] * 4 + [ctypes.c_int64]
        L.or_apt1d.restype = ctypes.c_int
        _lib = L
    return _lib


def _pulse_struct(d):
    p = _Pulse()
    p.kind = KINDS[d.get("kind", "plane")]
    p.pol = POLS[d.get("pol", "x")]
    p.env = ENVS[d.get("env", "cw")]
    p.sg_order = int(d.get("sg_order", 1))
    p.lg_p = int(d.get("lg_p", 0))
    p.lg_l = int(d.get("lg_l", 0))
    p.n_comp = int(d.get("n_comp", 0))
    p.longitudinal = 1 if d.get("longitudinal", False) else 0
    p.yee = 1 if d.get("yee", False) else 0
    p.one_d = 1 if d.get("one_d", False) else 0
    for name in ("a0", "omega", "w0", "z_focus", "t_focus", "env_len", "phase0", "beta_f",
                 "bw_frac", "ff_length", "yee_dx", "yee_dt", "omega_p"):
        default = 1.0 if name == "omega" else 0.0
        setattr(p, name, float(d.get(name, default)))
    return p


def prepare(pulse):
    """Derive the oracle's constants for a pulse dict; returns the C state."""
    st = _State()
    rc = lib().or_prepare(ctypes.byref(_pulse_struct(pulse)), ctypes.byref(st))
    if rc != 0:
        raise ValueError("oracle: invalid pulse description %r" % (pulse,))
    return st


def state(pulse):
    """Derived constants as a dict (k, vphi, vg, bratio, zR, amp and, for the
    flying focus, the component table)."""
    st = prepare(pulse)
    out = {k: getattr(st, k) for k in ("k", "vphi", "vg", "bratio", "zR", "amp", "n", "z_mid", "t_mid",
                                       "zeta", "jamp", "fdc")}
    n = st.n
    for k in ("fw", "fk", "fz", "ft", "fphi", "fzR"):
        out[k] = np.array(getattr(st, k)[:n])
    return out


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def fields(pulse, x, y, z, t):
    """E1, B1 at points; returns array [6, n] (Ex, Ey, Ez, Bx, By, Bz)."""
    st = prepare(pulse)
    x, y, z, t = np.broadcast_arrays(*[np.asarray(v, dtype=np.float64) for v in (x, y, z, t)])
    shape = x.shape
    x, y, z, t = [np.ascontiguousarray(v).ravel() for v in (x, y, z, t)]
    out = np.empty((6, x.size))
    buf = np.empty(6)
    L = lib()
    for i in range(x.size):
        L.or_fields(ctypes.byref(st), x[i], y[i], z[i], t[i], _dp(buf))
        out[:, i] = buf
    return out.reshape((6,) + shape)


def current(pulse, x, y, z, t):
    """Analytic current J1 (Eq. j1) at points; returns [3, n] (Jx, Jy, Jz)."""
    st = prepare(pulse)
    x, y, z, t = np.broadcast_arrays(*[np.asarray(v, dtype=np.float64) for v in (x, y, z, t)])
    shape = x.shape
    x, y, z, t = [np.ascontiguousarray(v).ravel() for v in (x, y, z, t)]
    out = np.empty((3, x.size))
    buf = np.empty(3)
    L = lib()
    for i in range(x.size):
        L.or_current(ctypes.byref(st), x[i], y[i], z[i], t[i], _dp(buf))
        out[:, i] = buf
    return out.reshape((3,) + shape)


def envelope_logd(pulse, eta):
    """(Gamma'/Gamma, Gamma''/Gamma) at each eta."""
    st = prepare(pulse)
    eta = np.atleast_1d(np.asarray(eta, dtype=np.float64))
    l1, l2 = np.empty(eta.size), np.empty(eta.size)
    a, b = ctypes.c_double(), ctypes.c_double()
    for i, e in enumerate(eta):
        if lib().or_envelope_logd(ctypes.byref(st), float(e), ctypes.byref(a), ctypes.byref(b)) != 0:
            raise ValueError("oracle: envelope without logarithmic derivatives")
        l1[i], l2[i] = a.value, b.value
    return l1, l2


def profile(pulse, x, y, z, j=0, t=0.0):
    """Complex transverse profile u at one point (t: closed-form flying focus)."""
    st = prepare(pulse)
    re, im = ctypes.c_double(), ctypes.c_double()
    lib().or_profile(ctypes.byref(st), j, x, y, z, t, ctypes.byref(re), ctypes.byref(im))
    return complex(re.value, im.value)


def envelope(pulse, eta):
    st = prepare(pulse)
    return np.array([lib().or_envelope(ctypes.byref(st), float(e)) for e in np.atleast_1d(eta)])


def grid_sample(grid, lo, hi, x, y, z):
    """Trilinear gather of a [6, nz, ny, nx] float32 grid at one point."""
    g = np.ascontiguousarray(grid, dtype=np.float32)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    out = np.empty(6)
    lib().or_grid_sample(g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), g.shape[3], g.shape[2],
                         g.shape[1], _dp(lo), _dp(hi), x, y, z, _dp(out))
    return out


def boris(u, E, B, dt):
    u = np.array(u, dtype=np.float64)
    E = np.asarray(E, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    lib().or_boris(_dp(u), _dp(E), _dp(B), dt)
    return u


def push(pulse, particles, t0, dt, n_steps, grid=None, lf=False, threads=1):
    """Push copies of the particle arrays (dict with x, y, z, ux, uy, uz).
    grid: None or (array [6, nz, ny, nx] float32, lo, hi).  Returns the new
    arrays as a dict (and the per-step light-front deviation if lf).
    threads > 1 runs contiguous chunks of particles concurrently (the C call
    releases the GIL); each particle is still pushed by the same plain loop."""
    if threads > 1 and np.asarray(particles["x"]).size > 1:
        import concurrent.futures
        n = np.asarray(particles["x"]).size
        bounds = np.linspace(0, n, min(threads, n) + 1).astype(int)
        chunks = [{k: np.asarray(particles[k])[a:b] for k in ("x", "y", "z", "ux", "uy", "uz")}
                  for a, b in zip(bounds[:-1], bounds[1:])]
        with concurrent.futures.ThreadPoolExecutor(max_workers=len(chunks)) as ex:
            res = list(ex.map(lambda c: push(pulse, c, t0, dt, n_steps, grid=grid, lf=lf), chunks))
        if lf:
            out = {k: np.concatenate([r[0][k] for r in res]) for k in res[0][0]}
            return out, np.max(np.stack([r[1] for r in res]), axis=0)
        return {k: np.concatenate([r[k] for r in res]) for k in res[0]}
    st = prepare(pulse)
    out = {k: np.array(particles[k], dtype=np.float64, copy=True) for k in ("x", "y", "z", "ux", "uy", "uz")}
    n = out["x"].size
    lf_buf = np.zeros(int(n_steps)) if lf else None
    if grid is not None:
        g, lo, hi = grid
        g = np.ascontiguousarray(g, dtype=np.float32)
        lo = np.asarray(lo, dtype=np.float64)
        hi = np.asarray(hi, dtype=np.float64)
        gp = g.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        nx, ny, nz = g.shape[3], g.shape[2], g.shape[1]
        lop, hip = _dp(lo), _dp(hi)
    else:
        gp, nx, ny, nz, lop, hip = None, 0, 0, 0, None, None
    lib().or_push(ctypes.byref(st), gp, nx, ny, nz, lop, hip, n, _dp(out["x"]), _dp(out["y"]),
                  _dp(out["z"]), _dp(out["ux"]), _dp(out["uy"]), _dp(out["uz"]), float(t0), float(dt),
                  int(n_steps), _dp(lf_buf) if lf else None)
    if lf:
        return out, lf_buf
    return out


def gamma_hist(ux, uy, uz, bins, lo, hi):
    ux, uy, uz = [np.ascontiguousarray(a, dtype=np.float64) for a in (ux, uy, uz)]
    counts = np.zeros(bins, dtype=np.uint32)
    lib().or_gamma_hist(ux.size, _dp(ux), _dp(uy), _dp(uz), bins, lo, hi,
                        counts.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    return counts


def set_gamma_sums(offsets, ux, uy, uz):
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    ux, uy, uz = [np.ascontiguousarray(a, dtype=np.float64) for a in (ux, uy, uz)]
    sums = np.zeros(off.size - 1)
    lib().or_set_gamma_sums(off.size - 1, off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                            _dp(ux), _dp(uy), _dp(uz), _dp(sums))
    return sums


def mean_gamma(pulse, particles, t0, dt, n_steps, grid=None):
    """Objective of the adjoint: mean final gamma of the particles."""
    out = push(pulse, particles, t0, dt, n_steps, grid=grid)
    off = np.array([0, out["x"].size], dtype=np.int64)
    return set_gamma_sums(off, out["ux"], out["uy"], out["uz"])[0] / out["x"].size


def grad_fd(pulse, particles, t0, dt, n_steps, names=("a0", "w0", "z_focus"), rel_h=1e-4,
            grid=None, scale=None):
    """Gradient of the mean final gamma with respect to pulse parameters by
    FP64 central differences with Richardson extrapolation:
      D(h) = (J(p + h) - J(p - h)) / (2h),  grad = (4 D(h/2) - D(h)) / 3,
    h = rel_h * scale[name] (default |p|, or 1 for a zero parameter)."""
    g = {}
    for name in names:
        p0 = float(pulse[name])
        sc = (scale or {}).get(name, abs(p0) if p0 != 0.0 else 1.0)
        h = rel_h * sc

        def J(v):
            q = dict(pulse)
            q[name] = v
            return mean_gamma(q, particles, t0, dt, n_steps, grid=grid)

        d1 = (J(p0 + h) - J(p0 - h)) / (2 * h)
        d2 = (J(p0 + h / 2) - J(p0 - h / 2)) / h
        g[name] = (4 * d2 - d1) / 3
    return g


def yee_nodes(pulse, shape, lo, d, t):
    """Analytic E1, B1 at the Yee-staggered nodes of a grid of shape
    (nz, ny, nx), node (i, j, k) at lo + (i, j, k) * d; returns [6, nz, ny, nx]
    (Ex, Ey, Ez, Bx, By, Bz), each at its own offset inside the cell."""
    st = prepare(pulse)
    nz, ny, nx = (int(v) for v in shape)
    lo = np.asarray(lo, dtype=np.float64)
    d = np.asarray(d, dtype=np.float64)
    out = np.empty((6, nz, ny, nx))
    lib().or_yee_nodes(ctypes.byref(st), nx, ny, nz, _dp(lo), _dp(d), float(t), _dp(out))
    return out


def yee1d(E, B, dz, dt, n_steps):
    """n_steps of the 1-D vacuum Yee scheme on copies of E (E_x at z_k) and B
    (B_y at z_{k+1/2}); returns the new (E, B)."""
    E = np.array(E, dtype=np.float64)
    B = np.array(B, dtype=np.float64)
    if E.shape != B.shape or E.ndim != 1:
        raise ValueError("E and B must be 1-D arrays of one length")
    lib().or_yee1d(E.size, _dp(E), _dp(B), float(dz), float(dt), int(n_steps))
    return E, B


def _line_arrays(E, B, J, wp2):
    E = np.array(E, dtype=np.float64)
    B = np.array(B, dtype=np.float64)
    J = np.array(J, dtype=np.float64)
    wp2 = np.ascontiguousarray(np.broadcast_to(np.asarray(wp2, dtype=np.float64), E.shape))
    if E.ndim != 1 or B.shape != E.shape or J.shape != E.shape:
        raise ValueError("E, B and J must be 1-D arrays of one length")
    return E, B, J, wp2


def plasma1d(E, B, J, wp2, dz, dt, n_steps):
    """n_steps of the 1-D Yee line with a linear cold-plasma current (E_x at
    z_k, B_y at z_{k+1/2}, J_x at z_k; wp2 = omega_p^2 per node or scalar);
    returns the new (E, B, J)."""
    E, B, J, wp2 = _line_arrays(E, B, J, wp2)
    lib().or_plasma1d(E.size, _dp(E), _dp(B), _dp(J), _dp(wp2), float(dz), float(dt), int(n_steps))
    return E, B, J


def apt1d(pulse, E2, B2, J, wp2, z0, dz, t0, dt, n_steps):
    """n_steps of the line in the split form of Sec. 4 with the pulse's
    analytic E1 and current J1; returns the new (E2, B2, J)."""
    st = prepare(pulse)
    E, B, J, wp2 = _line_arrays(E2, B2, J, wp2)
    rc = lib().or_apt1d(ctypes.byref(st), E.size, _dp(E), _dp(B), _dp(J), _dp(wp2), float(z0),
                        float(dz), float(t0), float(dt), int(n_steps))
    if rc != 0:
        raise ValueError("oracle: the line carries E_x: the pulse must be polarised along x")
    return E, B, J
