"""Plain FP64 CPU oracle for the analytic-pulse push (arXiv:2307.04843).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it; the product package never imports it.
The C core (``oracle.c``) is built with plain gcc, no fast-math, no FMA
contraction (``build()``), and wrapped with ctypes here.  Pulses are plain
dicts of physical parameters (the same dicts the product binding takes); this
module maps them onto the oracle's own structure.

Functions: ``fields``, ``push``, ``boris``, ``grid_sample``, ``gamma_hist``,
``set_gamma_sums``, ``profile``, ``envelope``, ``state``,
``grad_fd`` (FP64 central finite differences with Richardson extrapolation of
the per-set mean final gamma), ``yee_nodes`` (E1, B1 at Yee-staggered grid
nodes), ``yee1d`` (the 1-D vacuum Yee scheme of Sec. 2.1), and for Sec. 4
``current`` (the analytic current J1), ``envelope_logd``, ``plasma1d`` (the
line with a linear cold-plasma current) and ``apt1d`` (the same line in the
split form with E1 and J1 analytic).
"""
from .core import (  # noqa: F401
    build,
    lib,
    prepare,
    state,
    fields,
    profile,
    envelope,
    grid_sample,
    boris,
    push,
    gamma_hist,
    set_gamma_sums,
    mean_gamma,
    grad_fd,
    yee_nodes,
    yee1d,
    current,
    envelope_logd,
    plasma1d,
    apt1d,
)
