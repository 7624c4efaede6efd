"""The dependency cone the full-size GPU parity test relies on.

After T steps a node's fields depend only on nodes within 2 T + 1 of it, so
the oracle on a periodic window of half-width h >= 2 T + 1 + r + 1 around a
patch of radius r reproduces the patch of the full domain.  Checked here on
the oracle alone: a 200^2 four-roll mill (the benchmark's parameters) against
its 181^2 window, T = 40, agree to round-off on the 9 x 9 patch, while a
window far too narrow for the step count (half-width 30) does not -- the
check can fail.  (The bound is conservative: the disturbance at the very
edge of the cone is far below round-off, so a window a few rings too
narrow still agrees in practice.)"""
import numpy as np

from oracle_helpers import oracle_sim
from paper_2508_16997_gb300 import workloads as wl


def _window(inst, cx, cy, h):
    N = inst.nx
    xs = np.arange(cx - h, cx + h + 1) % N
    ys = np.arange(cy - h, cy + h + 1) % N
    F = inst.force_field[:, ys][:, :, xs]
    return wl.Instance(2 * h + 1, 2 * h + 1, True, inst.beta, inst.Wi, inst.Re, inst.Sc,
                       inst.Ma, inst.Lc, inst.Lambda_s, inst.Lambda_p, 0.0, 0.0, "window",
                       np.ascontiguousarray(F), inst.seed)


def _patch_error(T, h, r=4):
    inst = wl.frm(200, beta=0.3, Wi=20.0, Re=0.01, Ma=1e-3)
    cx, cy = 37, 151
    full = oracle_sim(inst)
    full.step(T)
    win = oracle_sim(_window(inst, cx, cy, h))
    win.step(T)
    xs = np.arange(cx - r, cx + r + 1) % 200
    ys = np.arange(cy - r, cy + r + 1) % 200
    a = full.fields()[:, ys][:, :, xs]
    b = win.fields()[:, h - r:h + r + 1, h - r:h + r + 1]
    return float(np.abs(a[1:3] - b[1:3]).max() / np.abs(a[1:3]).max())


def test_window_reproduces_patch():
    assert _patch_error(40, 90) <= 1e-12


def test_too_narrow_window_differs():
    assert _patch_error(40, 30) > 1e-6
