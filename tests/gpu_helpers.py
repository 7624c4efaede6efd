"""Helpers for the GPU parity tests: relative L2 distances of the CUDA path's
fields from the oracle's on the same seeded inputs."""
from __future__ import annotations

import numpy as np


def rel_l2(a: np.ndarray, b: np.ndarray) -> float:
    """||a - b||_2 / ||b||_2 (absolute when ||b|| = 0)."""
    den = float(np.linalg.norm(b))
    num = float(np.linalg.norm(a - b))
    return num / den if den > 0 else num


def parity_errors(gpu: np.ndarray, ref: np.ndarray) -> dict:
    """Relative L2 errors on u = (ux, uy), on C = (Axx, Axy, Ayy), on the
    polymer deformation C - I, and on rho - 1."""
    I = np.zeros_like(ref[3:6])
    I[0] = 1.0
    I[2] = 1.0
    return {
        "u": rel_l2(gpu[1:3], ref[1:3]),
        "C": rel_l2(gpu[3:6], ref[3:6]),
        "C-I": rel_l2(gpu[3:6] - I, ref[3:6] - I),
        "rho-1": rel_l2(gpu[0] - 1.0, ref[0] - 1.0),
    }
