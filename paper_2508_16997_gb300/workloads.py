"""Seeded synthetic inputs shaped like the paper's benchmark workloads.

This module is shared by the tests (oracle and CUDA sides alike) and by the
benchmark.  It holds only the *workload definitions* -- grid sizes, the
dimensionless groups, the body-force fields the paper prescribes and seeded
random perturbations -- and none of the lattice Boltzmann arithmetic.  It
imports nothing else from this package.

Workloads (Sec. 4 of the paper; sizes as used by this project):

* four-roll mill (Sec. 4.1): N x N doubly periodic grid, x~ = 2 pi x / N,
  body force F = F0 (sin x~ cos y~, -cos x~ sin y~) (eq. eq-force) with
  F0 = 2 nu U_c (2 pi / N)^2; the paper writes the solvent viscosity mu_s,
  the four-roll-mill workload of this project uses the total viscosity nu_0
  (``force_visc="nu0"``) unless asked otherwise.
* Poiseuille channel (Sec. 4.2): periodic in x, wet-node walls on rows
  y = 0 and y = H (ny = H + 1), L_c = H, uniform force
  F_x = 8 (nu_s + nu_p) U_c / L_c^2.
* batched mix: instances of both kinds with seeded random sizes, Wi and beta.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict

import numpy as np

CS = 1.0 / math.sqrt(3.0)  # lattice speed of sound for c = 1 (D2Q9)


@dataclass
class Instance:
    """One simulation's problem statement (grid, groups, force)."""
    nx: int
    ny: int
    periodic_y: bool
    beta: float
    Wi: float
    Re: float
    Sc: float
    Ma: float
    Lc: float
    Lambda_s: float = 0.25
    Lambda_p: float = 1e-6
    Fx: float = 0.0          # uniform force (channel)
    Fy: float = 0.0
    kind: str = "custom"     # "frm" | "channel" | "custom"
    force_field: np.ndarray | None = field(default=None, repr=False)  # (2, ny, nx) or None
    seed: int = 0

    @property
    def n_nodes(self) -> int:
        return self.nx * self.ny

    def scalars(self) -> dict:
        d = asdict(self)
        d.pop("force_field")
        return d


def velocity_scale(Ma: float) -> float:
    """U_c from the Mach number (eq_Mach)."""
    return Ma * CS


def total_viscosity(Ma: float, Lc: float, Re: float) -> float:
    """nu_0 = U_c L_c / Re (eqb5 with rho = 1)."""
    return velocity_scale(Ma) * Lc / Re


def frm(N: int, beta=0.5, Wi=5.0, Re=0.01, Sc=1e5, Ma=1e-3, Lambda_s=0.25, Lambda_p=1e-6,
        force_visc: str = "nu0", seed: int = 0) -> Instance:
    """Simplified four-roll mill on an N x N periodic grid (Sec. 4.1)."""
    Lc = N / (2.0 * math.pi)
    Uc = velocity_scale(Ma)
    nu0 = total_viscosity(Ma, Lc, Re)
    nu = nu0 if force_visc == "nu0" else beta * nu0
    F0 = 2.0 * nu * Uc * (2.0 * math.pi / N) ** 2
    xt = 2.0 * math.pi * np.arange(N) / N
    X, Y = np.meshgrid(xt, xt, indexing="xy")  # X[y, x] = x~, Y[y, x] = y~
    F = np.empty((2, N, N))
    F[0] = F0 * np.sin(X) * np.cos(Y)
    F[1] = -F0 * np.cos(X) * np.sin(Y)
    return Instance(N, N, True, beta, Wi, Re, Sc, Ma, Lc, Lambda_s, Lambda_p, 0.0, 0.0, "frm",
                    F, seed)


def channel(H: int, nx: int = 4, beta=0.5, Wi=1.0, Re=1.0, Sc=1e6, Ma=0.1, Lambda_s=0.25,
            Lambda_p=2.5e-7, seed: int = 0) -> Instance:
    """Body-force-driven Poiseuille channel, walls on rows 0 and H (Sec. 4.2)."""
    Lc = float(H)
    nu0 = total_viscosity(Ma, Lc, Re)
    Fx = 8.0 * nu0 * velocity_scale(Ma) / Lc ** 2
    return Instance(nx, H + 1, False, beta, Wi, Re, Sc, Ma, Lc, Lambda_s, Lambda_p, Fx, 0.0,
                    "channel", None, seed)


def batch_mix(n: int = 256, base_seed: int = 20250823, frac_channel: float = 0.5,
              H_range=(32, 512), N_range=(64, 512), Wi_log10=(0.0, 4.0),
              beta_range=(0.1, 0.9)) -> list[Instance]:
    """Seeded mix of channel and four-roll-mill instances of uneven sizes.

    Instance i draws from ``np.random.default_rng(base_seed + i)``:
    channel height H ~ U{H_range}, square four-roll-mill side N ~ U{N_range},
    Wi = 10^U(Wi_log10), beta ~ U(beta_range).  The first ``frac_channel * n``
    instances are channels, the rest four-roll mills."""
    out = []
    n_ch = int(round(frac_channel * n))
    for i in range(n):
        rng = np.random.default_rng(base_seed + i)
        Wi = float(10.0 ** rng.uniform(*Wi_log10))
        beta = float(rng.uniform(*beta_range))
        if i < n_ch:
            H = int(rng.integers(H_range[0], H_range[1] + 1))
            out.append(channel(H, beta=beta, Wi=Wi, seed=base_seed + i))
        else:
            N = int(rng.integers(N_range[0], N_range[1] + 1))
            out.append(frm(N, beta=beta, Wi=Wi, seed=base_seed + i))
    return out


def random_fields(nx: int, ny: int, seed: int, du: float = 1e-2, drho: float = 1e-3,
                  dA: float = 0.1) -> np.ndarray:
    """Smooth-free random initial fields (6, ny, nx): rho, ux, uy, Axx, Axy, Ayy.

    A = I + M M^T-type perturbation so that it stays symmetric positive
    definite: Axx = 1 + a^2 + b^2, Axy = a c, Ayy = 1 + c^2 with a, b, c
    uniform in [-sqrt(dA), sqrt(dA)]."""
    rng = np.random.default_rng(seed)
    out = np.empty((6, ny, nx))
    out[0] = 1.0 + drho * rng.uniform(-1, 1, (ny, nx))
    out[1] = du * rng.uniform(-1, 1, (ny, nx))
    out[2] = du * rng.uniform(-1, 1, (ny, nx))
    s = math.sqrt(dA)
    a, b, c = (s * rng.uniform(-1, 1, (ny, nx)) for _ in range(3))
    out[3] = 1.0 + a * a + b * b
    out[4] = a * c
    out[5] = 1.0 + c * c
    return out


def random_force(nx: int, ny: int, seed: int, amp: float = 1e-5) -> np.ndarray:
    """Random per-node body force (2, ny, nx), uniform in [-amp, amp]."""
    rng = np.random.default_rng(seed)
    return amp * rng.uniform(-1, 1, (2, ny, nx))
