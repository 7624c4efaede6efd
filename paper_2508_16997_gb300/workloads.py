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
* solid obstacles (Sec. 4.3 geometry): a solid mask and, for curved walls,
  the fraction q of each wall link at which the wall lies; a cylinder in a
  periodic channel, a rectangular block in a periodic box, and a channel
  bounded by a solid row at a chosen wall distance.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict

import numpy as np

CS = 1.0 / math.sqrt(3.0)  # lattice speed of sound for c = 1 (D2Q9)

# D2Q9 directions in the order both implementations use; the geometry below
# needs them to name wall links (link (k, i): fluid node k, solid k - e_i).
EX = (0, 1, 0, -1, 0, 1, -1, -1, 1)
EY = (0, 0, 1, 0, -1, 1, 1, -1, -1)


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
    solid: np.ndarray | None = field(default=None, repr=False)   # (ny, nx) uint8, 1 = solid
    wall_q: np.ndarray | None = field(default=None, repr=False)  # (9, ny, nx) link fractions
    open_x: bool = False     # inlet column x = 0, outlet column x = nx - 1
    model: int = 0           # 0 Oldroyd-B, 1 FENE-P, 2 FENE-CR
    L2: float = 0.0          # FENE extensibility L^2 (models 1, 2)
    gtilde: int = 0          # G~_i: 0 eq_p_G_1, 1 eq_p_G (density gradient)
    inlet: np.ndarray | None = field(default=None, repr=False)   # (5, ny) ux, uy, Axx, Axy, Ayy

    @property
    def n_nodes(self) -> int:
        return self.nx * self.ny

    def scalars(self) -> dict:
        d = asdict(self)
        for k in ("force_field", "solid", "wall_q", "inlet"):
            d.pop(k)
        return d

    def wall_links(self):
        """Wall links of the mask as (node k, direction i, q): fluid node k
        whose neighbour k - e_i is solid, q from ``wall_q`` (1/2 if None)."""
        if self.solid is None:
            return []
        out = []
        nx, ny = self.nx, self.ny
        for y in range(ny):
            for x in range(nx):
                if self.solid[y, x]:
                    continue
                for i in range(1, 9):
                    ys = y - EY[i]
                    if self.periodic_y:
                        ys %= ny
                    elif not 0 <= ys < ny:
                        continue
                    if self.solid[ys, (x - EX[i]) % nx]:
                        q = 0.5 if self.wall_q is None else float(self.wall_q[i, y, x])
                        out.append((y * nx + x, i, q))
        return out


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


def _circle_links(solid: np.ndarray, cx: float, cy: float, R: float, periodic_y: bool):
    """Link fractions q (9, ny, nx) for a circle of radius R centred at
    (cx, cy): for fluid node x_b and solid neighbour x_b - e_i, the first
    crossing x_b + t (x_s - x_b) of the circle, t in (0, 1]."""
    ny, nx = solid.shape
    q = np.full((9, ny, nx), 0.5)
    for y in range(ny):
        for x in range(nx):
            if solid[y, x]:
                continue
            for i in range(1, 9):
                ys, xs = y - EY[i], (x - EX[i]) % nx
                if periodic_y:
                    ys %= ny
                elif not 0 <= ys < ny:
                    continue
                if not solid[ys, xs]:
                    continue
                px, py = x - cx, y - cy
                dx, dy = -EX[i], -EY[i]
                a = dx * dx + dy * dy
                b = px * dx + py * dy
                c = px * px + py * py - R * R
                t = (-b - math.sqrt(max(b * b - a * c, 0.0))) / a
                q[i, y, x] = min(max(t, 1e-6), 1.0)
    return q


def poiseuille_inlet(H: int, Umax: float, lam: float) -> np.ndarray:
    """Fully developed Oldroyd-B channel profile on rows y = 0..H (walls at 0
    and H): u_x = 4 Umax y (H - y) / H^2, u_y = 0, A_xy = lam du/dy,
    A_xx = 1 + 2 (lam du/dy)^2, A_yy = 1 (Sec. 4.2 closed form, used as the
    inlet profile of Sec. 4.3).  Returns (5, H + 1)."""
    y = np.arange(H + 1, dtype=float)
    u = 4.0 * Umax * y * (H - y) / H ** 2
    du = 4.0 * Umax * (H - 2.0 * y) / H ** 2
    out = np.zeros((5, H + 1))
    out[0] = u
    out[2] = 1.0 + 2.0 * (lam * du) ** 2
    out[3] = lam * du
    out[4] = 1.0
    return out


def cylinder_channel(R: int, L: int | None = None, H: int | None = None, beta=0.59, Wi=0.5,
                     Re=1.0, Sc=1e6, Ma=0.01, Lambda_s=0.25, Lambda_p=2.5e-7,
                     curved: bool = True, open_x: bool = False, seed: int = 0) -> Instance:
    """Cylinder of radius R in a channel (Sec. 4.3 geometry): L x (H + 1)
    nodes, wet-node walls on rows 0 and H, cylinder centred at (L/2, H/2),
    solid where (x - cx)^2 + (y - cy)^2 <= R^2, L_c = R, U_max = 1.5 U_c.
    open_x: the paper's set-up -- inlet column x = 0 with the fully
    developed profile (poiseuille_inlet, lambda = Wi R / U_c), zero-gradient
    outlet x = L - 1, no body force.  Otherwise periodic in x and driven by
    the uniform force F_x = 8 nu_0 U_max / H^2 of that profile.  curved:
    exact link fractions of the circle, else staircase (q = 1/2)."""
    L = 30 * R if L is None else L
    H = 4 * R if H is None else H
    ny = H + 1
    cx, cy = 0.5 * L, 0.5 * H
    Y, X = np.mgrid[0:ny, 0:L]
    solid = (((X - cx) ** 2 + (Y - cy) ** 2) <= R * R).astype(np.uint8)
    Lc = float(R)
    nu0 = total_viscosity(Ma, Lc, Re)
    Uc = velocity_scale(Ma)
    Fx = 0.0 if open_x else 8.0 * nu0 * 1.5 * Uc / float(H) ** 2
    inst = Instance(L, ny, False, beta, Wi, Re, Sc, Ma, Lc, Lambda_s, Lambda_p, Fx, 0.0,
                    "cylinder", None, seed)
    inst.solid = solid
    inst.wall_q = _circle_links(solid, cx, cy, R, False) if curved else None
    if open_x:
        inst.open_x = True
        inst.inlet = poiseuille_inlet(H, 1.5 * Uc, Wi * Lc / Uc)
    return inst


def obstacle_box(nx: int, ny: int, block=(0.25, 0.5, 0.375, 0.625), Fx=1e-5, Fy=0.0,
                 beta=0.5, Wi=1.0, Re=1.0, Sc=1e4, Ma=0.1, Lambda_s=0.25, Lambda_p=1e-6,
                 seed: int = 0) -> Instance:
    """Doubly periodic nx x ny box with a solid rectangle covering the
    fractions block = (x0, x1, y0, y1) of the box, uniform force (Fx, Fy),
    L_c = ny (half-way walls, q = 1/2)."""
    x0, x1 = int(round(block[0] * nx)), int(round(block[1] * nx))
    y0, y1 = int(round(block[2] * ny)), int(round(block[3] * ny))
    solid = np.zeros((ny, nx), np.uint8)
    solid[y0:y1, x0:x1] = 1
    inst = Instance(nx, ny, True, beta, Wi, Re, Sc, Ma, float(ny), Lambda_s, Lambda_p, Fx, Fy,
                    "obstacle", None, seed)
    inst.solid = solid
    return inst


def staircase_channel(H: int, q: float = 0.5, nx: int = 3, beta=1.0, Wi=1.0, Re=1.0,
                      Sc=1e6, Ma=0.1, Lambda_s=0.25, Lambda_p=2.5e-7) -> Instance:
    """Channel bounded by one solid row: doubly periodic nx x (H + 1) grid,
    row 0 solid, fluid rows 1..H; every wall link crosses the wall at
    fraction q, so the walls lie at y = 1 - q and y = H + q and the channel
    width is W = H - 1 + 2q (= L_c).  Uniform force F_x = 8 nu_0 U_c / W^2."""
    ny = H + 1
    solid = np.zeros((ny, nx), np.uint8)
    solid[0, :] = 1
    W = H - 1 + 2.0 * q
    nu0 = total_viscosity(Ma, W, Re)
    Fx = 8.0 * nu0 * velocity_scale(Ma) / W ** 2
    inst = Instance(nx, ny, True, beta, Wi, Re, Sc, Ma, W, Lambda_s, Lambda_p, Fx, 0.0,
                    "staircase", None, 0)
    inst.solid = solid
    inst.wall_q = np.full((9, ny, nx), float(q))
    return inst


def circle_box(nx: int, ny: int, R: float, cx: float, cy: float, Fx=1e-5, Fy=0.0, beta=0.5,
               Wi=1.0, Re=1.0, Sc=1e4, Ma=0.1, Lambda_s=0.25, Lambda_p=1e-6,
               curved: bool = True) -> Instance:
    """Doubly periodic nx x ny box with a solid disc of radius R centred at
    (cx, cy), uniform force (Fx, Fy), L_c = 2R; curved: exact link
    fractions of the circle, else q = 1/2."""
    Y, X = np.mgrid[0:ny, 0:nx]
    solid = (((X - cx) ** 2 + (Y - cy) ** 2) <= R * R).astype(np.uint8)
    inst = Instance(nx, ny, True, beta, Wi, Re, Sc, Ma, 2.0 * R, Lambda_s, Lambda_p, Fx, Fy,
                    "obstacle", None, 0)
    inst.solid = solid
    inst.wall_q = _circle_links(solid, cx, cy, R, True) if curved else None
    return inst
