"""Closed-form solutions used to pin the FP64 oracle.

Each function states the mathematics it evaluates and where it comes from.
Nothing here calls the oracle or the CUDA library.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.linalg import expm

CS2 = 1.0 / 3.0
# D2Q9 velocities and weights, retyped from the paper's definition (Sec. 3.1)
E = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]],
             dtype=float)
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def hermite(i: int):
    """Hermite tensors H1 (2,), H2 (2,2), H3 (2,2,2) of direction i."""
    e = E[i]
    d = np.eye(2)
    H1 = e.copy()
    H2 = np.outer(e, e) - CS2 * d
    H3 = (np.einsum("a,b,c->abc", e, e, e)
          - CS2 * (np.einsum("a,bc->abc", e, d) + np.einsum("b,ac->abc", e, d)
                   + np.einsum("c,ab->abc", e, d)))
    return H1, H2, H3


def poiseuille_steady(H: int, Wi: float, Uc: float):
    """Steady Oldroyd-B plane Poiseuille flow (Sec. 4.2, eq_ux_ana, eq_Tab_ana).

    With y* = y/H, u* = 4 y*(1-y*); the stresses tau*_xx = 2 Wi (1-beta) u*'^2,
    tau*_xy = (1-beta) u*' and tau*_yy = 0 become, through the Kramers
    relation tau = (mu_p/lambda)(A - I) (eq_kramer, eqb4) with lambda = Wi H/U_c,
        A_xy = Wi u*',  A_xx = 1 + 2 (Wi u*')^2,  A_yy = 1.
    Returns (ux, Axx, Axy, Ayy) on rows y = 0..H."""
    ys = np.arange(H + 1) / H
    u = 4.0 * ys * (1.0 - ys)
    du = 4.0 - 8.0 * ys
    return Uc * u, 1.0 + 2.0 * (Wi * du) ** 2, Wi * du, np.ones_like(ys)


def waters_king_u(ystar: float, tstar, Wi: float, Re: float, beta: float,
                  n_terms: int = 400):
    """Start-up Oldroyd-B Poiseuille velocity u*(y*, t*) (Sec. 4.2, Waters-King).

    u* = 4y*(1-y*) - 32 sum_n sin(N y*)/N^3 G_N(E, t*),  N = (2n-1) pi, E = Wi/Re,
    G_N = exp(-a t*/(2Wi)) [cosh(b t*/(2Wi)) + (g/b) sinh(b t*/(2Wi))],
    a = 1 + beta E N^2, b^2 = a^2 - 4 N^2 E, g = 1 + (beta - 2) E N^2,
    with cos/sin in place of cosh/sinh when b^2 < 0.  (Checked independently:
    it solves Re u_t = 8 + beta u_yy + s_y, Wi s_t + s = (1-beta) u_y from rest.)"""
    t = np.asarray(tstar, dtype=float)
    E_ = Wi / Re
    u = 4.0 * ystar * (1.0 - ystar) * np.ones_like(t)
    for n in range(1, n_terms + 1):
        N = (2 * n - 1) * math.pi
        a = 1.0 + beta * E_ * N * N
        b2 = a * a - 4.0 * N * N * E_
        g = 1.0 + (beta - 2.0) * E_ * N * N
        b = math.sqrt(abs(b2))
        x = b * t / (2.0 * Wi)
        decay = np.exp(-a * t / (2.0 * Wi))
        if b2 >= 0:
            # cosh + (g/b) sinh, written with exponentials that cannot overflow
            # (b < a, so the growth is dominated by the decay)
            G = 0.5 * (np.exp(-(a - b) * t / (2 * Wi)) * (1 + g / b)
                       + np.exp(-(a + b) * t / (2 * Wi)) * (1 - g / b))
        else:
            G = decay * (np.cos(x) + (g / b) * np.sin(x))
        u = u - 32.0 * math.sin(N * ystar) / N ** 3 * G
    return u


def frm_newtonian(N: int, Uc: float):
    """Newtonian steady four-roll-mill velocity (eq-steady):
    u = U_c (sin x~ cos y~, -cos x~ sin y~), x~ = 2 pi x / N.  Arrays [y][x]."""
    xt = 2 * math.pi * np.arange(N) / N
    X, Y = np.meshgrid(xt, xt, indexing="xy")
    return Uc * np.sin(X) * np.cos(Y), -Uc * np.cos(X) * np.sin(Y)


def oldroyd_b_point_ode(A0, grad, lam, t):
    """Conformation at a point where u = 0, with a frozen velocity gradient.

    From the constitutive equation (eq_Constitutive with eqb4, kappa = 0, u = 0
    at the point): dA/dt = A L + L^T A + (tr L) A - (A - I)/lambda, where
    L[g][b] = d_g u_b, i.e. dA_ab/dt = A_ag d_g u_b + A_gb d_g u_a + A_ab d_g u_g
    - (A_ab - d_ab)/lambda.  Linear in vec(A) = (Axx, Axy, Ayy); solved exactly
    with a matrix exponential.  Returns an array (len(t), 3)."""
    L = np.asarray(grad, float).reshape(2, 2)
    idx = [(0, 0), (0, 1), (1, 1)]
    M = np.zeros((3, 3))
    c = np.zeros(3)

    def comp(a, b):
        return idx.index((min(a, b), max(a, b)))

    for r, (a, b) in enumerate(idx):
        c[r] = (1.0 if a == b else 0.0) / lam
        M[r, r] += -1.0 / lam + (L[0, 0] + L[1, 1])
        for g in range(2):
            M[r, comp(a, g)] += L[g, b]
            M[r, comp(g, b)] += L[g, a]
    Xinf = -np.linalg.solve(M, c)
    X0 = np.asarray(A0, float)
    return np.array([Xinf + expm(M * tt) @ (X0 - Xinf) for tt in np.atleast_1d(t)])
