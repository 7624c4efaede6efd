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


def poiseuille_steady_diffusive(H: int, Wi: float, Uc: float, beta: float, kappa: float,
                                y=None):
    """Steady Oldroyd-B plane Poiseuille flow WITH the stress diffusion of the
    conformation equation (eq_Constitutive with kappa > 0, Sec. 2) and
    zero-flux walls (the conservation CNEBB enforces, Sec. 3.3).

    The kappa = 0 profile of poiseuille_steady() cannot meet a zero-flux wall
    (its A_xy = lambda u' has a non-zero wall gradient), so a boundary layer
    of width delta = sqrt(kappa beta lambda) forms.  With x-invariance,
    A_yy = 1 exactly, and with eta = H/2 - y, F/mu_0 = 8 U_c/H^2 (the
    channel force of Sec. 4.2), lambda = Wi H/U_c, r = (1-beta)/beta:
      momentum:  mu_s u' + (mu_p/lambda) a = F eta            (a = A_xy)
      A_xy:      kappa a'' - a/lambda + u' = 0,   a' = 0 at the walls
      A_xx - 1:  kappa b'' - b/lambda + 2 a u' = 0, b' = 0 at the walls
    Eliminating u' gives kappa a'' - a/(beta lambda) = -F eta/mu_s, so
      a   = lambda (F/mu_0) [eta - delta sinh(eta/delta)/cosh(H/2delta)],
      u'  = (F/mu_0) [eta + r delta sinh(eta/delta)/cosh(H/2delta)],
      u   = (F/mu_0) [y (H - y)/2 + r delta^2 (cosh(H/2delta) - cosh(eta/delta))/cosh(H/2delta)],
    and b solves l^2 b'' - b = -2 lambda^2 (F/mu_0)^2 [eta^2 + (r-1) delta eta s/c - r delta^2 s^2/c^2]
    (s = sinh(eta/delta), c = cosh(H/2delta), l^2 = kappa lambda) with
    b'(+-H/2) = 0: a particular solution term by term (eta^2, eta s and
    cosh(eta/delta), cosh(2 eta/delta), a constant) plus D cosh(eta/l).
    Needs 0 < beta < 1 and kappa > 0.  As kappa -> 0 it reduces to
    poiseuille_steady().  Returns (ux, Axx, Axy, Ayy) on rows y (default
    0..H)."""
    ys = np.arange(H + 1, dtype=float) if y is None else np.asarray(y, dtype=float)
    eta = H / 2.0 - ys
    lam = Wi * H / Uc
    Fm = 8.0 * Uc / H ** 2
    r = (1.0 - beta) / beta
    d = math.sqrt(kappa * beta * lam)
    l2 = kappa * lam
    l = math.sqrt(l2)
    E = H / 2.0
    # ratios of hyperbolic functions written so that they cannot overflow
    def sc(x):   # sinh(x/d) / cosh(E/d)
        return 0.5 * (np.exp((x - E) / d) - np.exp((-x - E) / d)) / (0.5 * (1 + math.exp(-2 * E / d)))

    def cc(x):   # cosh(x/d) / cosh(E/d)
        return 0.5 * (np.exp((x - E) / d) + np.exp((-x - E) / d)) / (0.5 * (1 + math.exp(-2 * E / d)))

    a = lam * Fm * (eta - d * sc(eta))
    u = Fm * (ys * (H - ys) / 2.0 + r * d * d * (1.0 - cc(eta)))
    K = 2.0 * lam ** 2 * Fm ** 2
    # particular solution of l^2 b'' - b = -K [eta^2 + (r-1) d eta s/c - r d^2 s^2/c^2]
    # in terms of the bounded ratios sc, cc and cc2(x) = cosh(2x/d)/cosh(E/d)^2
    P = -K * (r - 1.0) * d * beta / (1.0 - beta)
    Q = -2.0 * P * d / (1.0 - beta)
    M = K * r * d * d / (2.0 * (4.0 / beta - 1.0))
    C0 = K * r * d * d / 2.0
    denom = (0.5 * (1 + math.exp(-2 * E / d))) ** 2

    def cc2(x):
        return 0.5 * (np.exp((2 * x - 2 * E) / d) + np.exp((-2 * x - 2 * E) / d)) / denom

    def sc2(x):
        return 0.5 * (np.exp((2 * x - 2 * E) / d) - np.exp((-2 * x - 2 * E) / d)) / denom

    c2 = 4.0 * math.exp(-2 * E / d) / (1 + math.exp(-2 * E / d)) ** 2  # 1/cosh(E/d)^2
    bp = K * (eta ** 2 + 2 * l2) + P * eta * sc(eta) + Q * cc(eta) + M * cc2(eta) + C0 * c2
    dbpE = (2 * K * E + P * (sc(E) + E / d * cc(E)) + Q / d * sc(E) + 2 * M / d * sc2(E))
    # homogeneous part D cosh(eta/l) with D l^-1 sinh(E/l) = -b_p'(E), written as
    # D cosh(eta/l) = -l b_p'(E) cosh(eta/l)/sinh(E/l)
    ratio = (np.exp((eta - E) / l) + np.exp((-eta - E) / l)) / (1 - math.exp(-2 * E / l))
    b = bp - l * dbpE * ratio
    return u, 1.0 + b, a, np.ones_like(ys)


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
