/*
 * lbve_oracle.c -- plain, slow, FP64 CPU oracle of the coupled viscoelastic
 * lattice Boltzmann time step of Yu, Chen, Wang, Yuan & Shu, "An improved
 * lattice Boltzmann method with a novel conservative boundary scheme for
 * viscoelastic fluid flows" (arXiv 2508.16997).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA path and never calls it.
 *
 * The oracle is written as the paper's algorithm, step by step, with no
 * blocking, fusion or algebraic shortcut: every Hermite moment is the literal
 * sum over the nine D2Q9 directions, every tensor contraction runs over all
 * index tuples, and streaming is an explicit push.  Precomputed tables hold
 * only the D2Q9 velocities, weights and Hermite polynomials themselves.
 *
 * State at the start of a step (time t): the completed post-streaming
 * populations f_i(x,t) and g^c_i(x,t) (c = xx, xy, yy), plus the history
 * S^c(x,t-1) and u(x,t-1) needed by the time derivative of the CDE source.
 *
 * One step (Sec. 3):
 *   1. moments:  rho = sum f, rho u = sum e f + F/2 (eq. eq_ev_f0),
 *                phi^c = sum g^c (Sec. 3.2, last relation)
 *   2. gradients of u and of rho u_x^3, rho u_y^3 by second-order finite
 *      differences (the paper does not state the scheme; reading: central
 *      differences, one-sided second order on wall rows)
 *   3. Oldroyd-B stress tau = mu_p/lambda (A - I) (eq_kramer, eqb4) and the
 *      constitutive source S = Phi_ab (Sec. 3.2, expression under eq_cde)
 *   4. hydrodynamic TRT-RLB collision with G_i, F_i, T_i (eq_ev_f, eq2, eq4,
 *      eq5, eq6 and the forcing term of Sec. 3.1)
 *   5. three CDE TRT-RLB collisions with G~_i (eq_p_G_1), F~_i (eq_p_F) and
 *      the backward difference of F~_i (eq_g0 and the difference formula of
 *      Sec. 3.2)
 *   6. push streaming; populations that would come from outside the domain
 *      are left unknown
 *   7. hydrodynamic wet-node non-equilibrium bounce-back (Zou-He) on flat
 *      walls (named in Secs. 4.2, 4.3; formulas are this oracle's reading)
 *  7b. at fluid nodes next to a solid-mask node: interpolated bounce-back of
 *      each unknown hydrodynamic population (the linear scheme of Bouzidi,
 *      Firdaouss & Lallemand 2001, standing in for the curved-wall scheme
 *      the paper cites in Sec. 4.3 without formulas; q = 1/2 is half-way
 *      bounce-back) and the momentum-exchange force on the solid (eq_F_x)
 *   8. CNEBB completion of each CDE lattice (Sec. 3.3) on the flat walls and
 *      at the solid-mask boundary nodes
 *  8b. open channels (inlet column x = 0, outlet column x = nx-1; Sec. 4.3):
 *      every population of all four lattices at the two columns by
 *      non-equilibrium extrapolation from the neighbouring column x_f, after
 *      7-8 completed it: inlet f = f^eq(rho_f, u_in) + f(x_f) - f^eq(rho_f,
 *      u_f), g = g^eq(A_in, u_in) + g(x_f) - g^eq(phi_f, u_f); outlet f =
 *      f^eq(1, u_f) + f(x_f) - f^eq(rho_f, u_f) (pressure rho_0 = 1,
 *      zero-gradient velocity) and g = g(x_f) (zero gradient).  Reading:
 *      the paper names NEBB for the hydro inlet/outlet and NEQE for the
 *      conformation lattices without formulas; NEBB's per-row knowns do not
 *      exist at the corner nodes, so both lattices use the extrapolation, and
 *      the outlet fixes the pressure (a velocity inlet with an outlet that
 *      also extrapolates the density leaves the pressure level free)
 *   9. history <- S(t), u(t)
 *
 * Domain: nx x ny nodes, row-major [y][x], periodic in x.  In y either
 * periodic, or wet-node walls on rows y = 0 and y = ny-1 (solid beyond).
 * Optionally a solid mask (orc_set_mask): solid nodes take no part in the
 * update and report zero fields; gradients next to them are one-sided.
 * Optionally open in x (orc_params.open_x): an inlet column x = 0 with the
 * profile of orc_set_inlet and a zero-gradient outlet column x = nx-1;
 * gradients along x are one-sided on those columns.
 *
 * Parity status: every function here is pinned by tests under tests/
 * (closed forms, invariants, special cases); see the per-function comments.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define Q 9
#define NC 3 /* conformation components: 0 = xx, 1 = xy, 2 = yy */

/* ---------------------------------------------------------------------- */
/* D2Q9 lattice (Sec. 3.1, velocity set and weights)                        */
/* ---------------------------------------------------------------------- */
static const int EX[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double W[Q] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,
                            1.0 / 9.0,  1.0 / 9.0,  1.0 / 36.0,
                            1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const int OPP[Q] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static const double CS2 = 1.0 / 3.0; /* c_s^2 with c = 1 */

/* Hermite polynomials of orders 1..3 for every direction (Sec. 3.1):
 *   H_a    = e_a
 *   H_ab   = e_a e_b - cs2 d_ab
 *   H_abc  = e_a e_b e_c - cs2 (e_a d_bc + e_b d_ac + e_c d_ab)         */
static double H1[Q][2], H2[Q][2][2], H3[Q][2][2][2];
static int tables_ready = 0;

static void build_tables(void) {
  if (tables_ready) return;
  for (int i = 0; i < Q; ++i) {
    const double e[2] = {(double)EX[i], (double)EY[i]};
    for (int a = 0; a < 2; ++a) {
      H1[i][a] = e[a];
      for (int b = 0; b < 2; ++b) {
        H2[i][a][b] = e[a] * e[b] - CS2 * (a == b);
        for (int c = 0; c < 2; ++c)
          H3[i][a][b][c] = e[a] * e[b] * e[c] -
                           CS2 * (e[a] * (b == c) + e[b] * (a == c) + e[c] * (a == b));
      }
    }
  }
  tables_ready = 1;
}

/* ---------------------------------------------------------------------- */
/* Parameters                                                               */
/* ---------------------------------------------------------------------- */
typedef struct {
  int32_t nx, ny;
  int32_t periodic_y; /* 0: wet-node walls on rows 0 and ny-1          */
  int32_t open_x;     /* 1: inlet column x = 0, outlet x = nx-1 (step 8b) */
  double beta, Wi, Re, Sc, Ma; /* Sec. 2.4-2.5                          */
  double Lc;                   /* characteristic length, lattice units  */
  double Lambda_s, Lambda_p;   /* magic parameters (Secs. 3.1, 3.2)      */
  double Fx, Fy;               /* uniform body force if no field given  */
  int32_t model;  /* constitutive function F(A) of eq_Constitutive / eq_kramer:
                     0 Oldroyd-B (eqb4), 1 FENE-P, 2 FENE-CR               */
  int32_t gtilde; /* G~_i: 0 incompressible form eq_p_G_1, 1 eq_p_G (with the
                     density gradient)                                      */
  double L2;      /* FENE extensibility L^2 (> 2), models 1 and 2           */
} orc_params;

/* Derived lattice coefficients (Sec. 2.4 and the relaxation-time relations
 * of Secs. 3.1-3.2), rho_0 = 1, dt = dx = 1:
 *   U_c = Ma c_s                                  (eq_Mach)
 *   nu_0 = U_c L_c / Re                           (eqb5)
 *   nu_s = beta nu_0, mu_p = (1-beta) nu_0         (eqb7, mu_0 = mu_s + mu_p)
 *   tau_s1 = nu_s / cs2 + 1/2                      (mu_s relation, Sec. 3.1)
 *   tau_s2 = Lambda_s/(tau_s1 - 1/2) + 1/2         (Lambda_s relation)
 *   kappa = nu_s / Sc                              (eqb8)
 *   tau_p1 = kappa / cs2 + 1/2                     (kappa relation, Sec. 3.2)
 *   tau_p2 = Lambda_p/(tau_p1 - 1/2) + 1/2         (tau_p2 relation)
 *   lambda = Wi L_c / U_c                          (eqb6)                 */
typedef struct {
  double Uc, nu0, nus, mup, tau_s1, tau_s2, kappa, tau_p1, tau_p2, lambda;
} orc_coeffs;

void orc_derive(const orc_params* p, orc_coeffs* c) {
  c->Uc = p->Ma * sqrt(CS2);
  c->nu0 = c->Uc * p->Lc / p->Re;
  c->nus = p->beta * c->nu0;
  c->mup = (1.0 - p->beta) * c->nu0;
  c->tau_s1 = c->nus / CS2 + 0.5;
  c->tau_s2 = p->Lambda_s / (c->tau_s1 - 0.5) + 0.5;
  c->kappa = c->nus / p->Sc;
  c->tau_p1 = c->kappa / CS2 + 0.5;
  c->tau_p2 = p->Lambda_p / (c->tau_p1 - 0.5) + 0.5;
  c->lambda = p->Wi * p->Lc / c->Uc;
}

/* ---------------------------------------------------------------------- */
/* Node-level building blocks                                               */
/* ---------------------------------------------------------------------- */

/* Third-order Hermite equilibrium of the hydrodynamic lattice (eq2). */
void orc_feq(double rho, double ux, double uy, double* feq) {
  build_tables();
  const double u[2] = {ux, uy};
  for (int i = 0; i < Q; ++i) {
    double s1 = 0, s2 = 0, s3 = 0;
    for (int a = 0; a < 2; ++a) {
      s1 += H1[i][a] * u[a];
      for (int b = 0; b < 2; ++b) {
        s2 += H2[i][a][b] * u[a] * u[b];
        for (int c = 0; c < 2; ++c) s3 += H3[i][a][b][c] * u[a] * u[b] * u[c];
      }
    }
    feq[i] = W[i] * rho *
             (1.0 + s1 / CS2 + s2 / (2.0 * CS2 * CS2) + s3 / (6.0 * CS2 * CS2 * CS2));
  }
}

/* Second-order Hermite equilibrium of a CDE lattice (eq_geq). */
void orc_geq(double phi, double ux, double uy, double* geq) {
  build_tables();
  const double u[2] = {ux, uy};
  for (int i = 0; i < Q; ++i) {
    double s1 = 0, s2 = 0;
    for (int a = 0; a < 2; ++a) {
      s1 += H1[i][a] * u[a];
      for (int b = 0; b < 2; ++b) s2 += H2[i][a][b] * u[a] * u[b];
    }
    geq[i] = W[i] * phi * (1.0 + s1 / CS2 + s2 / (2.0 * CS2 * CS2));
  }
}

/* Hydrodynamic moments (eq_ev_f0): rho = sum f, rho u = sum e f + F/2. */
void orc_hydro_moments(const double* f, double Fx, double Fy, double* rho, double* ux,
                       double* uy) {
  double r = 0, jx = 0, jy = 0;
  for (int i = 0; i < Q; ++i) {
    r += f[i];
    jx += EX[i] * f[i];
    jy += EY[i] * f[i];
  }
  *rho = r;
  *ux = (jx + 0.5 * Fx) / r;
  *uy = (jy + 0.5 * Fy) / r;
}

/* Hydrodynamic TRT-RLB collision (eq_ev_f) with
 *   off-equilibrium Hermite moments A0, A_a, A_ab, A_abc (eq4a-d),
 *   Galilean correction G_i (eq5) with d_g Phi_abg given by its two nonzero
 *     components dPhi[0] = d_x(rho u_x^3), dPhi[1] = d_y(rho u_y^3),
 *   viscoelastic source T_i (eq6) with tau = {tau_xx, tau_xy, tau_yy},
 *   first-order Hermite forcing F_i (Sec. 3.1), dt = 1.
 * Input f is the completed post-streaming population at time t; out is f^dagger. */
void orc_hydro_collide(const double* f, double Fx, double Fy, const double* tau,
                       const double* dPhi, double tau_s1, double tau_s2, double* out) {
  build_tables();
  double rho, ux, uy;
  orc_hydro_moments(f, Fx, Fy, &rho, &ux, &uy);
  double feq[Q];
  orc_feq(rho, ux, uy, feq);

  double A0 = 0, A1[2] = {0, 0}, A2[2][2] = {{0, 0}, {0, 0}};
  double A3[2][2][2] = {{{0, 0}, {0, 0}}, {{0, 0}, {0, 0}}};
  for (int i = 0; i < Q; ++i) {
    const double fneq = f[i] - feq[i];
    A0 += fneq;
    for (int a = 0; a < 2; ++a) {
      A1[a] += H1[i][a] * fneq;
      for (int b = 0; b < 2; ++b) {
        A2[a][b] += H2[i][a][b] * fneq;
        for (int c = 0; c < 2; ++c) A3[a][b][c] += H3[i][a][b][c] * fneq;
      }
    }
  }
  const double T2[2][2] = {{tau[0], tau[1]}, {tau[1], tau[2]}};
  const double dP[2][2] = {{dPhi[0], 0.0}, {0.0, dPhi[1]}}; /* d_g Phi_abg */
  const double F[2] = {Fx, Fy};
  const double cs4 = CS2 * CS2, cs6 = CS2 * CS2 * CS2;

  for (int i = 0; i < Q; ++i) {
    double r1 = A0, r3 = 0, g2 = 0, t2 = 0, f1 = 0;
    for (int a = 0; a < 2; ++a) {
      r1 += H1[i][a] * A1[a] / CS2;
      f1 += H1[i][a] * F[a] / CS2;
      for (int b = 0; b < 2; ++b) {
        r1 += H2[i][a][b] * A2[a][b] / (2.0 * cs4);
        g2 += H2[i][a][b] * dP[a][b];
        t2 += H2[i][a][b] * T2[a][b];
        for (int c = 0; c < 2; ++c) r3 += H3[i][a][b][c] * A3[a][b][c];
      }
    }
    const double Gi = -W[i] * (1.0 - 1.0 / (2.0 * tau_s1)) * g2 / (6.0 * cs6);
    const double Ti = -W[i] * t2 / (2.0 * cs4 * tau_s1);
    const double Fi = (1.0 - 1.0 / (2.0 * tau_s1)) * W[i] * f1;
    out[i] = feq[i] + W[i] * (1.0 - 1.0 / tau_s1) * r1 +
             W[i] * (1.0 - 1.0 / tau_s2) * r3 / (6.0 * cs6) + Gi + Fi + Ti;
  }
}

/* CDE source term F~_i (eq_p_F) for source S and velocity u.  Its e.u S
 * part cancels the U S share of the flux error (tau_p1 - 1/2) d_t(phi u);
 * pinned by test_source_velocity_term_removes_the_relaxation_drift. */
static void cde_source(double S, double ux, double uy, double tau_p1, double* Ft) {
  const double u[2] = {ux, uy};
  for (int i = 0; i < Q; ++i) {
    double eu = 0;
    for (int a = 0; a < 2; ++a) eu += H1[i][a] * u[a];
    Ft[i] = W[i] * S + (1.0 - 1.0 / (2.0 * tau_p1)) * W[i] * eu * S / CS2;
  }
}

/* CDE TRT-RLB collision (eq_g0) of one conformation lattice:
 *   off-equilibrium moments B0, B_a, B_ab (Sec. 3.2, eq_p_neq_m),
 *   auxiliary term G~_i (eq_p_G_1), source F~_i(t) (eq_p_F) and
 *   (dt^2/2) d_t F~_i with the backward difference of Sec. 3.2, dt = 1.
 * u, rho, F are the hydrodynamic velocity, density and body force at t;
 * S, S_old are the source at t and t-1; uold the velocity at t-1.
 * G~_i cancels the phi a share of the flux error (tau_p1 - 1/2) d_t(phi u);
 * pinned by test_gtilde_removes_the_acceleration_drift. */
void orc_cde_collide(const double* g, double rho, double ux, double uy, double Fx,
                     double Fy, double S, double S_old, double uxo, double uyo,
                     double tau_p1, double tau_p2, double* out) {
  build_tables();
  double phi = 0;
  for (int i = 0; i < Q; ++i) phi += g[i];
  double geq[Q];
  orc_geq(phi, ux, uy, geq);
  double B0 = 0, B1[2] = {0, 0}, B2[2][2] = {{0, 0}, {0, 0}};
  for (int i = 0; i < Q; ++i) {
    const double gneq = g[i] - geq[i];
    B0 += gneq;
    for (int a = 0; a < 2; ++a) {
      B1[a] += H1[i][a] * gneq;
      for (int b = 0; b < 2; ++b) B2[a][b] += H2[i][a][b] * gneq;
    }
  }
  double Ft[Q], Ft_old[Q];
  cde_source(S, ux, uy, tau_p1, Ft);
  cde_source(S_old, uxo, uyo, tau_p1, Ft_old);
  const double F[2] = {Fx, Fy};
  const double cs4 = CS2 * CS2;
  for (int i = 0; i < Q; ++i) {
    double r1 = B0, r2 = 0, eF = 0;
    for (int a = 0; a < 2; ++a) {
      r1 += H1[i][a] * B1[a] / CS2;
      eF += H1[i][a] * F[a];
      for (int b = 0; b < 2; ++b) r2 += H2[i][a][b] * B2[a][b] / (2.0 * cs4);
    }
    const double Gt = W[i] * (1.0 - 1.0 / (2.0 * tau_p1)) * (eF / CS2) * (phi / rho);
    out[i] = geq[i] + W[i] * (1.0 - 1.0 / tau_p1) * r1 + W[i] * (1.0 - 1.0 / tau_p2) * r2 +
             Gt + Ft[i] + 0.5 * (Ft[i] - Ft_old[i]);
  }
}

/* Constitutive function F(A) (eq_Constitutive, eq_kramer; Sec. 2 lists the
 * models the formalism takes).  The two FENE models fit the paper's single-F
 * form exactly (the same F relaxes A and gives the stress):
 *   model 0, Oldroyd-B (eqb4): F = A - I
 *   model 1, FENE-P:  F = A / (1 - tr A / L2) - I / (1 - 2 / L2)
 *                     (the 2-D form: F(I) = 0)
 *   model 2, FENE-CR: F = (A - I) L2 / (L2 - tr A)
 * A and F are {xx, xy, yy}. */
void orc_model_F(const double* A, int model, double L2, double* F) {
  const double tr = A[0] + A[2];
  if (model == 1) {
    const double f = 1.0 / (1.0 - tr / L2), a = 1.0 / (1.0 - 2.0 / L2);
    F[0] = f * A[0] - a;
    F[1] = f * A[1];
    F[2] = f * A[2] - a;
  } else if (model == 2) {
    const double f = L2 / (L2 - tr);
    F[0] = f * (A[0] - 1.0);
    F[1] = f * A[1];
    F[2] = f * (A[2] - 1.0);
  } else {
    F[0] = A[0] - 1.0;
    F[1] = A[1];
    F[2] = A[2] - 1.0;
  }
}

/* Constitutive source of eq_Constitutive (Sec. 3.2, Phi_ab) for a model:
 *   S_ab = -F_ab(A)/lambda + A_ag d_g u_b + A_gb d_g u_a + A_ab d_g u_g
 * grad[g][b] = d_g u_b.  A and S are {xx, xy, yy}. */
void orc_source_model(const double* A, const double* grad, double lambda, int model, double L2,
                      double* S) {
  const double A2[2][2] = {{A[0], A[1]}, {A[1], A[2]}};
  const double (*G)[2] = (const double (*)[2])grad;
  const int ab[3][2] = {{0, 0}, {0, 1}, {1, 1}};
  const double div = G[0][0] + G[1][1];
  double F[3];
  orc_model_F(A, model, L2, F);
  for (int c = 0; c < NC; ++c) {
    const int a = ab[c][0], b = ab[c][1];
    double s = -F[c] / lambda;
    for (int g = 0; g < 2; ++g) s += A2[a][g] * G[g][b] + A2[g][b] * G[g][a];
    s += A2[a][b] * div;
    S[c] = s;
  }
}

/* Oldroyd-B constitutive source (Sec. 3.2, expression for Phi_ab):
 *   S_ab = -(A_ab - d_ab)/lambda + A_ag d_g u_b + A_gb d_g u_a + A_ab d_g u_g
 * grad[g][b] = d_g u_b.  A and S are {xx, xy, yy}. */
void orc_source(const double* A, const double* grad, double lambda, double* S) {
  const double A2[2][2] = {{A[0], A[1]}, {A[1], A[2]}};
  const double (*G)[2] = (const double (*)[2])grad;
  const int ab[3][2] = {{0, 0}, {0, 1}, {1, 1}};
  const double div = G[0][0] + G[1][1];
  for (int c = 0; c < NC; ++c) {
    const int a = ab[c][0], b = ab[c][1];
    double s = -(A2[a][b] - (a == b)) / lambda;
    for (int g = 0; g < 2; ++g) s += A2[a][g] * G[g][b] + A2[g][b] * G[g][a];
    s += A2[a][b] * div;
    S[c] = s;
  }
}

/* Hydrodynamic wet-node bounce-back of the non-equilibrium part with the
 * two tangential/normal moment conditions (Zou-He), wall velocity 0, on a
 * flat wall.  The paper names the hydrodynamic NEBB scheme (Secs. 4.2, 4.3)
 * without formulas; this oracle's reading: the completed populations satisfy
 *   sum_i f_i = rho and sum_i e_i f_i = -F/2   (so u = 0 through eq_ev_f0),
 *   f_n - f_nbar = 0 for the wall-normal pair,
 * with rho solved from the known populations.  side = 0: bottom wall (unknown
 * 2, 5, 6), side = 1: top wall (unknown 4, 7, 8). */
void orc_zou_he(double* f, double Fx, double Fy, int side) {
  if (side == 0) {
    /* sum e_y f = f2+f5+f6 - (f4+f7+f8) = -Fy/2  and  sum f = rho          */
    f[2] = f[4];
    f[5] = f[7] - 0.5 * (f[1] - f[3]) - 0.25 * Fx - 0.25 * Fy;
    f[6] = f[8] + 0.5 * (f[1] - f[3]) + 0.25 * Fx - 0.25 * Fy;
  } else {
    f[4] = f[2];
    f[7] = f[5] + 0.5 * (f[1] - f[3]) + 0.25 * Fx + 0.25 * Fy;
    f[8] = f[6] - 0.5 * (f[1] - f[3]) - 0.25 * Fx + 0.25 * Fy;
  }
}

/* CNEBB completion of one CDE lattice at a boundary node (Sec. 3.3).
 *   known[i]   : 1 if g_i(x_b,t+1) arrived by streaming, 0 if unknown
 *   g          : post-streaming populations at (x_b,t+1), unknown slots ignored
 *   gpost      : post-collision populations at (x_b,t)
 *   ux, uy     : hydrodynamic velocity at (x_b,t+1) after the hydro completion
 * H is the set of directions pointing toward the solid, i.e. the opposites of
 * the unknown directions.  Returns the wall "in" and "out" amounts:
 *   out = sum_{eta in H} g^dagger_eta(x_b,t)   (sent toward the wall),
 *   in  = what the completion adds back = phi_b - sum_{gamma in Gamma} g_gamma. */
void orc_cnebb(double* g, const double* gpost, const int* known, double ux, double uy,
               double* in_amount, double* out_amount) {
  double phi = 0, out = 0;
  for (int i = 0; i < Q; ++i)
    if (known[i]) phi += g[i];
  double known_sum = phi;
  for (int i = 0; i < Q; ++i)
    if (!known[i]) {
      const int eta = OPP[i]; /* points toward the solid */
      phi += gpost[eta];
      out += gpost[eta];
    }
  double geq[Q];
  orc_geq(phi, ux, uy, geq);
  for (int i = 0; i < Q; ++i)
    if (!known[i]) g[i] = geq[i] + (g[OPP[i]] - geq[OPP[i]]);
  double rest = 0;
  for (int i = 1; i < Q; ++i) rest += g[i];
  g[0] = phi - rest;
  *in_amount = phi - known_sum;
  *out_amount = out;
}

/* ---------------------------------------------------------------------- */
/* Whole-domain simulation                                                  */
/* ---------------------------------------------------------------------- */
typedef struct {
  orc_params p;
  orc_coeffs c;
  int nx, ny, n;
  double* f;     /* [Q][n]      completed post-streaming, time t          */
  double* g;     /* [NC][Q][n]                                             */
  double* fpost; /* [Q][n]      post-collision (scratch)                   */
  double* gpost; /* [NC][Q][n]                                             */
  double* Sold;  /* [NC][n]     S(t-1)                                     */
  double* uold;  /* [2][n]      u(t-1)                                     */
  double* F;     /* [2][n]      body force                                 */
  double* mom;   /* [6][n]      rho, ux, uy, phi_xx, phi_xy, phi_yy at t   */
  double* grad;  /* [8][n]      dxux, dxuy, dyux, dyuy, dx(rho ux^3), dy(rho uy^3),
                                dx rho, dy rho (eq_p_G) */
  double* S;     /* [NC][n]                                                */
  int64_t t;
  double wall_in[NC], wall_out[NC];
  uint8_t* solid; /* [n] 1 = solid node, or NULL (no mask)                 */
  double* qlink;  /* [Q][n] wall distance fraction of link (x, i), i unknown */
  double drag[2]; /* momentum-exchange force on the solid mask, last step   */
  double* inlet;  /* [5][ny] u_x, u_y, A_xx, A_xy, A_yy of the inlet (open_x) */
} orc_sim;

static inline int wrap(int a, int n) { return ((a % n) + n) % n; }

/* 1 if (x, y) is a solid node of the mask.  x wraps; y wraps when periodic;
 * rows outside a walled domain are not mask nodes. */
static int is_solid(const orc_sim* s, int x, int y) {
  if (!s->solid) return 0;
  x = wrap(x, s->nx);
  if (s->p.periodic_y) y = wrap(y, s->ny);
  else if (y < 0 || y >= s->ny) return 0;
  return s->solid[y * s->nx + x] != 0;
}

/* 1 if (x, y) is a fluid node inside the domain. */
static int is_fluid(const orc_sim* s, int x, int y) {
  if (!s->p.periodic_y && (y < 0 || y >= s->ny)) return 0;
  return !is_solid(s, x, y);
}

/* Value of field q at (x, y) with the periodic wraps. */
static double at(const orc_sim* s, const double* q, int x, int y) {
  x = wrap(x, s->nx);
  if (s->p.periodic_y) y = wrap(y, s->ny);
  return q[y * s->nx + x];
}

static void compute_moments(orc_sim* s) {
  const int n = s->n;
  for (int k = 0; k < n; ++k) {
    if (s->solid && s->solid[k]) {
      for (int j = 0; j < 6; ++j) s->mom[j * n + k] = 0.0;
      continue;
    }
    double fk[Q];
    for (int i = 0; i < Q; ++i) fk[i] = s->f[i * n + k];
    double rho, ux, uy;
    orc_hydro_moments(fk, s->F[k], s->F[n + k], &rho, &ux, &uy);
    s->mom[0 * n + k] = rho;
    s->mom[1 * n + k] = ux;
    s->mom[2 * n + k] = uy;
    for (int c = 0; c < NC; ++c) {
      double phi = 0;
      for (int i = 0; i < Q; ++i) phi += s->g[(c * Q + i) * n + k];
      s->mom[(3 + c) * n + k] = phi;
    }
  }
}

/* Second-order finite difference of field q along x (dir 0) or y (dir 1)
 * at fluid node (x,y) (reading of the paper, which does not state how these
 * gradients are discretised):
 *   - central, (q(+1) - q(-1))/2, in the interior and across periodic wraps;
 *   - one-sided (-3 q0 + 4 q1 - q2)/2 on a wall row (and along x on the
 *     inlet and outlet columns), toward the interior;
 *   - next to a solid-mask node on one side: the one-sided second-order
 *     difference toward the fluid side when two fluid nodes lie there, else
 *     the first-order difference with the one fluid neighbour;
 *   - zero when both neighbours along the axis are solid. */
static double fd(const orc_sim* s, const double* q, int x, int y, int dir) {
  const int nx = s->nx, ny = s->ny, dx = dir == 0, dy = dir == 1;
  if (dir == 1 && !s->p.periodic_y && (y == 0 || y == ny - 1)) {
    const int t = y == 0 ? 1 : -1; /* toward the interior */
    return 0.5 * t * (-3.0 * at(s, q, x, y) + 4.0 * at(s, q, x, y + t) - at(s, q, x, y + 2 * t));
  }
  if (dir == 0 && s->p.open_x && (x == 0 || x == nx - 1)) {
    const int t = x == 0 ? 1 : -1; /* toward the interior */
    return 0.5 * t * (-3.0 * at(s, q, x, y) + 4.0 * at(s, q, x + t, y) - at(s, q, x + 2 * t, y));
  }
  const int sp = is_solid(s, x + dx, y + dy), sm = is_solid(s, x - dx, y - dy);
  if (!sp && !sm) return 0.5 * (at(s, q, x + dx, y + dy) - at(s, q, x - dx, y - dy));
  if (sp && sm) return 0.0;
  const int t = sp ? -1 : 1; /* toward the fluid side */
  if (is_fluid(s, x + 2 * t * dx, y + 2 * t * dy))
    return 0.5 * t *
           (-3.0 * at(s, q, x, y) + 4.0 * at(s, q, x + t * dx, y + t * dy) -
            at(s, q, x + 2 * t * dx, y + 2 * t * dy));
  return t * (at(s, q, x + t * dx, y + t * dy) - at(s, q, x, y));
}

static void compute_gradients_and_source(orc_sim* s) {
  const int n = s->n, nx = s->nx, ny = s->ny;
  double* cube_x = (double*)malloc(sizeof(double) * n);
  double* cube_y = (double*)malloc(sizeof(double) * n);
  for (int k = 0; k < n; ++k) {
    const double rho = s->mom[k], ux = s->mom[n + k], uy = s->mom[2 * n + k];
    cube_x[k] = rho * ux * ux * ux; /* Phi_xxx (eq5) */
    cube_y[k] = rho * uy * uy * uy; /* Phi_yyy */
  }
  const double* ux = s->mom + n;
  const double* uy = s->mom + 2 * n;
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      const int k = y * nx + x;
      if (s->solid && s->solid[k]) {
        for (int j = 0; j < 8; ++j) s->grad[j * n + k] = 0.0;
        for (int c = 0; c < NC; ++c) s->S[c * n + k] = 0.0;
        continue;
      }
      s->grad[0 * n + k] = fd(s, ux, x, y, 0);
      s->grad[1 * n + k] = fd(s, uy, x, y, 0);
      s->grad[2 * n + k] = fd(s, ux, x, y, 1);
      s->grad[3 * n + k] = fd(s, uy, x, y, 1);
      s->grad[4 * n + k] = fd(s, cube_x, x, y, 0);
      s->grad[5 * n + k] = fd(s, cube_y, x, y, 1);
      s->grad[6 * n + k] = fd(s, s->mom, x, y, 0); /* density gradient (eq_p_G) */
      s->grad[7 * n + k] = fd(s, s->mom, x, y, 1);
      /* grad[g][b] = d_g u_b */
      const double G[2][2] = {{s->grad[k], s->grad[n + k]}, {s->grad[2 * n + k], s->grad[3 * n + k]}};
      const double A[3] = {s->mom[3 * n + k], s->mom[4 * n + k], s->mom[5 * n + k]};
      double S[3];
      orc_source_model(A, &G[0][0], s->c.lambda, s->p.model, s->p.L2, S);
      for (int c = 0; c < NC; ++c) s->S[c * n + k] = S[c];
    }
  free(cube_x);
  free(cube_y);
}

static void fill_history(orc_sim* s) {
  const int n = s->n;
  for (int k = 0; k < n; ++k) {
    for (int c = 0; c < NC; ++c) s->Sold[c * n + k] = s->S[c * n + k];
    s->uold[k] = s->mom[n + k];
    s->uold[n + k] = s->mom[2 * n + k];
  }
}

static void free_sim(orc_sim* s) {
  if (!s) return;
  free(s->f); free(s->g); free(s->fpost); free(s->gpost); free(s->Sold);
  free(s->uold); free(s->F); free(s->mom); free(s->grad); free(s->S);
  free(s->solid); free(s->qlink); free(s->inlet);
  free(s);
}

/* Create a simulation.  force: [2][ny][nx] or NULL (uniform p->Fx, p->Fy).
 * init: [6][ny][nx] = rho, ux, uy, Axx, Axy, Ayy, or NULL for rho = 1, u = 0,
 * A = I (Sec. 4.2 initial state).  Populations start at equilibrium (eq2,
 * eq_geq) of the initial fields; history S(-1) := S(0), u(-1) := u(0), i.e.
 * the backward difference of F~ is zero on the first step. */
orc_sim* orc_create(const orc_params* p, const double* force, const double* init) {
  build_tables();
  if (p->nx < 1 || p->ny < 1 || (!p->periodic_y && p->ny < 3)) return NULL;
  if (p->open_x != 0 && (p->open_x != 1 || p->nx < 5)) return NULL;
  if (p->model < 0 || p->model > 2 || (p->model != 0 && !(p->L2 > 2.0))) return NULL;
  if (p->gtilde != 0 && p->gtilde != 1) return NULL;
  orc_sim* s = (orc_sim*)calloc(1, sizeof(orc_sim));
  s->p = *p;
  orc_derive(p, &s->c);
  s->nx = p->nx;
  s->ny = p->ny;
  s->n = p->nx * p->ny;
  const int n = s->n;
  s->f = (double*)calloc((size_t)Q * n, sizeof(double));
  s->g = (double*)calloc((size_t)NC * Q * n, sizeof(double));
  s->fpost = (double*)calloc((size_t)Q * n, sizeof(double));
  s->gpost = (double*)calloc((size_t)NC * Q * n, sizeof(double));
  s->Sold = (double*)calloc((size_t)NC * n, sizeof(double));
  s->uold = (double*)calloc((size_t)2 * n, sizeof(double));
  s->F = (double*)calloc((size_t)2 * n, sizeof(double));
  s->mom = (double*)calloc((size_t)6 * n, sizeof(double));
  s->grad = (double*)calloc((size_t)8 * n, sizeof(double));
  s->S = (double*)calloc((size_t)NC * n, sizeof(double));
  s->inlet = (double*)calloc((size_t)5 * p->ny, sizeof(double));
  if (!s->f || !s->g || !s->fpost || !s->gpost || !s->Sold || !s->uold || !s->F || !s->mom ||
      !s->grad || !s->S || !s->inlet) {
    free_sim(s);
    return NULL;
  }
  for (int y = 0; y < p->ny; ++y) s->inlet[2 * p->ny + y] = s->inlet[4 * p->ny + y] = 1.0;
  for (int k = 0; k < n; ++k) {
    s->F[k] = force ? force[k] : p->Fx;
    s->F[n + k] = force ? force[n + k] : p->Fy;
    const double rho = init ? init[k] : 1.0;
    const double ux = init ? init[n + k] : 0.0;
    const double uy = init ? init[2 * n + k] : 0.0;
    const double A[3] = {init ? init[3 * n + k] : 1.0, init ? init[4 * n + k] : 0.0,
                         init ? init[5 * n + k] : 1.0};
    double eq[Q];
    orc_feq(rho, ux, uy, eq);
    for (int i = 0; i < Q; ++i) s->f[i * n + k] = eq[i];
    for (int c = 0; c < NC; ++c) {
      orc_geq(A[c], ux, uy, eq);
      for (int i = 0; i < Q; ++i) s->g[(c * Q + i) * n + k] = eq[i];
    }
  }
  compute_moments(s);
  compute_gradients_and_source(s);
  fill_history(s);
  return s;
}

void orc_destroy(orc_sim* s) { free_sim(s); }

void orc_get_coeffs(const orc_sim* s, orc_coeffs* c) { *c = s->c; }

/* Advance n_steps time steps (steps 1-9 of the header). */
void orc_step(orc_sim* s, int64_t n_steps) {
  const int n = s->n, nx = s->nx, ny = s->ny;
  for (int64_t it = 0; it < n_steps; ++it) {
    /* 1-3: moments, gradients, stress and source at time t */
    compute_moments(s);
    compute_gradients_and_source(s);
    /* 4-5: collisions (fluid nodes only) */
    for (int k = 0; k < n; ++k) {
      if (s->solid && s->solid[k]) continue;
      const double rho = s->mom[k], ux = s->mom[n + k], uy = s->mom[2 * n + k];
      const double Fx = s->F[k], Fy = s->F[n + k];
      const double A[3] = {s->mom[3 * n + k], s->mom[4 * n + k], s->mom[5 * n + k]};
      double Fm[3];
      orc_model_F(A, s->p.model, s->p.L2, Fm);
      const double tau[3] = {s->c.mup / s->c.lambda * Fm[0], s->c.mup / s->c.lambda * Fm[1],
                             s->c.mup / s->c.lambda * Fm[2]}; /* eq_kramer */
      const double dPhi[2] = {s->grad[4 * n + k], s->grad[5 * n + k]};
      double fk[Q], out[Q];
      for (int i = 0; i < Q; ++i) fk[i] = s->f[i * n + k];
      orc_hydro_collide(fk, Fx, Fy, tau, dPhi, s->c.tau_s1, s->c.tau_s2, out);
      for (int i = 0; i < Q; ++i) s->fpost[i * n + k] = out[i];
      for (int c = 0; c < NC; ++c) {
        double gk[Q];
        for (int i = 0; i < Q; ++i) gk[i] = s->g[(c * Q + i) * n + k];
        /* G~_i sees F (eq_p_G_1) or F - c_s^2 grad rho (eq_p_G) */
        const double Gx = s->p.gtilde ? Fx - CS2 * s->grad[6 * n + k] : Fx;
        const double Gy = s->p.gtilde ? Fy - CS2 * s->grad[7 * n + k] : Fy;
        orc_cde_collide(gk, rho, ux, uy, Gx, Gy, s->S[c * n + k], s->Sold[c * n + k],
                        s->uold[k], s->uold[n + k], s->c.tau_p1, s->c.tau_p2, out);
        for (int i = 0; i < Q; ++i) s->gpost[(c * Q + i) * n + k] = out[i];
      }
    }
    /* 9 (done now, the values are no longer needed): history <- S(t), u(t) */
    fill_history(s);
    /* 6: push streaming between fluid nodes; unknown slots are overwritten
     * by 7-8 */
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const int k = y * nx + x;
        if (s->solid && s->solid[k]) continue;
        for (int i = 0; i < Q; ++i) {
          int yd = y + EY[i];
          if (s->p.periodic_y) yd = wrap(yd, ny);
          else if (yd < 0 || yd >= ny) continue; /* leaves toward the wall */
          const int xd = x + EX[i];
          if (s->p.open_x && (xd < 0 || xd >= nx)) continue; /* leaves the open channel */
          const int kd = yd * nx + wrap(xd, nx);
          if (s->solid && s->solid[kd]) continue; /* leaves toward the mask */
          s->f[i * n + kd] = s->fpost[i * n + k];
          for (int c = 0; c < NC; ++c) s->g[(c * Q + i) * n + kd] = s->gpost[(c * Q + i) * n + k];
        }
      }
    for (int c = 0; c < NC; ++c) s->wall_in[c] = s->wall_out[c] = 0.0;
    if (!s->p.periodic_y) {
      /* 7-8 on the two wall rows */
      for (int side = 0; side < 2; ++side) {
        const int y = side == 0 ? 0 : ny - 1;
        int known[Q];
        for (int i = 0; i < Q; ++i) {
          const int ys = y - EY[i]; /* source row of direction i */
          known[i] = (ys >= 0 && ys < ny);
        }
        /* the open columns' corner nodes are completed by 8b instead */
        const int xa = s->p.open_x ? 1 : 0, xb = s->p.open_x ? nx - 1 : nx;
        for (int x = xa; x < xb; ++x) {
          const int k = y * nx + x;
          const double Fx = s->F[k], Fy = s->F[n + k];
          double fk[Q];
          for (int i = 0; i < Q; ++i) fk[i] = s->f[i * n + k];
          orc_zou_he(fk, Fx, Fy, side);
          for (int i = 0; i < Q; ++i) s->f[i * n + k] = fk[i];
          double rho, ux, uy;
          orc_hydro_moments(fk, Fx, Fy, &rho, &ux, &uy);
          for (int c = 0; c < NC; ++c) {
            double gk[Q], gp[Q], win, wout;
            for (int i = 0; i < Q; ++i) {
              gk[i] = s->g[(c * Q + i) * n + k];
              gp[i] = s->gpost[(c * Q + i) * n + k];
            }
            orc_cnebb(gk, gp, known, ux, uy, &win, &wout);
            for (int i = 0; i < Q; ++i) s->g[(c * Q + i) * n + k] = gk[i];
            s->wall_in[c] += win;
            s->wall_out[c] += wout;
          }
        }
      }
    }
    s->drag[0] = s->drag[1] = 0.0;
    if (s->solid) {
      /* 7b and 8 at the fluid nodes next to the solid mask */
      for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
          const int k = y * nx + x;
          if (s->solid[k]) continue;
          int known[Q], any = 0;
          for (int i = 0; i < Q; ++i) {
            known[i] = !(i != 0 && is_solid(s, x - EX[i], y - EY[i]));
            any |= !known[i];
          }
          if (!any) continue;
          for (int i = 1; i < Q; ++i) {
            if (known[i]) continue;
            const int ib = OPP[i]; /* points toward the wall */
            const double q = s->qlink[i * n + k];
            const double fb = s->fpost[ib * n + k];
            double v;
            if (q < 0.5) {
              if (is_fluid(s, x + EX[i], y + EY[i])) {
                const int kf = wrap(y + EY[i], ny) * nx + wrap(x + EX[i], nx);
                v = 2.0 * q * fb + (1.0 - 2.0 * q) * s->fpost[ib * n + kf];
              } else {
                v = fb; /* no second fluid node: half-way bounce-back */
              }
            } else {
              v = fb / (2.0 * q) + (1.0 - 1.0 / (2.0 * q)) * s->fpost[i * n + k];
            }
            s->f[i * n + k] = v;
            /* eq_F_x: e_ib (f^dagger_ib(x,t) + f_i(x,t+1)) over links to the wall */
            s->drag[0] += EX[ib] * (fb + v);
            s->drag[1] += EY[ib] * (fb + v);
          }
          const double Fx = s->F[k], Fy = s->F[n + k];
          double fk[Q], rho, ux, uy;
          for (int i = 0; i < Q; ++i) fk[i] = s->f[i * n + k];
          orc_hydro_moments(fk, Fx, Fy, &rho, &ux, &uy);
          for (int c = 0; c < NC; ++c) {
            double gk[Q], gp[Q], win, wout;
            for (int i = 0; i < Q; ++i) {
              gk[i] = s->g[(c * Q + i) * n + k];
              gp[i] = s->gpost[(c * Q + i) * n + k];
            }
            orc_cnebb(gk, gp, known, ux, uy, &win, &wout);
            for (int i = 0; i < Q; ++i) s->g[(c * Q + i) * n + k] = gk[i];
            s->wall_in[c] += win;
            s->wall_out[c] += wout;
          }
        }
    }
    if (s->p.open_x) {
      /* 8b: inlet and outlet columns from their completed neighbours */
      for (int side = 0; side < 2; ++side) {
        const int xb = side == 0 ? 0 : nx - 1, xf = side == 0 ? 1 : nx - 2;
        for (int y = 0; y < ny; ++y) {
          const int kb = y * nx + xb, kf = y * nx + xf;
          double ff[Q], rho_f, ux_f, uy_f;
          for (int i = 0; i < Q; ++i) ff[i] = s->f[i * n + kf];
          orc_hydro_moments(ff, s->F[kf], s->F[n + kf], &rho_f, &ux_f, &uy_f);
          double eqb[Q], eqf[Q];
          if (side == 1) {
            /* outlet: reference pressure rho_0 = 1, zero-gradient velocity;
             * the conformation lattices copy the neighbour (zero gradient) */
            orc_feq(1.0, ux_f, uy_f, eqb);
            orc_feq(rho_f, ux_f, uy_f, eqf);
            for (int i = 0; i < Q; ++i) s->f[i * n + kb] = eqb[i] + (ff[i] - eqf[i]);
            for (int j = 0; j < NC * Q; ++j) s->g[j * n + kb] = s->g[j * n + kf];
            continue;
          }
          /* inlet: prescribed velocity and conformation, density extrapolated */
          const double ubx = s->inlet[y], uby = s->inlet[ny + y];
          orc_feq(rho_f, ubx, uby, eqb);
          orc_feq(rho_f, ux_f, uy_f, eqf);
          for (int i = 0; i < Q; ++i) s->f[i * n + kb] = eqb[i] + (ff[i] - eqf[i]);
          for (int c = 0; c < NC; ++c) {
            double gf[Q], phi_f = 0.0;
            for (int i = 0; i < Q; ++i) {
              gf[i] = s->g[(c * Q + i) * n + kf];
              phi_f += gf[i];
            }
            const double phib = s->inlet[(2 + c) * ny + y];
            orc_geq(phib, ubx, uby, eqb);
            orc_geq(phi_f, ux_f, uy_f, eqf);
            for (int i = 0; i < Q; ++i) s->g[(c * Q + i) * n + kb] = eqb[i] + (gf[i] - eqf[i]);
          }
        }
      }
    }
    s->t += 1;
  }
}

/* Inlet profile of an open channel: in [5][ny] = u_x, u_y, A_xx, A_xy,
 * A_yy at the inlet column (the zero velocity and A = I until set).
 * Returns 0, or -1 if the domain is not open in x. */
int orc_set_inlet(orc_sim* s, const double* in) {
  if (!s->p.open_x) return -1;
  memcpy(s->inlet, in, sizeof(double) * 5 * (size_t)s->ny);
  return 0;
}

/* Install a solid mask before the first step.  solid: [ny][nx], nonzero =
 * solid node.  q: [Q][ny][nx] or NULL; q[i][k] in (0, 1] is the fraction of
 * the link from fluid node k toward its solid neighbour k - e_i at which the
 * wall lies (used only where k is fluid and k - e_i solid; NULL = 1/2
 * everywhere, the staircase wall).  The moments, gradients, source and
 * history of the initial state are recomputed with the mask.
 * Returns 0, or -1 if the simulation already stepped, -2 if a walled domain
 * has solid nodes on rows 0..2 or ny-3..ny-1 (or an open channel on columns
 * 0..2 or nx-3..nx-1), -3 if a fluid node has solid
 * neighbours on both ends of one lattice line, -4 for q outside (0, 1]. */
int orc_set_mask(orc_sim* s, const uint8_t* solid, const double* q) {
  const int n = s->n, nx = s->nx, ny = s->ny;
  if (s->t != 0) return -1;
  uint8_t* m = (uint8_t*)malloc((size_t)n);
  double* ql = (double*)malloc(sizeof(double) * Q * (size_t)n);
  if (!m || !ql) {
    free(m);
    free(ql);
    return -5;
  }
  for (int k = 0; k < n; ++k) m[k] = solid[k] ? 1 : 0;
  for (int k = 0; k < Q * n; ++k) ql[k] = 0.5;
  uint8_t* old_solid = s->solid;
  double* old_q = s->qlink;
  s->solid = m;
  s->qlink = ql;
  int rc = 0;
  if (!s->p.periodic_y)
    for (int x = 0; x < nx && !rc; ++x)
      for (int r = 0; r < 3 && !rc; ++r)
        if (m[r * nx + x] || m[(ny - 1 - r) * nx + x]) rc = -2;
  if (s->p.open_x)
    for (int y = 0; y < ny && !rc; ++y)
      for (int r = 0; r < 3 && !rc; ++r)
        if (m[y * nx + r] || m[y * nx + nx - 1 - r]) rc = -2;
  for (int y = 0; y < ny && !rc; ++y)
    for (int x = 0; x < nx && !rc; ++x) {
      const int k = y * nx + x;
      if (m[k]) continue;
      for (int i = 1; i < Q && !rc; ++i) {
        if (!is_solid(s, x - EX[i], y - EY[i])) continue;
        if (is_solid(s, x + EX[i], y + EY[i])) rc = -3;
        if (q) {
          const double v = q[i * n + k];
          if (!(v > 0.0 && v <= 1.0)) rc = -4;
          ql[i * n + k] = v;
        }
      }
    }
  if (rc) {
    s->solid = old_solid;
    s->qlink = old_q;
    free(m);
    free(ql);
    return rc;
  }
  free(old_solid);
  free(old_q);
  compute_moments(s);
  compute_gradients_and_source(s);
  fill_history(s);
  return 0;
}

/* Macroscopic fields at the current time t: [6][ny][nx] =
 * rho, ux, uy (eq_ev_f0), Axx, Axy, Ayy (phi of each CDE lattice). */
void orc_fields(orc_sim* s, double* out) {
  compute_moments(s);
  memcpy(out, s->mom, sizeof(double) * 6 * (size_t)s->n);
}

/* Domain totals at time t and the wall balances of the last step:
 * out[0..2]  = sum rho, sum rho ux, sum rho uy      (fluid nodes)
 * out[3..5]  = sum phi_xx, sum phi_xy, sum phi_yy
 * out[6..8]  = CNEBB wall "in" per lattice, out[9..11] = wall "out"
 * out[12..13] = momentum-exchange force on the solid mask (eq_F_x). */
void orc_totals(orc_sim* s, double* out) {
  compute_moments(s);
  const int n = s->n;
  for (int j = 0; j < 14; ++j) out[j] = 0;
  out[12] = s->drag[0];
  out[13] = s->drag[1];
  for (int k = 0; k < n; ++k) {
    const double rho = s->mom[k];
    out[0] += rho;
    out[1] += rho * s->mom[n + k];
    out[2] += rho * s->mom[2 * n + k];
    for (int c = 0; c < NC; ++c) out[3 + c] += s->mom[(3 + c) * n + k];
  }
  for (int c = 0; c < NC; ++c) {
    out[6 + c] = s->wall_in[c];
    out[9 + c] = s->wall_out[c];
  }
}

/* Source S(t) of the last moment/gradient evaluation, and the history. */
void orc_get_source(const orc_sim* s, double* S_out) {
  memcpy(S_out, s->S, sizeof(double) * NC * (size_t)s->n);
}

/* Raw state access for tests: f [Q][n], g [NC][Q][n]. */
void orc_get_state(const orc_sim* s, double* f, double* g) {
  memcpy(f, s->f, sizeof(double) * Q * (size_t)s->n);
  memcpy(g, s->g, sizeof(double) * NC * Q * (size_t)s->n);
}
void orc_set_state(orc_sim* s, const double* f, const double* g) {
  memcpy(s->f, f, sizeof(double) * Q * (size_t)s->n);
  memcpy(s->g, g, sizeof(double) * NC * Q * (size_t)s->n);
}
int64_t orc_time(const orc_sim* s) { return s->t; }
