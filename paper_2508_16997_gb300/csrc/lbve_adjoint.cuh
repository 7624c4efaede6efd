// lbve_adjoint.cuh -- hand-written discrete adjoint of the coupled step.
//
// The forward step maps the stored state X_t (36 post-collision populations
// and 5 history values per node) and the body force F to X_{t+1}.  Its
// adjoint maps lambda_{t+1} = dL/dX_{t+1} to lambda_t = dL/dX_t and adds the
// step's contribution to dL/dF.  Every stage of the forward step (see
// lbve_step.cuh) is reversed by hand, in reverse order:
//   reconstruction (linear)          -> weighted moments of lambda
//   collision coefficients b, c      -> lambda of moments, u, rho, F, S, dPhi, tau
//   Oldroyd-B source Phi_ab          -> lambda of A and of the velocity gradient
//   finite-difference gradients      -> transposed stencils (a gather)
//   u = (j + F/2)/rho, moments       -> lambda of the completed populations
//   Zou-He and CNEBB completions     -> lambda of pulled populations, own wall slots, u_b
//   pull streaming                   -> reverse pull (a gather from x + e_i)
// Three passes per step, each one thread per node:
//   adj_local   collision/source/CNEBB reverse at the node; writes lambda of the
//               conformation pulls, the gradient adjoints and the direct
//               adjoints of rho and u; writes lambda_t's history part
//   adj_gather  transposed gradient stencils + u/rho chain + Zou-He reverse;
//               writes lambda of the hydro pulls, accumulates dL/dF
//   adj_pull    reverse pull into lambda_t's populations
// A fourth kernel (adj_moments) recomputes rho, u of the forward state so the
// gather can read its neighbours.  Open channels add a fifth between the
// gather and the pull (adj_column): the inlet and outlet nodes' completed
// populations are built from the neighbouring column, so their lambda goes
// back to that column's pulled populations, moments and force.  Modes: a normal step; the final fields
// (the loss enters through rho, u, A of the last step); the initial collision
// (equilibrium populations do not depend on F; history = current values).
#pragma once
#include "lbve_step.cuh"

namespace lbve {

// Plane counts of the adjoint buffers (all with the instance's stride).
constexpr int kStateVals = 41;  // 36 populations + 5 history

template <typename R>
struct AdjArgs {
  const R* X;         // [41][S] forward state X_t (pops, then history); kAdjInit: unused
  const double* init; // kAdjInit: staged initial fields float64 [6][S]
  const R* force;     // [2][S] per-node force or null (uniform)
  R* M;               // [3][S] rho, ux, uy of the forward state at time t+1 moments
  const R* lam_next;  // [41][S] lambda_{t+1}; kAdjFields: null
  const double* lam_fields;  // kAdjFields: dL/d(rho, ux, uy, Axx, Axy, Ayy) [6][n] (n = nx*ny)
  R* lam_pulled;      // [36][S] lambda of the pulled (pre-completion) populations
  R* lam_G;           // [6][S]  lambda of G00, G01, G10, G11, dPx, dPy
  R* lam_dir;         // [3][S]  direct lambda of rho, ux, uy
  R* lam_mh;          // [8][S]  direct lambda of the raw hydro moments
  R* lam_cur;         // [41][S] lambda_t
  double* dF;         // [2][n]  accumulated dL/dF
  const uint8_t* mask;     // [S] solid nodes, or null (no mask)
  const int32_t* widx;     // [S] wall record of a fluid node next to the mask, -1 if none
  const WallDev* walls;    // the records (instance index 0)
  double* dq;              // [8][n] accumulated dL/dq of the wall fractions, or null
  double drag_w[2];        // dL/d(force on the solid) of the final step (final pass)
  int final_pass;          // 1 in the pass that carries the loss
};

// D2Q9 velocities, opposites and weights for the mask code below.
__device__ __forceinline__ constexpr int aex(int i) {
  return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__device__ __forceinline__ constexpr int aey(int i) {
  return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
__device__ __forceinline__ constexpr int aopp(int i) {
  return i == 0 ? 0 : (i <= 4 ? (i + 1) % 4 + 1 : (i + 1) % 4 + 5);
}
__device__ __forceinline__ constexpr double awt(int i) {
  return i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
}

// v wrapped into [0, n) when it lies at most two nodes outside (every caller
// offsets an in-domain coordinate by -2..2): at most two corrections, even
// for n = 1.
__device__ __forceinline__ int adj_wrap(int v, int n) {
  if (v < 0) {
    v += n;
    if (v < 0) v += n;
  } else if (v >= n) {
    v -= n;
    if (v >= n) v -= n;
  }
  return v;
}

// Node index of (x, y), x and y at most two nodes outside the domain, with
// the periodic wraps; -1 outside a walled domain.
// In an open channel x still wraps: the wrapped node is the far open column,
// whose lambda of pulled populations adj_column has cleared and whose
// difference coefficients toward the wrap are zero, so nothing flows
// through the open ends.
__device__ __forceinline__ int adj_node(const InstDev& D, int x, int y) {
  x = adj_wrap(x, D.nx);
  if (D.periodic_y) y = adj_wrap(y, D.ny);
  else if (y < 0 || y >= D.ny) return -1;
  return y * D.nx + x;
}
__device__ __forceinline__ bool adj_solid(const uint8_t* M, int k) { return M && k >= 0 && M[k]; }
__device__ __forceinline__ bool adj_fluid(const uint8_t* M, int k) { return k >= 0 && !(M && M[k]); }

// Coefficients c[j + 2], j = -2..2, of the second-order difference along one
// axis at fluid node (x, y): D q = sum_j c[j + 2] q(x + j e).  The same rule
// as the forward step: central inside and across periodic wraps, one-sided on
// wall rows (y), next to a solid node one-sided second order when two fluid
// nodes lie on the fluid side, else first order, zero between two solids.
__device__ __forceinline__ void diff_coefs(const InstDev& D, const uint8_t* M, int x, int y,
                                           int axis, double c[5]) {
  for (int j = 0; j < 5; ++j) c[j] = 0.0;
  const int dx = axis == 0, dy = axis == 1;
  if (axis == 1 && !D.periodic_y && (y == 0 || y == D.ny - 1)) {
    if (y == 0) {
      c[2] = -1.5; c[3] = 2.0; c[4] = -0.5;
    } else {
      c[2] = 1.5; c[1] = -2.0; c[0] = 0.5;
    }
    return;
  }
  // beyond an open channel's inlet or outlet column counts as blocked
  const bool sp = adj_solid(M, adj_node(D, x + dx, y + dy)) || (dx && D.open_x && x == D.nx - 1);
  const bool sm = adj_solid(M, adj_node(D, x - dx, y - dy)) || (dx && D.open_x && x == 0);
  if (!sp && !sm) {
    c[1] = -0.5; c[3] = 0.5;
  } else if (sp && sm) {
    return;
  } else if (sp) {
    if (adj_fluid(M, adj_node(D, x - 2 * dx, y - 2 * dy))) {
      c[2] = 1.5; c[1] = -2.0; c[0] = 0.5;
    } else {
      c[2] = 1.0; c[1] = -1.0;
    }
  } else {
    if (adj_fluid(M, adj_node(D, x + 2 * dx, y + 2 * dy))) {
      c[2] = -1.5; c[3] = 2.0; c[4] = -0.5;
    } else {
      c[2] = -1.0; c[3] = 1.0;
    }
  }
}

// Completed wall-link populations of a fluid node next to the mask:
// interpolated bounce-back at wall fraction q from the raw state X.
template <typename R>
__device__ __forceinline__ R bouzidi(const InstDev& D, const R* X, const WallDev& W, int k, int x,
                                     int y, int i) {
  const int S = D.stride, ib = aopp(i);
  const double q = W.q[i - 1];
  const R fb = X[(size_t)ib * S + k];
  if (q < 0.5) {
    if ((W.fmask >> i) & 1) {
      const int kf = adj_node(D, x + aex(i), y + aey(i));
      return (R)(2.0 * q) * fb + (R)(1.0 - 2.0 * q) * X[(size_t)ib * S + kf];
    }
    return fb;
  }
  const double a = 1.0 / (2.0 * q);
  return (R)a * fb + (R)(1.0 - a) * X[(size_t)i * S + k];
}

// Open channels: the inlet (x = 0) and outlet (x = nx - 1) nodes' completed
// populations come from the neighbouring column x_f = 1 or nx - 2, as the
// forward column pass builds them: the neighbour's pull, Zou-He and CNEBB on
// wall rows, its rho, u and phi, then
//   inlet:  f = f_f + f^eq(rho_f, u_in) - f^eq(rho_f, u_f),
//           g = g_f + g^eq(A_in, u_in) - g^eq(phi_f, u_f);
//   outlet: f = f_f + f^eq(1, u_f) - f^eq(rho_f, u_f), g = g_f
// (the equilibrium differences as Hermite coefficient differences).
__device__ __forceinline__ bool adj_open_column(const InstDev& D, int x) {
  return D.open_x && (x == 0 || x == D.nx - 1);
}

template <typename R>
struct ColState {
  R dp[9], d[9];        // the neighbour's pulled and completed hydro populations
  R gp[3][9], g[3][9];  // the same for the conformation lattices
  R post[3][3];         // the neighbour's own outgoing-to-wall slots (wall rows)
  R Fx, Fy, rho, ux, uy;
  R phi[3];             // delta + sum of the completed g
  bool wb, wt;
  int kf;               // the neighbour's node index
};

template <typename R>
__device__ __forceinline__ void adj_column_state(const InstDev& D, const R* X, const R* force,
                                                 int side, int y, ColState<R>& C) {
  const int nx = D.nx, ny = D.ny, S = D.stride;
  const bool py = D.periodic_y != 0;
  const int xf = side == 0 ? 1 : nx - 2, rc = y * nx;
  C.kf = rc + xf;
  int rm, rp;
  neighbour_rows(y, nx, ny, py, rm, rp);
  C.wb = !py && y == 0;
  C.wt = !py && y == ny - 1;
  C.Fx = force ? force[C.kf] : coef<R>(D, kCoefFx);
  C.Fy = force ? force[S + C.kf] : coef<R>(D, kCoefFy);
  pull9<R>(X, S, rc, rm, rp, xf, xf - 1, xf + 1, C.dp);
#pragma unroll
  for (int i = 0; i < 9; ++i) C.d[i] = C.dp[i];
  if (C.wb || C.wt) zou_he<R>(C.d, C.Fx, C.Fy, C.wb);
  HydroM<R> hm;
  hydro_moments<R>(C.d, hm);
  C.rho = R(1) + hm.drho;
  C.ux = (hm.jx + R(0.5) * C.Fx) / C.rho;
  C.uy = (hm.jy + R(0.5) * C.Fy) / C.rho;
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    pull9<R>(X + (size_t)(9 + 9 * l) * S, S, rc, rm, rp, xf, xf - 1, xf + 1, C.gp[l]);
#pragma unroll
    for (int i = 0; i < 9; ++i) C.g[l][i] = C.gp[l][i];
    C.post[l][0] = C.post[l][1] = C.post[l][2] = R(0);
    if (C.wb || C.wt) {
      const R* own = X + (size_t)(9 + 9 * l) * S + C.kf;
      C.post[l][0] = own[(C.wb ? 4 : 2) * S];
      C.post[l][1] = own[(C.wb ? 7 : 5) * S];
      C.post[l][2] = own[(C.wb ? 8 : 6) * S];
      double wi, wo;
      cnebb<R>(C.g[l], C.post[l][0], C.post[l][1], C.post[l][2], (l == 1) ? R(0) : R(1), C.ux,
               C.uy, C.wb, wi, wo);
    }
    CdeM<R> m;
    cde_moments<R>(C.g[l], m);
    C.phi[l] = ((l == 1) ? R(0) : R(1)) + m.dphi;
  }
}

// The open node's completed populations from the column state.
template <typename R>
__device__ __forceinline__ void column_complete(const InstDev& D, int side, int y,
                                                const ColState<R>& C, R d[9], R g[3][9]) {
  const int ny = D.ny;
  const R rho = C.rho, ux = C.ux, uy = C.uy;
  R e[9];
  if (side == 0) {
    const double* in = D.inlet;
    const R bx = (R)in[y], by = (R)in[ny + y];
    reconstruct<R>(R(0), rho * (bx - ux), rho * (by - uy), rho * (bx * bx - ux * ux),
                   rho * (by * by - uy * uy), rho * (bx * by - ux * uy),
                   rho * (bx * bx * by - ux * ux * uy), rho * (bx * by * by - ux * uy * uy), e);
#pragma unroll
    for (int i = 0; i < 9; ++i) d[i] = C.d[i] + e[i];
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      const R phif = C.phi[l], phib = (R)in[(2 + l) * ny + y];
      reconstruct<R>(phib - phif, phib * bx - phif * ux, phib * by - phif * uy,
                     phib * bx * bx - phif * ux * ux, phib * by * by - phif * uy * uy,
                     phib * bx * by - phif * ux * uy, R(0), R(0), e);
#pragma unroll
      for (int i = 0; i < 9; ++i) g[l][i] = C.g[l][i] + e[i];
    }
  } else {
    const R dr = R(1) - rho;
    reconstruct<R>(dr, dr * ux, dr * uy, dr * ux * ux, dr * uy * uy, dr * ux * uy,
                   dr * ux * ux * uy, dr * ux * uy * uy, e);
#pragma unroll
    for (int i = 0; i < 9; ++i) d[i] = C.d[i] + e[i];
#pragma unroll
    for (int l = 0; l < 3; ++l)
#pragma unroll
      for (int i = 0; i < 9; ++i) g[l][i] = C.g[l][i];
  }
}

// Reverse of zou_he(): lambda of the completed populations ld (in place) to
// lambda of the pulled ones, and the force's share.
template <typename R>
__device__ __forceinline__ void zou_he_T(R ld[9], R& lFx, R& lFy, bool bottom) {
  if (bottom) {
    // d2 = d4; d5 = d7 - h - Fx/4 - Fy/4; d6 = d8 + h + Fx/4 - Fy/4, h = (d1 - d3)/2
    ld[4] += ld[2];
    ld[7] += ld[5];
    ld[8] += ld[6];
    ld[1] += R(0.5) * (ld[6] - ld[5]);
    ld[3] += R(0.5) * (ld[5] - ld[6]);
    lFx += R(0.25) * (ld[6] - ld[5]);
    lFy += R(-0.25) * (ld[5] + ld[6]);
    ld[2] = ld[5] = ld[6] = R(0);
  } else {
    // d4 = d2; d7 = d5 + h + Fx/4 + Fy/4; d8 = d6 - h - Fx/4 + Fy/4
    ld[2] += ld[4];
    ld[5] += ld[7];
    ld[6] += ld[8];
    ld[1] += R(0.5) * (ld[7] - ld[8]);
    ld[3] += R(0.5) * (ld[8] - ld[7]);
    lFx += R(0.25) * (ld[7] - ld[8]);
    lFy += R(0.25) * (ld[7] + ld[8]);
    ld[4] = ld[7] = ld[8] = R(0);
  }
}

// Forward recompute at one node: completed hydro populations (deviations),
// force, raw moments and rho, u.  kAdjInit takes the equilibria of the
// staged initial fields instead of a pull and completes no wall.
template <typename R, int MODE, bool OPEN>
__device__ __forceinline__ void adj_hydro_node(const InstDev& D, const AdjArgs<R>& A, int x, int y,
                                               R d[9], R& Fx, R& Fy, HydroM<R>& hm, R& rho, R& ux,
                                               R& uy) {
  const int nx = D.nx, ny = D.ny, S = D.stride;
  const bool py = D.periodic_y != 0;
  const int k = y * nx + x;
  int rm, rp;
  neighbour_rows(y, nx, ny, py, rm, rp);
  const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
  Fx = A.force ? A.force[k] : coef<R>(D, kCoefFx);
  Fy = A.force ? A.force[S + k] : coef<R>(D, kCoefFy);
  if (MODE == kAdjInit) {
    PopSource<R, kModeInit>::hydro(A.init, S, nx, k, y * nx, rm, rp, x, xm, xp, d);
  } else if (OPEN && adj_open_column(D, x)) {
    ColState<R> C;
    adj_column_state<R>(D, A.X, A.force, x == 0 ? 0 : 1, y, C);
    R g[3][9];
    column_complete<R>(D, x == 0 ? 0 : 1, y, C, d, g);
  } else {
    pull9<R>(A.X, S, y * nx, rm, rp, x, xm, xp, d);
    if (!py && (y == 0 || y == ny - 1)) zou_he<R>(d, Fx, Fy, y == 0);
    if (A.widx && A.widx[k] >= 0) {
      // the wall pass: interpolated bounce-back of the wall links
      const WallDev& W = A.walls[A.widx[k]];
#pragma unroll
      for (int i = 1; i < 9; ++i)
        if ((W.umask >> i) & 1) d[i] = bouzidi<R>(D, A.X, W, k, x, y, i);
    }
  }
  hydro_moments<R>(d, hm);
  rho = R(1) + hm.drho;
  ux = (hm.jx + R(0.5) * Fx) / rho;
  uy = (hm.jy + R(0.5) * Fy) / rho;
}

// rho, u of every node of the forward state (for the neighbours' gradients).
template <typename R, int MODE, bool OPEN>
__global__ void adj_moments(const InstDev* __restrict__ Dp, AdjArgs<R> A) {
  const InstDev& D = *Dp;
  const int n = D.nx * D.ny;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int x = k % D.nx, y = k / D.nx, S = D.stride;
  if (A.mask && A.mask[k]) {  // solid: never read with a nonzero coefficient
    A.M[k] = R(1);
    A.M[S + k] = A.M[2 * S + k] = R(0);
    return;
  }
  R d[9], Fx, Fy, rho, ux, uy;
  HydroM<R> hm;
  adj_hydro_node<R, MODE, OPEN>(D, A, x, y, d, Fx, Fy, hm, rho, ux, uy);
  A.M[k] = rho;
  A.M[S + k] = ux;
  A.M[2 * S + k] = uy;
}

// Transpose of reconstruct(): lambda of the Hermite coefficients from the
// lambda of the nine rebuilt populations (weighted moments).
template <typename R>
__device__ __forceinline__ void reconstruct_T(const R l[9], R& b0, R& bx, R& by, R& bxx, R& byy,
                                              R& bxy, R& bxxy, R& bxyy) {
  const R w0 = R(4.0 / 9.0), w1 = R(1.0 / 9.0), w5 = R(1.0 / 36.0);
  const R a0 = w0 * l[0], a1 = w1 * l[1], a2 = w1 * l[2], a3 = w1 * l[3], a4 = w1 * l[4];
  const R a5 = w5 * l[5], a6 = w5 * l[6], a7 = w5 * l[7], a8 = w5 * l[8];
  const R s58 = (a5 + a6) + (a7 + a8);
  b0 = ((a0 + a1) + (a2 + a3)) + (a4 + s58);
  bx = R(3) * ((a1 - a3) + ((a5 - a6) + (a8 - a7)));
  by = R(3) * ((a2 - a4) + ((a5 + a6) - (a7 + a8)));
  // H_xx = e_x^2 - 1/3, H_yy = e_y^2 - 1/3, 2 H_xy = 2 e_x e_y
  const R sall = b0;
  bxx = R(4.5) * (((a1 + a3) + s58) - sall / R(3));
  byy = R(4.5) * (((a2 + a4) + s58) - sall / R(3));
  bxy = R(9) * ((a5 + a7) - (a6 + a8));
  // H_xxy = e_y (e_x^2 - 1/3), H_xyy = e_x (e_y^2 - 1/3)
  const R ey_all = (a2 - a4) + ((a5 + a6) - (a7 + a8));
  const R ex_all = (a1 - a3) + ((a5 - a6) + (a8 - a7));
  bxxy = R(13.5) * (((a5 + a6) - (a7 + a8)) - ey_all / R(3));
  bxyy = R(13.5) * (((a5 + a8) - (a6 + a7)) - ex_all / R(3));
}

// Transpose of hydro_moments / cde_moments: lambda of the nine populations
// from lambda of (drho, jx, jy, pxx, pyy, pxy, qxxy, qxyy).
template <typename R>
__device__ __forceinline__ void moments_T(R l0, R lx, R ly, R lxx, R lyy, R lxy, R lxxy, R lxyy,
                                          R out[9]) {
  out[0] = l0;
  out[1] = l0 + lx + lxx;
  out[3] = l0 - lx + lxx;
  out[2] = l0 + ly + lyy;
  out[4] = l0 - ly + lyy;
  // diagonals: e_x^2 = e_y^2 = 1
  out[5] = l0 + lx + ly + lxx + lyy + lxy + lxxy + lxyy;
  out[6] = l0 - lx + ly + lxx + lyy - lxy + lxxy - lxyy;
  out[7] = l0 - lx - ly + lxx + lyy + lxy - lxxy - lxyy;
  out[8] = l0 + lx - ly + lxx + lyy - lxy - lxxy + lxyy;
}

// Reverse of cnebb() at a wall node: given lambda of the completed
// populations lg[9], add to lambda of the pulled known populations (ld),
// of the node's own outgoing-to-wall slots (lpost[3], in H order) and of u_b.
template <typename R>
__device__ __forceinline__ void cnebb_T(const R d[9], R pa, R pb, R pc, R delta, R ubx, R uby,
                                        bool bottom, const R lg[9], R ld[9], R lpost[3], R& lubx,
                                        R& luby) {
  // forward intermediates
  R dphi;
  if (bottom) dphi = ((d[0] + d[1]) + (d[3] + d[4])) + ((d[7] + d[8]) + ((pa + pb) + pc));
  else dphi = ((d[0] + d[1]) + (d[3] + d[2])) + ((d[5] + d[6]) + ((pa + pb) + pc));
  const R phib = delta + dphi;
  const R a2 = R(6.0 / 9.0) * phib, a5 = R(6.0 / 36.0) * phib;
  // g0 = dphi - sum_{i != 0} g_i, so every other completed slot also feeds -lg[0]
  R lt[9];
#pragma unroll
  for (int i = 1; i < 9; ++i) lt[i] = lg[i] - lg[0];
  R ldphi = lg[0];
  R la2 = R(0), la5 = R(0);
  if (bottom) {
    // known: 0? (g0 is rebuilt), 1, 3, 4, 7, 8; unknown rebuilt: 2, 5, 6
    ld[1] += lt[1];
    ld[3] += lt[3];
    ld[4] += lt[4] + lt[2];
    ld[7] += lt[7] + lt[5];
    ld[8] += lt[8] + lt[6];
    la2 += uby * lt[2];
    luby += a2 * lt[2];
    la5 += (ubx + uby) * lt[5] + (uby - ubx) * lt[6];
    lubx += a5 * (lt[5] - lt[6]);
    luby += a5 * (lt[5] + lt[6]);
  } else {
    // known: 1, 2, 3, 5, 6; rebuilt: 4 = d2 - a2 uy, 7 = d5 - a5 (ux+uy), 8 = d6 + a5 (ux-uy)
    ld[1] += lt[1];
    ld[3] += lt[3];
    ld[2] += lt[2] + lt[4];
    ld[5] += lt[5] + lt[7];
    ld[6] += lt[6] + lt[8];
    la2 += -uby * lt[4];
    luby += -a2 * lt[4];
    la5 += -(ubx + uby) * lt[7] + (ubx - uby) * lt[8];
    lubx += a5 * (lt[8] - lt[7]);
    luby += -a5 * (lt[7] + lt[8]);
  }
  ldphi += R(6.0 / 9.0) * la2 + R(6.0 / 36.0) * la5;
  // dphi = sum of the known slots (0 included) and the three own post slots
  ld[0] += ldphi;
  if (bottom) {
    ld[1] += ldphi;
    ld[3] += ldphi;
    ld[4] += ldphi;
    ld[7] += ldphi;
    ld[8] += ldphi;
  } else {
    ld[1] += ldphi;
    ld[3] += ldphi;
    ld[2] += ldphi;
    ld[5] += ldphi;
    ld[6] += ldphi;
  }
  lpost[0] += ldphi;
  lpost[1] += ldphi;
  lpost[2] += ldphi;
}

// CNEBB at a fluid node next to the mask (Sec. 3.3), unknown set U = umask,
// as the wall pass does it: pm[i] (i in U) is the node's own post-collision
// slot opposite i.
template <typename R>
__device__ __forceinline__ void cnebb_mask(R g[9], const R pm[9], R delta, R ubx, R uby,
                                           int umask) {
  R dphi = R(0);
#pragma unroll
  for (int i = 0; i < 9; ++i) dphi += (i != 0 && ((umask >> i) & 1)) ? pm[i] : g[i];
  const R phib = delta + dphi;
#pragma unroll
  for (int i = 1; i < 9; ++i)
    if ((umask >> i) & 1)
      g[i] = g[aopp(i)] + (R)(6.0 * awt(i)) * phib * ((R)aex(i) * ubx + (R)aey(i) * uby);
  R rest = R(0);
#pragma unroll
  for (int i = 1; i < 9; ++i) rest += g[i];
  g[0] = dphi - rest;
}

// Reverse of cnebb_mask(): from lambda of the completed populations lg,
// add to lambda of the pulled known populations (ld), of the own posts
// (lpm, i in U) and of u_b.  gp: the pulled populations before completion.
template <typename R>
__device__ __forceinline__ void cnebb_mask_T(const R gp[9], const R pm[9], R delta, R ubx, R uby,
                                             int umask, const R lg[9], R ld[9], R lpm[9],
                                             R& lubx, R& luby) {
  R dphi = R(0);
#pragma unroll
  for (int i = 0; i < 9; ++i) dphi += (i != 0 && ((umask >> i) & 1)) ? pm[i] : gp[i];
  const R phib = delta + dphi;
  R ldphi = lg[0], lphib = R(0);  // g0 = dphi - sum_{i != 0} g_i
#pragma unroll
  for (int i = 1; i < 9; ++i) {
    const R lt = lg[i] - lg[0];
    if ((umask >> i) & 1) {
      const R a = (R)(6.0 * awt(i));
      ld[aopp(i)] += lt;
      lphib += a * ((R)aex(i) * ubx + (R)aey(i) * uby) * lt;
      lubx += a * phib * (R)aex(i) * lt;
      luby += a * phib * (R)aey(i) * lt;
    } else {
      ld[i] += lt;
    }
  }
  ldphi += lphib;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    if (i != 0 && ((umask >> i) & 1)) lpm[i] += ldphi;
    else ld[i] += ldphi;
  }
}

// Pass 1: local reverse of the collision, source, history and CNEBB.
// float32: a budget of 128 registers (two CTAs per SM) trades a few spills
// for twice the warps in flight; float64 keeps its full register file.
template <typename R, int MODE, bool OPEN>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 2 : 1)
    adj_local(const InstDev* __restrict__ Dp, AdjArgs<R> A) {
  const InstDev& D = *Dp;
  const int nx = D.nx, ny = D.ny, S = D.stride, n = nx * ny;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int x = k % nx, y = k / nx;
  const bool py = D.periodic_y != 0;
  const bool wb = !py && y == 0, wt = !py && y == ny - 1;
  // an open column's node takes completed populations (no wall completion)
  const bool ocol = OPEN && MODE != kAdjInit && adj_open_column(D, x);
  const bool walls = (MODE != kAdjInit) && (wb || wt) && !ocol;
  if (A.mask && A.mask[k]) {
    // a solid node takes no part: every lambda it would carry is zero
#pragma unroll
    for (int q = 9; q < 36; ++q) A.lam_pulled[(size_t)q * S + k] = R(0);
#pragma unroll
    for (int j = 0; j < 6; ++j) A.lam_G[(size_t)j * S + k] = R(0);
#pragma unroll
    for (int j = 0; j < 3; ++j) A.lam_dir[(size_t)j * S + k] = R(0);
#pragma unroll
    for (int j = 0; j < 8; ++j) A.lam_mh[(size_t)j * S + k] = R(0);
    if (MODE != kAdjInit) {
#pragma unroll
      for (int j = 0; j < 5; ++j) A.lam_cur[(size_t)(36 + j) * S + k] = R(0);
    }
    return;
  }
  const int wrec = (MODE != kAdjInit && A.widx) ? A.widx[k] : -1;  // wall record (mask)
  const int umask = wrec >= 0 ? A.walls[wrec].umask : 0;

  // ---- forward recompute ----
  R d[9], Fx, Fy, rho, ux, uy;
  HydroM<R> hm;
  adj_hydro_node<R, MODE, OPEN>(D, A, x, y, d, Fx, Fy, hm, rho, ux, uy);
  int rm, rp;
  neighbour_rows(y, nx, ny, py, rm, rp);
  const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
  R g[3][9], gp[3][9], post[3][3], pm[3][9];
  CdeM<R> cm[3];
  if (ocol) {
    ColState<R> C;
    adj_column_state<R>(D, A.X, A.force, x == 0 ? 0 : 1, y, C);
    R dd[9];
    column_complete<R>(D, x == 0 ? 0 : 1, y, C, dd, g);
  }
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    if (MODE == kAdjInit) {
      PopSource<R, kModeInit>::cde(A.init, l, S, nx, k, y * nx, rm, rp, x, xm, xp, g[l]);
    } else if (!ocol) {
      pull9<R>(A.X + (size_t)(9 + 9 * l) * S, S, y * nx, rm, rp, x, xm, xp, g[l]);
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) gp[l][i] = g[l][i];  // pulled, before completion
    post[l][0] = post[l][1] = post[l][2] = R(0);
    if (walls) {
      const R* own = A.X + (size_t)(9 + 9 * l) * S + k;
      post[l][0] = own[(wb ? 4 : 2) * S];
      post[l][1] = own[(wb ? 7 : 5) * S];
      post[l][2] = own[(wb ? 8 : 6) * S];
      double wi, wo;
      cnebb<R>(g[l], post[l][0], post[l][1], post[l][2], (l == 1) ? R(0) : R(1), ux, uy, wb, wi,
               wo);
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) pm[l][i] = R(0);
    if (umask) {
      const R* own = A.X + (size_t)(9 + 9 * l) * S + k;
#pragma unroll
      for (int i = 1; i < 9; ++i)
        if ((umask >> i) & 1) pm[l][i] = own[(size_t)aopp(i) * S];
      cnebb_mask<R>(g[l], pm[l], (l == 1) ? R(0) : R(1), ux, uy, umask);
    }
    cde_moments<R>(g[l], cm[l]);
  }

  R lrho = R(0), lux = R(0), luy = R(0);         // direct lambdas of rho, u
  R lm[8] = {R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0)};  // raw hydro moments
  R lG[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};                // G00 G01 G10 G11 dPx dPy
  R lcm[3][6];                                                   // raw CDE moments
  R lFx = R(0), lFy = R(0);
#pragma unroll
  for (int l = 0; l < 3; ++l)
#pragma unroll
    for (int j = 0; j < 6; ++j) lcm[l][j] = R(0);

  if (MODE == kAdjFields) {
    // the loss enters through the fields of this step; nothing flows to the history
    R* lh = A.lam_cur + (size_t)36 * S;
#pragma unroll
    for (int j = 0; j < 5; ++j) lh[(size_t)j * S + k] = R(0);
    lrho = (R)A.lam_fields[k];
    lux = (R)A.lam_fields[n + k];
    luy = (R)A.lam_fields[2 * n + k];
#pragma unroll
    for (int l = 0; l < 3; ++l) lcm[l][0] = (R)A.lam_fields[(3 + l) * n + k];
  } else {
    // ---- forward recompute of gradients, source, coefficients ----
    const R* Mr = A.M;
    const R* Mx = A.M + S;
    const R* My = A.M + 2 * S;
    // the step's difference rules (central, wall rows, next to solids)
    R G00 = R(0), G01 = R(0), dPx = R(0), G10 = R(0), G11 = R(0), dPy = R(0);
    if (!A.mask && !wb && !wt && !(OPEN && adj_open_column(D, x))) {
      // central differences along both axes: the general rule's result, term
      // by term in the same order, without looking the rule up
      const int kxm = y * nx + adj_wrap(x - 1, nx), kxp = y * nx + adj_wrap(x + 1, nx);
      const int kym = adj_node(D, x, y - 1), kyp = adj_node(D, x, y + 1);
      const R cm_ = R(-0.5), cp_ = R(0.5);
      G00 += cm_ * Mx[kxm];
      G01 += cm_ * My[kxm];
      dPx += cm_ * (Mr[kxm] * Mx[kxm] * Mx[kxm] * Mx[kxm]);
      G10 += cm_ * Mx[kym];
      G11 += cm_ * My[kym];
      dPy += cm_ * (Mr[kym] * My[kym] * My[kym] * My[kym]);
      G00 += cp_ * Mx[kxp];
      G01 += cp_ * My[kxp];
      dPx += cp_ * (Mr[kxp] * Mx[kxp] * Mx[kxp] * Mx[kxp]);
      G10 += cp_ * Mx[kyp];
      G11 += cp_ * My[kyp];
      dPy += cp_ * (Mr[kyp] * My[kyp] * My[kyp] * My[kyp]);
    } else {
      double cx[5], cy[5];
      diff_coefs(D, A.mask, x, y, 0, cx);
      diff_coefs(D, A.mask, x, y, 1, cy);
#pragma unroll
      for (int j = -2; j <= 2; ++j) {
        if (cx[j + 2] != 0.0) {
          const int kj = adj_node(D, x + j, y);
          const R c = (R)cx[j + 2];
          G00 += c * Mx[kj];
          G01 += c * My[kj];
          dPx += c * (Mr[kj] * Mx[kj] * Mx[kj] * Mx[kj]);
        }
        if (cy[j + 2] != 0.0) {
          const int kj = adj_node(D, x, y + j);
          const R c = (R)cy[j + 2];
          G10 += c * Mx[kj];
          G11 += c * My[kj];
          dPy += c * (Mr[kj] * My[kj] * My[kj] * My[kj]);
        }
      }
    }
    const R Axx = R(1) + cm[0].dphi, Axy = cm[1].dphi, Ayy = R(1) + cm[2].dphi;
    const R mpl = coef<R>(D, kCoefMupLam), il = coef<R>(D, kCoefInvLam);
    const R div = G00 + G11;
    R Sc[3];
    Sc[0] = -cm[0].dphi * il + R(2) * (Axx * G00 + Axy * G10) + Axx * div;
    Sc[1] = -cm[1].dphi * il + (Axx * G01 + Axy * G11) + (Axy * G00 + Ayy * G10) + Axy * div;
    Sc[2] = -cm[2].dphi * il + R(2) * (Axy * G01 + Ayy * G11) + Ayy * div;
    R So[3], uxo, uyo;
    if (MODE == kAdjInit) {
      So[0] = Sc[0];
      So[1] = Sc[1];
      So[2] = Sc[2];
      uxo = ux;
      uyo = uy;
    } else {
      const R* h = A.X + (size_t)36 * S;
      So[0] = h[k];
      So[1] = h[S + k];
      So[2] = h[2 * S + k];
      uxo = h[3 * S + k];
      uyo = h[4 * S + k];
    }

    // ---- lambda of the step outputs ----
    R lout[4][9], lH[5];
#pragma unroll
    for (int q = 0; q < 36; ++q) lout[q / 9][q % 9] = A.lam_next[(size_t)q * S + k];
#pragma unroll
    for (int j = 0; j < 5; ++j) lH[j] = A.lam_next[(size_t)(36 + j) * S + k];
    // history out = (S, u)
    R lS[3] = {lH[0], lH[1], lH[2]};
    lux += lH[3];
    luy += lH[4];
    R lSo[3] = {R(0), R(0), R(0)}, luxo = R(0), luyo = R(0);

    // ---- hydro collision reverse ----
    {
      const R cs2 = R(1.0 / 3.0);
      const R c1 = coef<R>(D, kCoefCs1), c2 = coef<R>(D, kCoefCs2);
      const R h1 = coef<R>(D, kCoefHs1), w1 = coef<R>(D, kCoefWs1);
      R lb0, lbx, lby, lbxx, lbyy, lbxy, lbxxy, lbxyy;
      reconstruct_T<R>(lout[0], lb0, lbx, lby, lbxx, lbyy, lbxy, lbxxy, lbxyy);
      // b0' = drho; bx = jx + Fx; by = jy + Fy
      lm[0] += lb0;
      lm[1] += lbx;
      lm[2] += lby;
      lFx += lbx;
      lFy += lby;
      // bxx = (1-c1) rho ux^2 + c1 pxx - c1 cs2 drho - h1 dPx - w1 mpl dphi_xx, etc.
      lm[3] += c1 * lbxx;
      lm[4] += c1 * lbyy;
      lm[5] += c1 * lbxy;
      lm[0] += -c1 * cs2 * (lbxx + lbyy);
      lG[4] += -h1 * lbxx;
      lG[5] += -h1 * lbyy;
      lcm[0][0] += -w1 * mpl * lbxx;
      lcm[1][0] += -w1 * mpl * lbxy;
      lcm[2][0] += -w1 * mpl * lbyy;
      // bxxy = (1-c2) rho ux^2 uy + c2 qxxy - c2 cs2 jy; bxyy likewise with jx
      lm[6] += c2 * lbxxy;
      lm[7] += c2 * lbxyy;
      lm[2] += -c2 * cs2 * lbxxy;
      lm[1] += -c2 * cs2 * lbxyy;
      const R q1 = (R(1) - c1) * lbxx, q2 = (R(1) - c1) * lbyy, q3 = (R(1) - c1) * lbxy;
      const R q4 = (R(1) - c2) * lbxxy, q5 = (R(1) - c2) * lbxyy;
      // Q1 = rho ux^2, Q2 = rho uy^2, Q3 = rho ux uy, Q4 = rho ux^2 uy, Q5 = rho ux uy^2
      lrho += ux * ux * q1 + uy * uy * q2 + ux * uy * q3 + ux * ux * uy * q4 + ux * uy * uy * q5;
      lux += R(2) * rho * ux * q1 + rho * uy * q3 + R(2) * rho * ux * uy * q4 + rho * uy * uy * q5;
      luy += R(2) * rho * uy * q2 + rho * ux * q3 + rho * ux * ux * q4 + R(2) * rho * ux * uy * q5;
    }

    // ---- conformation collision reverse ----
    {
      const R cs2 = R(1.0 / 3.0);
      const R ep = coef<R>(D, kCoefEp1), c2 = coef<R>(D, kCoefCp2), h1 = coef<R>(D, kCoefHp1);
      const R e1 = ep - R(1);  // 1 - 1/tau_p1
#pragma unroll
      for (int l = 0; l < 3; ++l) {
        const R phi = (l == 1 ? R(0) : R(1)) + cm[l].dphi;
        R lc0, lcx, lcy, lcxx, lcyy, lcxy, u1, u2;
        reconstruct_T<R>(lout[1 + l], lc0, lcx, lcy, lcxx, lcyy, lcxy, u1, u2);
        R lphi = R(0);
        // c0p = dphi + 1.5 S - 0.5 So
        lcm[l][0] += lc0;
        lS[l] += R(1.5) * lc0;
        lSo[l] += R(-0.5) * lc0;
        // cx = (1-e1) phi ux + e1 jx + h1 phi Fx / rho + 1.5 h1 ux S - 0.5 h1 uxo So
        lphi += ((R(1) - e1) * ux + h1 * Fx / rho) * lcx + ((R(1) - e1) * uy + h1 * Fy / rho) * lcy;
        lux += ((R(1) - e1) * phi + R(1.5) * h1 * Sc[l]) * lcx;
        luy += ((R(1) - e1) * phi + R(1.5) * h1 * Sc[l]) * lcy;
        lcm[l][1] += e1 * lcx;
        lcm[l][2] += e1 * lcy;
        lFx += h1 * phi / rho * lcx;
        lFy += h1 * phi / rho * lcy;
        lrho += -h1 * phi * (Fx * lcx + Fy * lcy) / (rho * rho);
        lS[l] += R(1.5) * h1 * (ux * lcx + uy * lcy);
        luxo += R(-0.5) * h1 * So[l] * lcx;
        luyo += R(-0.5) * h1 * So[l] * lcy;
        lSo[l] += R(-0.5) * h1 * (uxo * lcx + uyo * lcy);
        // cxx = (1-c2) phi ux^2 + c2 pxx - c2 cs2 dphi, cyy, cxy = (1-c2) phi ux uy + c2 pxy
        const R k2 = R(1) - c2;
        lphi += k2 * (ux * ux * lcxx + uy * uy * lcyy + ux * uy * lcxy);
        lux += k2 * phi * (R(2) * ux * lcxx + uy * lcxy);
        luy += k2 * phi * (R(2) * uy * lcyy + ux * lcxy);
        lcm[l][3] += c2 * lcxx;
        lcm[l][4] += c2 * lcyy;
        lcm[l][5] += c2 * lcxy;
        lcm[l][0] += -c2 * cs2 * (lcxx + lcyy) + lphi;
      }
    }
    if (MODE == kAdjInit) {
      // history = current values: So = S, uo = u
#pragma unroll
      for (int l = 0; l < 3; ++l) lS[l] += lSo[l];
      lux += luxo;
      luy += luyo;
    } else {
      // lambda_t's history part
      R* lh = A.lam_cur + (size_t)36 * S;
      lh[k] = lSo[0];
      lh[S + k] = lSo[1];
      lh[2 * S + k] = lSo[2];
      lh[3 * S + k] = luxo;
      lh[4 * S + k] = luyo;
    }

    // ---- source reverse: S(A, grad u) ----
    {
      // S0
      lcm[0][0] += (-il + R(3) * G00 + G11) * lS[0];
      lcm[1][0] += R(2) * G10 * lS[0];
      lG[0] += R(3) * Axx * lS[0];
      lG[2] += R(2) * Axy * lS[0];
      lG[3] += Axx * lS[0];
      // S1
      lcm[0][0] += G01 * lS[1];
      lcm[1][0] += (-il + R(2) * G00 + R(2) * G11) * lS[1];
      lcm[2][0] += G10 * lS[1];
      lG[1] += Axx * lS[1];
      lG[3] += R(2) * Axy * lS[1];
      lG[0] += R(2) * Axy * lS[1];
      lG[2] += Ayy * lS[1];
      // S2
      lcm[1][0] += R(2) * G01 * lS[2];
      lcm[2][0] += (-il + G00 + R(3) * G11) * lS[2];
      lG[1] += R(2) * Axy * lS[2];
      lG[3] += R(3) * Ayy * lS[2];
      lG[0] += Ayy * lS[2];
    }
  }

  // ---- conformation moments -> completed populations -> CNEBB -> pulls ----
  if (MODE != kAdjInit) {
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      R lg[9];
      moments_T<R>(lcm[l][0], lcm[l][1], lcm[l][2], lcm[l][3], lcm[l][4], lcm[l][5], R(0), R(0),
                   lg);
      R ld[9];
      if (umask) {
        R lpm[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) ld[i] = lpm[i] = R(0);
        cnebb_mask_T<R>(gp[l], pm[l], (l == 1) ? R(0) : R(1), ux, uy, umask, lg, ld, lpm, lux,
                        luy);
        // unknown slots carry lambda of the own posts toward the wall
#pragma unroll
        for (int i = 1; i < 9; ++i)
          if ((umask >> i) & 1) ld[i] = lpm[i];
      } else if (walls) {
#pragma unroll
        for (int i = 0; i < 9; ++i) ld[i] = R(0);
        R lpost[3] = {R(0), R(0), R(0)};
        cnebb_T<R>(gp[l], post[l][0], post[l][1], post[l][2], (l == 1) ? R(0) : R(1), ux, uy,
                   wb, lg, ld, lpost, lux, luy);
        // unknown slots carry lambda of the own outgoing-to-wall slots (opposites)
        if (wb) {  // U = {2, 5, 6} <- H = {4, 7, 8}
          ld[2] = lpost[0];
          ld[5] = lpost[1];
          ld[6] = lpost[2];
        } else {  // U = {4, 7, 8} <- H = {2, 5, 6}
          ld[4] = lpost[0];
          ld[7] = lpost[1];
          ld[8] = lpost[2];
        }
      } else {
#pragma unroll
        for (int i = 0; i < 9; ++i) ld[i] = lg[i];
      }
      R* lp = A.lam_pulled + (size_t)(9 + 9 * l) * S + k;
#pragma unroll
      for (int i = 0; i < 9; ++i) lp[(size_t)i * S] = ld[i];
    }
  }
  A.lam_G[k] = lG[0];
  A.lam_G[S + k] = lG[1];
  A.lam_G[2 * S + k] = lG[2];
  A.lam_G[3 * S + k] = lG[3];
  A.lam_G[4 * S + k] = lG[4];
  A.lam_G[5 * S + k] = lG[5];
  A.lam_dir[k] = lrho;
  A.lam_dir[S + k] = lux;
  A.lam_dir[2 * S + k] = luy;
#pragma unroll
  for (int j = 0; j < 8; ++j) A.lam_mh[(size_t)j * S + k] = lm[j];
  A.dF[k] += (double)lFx;
  A.dF[n + k] += (double)lFy;
}

// Pass 2: gather the transposed gradient stencils, reverse u = (j + F/2)/rho
// and the hydro moments, reverse Zou-He; writes lambda of the hydro pulls and
// accumulates dL/dF.
template <typename R, int MODE, bool OPEN>
__global__ void adj_gather(const InstDev* __restrict__ Dp, AdjArgs<R> A) {
  const InstDev& D = *Dp;
  const int nx = D.nx, ny = D.ny, S = D.stride, n = nx * ny;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int x = k % nx, y = k / nx;
  const bool py = D.periodic_y != 0;
  if (A.mask && A.mask[k]) {
#pragma unroll
    for (int i = 0; i < 9; ++i) A.lam_pulled[(size_t)i * S + k] = R(0);
    return;
  }
  const R rho = A.M[k], ux = A.M[S + k], uy = A.M[2 * S + k];
  R lrho = A.lam_dir[k], lux = A.lam_dir[S + k], luy = A.lam_dir[2 * S + k];
  // transposed difference stencils: every fluid node kk within two nodes
  // along an axis whose difference reads this node with coefficient c
  {
    R lcx = R(0), lcy = R(0);
    if (!A.mask && (py || (y >= 3 && y <= ny - 4)) && !(OPEN && (x < 3 || x > nx - 4))) {
      // every stencil reaching this node is central (no mask, no wall row
      // within two rows): the general loop's terms in the same order
      const int kxp = y * nx + adj_wrap(x + 1, nx), kxm = y * nx + adj_wrap(x - 1, nx);
      const int kyp = adj_node(D, x, y + 1), kym = adj_node(D, x, y - 1);
      const R cm_ = R(-0.5), cp_ = R(0.5);
      lux += cm_ * A.lam_G[kxp];
      luy += cm_ * A.lam_G[S + kxp];
      lcx += cm_ * A.lam_G[4 * S + kxp];
      lux += cp_ * A.lam_G[kxm];
      luy += cp_ * A.lam_G[S + kxm];
      lcx += cp_ * A.lam_G[4 * S + kxm];
      lux += cm_ * A.lam_G[2 * S + kyp];
      luy += cm_ * A.lam_G[3 * S + kyp];
      lcy += cm_ * A.lam_G[5 * S + kyp];
      lux += cp_ * A.lam_G[2 * S + kym];
      luy += cp_ * A.lam_G[3 * S + kym];
      lcy += cp_ * A.lam_G[5 * S + kym];
    } else {
#pragma unroll
    for (int axis = 0; axis < 2; ++axis)
#pragma unroll
      for (int j = -2; j <= 2; ++j) {
        const int xk = x - (axis == 0 ? j : 0), yk = y - (axis == 1 ? j : 0);
        const int kk = adj_node(D, xk, yk);
        if (kk < 0 || (A.mask && A.mask[kk])) continue;
        double c[5];
        diff_coefs(D, A.mask, adj_wrap(xk, nx), kk / nx, axis, c);
        const R cj = (R)c[j + 2];
        if (cj == R(0)) continue;
        if (axis == 0) {
          lux += cj * A.lam_G[kk];
          luy += cj * A.lam_G[S + kk];
          lcx += cj * A.lam_G[4 * S + kk];
        } else {
          lux += cj * A.lam_G[2 * S + kk];
          luy += cj * A.lam_G[3 * S + kk];
          lcy += cj * A.lam_G[5 * S + kk];
        }
      }
    }
    // cx = rho ux^3, cy = rho uy^3
    lrho += ux * ux * ux * lcx + uy * uy * uy * lcy;
    lux += R(3) * rho * ux * ux * lcx;
    luy += R(3) * rho * uy * uy * lcy;
  }
  // u = (j + F/2) / rho, rho = 1 + drho
  R lm[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) lm[j] = (MODE == kAdjFields) ? R(0) : A.lam_mh[(size_t)j * S + k];
  lm[1] += lux / rho;
  lm[2] += luy / rho;
  lm[0] += lrho - (ux * lux + uy * luy) / rho;
  R lFx = R(0.5) * lux / rho, lFy = R(0.5) * luy / rho;
  if (MODE != kAdjInit) {
    R ld[9];
    moments_T<R>(lm[0], lm[1], lm[2], lm[3], lm[4], lm[5], lm[6], lm[7], ld);
    // Zou-He on wall rows; an open column's node is completed by the column
    // pass instead (adj_column takes its lambda back to the neighbour)
    const bool wb = !py && y == 0, wt = !py && y == ny - 1;
    if ((wb || wt) && !(OPEN && adj_open_column(D, x))) zou_he_T<R>(ld, lFx, lFy, wb);
    if (A.final_pass && A.widx && A.widx[k] >= 0) {
      // the loss's share of the final step's force on the solid: e_ib (f^dagger_ib +
      // f_i) over the wall links (eq_F_x); here the f_i part (the completed links)
      const int um = A.walls[A.widx[k]].umask;
#pragma unroll
      for (int i = 1; i < 9; ++i)
        if ((um >> i) & 1) ld[i] -= (R)(A.drag_w[0] * aex(i) + A.drag_w[1] * aey(i));
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) A.lam_pulled[(size_t)i * S + k] = ld[i];
  }
  A.dF[k] += (double)lFx;
  A.dF[n + k] += (double)lFy;
}

// Pass 2b (open channels, after the gather): reverse of the column pass.
// One thread per open-column node (side, y).  The gather and the local pass
// left there lambda of the node's completed populations; they go back to the
// neighbour x_f's pulled populations (the unknown slots of a wall row carry
// lambda of its own outgoing-to-wall slots, as in adj_local), and through the
// neighbour's rho, u and phi to its moments and force.  The open node's own
// entries are then cleared: it pulls nothing.
template <typename R, int MODE>
__global__ void adj_column(const InstDev* __restrict__ Dp, AdjArgs<R> A) {
  const InstDev& D = *Dp;
  const int nx = D.nx, ny = D.ny, S = D.stride, n = nx * ny;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (!D.open_x || t >= 2 * ny) return;
  const int side = t / ny, y = t % ny;
  const int kc = y * nx + (side == 0 ? 0 : nx - 1);
  R lc[36];
#pragma unroll
  for (int q = 0; q < 36; ++q) {
    lc[q] = A.lam_pulled[(size_t)q * S + kc];
    A.lam_pulled[(size_t)q * S + kc] = R(0);
  }
  ColState<R> C;
  adj_column_state<R>(D, A.X, A.force, side, y, C);
  const R rho = C.rho, ux = C.ux, uy = C.uy;
  R lrho = R(0), lux = R(0), luy = R(0);
  R ld[9], lg[3][9];
#pragma unroll
  for (int i = 0; i < 9; ++i) ld[i] = lc[i];
#pragma unroll
  for (int l = 0; l < 3; ++l)
#pragma unroll
    for (int i = 0; i < 9; ++i) lg[l][i] = lc[9 + 9 * l + i];
  R b0, b1, b2, b3, b4, b5, b6, b7;
  reconstruct_T<R>(lc, b0, b1, b2, b3, b4, b5, b6, b7);
  if (side == 0) {
    const double* in = D.inlet;
    const R bx = (R)in[y], by = (R)in[ny + y];
    // coefficients rho (b - u) ... of the hydrodynamic equilibrium difference
    lrho += (bx - ux) * b1 + (by - uy) * b2 + (bx * bx - ux * ux) * b3 + (by * by - uy * uy) * b4 +
            (bx * by - ux * uy) * b5 + (bx * bx * by - ux * ux * uy) * b6 +
            (bx * by * by - ux * uy * uy) * b7;
    lux += -rho * b1 - R(2) * rho * ux * b3 - rho * uy * b5 - R(2) * rho * ux * uy * b6 -
           rho * uy * uy * b7;
    luy += -rho * b2 - R(2) * rho * uy * b4 - rho * ux * b5 - rho * ux * ux * b6 -
           R(2) * rho * ux * uy * b7;
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      R m0, m1, m2, m3, m4, m5, m6, m7;
      reconstruct_T<R>(lc + 9 + 9 * l, m0, m1, m2, m3, m4, m5, m6, m7);
      const R phif = C.phi[l];
      // coefficients phi_b b - phi_f u ...: d/dphi_f and d/du
      const R lphif = -m0 - ux * m1 - uy * m2 - ux * ux * m3 - uy * uy * m4 - ux * uy * m5;
      lux += -phif * m1 - R(2) * phif * ux * m3 - phif * uy * m5;
      luy += -phif * m2 - R(2) * phif * uy * m4 - phif * ux * m5;
      // phi_f = delta + sum of the completed g_f
#pragma unroll
      for (int i = 0; i < 9; ++i) lg[l][i] += lphif;
    }
  } else {
    // coefficients (1 - rho) (1, u, u u, u u u) of the outlet's difference
    const R dr = R(1) - rho;
    const R ldr = b0 + ux * b1 + uy * b2 + ux * ux * b3 + uy * uy * b4 + ux * uy * b5 +
                  ux * ux * uy * b6 + ux * uy * uy * b7;
    lrho += -ldr;
    lux += dr * (b1 + R(2) * ux * b3 + uy * b5 + R(2) * ux * uy * b6 + uy * uy * b7);
    luy += dr * (b2 + R(2) * uy * b4 + ux * b5 + ux * ux * b6 + R(2) * ux * uy * b7);
  }
  // the neighbour's CNEBB on wall rows (u_b = its u)
  R lgp[3][9];
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    if (C.wb || C.wt) {
#pragma unroll
      for (int i = 0; i < 9; ++i) lgp[l][i] = R(0);
      R lpost[3] = {R(0), R(0), R(0)};
      cnebb_T<R>(C.gp[l], C.post[l][0], C.post[l][1], C.post[l][2], (l == 1) ? R(0) : R(1), ux,
                 uy, C.wb, lg[l], lgp[l], lpost, lux, luy);
      if (C.wb) {  // U = {2, 5, 6} <- H = {4, 7, 8}
        lgp[l][2] = lpost[0];
        lgp[l][5] = lpost[1];
        lgp[l][6] = lpost[2];
      } else {     // U = {4, 7, 8} <- H = {2, 5, 6}
        lgp[l][4] = lpost[0];
        lgp[l][7] = lpost[1];
        lgp[l][8] = lpost[2];
      }
    } else {
#pragma unroll
      for (int i = 0; i < 9; ++i) lgp[l][i] = lg[l][i];
    }
  }
  // u = (j + F/2) / rho, rho = 1 + drho, moments of the completed d_f
  R lFx = R(0.5) * lux / rho, lFy = R(0.5) * luy / rho;
  R lm[9];
  moments_T<R>(lrho - (ux * lux + uy * luy) / rho, lux / rho, luy / rho, R(0), R(0), R(0), R(0),
               R(0), lm);
#pragma unroll
  for (int i = 0; i < 9; ++i) ld[i] += lm[i];
  if (C.wb || C.wt) zou_he_T<R>(ld, lFx, lFy, C.wb);
  const int kf = C.kf;
#pragma unroll
  for (int i = 0; i < 9; ++i) A.lam_pulled[(size_t)i * S + kf] += ld[i];
#pragma unroll
  for (int l = 0; l < 3; ++l)
#pragma unroll
    for (int i = 0; i < 9; ++i) A.lam_pulled[(size_t)(9 + 9 * l + i) * S + kf] += lgp[l][i];
  A.dF[kf] += (double)lFx;
  A.dF[n + kf] += (double)lFy;
}

// Pass 3: reverse pull.  lambda_t(y, i) = lambda_pulled(y + e_i, i).  A
// population that leaves toward a flat wall or a solid node is not pulled by
// anyone; instead:
//   conformation lattices: CNEBB's lambda of the own post, kept in the
//     opposite (unknown) slot of y;
//   hydrodynamic lattice at a mask wall: the interpolated bounce-back
//     weights -- 2q, 1 or 1/(2q) on the own opposite post -- plus, on the
//     final pass, the loss's share of the force on the solid.
// The interpolation's other operands add 1 - 1/(2q) (the own post in the
// same direction, q >= 1/2) and 1 - 2q (the next node's post, q < 1/2), and
// each wall link adds lambda of its completed population times dv/dq to
// dL/dq.  A population that leaves an open channel through its inlet or
// outlet reads the (cleared) entries of the far open column: zero.
template <typename R>
__global__ void adj_pull(const InstDev* __restrict__ Dp, AdjArgs<R> A) {
  const InstDev& D = *Dp;
  const int nx = D.nx, S = D.stride, n = nx * D.ny;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int x = k % nx, y = k / nx;
  if (A.mask && A.mask[k]) {
#pragma unroll
    for (int q = 0; q < 36; ++q) A.lam_cur[(size_t)q * S + k] = R(0);
    return;
  }
  const int wrec = A.widx ? A.widx[k] : -1;
  const WallDev* W = wrec >= 0 ? &A.walls[wrec] : nullptr;
  // every value is gathered before the first store: lam_cur and lam_pulled
  // are distinct buffers, but the compiler cannot know it, and interleaved
  // stores would hold each load back behind the previous one
  R vals[36];
#pragma unroll
  for (int l = 0; l < 4; ++l) {
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const int kd = adj_node(D, x + aex(i), y + aey(i));
      const R* lp = A.lam_pulled + (size_t)(9 * l) * S;
      R v = R(0);
      if (kd >= 0 && !(A.mask && A.mask[kd])) {
        v = lp[(size_t)i * S + kd];
      } else if (l > 0) {
        v = lp[(size_t)aopp(i) * S + k];  // CNEBB's own slot
      } else if (kd >= 0 && W) {
        // into the mask: the wall link aopp(i) of this node
        const int j = aopp(i);
        const double q = W->q[j - 1];
        const double c = q < 0.5 ? (((W->fmask >> j) & 1) ? 2.0 * q : 1.0) : 1.0 / (2.0 * q);
        v = (R)c * lp[(size_t)j * S + k];
        if (A.final_pass) v += (R)(A.drag_w[0] * aex(i) + A.drag_w[1] * aey(i));
      }
      if (l == 0) {
        // the "same direction" operand of this node's own link i (q >= 1/2)
        if (W && i != 0 && ((W->umask >> i) & 1) && W->q[i - 1] >= 0.5)
          v += (R)(1.0 - 1.0 / (2.0 * W->q[i - 1])) * lp[(size_t)i * S + k];
        // the "next node" operand of the link aopp(i) of node k + e_i (q < 1/2)
        if (i != 0 && kd >= 0 && A.widx && !(A.mask && A.mask[kd]) && A.widx[kd] >= 0) {
          const WallDev& Wb = A.walls[A.widx[kd]];
          const int j = aopp(i);
          if (((Wb.umask >> j) & 1) && ((Wb.fmask >> j) & 1) && Wb.q[j - 1] < 0.5)
            v += (R)(1.0 - 2.0 * Wb.q[j - 1]) * lp[(size_t)j * S + kd];
        }
      }
      vals[9 * l + i] = v;
    }
  }
#pragma unroll
  for (int q = 0; q < 36; ++q) A.lam_cur[(size_t)q * S + k] = vals[q];
  if (W && A.dq) {
    // dL/dq of this node's wall links: lambda of the completed population
    // times its derivative in q (the raw state X of this step)
#pragma unroll
    for (int j = 1; j < 9; ++j) {
      if (!((W->umask >> j) & 1)) continue;
      const double q = W->q[j - 1];
      const double fb = (double)A.X[(size_t)aopp(j) * S + k];
      double dv = 0.0;
      if (q < 0.5) {
        if ((W->fmask >> j) & 1) {
          const int kf = adj_node(D, x + aex(j), y + aey(j));
          dv = 2.0 * (fb - (double)A.X[(size_t)aopp(j) * S + kf]);
        }
      } else {
        dv = ((double)A.X[(size_t)j * S + k] - fb) / (2.0 * q * q);
      }
      A.dq[(size_t)(j - 1) * n + k] += (double)A.lam_pulled[(size_t)j * S + k] * dv;
    }
  }
}

}  // namespace lbve
