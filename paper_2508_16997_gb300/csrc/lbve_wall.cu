// lbve_wall.cu -- wall pass of the solid mask and column pass of open
// channels (hand-written CUDA, sm_103a).
//
// Runs before every step on the compact list of fluid nodes next to solid
// nodes (one thread per node).  For each wall link (x_b, i), i.e. x_b - e_i
// solid, it computes the population that arrives at x_b along e_i and
// stores it in the solid node's slot i, which is exactly where the step
// kernel's pull of x_b reads it.  So the fused step needs no wall logic for
// the mask: it pulls completed populations everywhere.
//   - Hydrodynamic lattice: linear interpolated bounce-back (Bouzidi,
//     Firdaouss & Lallemand 2001) at wall fraction q; q = 1/2 is half-way
//     bounce-back.  It stands in for the curved-wall scheme of Sec. 4.3.
//   - Conformation lattices: CNEBB (Sec. 3.3) with u_b from the completed
//     hydrodynamic populations; the closing rest population is written to
//     the node's own rest slot (only this node pulls it).
//   - Final step: the momentum-exchange force on the solid (eq_F_x) and the
//     CNEBB wall in/out amounts, float64, one record per wall node.
// Reads touch only fluid nodes' slots and writes only solid nodes' slots and
// the node's own rest slots, so the threads never race.
#include <cuda_runtime.h>

#include "lbve_internal.h"
#include "lbve_step.cuh"

namespace lbve {
namespace {

// D2Q9 velocities, opposites and weights (Sec. 3.1); with unrolled loops the
// index is a constant and these fold away.
__device__ __forceinline__ constexpr int ex(int i) {
  return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__device__ __forceinline__ constexpr int ey(int i) {
  return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
__device__ __forceinline__ constexpr int opp(int i) {
  return i == 0 ? 0 : (i <= 4 ? (i + 1) % 4 + 1 : (i + 1) % 4 + 5);
}
__device__ __forceinline__ constexpr double wt(int i) {
  return i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
}

constexpr int kWallThreads = 128;

template <typename R, bool FINAL>
__global__ void __launch_bounds__(kWallThreads)
    wall_kernel(const InstDev* __restrict__ insts, const WallDev* __restrict__ walls, int n,
                int parity, double* __restrict__ rec) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const WallDev W = walls[t];
  if (W.inst < 0) return;
  const InstDev& D = insts[W.inst];
  const int nx = D.nx, ny = D.ny, S = D.stride;
  const bool py = D.periodic_y != 0;
  R* __restrict__ p = (R*)D.pop[parity];
  const int k = W.k, x = k % nx, y = k / nx;
  // node k + s e_i; mask nodes lie at least three rows from a flat wall, so
  // no neighbour leaves a walled domain
  int nb_m[9], nb_p[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    int xm = x - ex(i), xp = x + ex(i), ym = y - ey(i), yp = y + ey(i);
    xm = xm < 0 ? xm + nx : (xm >= nx ? xm - nx : xm);
    xp = xp < 0 ? xp + nx : (xp >= nx ? xp - nx : xp);
    if (py) {
      ym = ym < 0 ? ym + ny : (ym >= ny ? ym - ny : ym);
      yp = yp < 0 ? yp + ny : (yp >= ny ? yp - ny : yp);
    }
    nb_m[i] = ym * nx + xm;
    nb_p[i] = yp * nx + xp;
  }
  const R Fx = D.force_field ? ((const R*)D.force)[k] : coef<R>(D, kCoefFx);
  const R Fy = D.force_field ? ((const R*)D.force)[S + k] : coef<R>(D, kCoefFy);

  // ---- every operand first: the loads issue together, before any store ----
  const R* __restrict__ ps = p;
  R d[9], a2[9];  // hydro: pulled population, or (wall link) own post toward the wall
                  // and the second interpolation operand
  R g[3][9];      // conformation: pulled population, or (wall link) own post
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    a2[i] = R(0);
    if (i != 0 && ((W.umask >> i) & 1)) {
      const int ib = opp(i);
      d[i] = ps[(size_t)ib * S + k];
      if (W.q[i - 1] < 0.5)
        a2[i] = ((W.fmask >> i) & 1) ? ps[(size_t)ib * S + nb_p[i]] : d[i];
      else
        a2[i] = ps[(size_t)i * S + k];
#pragma unroll
      for (int l = 0; l < 3; ++l) g[l][i] = ps[(size_t)(9 + 9 * l + ib) * S + k];
    } else {
      d[i] = ps[(size_t)i * S + nb_m[i]];
#pragma unroll
      for (int l = 0; l < 3; ++l) g[l][i] = ps[(size_t)(9 + 9 * l + i) * S + nb_m[i]];
    }
  }

  // ---- hydrodynamic lattice: interpolated bounce-back -----------------------
  double fdx = 0.0, fdy = 0.0;
#pragma unroll
  for (int i = 1; i < 9; ++i) {
    if (!((W.umask >> i) & 1)) continue;
    const double q = W.q[i - 1];
    const R fb = d[i];  // own post-collision toward the wall
    R v;
    if (q < 0.5) {
      // second operand: the next fluid node's post toward the wall (half-way
      // bounce-back, a2 = fb, where there is none)
      v = (R)(2.0 * q) * fb + (R)(1.0 - 2.0 * q) * a2[i];
    } else {
      const double a = 1.0 / (2.0 * q);
      v = (R)a * fb + (R)(1.0 - a) * a2[i];
    }
    p[(size_t)i * S + nb_m[i]] = v;
    d[i] = v;
    if (FINAL) {
      // eq_F_x: e_ib (f^dagger_ib + f_i) over the links to the wall
      const double sum = 2.0 * wt(i) + (double)fb + (double)v;
      fdx -= ex(i) * sum;
      fdy -= ey(i) * sum;
    }
  }
  HydroM<R> hm;
  hydro_moments<R>(d, hm);
  const R rho = R(1) + hm.drho;
  const R irho = R(1) / rho;
  const R ux = (hm.jx + R(0.5) * Fx) * irho;
  const R uy = (hm.jy + R(0.5) * Fy) * irho;

  // ---- conformation lattices: CNEBB -----------------------------------------
  double wio[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    R* __restrict__ pl = p + (size_t)(9 + 9 * l) * S;
    const R delta = (l == 1) ? R(0) : R(1);
    // phi_b = known pulled populations + own posts toward the wall
    R dphi = R(0);
    double out = 0.0;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      dphi += g[l][i];
      if (FINAL && i != 0 && ((W.umask >> i) & 1)) out += wt(i) * (double)delta + (double)g[l][i];
    }
    const R phib = delta + dphi;
    // g_i = g_ibar + g^eq_i - g^eq_ibar = g_ibar + 6 w_i phi_b (e_i . u_b); the
    // opposite of a wall link is never one
#pragma unroll
    for (int i = 1; i < 9; ++i)
      if ((W.umask >> i) & 1)
        g[l][i] = g[l][opp(i)] + (R)(6.0 * wt(i)) * phib * ((R)ex(i) * ux + (R)ey(i) * uy);
    R rest = R(0);
#pragma unroll
    for (int i = 1; i < 9; ++i) rest += g[l][i];
    const R g0_old = g[l][0];
    const R g0 = dphi - rest;
    double in = 0.0;
#pragma unroll
    for (int i = 1; i < 9; ++i)
      if ((W.umask >> i) & 1) {
        pl[(size_t)i * S + nb_m[i]] = g[l][i];
        if (FINAL) in += wt(i) * (double)delta + (double)g[l][i];
      }
    pl[k] = g0;
    if (FINAL) {
      wio[l] = in + ((double)g0 - (double)g0_old);
      wio[3 + l] = out;
    }
  }
  if (FINAL) {
    double* r = rec + (size_t)t * kWallRec;
    r[0] = fdx;
    r[1] = fdy;
#pragma unroll
    for (int j = 0; j < 6; ++j) r[2 + j] = wio[j];
  }
}

// ---------------------------------------------------------------------------
// Column pass of an open channel (Sec. 4.3 inlet/outlet), one thread per node
// of the two open columns.  The node's neighbour x_f (column 1 or nx - 2) is
// pulled and, on a wall row, completed (Zou-He, CNEBB) exactly as the step
// does; then every population of the open-column node follows by
// non-equilibrium extrapolation:
//   inlet:  f = f^eq(rho_f, u_in) - f^eq(rho_f, u_f) + f(x_f),
//           g = g^eq(A_in, u_in) - g^eq(phi_f, u_f) + g(x_f);
//   outlet: f = f^eq(1, u_f) - f^eq(rho_f, u_f) + f(x_f), g = g(x_f).
// The equilibrium differences are Hermite reconstructions of coefficient
// differences.  The result goes to the instance's colbuf, which the masked
// step reads in place of pulling these nodes; src is only read.
template <typename R>
__global__ void __launch_bounds__(kWallThreads)
    column_kernel(const InstDev* __restrict__ insts, const ColTask* __restrict__ tasks, int n,
                  int parity) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const ColTask T = tasks[t];
  if (T.inst < 0) return;
  const InstDev& D = insts[T.inst];
  const int nx = D.nx, ny = D.ny, S = D.stride, y = T.y, side = T.side;
  const bool py = D.periodic_y != 0;
  const R* __restrict__ src = (const R*)D.pop[parity];
  const int xf = side == 0 ? 1 : nx - 2;
  const int rc = y * nx, k = rc + xf;
  int rm, rp;
  neighbour_rows(y, nx, ny, py, rm, rp);
  const bool wb = !py && y == 0, wt = !py && y == ny - 1;
  const R Fx = D.force_field ? ((const R*)D.force)[k] : coef<R>(D, kCoefFx);
  const R Fy = D.force_field ? ((const R*)D.force)[S + k] : coef<R>(D, kCoefFy);
  R d[9], g[3][9];
  pull9<R>(src, S, rc, rm, rp, xf, xf - 1, xf + 1, d);
#pragma unroll
  for (int l = 0; l < 3; ++l)
    pull9<R>(src + (size_t)(9 + 9 * l) * S, S, rc, rm, rp, xf, xf - 1, xf + 1, g[l]);
  if (wb || wt) zou_he<R>(d, Fx, Fy, wb);
  HydroM<R> hm;
  hydro_moments<R>(d, hm);
  const R rho = R(1) + hm.drho;
  const R irho = R(1) / rho;
  const R ux = (hm.jx + R(0.5) * Fx) * irho, uy = (hm.jy + R(0.5) * Fy) * irho;
  if (wb || wt) {
    // bottom wall: H = {4, 7, 8}; top wall: H = {2, 5, 6}
    const int h0 = wb ? 4 : 2, h1 = wb ? 7 : 5, h2 = wb ? 8 : 6;
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      const R* own = src + (size_t)(9 + 9 * l) * S + k;
      double win, wout;
      cnebb<R>(g[l], own[h0 * S], own[h1 * S], own[h2 * S], (l == 1) ? R(0) : R(1), ux, uy, wb,
               win, wout);
    }
  }
  R* __restrict__ cb = (R*)D.colbuf;
  const int c = side * ny + y, ld = 2 * ny;
  R e[9];
  if (side == 0) {
    const double* in = D.inlet;
    const R bx = (R)in[y], by = (R)in[ny + y];
    reconstruct<R>(R(0), rho * (bx - ux), rho * (by - uy), rho * (bx * bx - ux * ux),
                   rho * (by * by - uy * uy), rho * (bx * by - ux * uy),
                   rho * (bx * bx * by - ux * ux * uy), rho * (bx * by * by - ux * uy * uy), e);
#pragma unroll
    for (int i = 0; i < 9; ++i) cb[(size_t)i * ld + c] = d[i] + e[i];
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      CdeM<R> m;
      cde_moments<R>(g[l], m);
      const R phif = ((l == 1) ? R(0) : R(1)) + m.dphi;
      const R phib = (R)in[(2 + l) * ny + y];
      reconstruct<R>(phib - phif, phib * bx - phif * ux, phib * by - phif * uy,
                     phib * bx * bx - phif * ux * ux, phib * by * by - phif * uy * uy,
                     phib * bx * by - phif * ux * uy, R(0), R(0), e);
#pragma unroll
      for (int i = 0; i < 9; ++i) cb[(size_t)(9 + 9 * l + i) * ld + c] = g[l][i] + e[i];
    }
  } else {
    const R dr = R(1) - rho;  // density rho_0 = 1 at the outlet
    reconstruct<R>(dr, dr * ux, dr * uy, dr * ux * ux, dr * uy * uy, dr * ux * uy,
                   dr * ux * ux * uy, dr * ux * uy * uy, e);
#pragma unroll
    for (int i = 0; i < 9; ++i) cb[(size_t)i * ld + c] = d[i] + e[i];
#pragma unroll
    for (int l = 0; l < 3; ++l)
#pragma unroll
      for (int i = 0; i < 9; ++i) cb[(size_t)(9 + 9 * l + i) * ld + c] = g[l][i];
  }
}

template <typename R>
int launch_wall_t(const InstDev* d_insts, const WallDev* d_walls, double* d_rec, int n,
                  int parity, int flags, cudaStream_t st) {
  if (n <= 0) return 0;
  const int grid = (n + kWallThreads - 1) / kWallThreads;
  if (flags & kFinal)
    wall_kernel<R, true><<<grid, kWallThreads, 0, st>>>(d_insts, d_walls, n, parity, d_rec);
  else
    wall_kernel<R, false><<<grid, kWallThreads, 0, st>>>(d_insts, d_walls, n, parity, d_rec);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;  // the caller reads and clears it
}

}  // namespace

int launch_column(int prec, const InstDev* d_insts, const ColTask* d_tasks, int n, int parity,
                  void* stream) {
  if (n <= 0) return 0;
  cudaStream_t st = (cudaStream_t)stream;
  const int grid = (n + kWallThreads - 1) / kWallThreads;
  if (prec == 0)
    column_kernel<double><<<grid, kWallThreads, 0, st>>>(d_insts, d_tasks, n, parity);
  else
    column_kernel<float><<<grid, kWallThreads, 0, st>>>(d_insts, d_tasks, n, parity);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;  // the caller reads and clears it
}

int launch_wall(int prec, const InstDev* d_insts, const WallDev* d_walls, double* d_rec, int n,
                int parity, int flags, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  if (prec == 0) return launch_wall_t<double>(d_insts, d_walls, d_rec, n, parity, flags, st);
  return launch_wall_t<float>(d_insts, d_walls, d_rec, n, parity, flags, st);
}

}  // namespace lbve
