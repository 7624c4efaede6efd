// lbve_step.cuh -- the fused coupled time step (hand-written CUDA, sm_103a).
//
// One CTA updates one tile of one instance.  Storage is structure-of-arrays,
// x fastest: 9 hydrodynamic planes then 3 x 9 conformation planes of
// post-collision populations, kept as deviations from the rest state
// (f_i - w_i, g^c_i - w_i delta_c), ping-pong between two buffers (pull
// scheme), plus 5 history planes (S_xx, S_xy, S_yy, ux, uy of the previous
// step) and an optional per-node body force.
//
// Per step, per node (paper Sec. 3):
//   pull-stream all 36 populations (eq_ev_f / eq_g0 left-hand sides);
//   complete wall rows: hydro wet-node bounce-back of the non-equilibrium part
//   (Zou-He, wall velocity 0), then CNEBB for each conformation lattice from
//   the node's own outgoing-to-wall post-collision slots (Sec. 3.3);
//   moments rho, u (eq_ev_f0), phi^c;
//   second-order finite differences of u, rho u_x^3, rho u_y^3 from a
//   one-node (two rows at walls) halo of moments held in shared memory;
//   Oldroyd-B stress (eq_kramer, eqb4) and source Phi_ab (Sec. 3.2);
//   TRT-RLB collisions of all four lattices, evaluated in Hermite moment
//   space: the regularised post-collision state is the projection onto
//   {1, H_a, H_ab, H_xxy, H_xyy} (the D2Q9 H_xxx, H_yyy vanish), so it is
//   rebuilt per direction from 8 (hydro) or 6 (conformation) coefficients.
//   This is algebraically identical to eq_ev_f / eq_g0 written per direction.
//
// Phase A computes rho, u on the tile plus halo into shared memory; phase B
// does the full update of the tile's own nodes.  Halo pulls hit L1/L2; each
// population is read from HBM once per step by the node that pulls it.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "lbve_df32.cuh"
#include "lbve_internal.h"

#ifndef LBVE_FP32_MIN_BLOCKS
#define LBVE_FP32_MIN_BLOCKS 7
#endif

namespace lbve {

// Exact float -> double conversion by integer operations: GB300 converts
// float to double on its float64 pipe (64 cycles per warp instruction),
// integer operations issue every cycle.  Zero, subnormal, normal, infinite
// and NaN inputs (IEEE 754 binary32 -> binary64: exponent rebiased by
// 1023 - 127, fraction shifted by 29 bits; subnormals normalised).
__device__ __forceinline__ double f2d_exact(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint64_t sign = (uint64_t)(b >> 31) << 63;
  const uint32_t e = (b >> 23) & 0xffu;
  const uint32_t m = b & 0x7fffffu;
  uint64_t r;
  if (e == 0xffu) {
    r = sign | 0x7ff0000000000000ull | ((uint64_t)m << 29);
  } else if (e != 0u) {
    r = sign | ((uint64_t)(e + 896u) << 52) | ((uint64_t)m << 29);
  } else if (m == 0u) {
    r = sign;
  } else {
    const int msb = 31 - __clz(m);  // 0..22: value 2^(msb - 149) (1 + fraction)
    r = sign | ((uint64_t)(msb + 874) << 52) | (((uint64_t)m << (52 - msb)) & 0xfffffffffffffull);
  }
  return __longlong_as_double((long long)r);
}
__device__ __forceinline__ double to_f64(float v) { return f2d_exact(v); }
__device__ __forceinline__ double to_f64(double v) { return v; }
__device__ __forceinline__ double to_f64(df32 v) { return f2d_exact(v.hi) + f2d_exact(v.lo); }

template <typename R>
struct HydroM {  // raw moments of the (deviation) populations
  R drho, jx, jy, pxx, pyy, pxy, qxxy, qxyy;
};
template <typename R>
struct CdeM {
  R dphi, jx, jy, pxx, pyy, pxy;
};

template <typename R>
__device__ __forceinline__ void hydro_moments(const R d[9], HydroM<R>& m) {
  const R s58 = (d[5] + d[6]) + (d[7] + d[8]);
  m.drho = ((d[0] + d[1]) + (d[2] + d[3])) + (d[4] + s58);
  m.jx = (d[1] - d[3]) + ((d[5] - d[6]) + (d[8] - d[7]));
  m.jy = (d[2] - d[4]) + ((d[5] + d[6]) - (d[7] + d[8]));
  m.pxx = (d[1] + d[3]) + s58;
  m.pyy = (d[2] + d[4]) + s58;
  m.pxy = (d[5] + d[7]) - (d[6] + d[8]);
  m.qxxy = (d[5] + d[6]) - (d[7] + d[8]);
  m.qxyy = (d[5] + d[8]) - (d[6] + d[7]);
}

template <typename R>
__device__ __forceinline__ void cde_moments(const R d[9], CdeM<R>& m) {
  const R s58 = (d[5] + d[6]) + (d[7] + d[8]);
  m.dphi = ((d[0] + d[1]) + (d[2] + d[3])) + (d[4] + s58);
  m.jx = (d[1] - d[3]) + ((d[5] - d[6]) + (d[8] - d[7]));
  m.jy = (d[2] - d[4]) + ((d[5] + d[6]) - (d[7] + d[8]));
  m.pxx = (d[1] + d[3]) + s58;
  m.pyy = (d[2] + d[4]) + s58;
  m.pxy = (d[5] + d[7]) - (d[6] + d[8]);
}

// Rebuild the nine (deviation) populations from Hermite coefficients:
//   d_i = w_i [ b0' + 3 e.b + 4.5 (H_xx bxx + 2 H_xy bxy + H_yy byy)
//               + 13.5 (H_xxy bxxy + H_xyy bxyy) ]
// with b0' the zeroth coefficient minus the rest value.
// Float32: the products with the weights are correctly rounded, w v =
// fmaf(v, w, v w_lo) with w + w_lo = 1/9 or 1/36 to 2^-48: multiplying by
// the rounded weights alone scales every moment the weights carry by
// sum_i fl(w_i) e_i e_i... = 1 + 7e-9 at every collision, a bias that the
// momentum (and the slowly relaxing conformation moments) accumulate over
// their relaxation times.  The rest population is taken as b0' minus the
// other eight, which equals its formula in exact arithmetic and keeps
// sum_i d_i = b0' up to unbiased rounding.  Float64 keeps the plain formula:
// its weight bias is ~1e-17, and the float64 step is bound by the FP64 pipe.
template <typename R>
__device__ __forceinline__ R wmul(R v, R w, R wlo) {
  if constexpr (sizeof(R) == 4)
    return fmaf(v, w, v * wlo);
  else
    return w * v;
}

template <typename R>
__device__ __forceinline__ void reconstruct(R b0p, R bx, R by, R bxx, R byy, R bxy, R bxxy,
                                            R bxyy, R out[9]) {
  const R w0 = R(4.0 / 9.0), w1 = R(1.0 / 9.0), w5 = R(1.0 / 36.0);
  // low parts of 1/9 and 1/36 below their float32 roundings
  constexpr float kW1lo = (float)(1.0 / 9.0 - (double)(float)(1.0 / 9.0));
  constexpr float kW5lo = (float)(1.0 / 36.0 - (double)(float)(1.0 / 36.0));
  const R w1lo = R(kW1lo), w5lo = R(kW5lo);
  const R s = bxx + byy;
  if constexpr (sizeof(R) == 8) out[0] = w0 * (b0p - R(1.5) * s);
  const R b13 = b0p + R(3.0) * bxx - R(1.5) * byy;
  const R o13 = R(3.0) * bx - R(4.5) * bxyy;
  out[1] = wmul<R>(b13 + o13, w1, w1lo);
  out[3] = wmul<R>(b13 - o13, w1, w1lo);
  const R b24 = b0p - R(1.5) * bxx + R(3.0) * byy;
  const R o24 = R(3.0) * by - R(4.5) * bxxy;
  out[2] = wmul<R>(b24 + o24, w1, w1lo);
  out[4] = wmul<R>(b24 - o24, w1, w1lo);
  const R bd = b0p + R(3.0) * s;
  const R xy9 = R(9.0) * bxy;
  const R o57 = R(3.0) * (bx + by) + R(9.0) * (bxxy + bxyy);
  const R o68 = R(3.0) * (by - bx) + R(9.0) * (bxxy - bxyy);
  out[5] = wmul<R>((bd + xy9) + o57, w5, w5lo);
  out[7] = wmul<R>((bd + xy9) - o57, w5, w5lo);
  out[6] = wmul<R>((bd - xy9) + o68, w5, w5lo);
  out[8] = wmul<R>((bd - xy9) - o68, w5, w5lo);
  if constexpr (sizeof(R) == 4)
    out[0] = b0p - (((out[1] + out[3]) + (out[2] + out[4])) + ((out[5] + out[7]) + (out[6] + out[8])));
}

// Pull the nine populations of one lattice arriving at (x, y): d_i(x) =
// post_i(x - e_i).  rm / rp are the row offsets of rows y-1 / y+1, or -1
// where that row is outside a walled domain (those directions stay unknown
// and are completed by the caller).
template <typename R>
__device__ __forceinline__ void pull9(const R* __restrict__ p, int S, int rc, int rm, int rp,
                                      int x, int xm, int xp, R d[9]) {
  d[0] = p[0 * S + rc + x];
  d[1] = p[1 * S + rc + xm];
  d[3] = p[3 * S + rc + xp];
  if (rm >= 0) {
    d[2] = p[2 * S + rm + x];
    d[5] = p[5 * S + rm + xm];
    d[6] = p[6 * S + rm + xp];
  } else {
    d[2] = d[5] = d[6] = R(0);
  }
  if (rp >= 0) {
    d[4] = p[4 * S + rp + x];
    d[7] = p[7 * S + rp + xp];
    d[8] = p[8 * S + rp + xm];
  } else {
    d[4] = d[7] = d[8] = R(0);
  }
}

// Hydrodynamic wet-node completion with zero wall velocity: sum e f = -F/2
// (so u = 0 through eq_ev_f0) and the wall-normal pair bounced back.  The
// paired weights are equal, so the formulas hold for deviations unchanged.
template <typename R>
__device__ __forceinline__ void zou_he(R d[9], R Fx, R Fy, bool bottom) {
  const R h = R(0.5) * (d[1] - d[3]);
  const R qx = R(0.25) * Fx, qy = R(0.25) * Fy;
  if (bottom) {
    d[2] = d[4];
    d[5] = d[7] - h - qx - qy;
    d[6] = d[8] + h + qx - qy;
  } else {
    d[4] = d[2];
    d[7] = d[5] + h + qx + qy;
    d[8] = d[6] - h - qx + qy;
  }
}

// CNEBB (Sec. 3.3) on deviations.  post_* are the node's own post-collision
// slots pointing toward the wall (H); the unknown directions U are their
// opposites.  phi_b = known incoming + sum_H post; unknown i gets
// g_i = g_ibar + (g^eq_i - g^eq_ibar) = g_ibar + 6 w_i phi_b (e_i . u_b);
// the rest population closes sum g = phi_b.  Returns the wall in/out amounts
// (full populations, float64).
template <typename R>
__device__ __forceinline__ void cnebb(R d[9], R post_a, R post_b, R post_c, R delta_c, R ubx,
                                      R uby, bool bottom, double& win, double& wout) {
  // bottom: H = {4, 7, 8}, U = {2, 5, 6};  top: H = {2, 5, 6}, U = {4, 7, 8}
  const R d0_old = d[0];
  R dphi;
  if (bottom) {
    dphi = ((d[0] + d[1]) + (d[3] + d[4])) + ((d[7] + d[8]) + ((post_a + post_b) + post_c));
  } else {
    dphi = ((d[0] + d[1]) + (d[3] + d[2])) + ((d[5] + d[6]) + ((post_a + post_b) + post_c));
  }
  const R phib = delta_c + dphi;
  const R a2 = R(6.0 / 9.0) * phib, a5 = R(6.0 / 36.0) * phib;
  if (bottom) {
    d[2] = d[4] + a2 * uby;
    d[5] = d[7] + a5 * (ubx + uby);
    d[6] = d[8] + a5 * (uby - ubx);
  } else {
    d[4] = d[2] - a2 * uby;
    d[7] = d[5] - a5 * (ubx + uby);
    d[8] = d[6] + a5 * (ubx - uby);
  }
  d[0] = dphi - (((d[1] + d[2]) + (d[3] + d[4])) + ((d[5] + d[6]) + (d[7] + d[8])));
  const double dc = to_f64(delta_c);
  wout = (to_f64(post_a) + to_f64(post_b) + to_f64(post_c)) + dc / 6.0;
  double added;
  if (bottom) added = to_f64(d[2]) + to_f64(d[5]) + to_f64(d[6]);
  else added = to_f64(d[4]) + to_f64(d[7]) + to_f64(d[8]);
  win = added + dc / 6.0 + (to_f64(d[0]) - to_f64(d0_old));
}

// One level of a transposed butterfly sum over a warp: each lane holds M
// partial sums; it keeps one half (the upper one when `up`), receives the
// partner's values of that half across lane distance o and adds them, so
// that after the levels 16, 8, 4, 2 (and a last pairwise sum across 1) lanes
// 2s and 2s + 1 hold the warp's total of value s, for 16 values with 16
// additions per lane instead of 5 per value.
template <int M>
__device__ __forceinline__ void fold_half(double* v, int o, bool up) {
#pragma unroll
  for (int j = 0; j < M / 2; ++j) {
    const double keep = up ? v[j + M / 2] : v[j];
    const double send = up ? v[j] : v[j + M / 2];
    v[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
  }
}

// Populations of one lattice at a node: pulled from the previous step
// (kModeStep) or the equilibrium of the staged initial fields (kModeInit).
template <typename R, int MODE>
struct PopSource;

template <typename R>
struct PopSource<R, kModeStep> {
  static __device__ __forceinline__ void hydro(const void* src, int S, int nx, int k, int rc,
                                               int rm, int rp, int x, int xm, int xp, R d[9]) {
    pull9<R>((const R*)src, S, rc, rm, rp, x, xm, xp, d);
  }
  static __device__ __forceinline__ void cde(const void* src, int l, int S, int nx, int k, int rc,
                                             int rm, int rp, int x, int xm, int xp, R d[9]) {
    pull9<R>((const R*)src + (size_t)(9 + 9 * l) * S, S, rc, rm, rp, x, xm, xp, d);
  }
};

template <typename R>
struct PopSource<R, kModeInit> {
  // staged fields: float64 [6][S] = rho, ux, uy, Axx, Axy, Ayy at node k
  static __device__ __forceinline__ void hydro(const void* src, int S, int nx, int k, int rc,
                                               int rm, int rp, int x, int xm, int xp, R d[9]) {
    const double* f = (const double*)src;
    const R r = (R)f[k], ux = (R)f[S + k], uy = (R)f[2 * S + k];
    // equilibrium (eq2): Hermite coefficients rho, rho u, rho uu, rho u_x^2 u_y, rho u_x u_y^2
    reconstruct<R>((R)(f[k] - 1.0), r * ux, r * uy, r * ux * ux, r * uy * uy, r * ux * uy,
                   r * ux * ux * uy, r * ux * uy * uy, d);
  }
  static __device__ __forceinline__ void cde(const void* src, int l, int S, int nx, int k, int rc,
                                             int rm, int rp, int x, int xm, int xp, R d[9]) {
    const double* f = (const double*)src;
    const R ux = (R)f[S + k], uy = (R)f[2 * S + k];
    const double A = f[(3 + l) * S + k];
    const R a = (R)A;
    const R ap = (R)(A - (l == 1 ? 0.0 : 1.0));
    // equilibrium (eq_geq): phi, phi u, phi uu
    reconstruct<R>(ap, a * ux, a * uy, a * ux * ux, a * uy * uy, a * ux * uy, R(0), R(0), d);
  }
};

// Row offsets of the rows y-1 and y+1 feeding the pull at row y (-1 outside
// a walled domain).
__device__ __forceinline__ void neighbour_rows(int y, int nx, int ny, bool py, int& rm, int& rp) {
  if (py) {
    rm = (y == 0 ? ny - 1 : y - 1) * nx;
    rp = (y == ny - 1 ? 0 : y + 1) * nx;
  } else {
    rm = y > 0 ? (y - 1) * nx : -1;
    rp = y < ny - 1 ? (y + 1) * nx : -1;
  }
}

// rho, u of node (gx, gy) at the current time: pull (or equilibrium at
// init), hydro wall completion, moments (eq_ev_f0).
template <typename R, int MODE>
__device__ __forceinline__ void node_rho_u(const void* src, const R* __restrict__ force,
                                           bool ffield, R Fx0, R Fy0, int S, int nx, int ny,
                                           bool py, int gx, int gy, R& rho, R& ux, R& uy) {
  const int k = gy * nx + gx;
  int rm, rp;
  neighbour_rows(gy, nx, ny, py, rm, rp);
  const int xm = gx == 0 ? nx - 1 : gx - 1, xp = gx == nx - 1 ? 0 : gx + 1;
  const R Fx = ffield ? force[k] : Fx0;
  const R Fy = ffield ? force[S + k] : Fy0;
  R d[9];
  PopSource<R, MODE>::hydro(src, S, nx, k, gy * nx, rm, rp, gx, xm, xp, d);
  if (MODE == kModeStep && !py && (gy == 0 || gy == ny - 1)) zou_he<R>(d, Fx, Fy, gy == 0);
  HydroM<R> m;
  hydro_moments<R>(d, m);
  rho = R(1) + m.drho;
  const R irho = R(1) / rho;
  ux = (m.jx + R(0.5) * Fx) * irho;
  uy = (m.jy + R(0.5) * Fy) * irho;
}

template <typename R>
__device__ __forceinline__ R coef(const InstDev& D, int i);
template <>
__device__ __forceinline__ double coef<double>(const InstDev& D, int i) {
  return D.cd[i];
}
template <>
__device__ __forceinline__ float coef<float>(const InstDev& D, int i) {
  return D.cf[i];
}
template <>
__device__ __forceinline__ df32 coef<df32>(const InstDev& D, int i) {
  return df32(D.cf[i], D.cl[i]);
}

// Position of halo-ring slot q in the (TX+2) x (TY+2hy) region: hy rows
// above and hy rows below the tile (its TX columns), one column left and one
// right of it.  The region's four corner blocks are never computed: every
// difference stencil runs along a single axis, so no node reads them.
__device__ __forceinline__ void ring_slot(int q, int RW, int TY, int hy, int& lx, int& ly) {
  const int TX = RW - 2;
  if (q < hy * TX) {
    ly = q / TX;
    lx = 1 + q % TX;
  } else if ((q -= hy * TX) < hy * TX) {
    ly = hy + TY + q / TX;
    lx = 1 + q % TX;
  } else if ((q -= hy * TX) < TY) {
    lx = 0;
    ly = hy + q;
  } else {
    lx = RW - 1;
    ly = hy + q - TY;
  }
}

// Global node of region slot (lx, ly); false if it lies outside a walled domain.
__device__ __forceinline__ bool region_node(int lx, int ly, int x0, int y0, int hy, int nx,
                                            int ny, bool py, int& gx, int& gy) {
  gx = x0 - 1 + lx;
  gx = ((gx % nx) + nx) % nx;
  gy = y0 - hy + ly;
  if (py) {
    gy = ((gy % ny) + ny) % ny;
    return true;
  }
  return gy >= 0 && gy < ny;
}

// v wrapped into [0, n) when it lies less than one period outside it.
__device__ __forceinline__ int wrap_once(int v, int n) {
  return v < 0 ? v + n : (v >= n ? v - n : v);
}

// region_node for a kTileTX-wide tile of an instance with D.t32 set: its
// halo columns x0-1 .. x0+kTileTX and (periodic) rows y0-2 .. y0+TY+1 lie
// less than one period outside the domain (nx >= kTileTX; ny >= TY + 2 when
// periodic), so one conditional wrap replaces the modulo.
__device__ __forceinline__ bool region_node_once(int lx, int ly, int x0, int y0, int hy, int nx,
                                                 int ny, bool py, int& gx, int& gy) {
  gx = wrap_once(x0 - 1 + lx, nx);
  gy = y0 - hy + ly;
  if (py) {
    gy = wrap_once(gy, ny);
    return true;
  }
  return gy >= 0 && gy < ny;
}

// Conformation tensor and constitutive function F(A) of a node from its
// raw conformation deviations dphi_c (Sec. 2: eqb4 for Oldroyd-B, FENE-P,
// FENE-CR), F in deviation form F = f (A - I) + (f - a) I.
template <typename R, bool MASKED>
__device__ __forceinline__ void polymer_terms(const InstDev& D, R d0, R d1, R d2, R& Axx,
                                              R& Axy, R& Ayy, R& Fxx, R& Fxy, R& Fyy) {
  Axx = R(1) + d0;
  Axy = d1;
  Ayy = R(1) + d2;
  Fxx = d0;
  Fxy = d1;
  Fyy = d2;
  if (MASKED && D.model != 0) {  // other models run in the general variant only
    const R tr = Axx + Ayy;
    const R f = R(1) / (R(1) - tr * coef<R>(D, kCoefInvL2));
    const R a = D.model == 2 ? f : coef<R>(D, kCoefAfene);
    Fxx = f * d0 + (f - a);
    Fxy = f * d1;
    Fyy = f * d2 + (f - a);
  }
}

// Component l (xx, xy, yy) of the source Phi_ab of the conformation
// equation (Sec. 3.2) with G** = d_g u_b.
template <typename R>
__device__ __forceinline__ R source_component(int l, R Axx, R Axy, R Ayy, R Fxx, R Fxy, R Fyy,
                                              R il, R G00, R G01, R G10, R G11) {
  const R div = G00 + G11;
  if (l == 0) return -Fxx * il + R(2) * (Axx * G00 + Axy * G10) + Axx * div;
  if (l == 1) return -Fxy * il + (Axx * G01 + Axy * G11) + (Axy * G00 + Ayy * G10) + Axy * div;
  return -Fyy * il + R(2) * (Axy * G01 + Ayy * G11) + Ayy * div;
}

// Hydrodynamic TRT-RLB collision of one node (eq_ev_f, eq4, eq5, eq6, F_i)
// and the store of its 9 post-collision populations.
template <typename R>
__device__ __forceinline__ void collide_hydro(const InstDev& D, int k, int S, R* __restrict__ dst,
                                              const HydroM<R>& hm, R rho, R ux, R uy, R dPx,
                                              R dPy, R txx, R txy, R tyy, R Fx, R Fy) {
  const R cs2 = R(1.0 / 3.0);
  const R c1 = coef<R>(D, kCoefCs1), c2 = coef<R>(D, kCoefCs2);
  const R h1 = coef<R>(D, kCoefHs1), w1 = coef<R>(D, kCoefWs1);
  const R ruxx = rho * ux * ux, ruyy = rho * uy * uy, ruxy = rho * ux * uy;
  const R ruxxy = ruxx * uy, ruxyy = ruxy * uy;
  const R nxx = hm.pxx - cs2 * hm.drho - ruxx;  // A_xx^neq
  const R nyy = hm.pyy - cs2 * hm.drho - ruyy;  // A_yy^neq
  const R nxy = hm.pxy - ruxy;                  // A_xy^neq
  const R nxxy = hm.qxxy - cs2 * hm.jy - ruxxy; // A_xxy^neq
  const R nxyy = hm.qxyy - cs2 * hm.jx - ruxyy; // A_xyy^neq
  const R bx = hm.jx + Fx, by = hm.jy + Fy;     // rho u + (1-1/tau)A_a + F-term
  const R bxx = ruxx + c1 * nxx - h1 * dPx - w1 * txx;
  const R byy = ruyy + c1 * nyy - h1 * dPy - w1 * tyy;
  const R bxy = ruxy + c1 * nxy - w1 * txy;
  const R bxxy = ruxxy + c2 * nxxy;
  const R bxyy = ruxyy + c2 * nxyy;
  R out[9];
  reconstruct<R>(hm.drho, bx, by, bxx, byy, bxy, bxxy, bxyy, out);
#pragma unroll
  for (int i = 0; i < 9; ++i) dst[(size_t)i * S + k] = out[i];
}

// Conformation TRT-RLB collision of lattice l at one node (eq_g0 with
// G~_i, F~_i and its backward time difference) and the store of its 9
// post-collision populations.  sl, so: the source now and one step back.
template <typename R, bool MASKED>
__device__ __forceinline__ void collide_cde(const InstDev& D, int k, int S, R* __restrict__ dst,
                                            int l, const CdeM<R>& m, R rho, R ux, R uy, R sl,
                                            R so, R uxo, R uyo, R Fx, R Fy, R dRx, R dRy) {
  const R cs2 = R(1.0 / 3.0);
  const R ep = coef<R>(D, kCoefEp1), c2 = coef<R>(D, kCoefCp2), h1 = coef<R>(D, kCoefHp1);
  const R irho = R(1) / rho;
  const R uxx = ux * ux, uyy = uy * uy, uxy = ux * uy;
  // the force G~_i sees: F (eq_p_G_1) or F - c_s^2 grad rho (eq_p_G)
  const bool gt = MASKED && D.gtilde;
  const R Gx = gt ? Fx - cs2 * dRx : Fx, Gy = gt ? Fy - cs2 * dRy : Fy;
  const R phi = (l == 1 ? R(0) : R(1)) + m.dphi;
  const R Bx = m.jx - phi * ux, By = m.jy - phi * uy;
  const R Bxx = m.pxx - cs2 * m.dphi - phi * uxx;
  const R Byy = m.pyy - cs2 * m.dphi - phi * uyy;
  const R Bxy = m.pxy - phi * uxy;
  // small source terms first, one rounding at the magnitude of phi
  const R c0p = m.dphi + (R(1.5) * sl - R(0.5) * so);
  const R pr = phi * irho;
  // (1 - 1/tau_p1) B = -B + ep B, kept split so float32 keeps the tiny
  // difference tau_p1 - 1/2 accurately
  const R cx = (phi * ux - Bx) + ep * Bx + h1 * (pr * Gx + ux * sl) +
               R(0.5) * h1 * (ux * sl - uxo * so);
  const R cy = (phi * uy - By) + ep * By + h1 * (pr * Gy + uy * sl) +
               R(0.5) * h1 * (uy * sl - uyo * so);
  const R cxx = phi * uxx + c2 * Bxx;
  const R cyy = phi * uyy + c2 * Byy;
  const R cxy = phi * uxy + c2 * Bxy;
  R out[9];
  reconstruct<R>(c0p, cx, cy, cxx, cyy, cxy, R(0), R(0), out);
  R* dl = dst + (size_t)(9 + 9 * l) * S;
#pragma unroll
  for (int i = 0; i < 9; ++i) dl[(size_t)i * S + k] = out[i];
}

// Final-step record of one node: its float64 fields and its contributions to
// the tile's partial record.  lattice -1 writes everything; 0 the
// hydrodynamic part (rho, u, momentum, residual), 1..3 conformation lattice
// lattice - 1 (A component, its sum; the wall balance is the caller's).  The
// sums of rho, A_xx and A_yy are kept as deviations from their rest value 1
// (added per tile from its node count) and the residual is scaled by 1/U_c
// per tile: GB300 issues a float64 instruction only every 64 cycles per
// warp, so the final step keeps them few.
// Type of the per-node contributions to a tile's partial record: float32
// instances keep float32 values (and exact float32 pairs) until the warp
// totals, float64 instances float64 values.
template <typename R>
using PartT = typename std::conditional<sizeof(R) == 4, float, double>::type;

// ux_prev, uy_prev: the velocity fields of the previous final step at node
// k, read by the caller before the collision (unused at init)
template <typename R, int MODE>
__device__ __forceinline__ void final_node(const InstDev& D, int k, int S, int lattice, R drho,
                                           R rho, R ux, R uy, const R* dphi, PartT<R> ux_prev,
                                           PartT<R> uy_prev, PartT<R>* part, PartT<R>* plo) {
  double* fl = D.fields;
  bool finite = true;
  if (lattice <= 0) {
    const double dr = to_f64(drho);
    const double vx = to_f64(ux), vy = to_f64(uy);
    fl[k] = 1.0 + dr;
    fl[S + k] = vx;
    fl[2 * S + k] = vy;
    if constexpr (sizeof(R) == 4) {
      // in float32: the previous fields are float32 values
      const float res =
          (MODE == kModeStep) ? fmaxf(fabsf(ux - ux_prev), fabsf(uy - uy_prev)) : 0.f;
      // rho u exactly, as a float32 pair (product and its rounding error)
      const float px = rho * ux, py = rho * uy;
      part[kSumRho] = drho;
      part[kSumJx] = px;
      part[kSumJy] = py;
      plo[kSumJx] = fmaf(rho, ux, -px);
      plo[kSumJy] = fmaf(rho, uy, -py);
      part[kResid] = res;
      finite = isfinite(drho) && isfinite(ux) && isfinite(uy);
    } else {
      const double res =
          (MODE == kModeStep) ? fmax(fabs(vx - ux_prev), fabs(vy - uy_prev)) : 0.0;
      part[kSumRho] = dr;
      part[kSumJx] = to_f64(rho) * vx;
      part[kSumJy] = to_f64(rho) * vy;
      part[kResid] = res;
      finite = isfinite(dr) && isfinite(vx) && isfinite(vy);
    }
  }
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    if (lattice >= 0 && lattice != 1 + l) continue;
    const double d = to_f64(dphi[l]);
    fl[(3 + l) * S + k] = l == 1 ? d : 1.0 + d;
    if constexpr (sizeof(R) == 4) {
      part[kSumPhi + l] = dphi[l];
      finite = finite && isfinite(dphi[l]);
    } else {
      part[kSumPhi + l] = d;
      finite = finite && isfinite(d);
    }
  }
  if (!finite) part[kResid] = 0;
  part[kNonFinite] = finite ? 0 : 1;
}

// Final step: start the previous velocity fields of node k (the residual's
// operands) on their way to L2 with the node's other loads; they are read
// just before the collision.  Read only after the collision, each warp
// stalled there for a full HBM round trip, which made the final step of a
// large batch take 1.8 times as long; loaded with the populations, they
// cost more registers than they save.
__device__ __forceinline__ void prefetch_prev_u(const InstDev& D, int k, int S) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(D.fields + S + k));
  asm volatile("prefetch.global.L2 [%0];" ::"l"(D.fields + 2 * S + k));
}

// Source, both collisions, stores and final-step bookkeeping of one node
// whose populations are already reduced to (wall-completed) moments:
//   hm      raw hydro moments, cm[3] raw conformation moments
//   rho, u  eq_ev_f0 moments; G** = d_g u_b; dPx, dPy = d_x(rho ux^3), d_y(rho uy^3)
//   So, uo  source and velocity of the previous step (ignored at init)
// Writes the 36 post-collision populations and the 5 history values of node k;
// on the final step also the float64 fields and this node's partial sums.
template <typename R, int MODE, bool FINAL, bool MASKED>
__device__ __forceinline__ void collide_node(const InstDev& D, int k, int S, R* __restrict__ dst,
                                             R* __restrict__ hist, const HydroM<R>& hm,
                                             const CdeM<R>* cm, R rho, R ux, R uy, R G00, R G01,
                                             R G10, R G11, R dPx, R dPy, R dRx, R dRy, R Fx,
                                             R Fy, R So0, R So1, R So2, R uxo, R uyo,
                                             PartT<R> ux_prev, PartT<R> uy_prev, PartT<R>* part,
                                             PartT<R>* plo) {
  // conformation tensor, constitutive function, polymer stress (eq_kramer),
  // source Phi_ab
  R Axx, Axy, Ayy, Fxx, Fxy, Fyy;
  polymer_terms<R, MASKED>(D, cm[0].dphi, cm[1].dphi, cm[2].dphi, Axx, Axy, Ayy, Fxx, Fxy, Fyy);
  const R mpl = coef<R>(D, kCoefMupLam), il = coef<R>(D, kCoefInvLam);
  const R txx = mpl * Fxx, txy = mpl * Fxy, tyy = mpl * Fyy;
  R Sc[3], So[3] = {So0, So1, So2};
#pragma unroll
  for (int l = 0; l < 3; ++l)
    Sc[l] = source_component<R>(l, Axx, Axy, Ayy, Fxx, Fxy, Fyy, il, G00, G01, G10, G11);
  if (MODE != kModeStep) {
    // first step: the backward difference of the CDE source is zero
    So[0] = Sc[0];
    So[1] = Sc[1];
    So[2] = Sc[2];
    uxo = ux;
    uyo = uy;
  }
  collide_hydro<R>(D, k, S, dst, hm, rho, ux, uy, dPx, dPy, txx, txy, tyy, Fx, Fy);
#pragma unroll
  for (int l = 0; l < 3; ++l)
    collide_cde<R, MASKED>(D, k, S, dst, l, cm[l], rho, ux, uy, Sc[l], So[l], uxo, uyo, Fx, Fy,
                           dRx, dRy);

  hist[k] = Sc[0];
  hist[S + k] = Sc[1];
  hist[2 * S + k] = Sc[2];
  hist[3 * S + k] = ux;
  hist[4 * S + k] = uy;

  if (FINAL) {
    const R dphi[3] = {cm[0].dphi, cm[1].dphi, cm[2].dphi};
    final_node<R, MODE>(D, k, S, -1, hm.drho, rho, ux, uy, dphi, ux_prev, uy_prev, part, plo);
  }
}

// Second-order differences in y of u and rho u_y^3 at a node, from the
// moments of rows y-2..y+2 (central inside, one-sided on wall rows).
template <typename R>
__device__ __forceinline__ void y_gradients(bool wb, bool wt, R rm2, R uxm2, R uym2, R rm1,
                                            R uxm1, R uym1, R r0, R ux0, R uy0, R rp1, R uxp1,
                                            R uyp1, R rp2, R uxp2, R uyp2, R& G10, R& G11,
                                            R& dPy) {
  const R half = R(0.5);
  if (wb) {
    G10 = half * (R(-3) * ux0 + R(4) * uxp1 - uxp2);
    G11 = half * (R(-3) * uy0 + R(4) * uyp1 - uyp2);
    dPy = half * (R(-3) * (r0 * uy0 * uy0 * uy0) + R(4) * (rp1 * uyp1 * uyp1 * uyp1) -
                  rp2 * uyp2 * uyp2 * uyp2);
  } else if (wt) {
    G10 = half * (R(3) * ux0 - R(4) * uxm1 + uxm2);
    G11 = half * (R(3) * uy0 - R(4) * uym1 + uym2);
    dPy = half * (R(3) * (r0 * uy0 * uy0 * uy0) - R(4) * (rm1 * uym1 * uym1 * uym1) +
                  rm2 * uym2 * uym2 * uym2);
  } else {
    G10 = half * (uxp1 - uxm1);
    G11 = half * (uyp1 - uym1);
    dPy = half * (rp1 * uyp1 * uyp1 * uyp1 - rm1 * uym1 * uym1 * uym1);
  }
}

// The same y difference of the density (for the eq_p_G form of G~).
template <typename R>
__device__ __forceinline__ R y_drho(bool wb, bool wt, R rm2, R rm1, R r0, R rp1, R rp2) {
  const R half = R(0.5);
  if (wb) return half * (R(-3) * r0 + R(4) * rp1 - rp2);
  if (wt) return half * (R(3) * r0 - R(4) * rm1 + rm2);
  return half * (rp1 - rm1);
}

// Resident CTAs per SM the register budget is sized for: the float32 step
// is HBM-bound and wants more loads in flight; the float64 step is bound by
// the FP64 pipe.
// Masked tiles carry the mask's one-sided differences: a budget of 5 CTAs
// per SM lets them keep their registers without spills.
#ifndef LBVE_FP32_MASKED_MIN_BLOCKS
#define LBVE_FP32_MASKED_MIN_BLOCKS 5
#endif
// Float64 CTAs: 256 threads two per SM (128 registers per thread).  The
// 64- and one-warp CTAs serve batches with fewer tiles than 4 and 2 per SM,
// so they are budgeted for that many and keep every value in registers.
// Float32 pairs: 3 CTAs per SM keep their registers (227 at most) without
// spills; 4 per SM spill a little and ran 1.4 % slower on the batched mix.
#ifndef LBVE_DF32_MIN_BLOCKS
#define LBVE_DF32_MIN_BLOCKS 3
#endif
template <typename R, bool MASKED, int NT>
struct MinBlocks {
  static constexpr int value =
      std::is_same<R, df32>::value
          ? LBVE_DF32_MIN_BLOCKS
          : sizeof(R) == 4 ? (MASKED ? LBVE_FP32_MASKED_MIN_BLOCKS : LBVE_FP32_MIN_BLOCKS)
                           : (NT <= 32 ? 2 : NT <= 64 ? 4 : (NT <= 512 ? 512 / NT : 1));
};

// One-sided differences along one axis next to the solid mask (same rule as
// the central and wall-row differences: second order on the fluid side when
// two fluid nodes lie there, else first order; zero between two solids).
//   t:        +1 toward +axis, -1 toward -axis (the fluid side)
//   q0, q1:   (rho, ux, uy) of the node and of its fluid neighbour at +t
//   has2:     whether the node at +2t is fluid; (r2, u2x, u2y) its values
//   axis:     0 = x (the cube is rho ux^3), 1 = y (rho uy^3)
template <typename R>
__device__ __forceinline__ void one_sided(int t, R r0, R ux0, R uy0, R r1, R ux1, R uy1,
                                          bool has2, R r2, R ux2, R uy2, int axis, R& dux,
                                          R& duy, R& dcube, R& drho) {
  const R v0 = axis == 0 ? ux0 : uy0, v1 = axis == 0 ? ux1 : uy1, v2 = axis == 0 ? ux2 : uy2;
  const R c0 = r0 * v0 * v0 * v0, c1 = r1 * v1 * v1 * v1, c2 = r2 * v2 * v2 * v2;
  const R ts = (R)t;
  if (has2) {
    const R h = R(0.5) * ts;
    dux = h * (R(-3) * ux0 + R(4) * ux1 - ux2);
    duy = h * (R(-3) * uy0 + R(4) * uy1 - uy2);
    dcube = h * (R(-3) * c0 + R(4) * c1 - c2);
    drho = h * (R(-3) * r0 + R(4) * r1 - r2);
  } else {
    dux = ts * (ux1 - ux0);
    duy = ts * (uy1 - uy0);
    dcube = ts * (c1 - c0);
    drho = ts * (r1 - r0);
  }
}

// Open channels: nodes of the inlet (x = 0) and outlet (x = nx - 1) columns
// take their completed populations from the column pass's colbuf during a
// step (the pull would miss the populations entering from outside).
__device__ __forceinline__ bool open_column(const InstDev& D, int gx) {
  return D.open_x && (gx == 0 || gx == D.nx - 1);
}
template <typename R>
__device__ __forceinline__ const R* colbuf_node(const InstDev& D, int gx, int gy) {
  return (const R*)D.colbuf + (gx == 0 ? 0 : D.ny) + gy;  // plane stride 2 ny
}

// rho, u of region node (gx, gy) for the masked variant: open-column nodes
// from colbuf during a step, every other node as node_rho_u.
template <typename R, int MODE>
__device__ __forceinline__ void region_rho_u(const InstDev& D, const void* src,
                                             const R* __restrict__ force, bool ffield, R Fx0,
                                             R Fy0, int S, int nx, int ny, bool py, int gx,
                                             int gy, R& rho, R& ux, R& uy) {
  if (MODE == kModeStep && open_column(D, gx)) {
    const R* cb = colbuf_node<R>(D, gx, gy);
    const int ld = 2 * ny;
    R d[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) d[i] = cb[(size_t)i * ld];
    const int k = gy * nx + gx;
    const R Fx = ffield ? force[k] : Fx0, Fy = ffield ? force[S + k] : Fy0;
    HydroM<R> m;
    hydro_moments<R>(d, m);
    rho = R(1) + m.drho;
    const R irho = R(1) / rho;
    ux = (m.jx + R(0.5) * Fx) * irho;
    uy = (m.jy + R(0.5) * Fy) * irho;
    return;
  }
  node_rho_u<R, MODE>(src, force, ffield, Fx0, Fy0, S, nx, ny, py, gx, gy, rho, ux, uy);
}

// Sum of two float32 pairs (hi + lo), renormalised (Knuth's two-sum of the
// high parts, the low parts added to its error, a fast two-sum at the end).
__device__ __forceinline__ void df_add(float& ah, float& al, float bh, float bl) {
  const float s = ah + bh, bv = s - ah;
  const float e = ((ah - (s - bv)) + (bh - bv)) + (al + bl);
  ah = s + e;
  al = e - (ah - s);
}

// One butterfly level (fold_half) on float32 pairs.
template <int M>
__device__ __forceinline__ void fold_half_df(float* h, float* l, int o, bool up) {
#pragma unroll
  for (int j = 0; j < M / 2; ++j) {
    const float kh = up ? h[j + M / 2] : h[j], kl = up ? l[j + M / 2] : l[j];
    const float sh = up ? h[j] : h[j + M / 2], sl = up ? l[j] : l[j + M / 2];
    const float rh = __shfl_xor_sync(0xffffffffu, sh, o), rl = __shfl_xor_sync(0xffffffffu, sl, o);
    h[j] = kh;
    l[j] = kl;
    df_add(h[j], l[j], rh, rl);
  }
}

// The tile's partial record of the final step in a fixed order: the 12
// sums by a transposed butterfly per warp, the residual (>= 0 and finite, so
// the order of its bit patterns is its numeric order) and the non-finite
// count as integers, then the warps in order and the rest values from the
// count of the tile's fluid nodes.  Every thread of the CTA calls it.  A
// float32 instance's values are float32 numbers or exact float32 pairs
// (part + plo), and its butterfly adds float32 pairs (a 48-bit sum; GB300
// issues a float64 addition only every 64 cycles per warp); the warp totals
// and everything after them are float64.  A float32 warp whose nodes carry no
// wall balance folds only the first 6 values (the order of the sum is fixed
// by the tile's own data, so totals stay reproducible).
template <int NT, typename P>
__device__ __forceinline__ void tile_partials(const InstDev& D, const TileDev& T, const P* part,
                                              const P* plo, bool active,
                                              double* __restrict__ partials,
                                              double (*s_red)[kPartial]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  static_assert(kNonFinite == 13 && kResid == 12, "12 sums, then residual and flag");
  double total;  // this lane's warp total of value slot
  double resid;  // the warp's largest residual
  int slot;   // the value slot this lane's total belongs to
  bool write;  // whether this lane writes it
  if constexpr (sizeof(P) == 4) {
    // a warp without wall nodes has zero wall balances (slots 6..11): its
    // butterfly sums the first 6 values only
    bool wall = false;
#pragma unroll
    for (int j = kWallIn; j < kResid; ++j) wall = wall || part[j] != 0.f || plo[j] != 0.f;
    if (__any_sync(0xffffffffu, wall)) {
      float h[16], l[16];
#pragma unroll
      for (int j = 0; j < 12; ++j) {
        h[j] = part[j];
        l[j] = plo[j];
      }
#pragma unroll
      for (int j = 12; j < 16; ++j) h[j] = l[j] = 0.f;
      fold_half_df<16>(h, l, 16, (lane & 16) != 0);
      fold_half_df<8>(h, l, 8, (lane & 8) != 0);
      fold_half_df<4>(h, l, 4, (lane & 4) != 0);
      fold_half_df<2>(h, l, 2, (lane & 2) != 0);
      const float rh = __shfl_xor_sync(0xffffffffu, h[0], 1);
      const float rl = __shfl_xor_sync(0xffffffffu, l[0], 1);
      df_add(h[0], l[0], rh, rl);
      total = f2d_exact(h[0]) + f2d_exact(l[0]);
      slot = (lane >> 1) & 15;
      write = (lane & 1) == 0 && slot < 12;
    } else {
      float h[8], l[8];
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        h[j] = part[j];
        l[j] = plo[j];
      }
      h[6] = h[7] = l[6] = l[7] = 0.f;
      fold_half_df<8>(h, l, 16, (lane & 16) != 0);
      fold_half_df<4>(h, l, 8, (lane & 8) != 0);
      fold_half_df<2>(h, l, 4, (lane & 4) != 0);
#pragma unroll
      for (int o = 2; o > 0; o >>= 1) {
        const float rh = __shfl_xor_sync(0xffffffffu, h[0], o);
        const float rl = __shfl_xor_sync(0xffffffffu, l[0], o);
        df_add(h[0], l[0], rh, rl);
      }
      // value (lane >> 2) & 7; lanes 4m write it, lanes 4m + 1 the zero of wall slot 6 + m
      const int s8 = (lane >> 2) & 7;
      total = (lane & 3) == 1 ? 0.0 : f2d_exact(h[0]) + f2d_exact(l[0]);
      slot = (lane & 3) == 1 ? kWallIn + s8 : s8;
      write = (lane & 3) <= 1 && s8 < 6;
    }
    int rb = __float_as_int(part[kResid]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rb = max(rb, __shfl_xor_sync(0xffffffffu, rb, o));
    resid = f2d_exact(__int_as_float(rb));
  } else {
    double v[16];
#pragma unroll
    for (int j = 0; j < 12; ++j) v[j] = part[j];
#pragma unroll
    for (int j = 12; j < 16; ++j) v[j] = 0.0;
    fold_half<16>(v, 16, (lane & 16) != 0);
    fold_half<8>(v, 8, (lane & 8) != 0);
    fold_half<4>(v, 4, (lane & 4) != 0);
    fold_half<2>(v, 2, (lane & 2) != 0);
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
    total = v[0];
    slot = (lane >> 1) & 15;
    write = (lane & 1) == 0 && slot < 12;
    long long rb = __double_as_longlong(part[kResid]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const long long ob = __shfl_xor_sync(0xffffffffu, rb, o);
      rb = ob > rb ? ob : rb;
    }
    resid = __longlong_as_double(rb);
  }
  const unsigned nf = __popc(__ballot_sync(0xffffffffu, part[kNonFinite] != P(0)));
  if (write) s_red[warp][slot] = total;
  if (lane == 0) {
    s_red[warp][kResid] = resid;
    s_red[warp][kNonFinite] = (double)nf;
  }
  const int nfluid = __syncthreads_count(active);
  if (threadIdx.x < 14) {
    const int j = threadIdx.x;
    double t = s_red[0][j];
    for (int w = 1; w < NT / 32; ++w) t = (j == kResid) ? fmax(t, s_red[w][j]) : t + s_red[w][j];
    if (j == kSumRho || j == kSumPhi || j == kSumPhi + 2) t += (double)nfluid;
    if (j == kResid) t *= D.inv_Uc;
    partials[(size_t)T.slot * kPartial + j] = t;
  }
}

template <typename R, int MODE, bool FINAL, bool MASKED, int NT>
__device__ __forceinline__ void process_tile(const InstDev* __restrict__ insts, const TileDev T,
                                             int parity, double* __restrict__ partials, R* s_rho,
                                             R* s_ux, R* s_uy, double (*s_red)[kPartial]) {
  const InstDev& D = insts[T.inst];
  const int nx = D.nx, ny = D.ny, S = D.stride, TX = D.TX, TY = D.TY, hy = D.hy;
  const bool py = D.periodic_y != 0;
  const void* src = D.pop[parity];
  const R* __restrict__ srcR = (const R*)src;
  R* __restrict__ dst = (R*)D.pop[parity ^ 1];
  const R* __restrict__ force = (const R*)D.force;
  R* __restrict__ hist = (R*)D.hist;
  const bool ffield = D.force_field != 0;
  const R Fx0 = coef<R>(D, kCoefFx), Fy0 = coef<R>(D, kCoefFy);
  const int RW = TX + 2;

  // ---- phase A --------------------------------------------------------------
  // Every load this thread needs -- one halo-ring node's hydro populations
  // and all of its own node's populations, history and force -- is issued
  // before any of them is used, so the tile's whole HBM traffic is in flight
  // together.  Own hydro and conformation populations are then reduced to
  // moments (walls completed first); rho and u go to shared memory.
  // Thread and halo-slot indices.  For plain kTileTX-wide tiles (D.t32) the
  // divisions by the width and the wraps use compile-time constants; the
  // arithmetic after this prologue is one code path for every width.
  const bool t32 = !MASKED && D.t32;
  int tx, ty;
  if (t32) {
    tx = threadIdx.x % kTileTX;
    ty = threadIdx.x / kTileTX;
  } else {
    tx = threadIdx.x % TX;
    ty = threadIdx.x / TX;
  }
  const bool in_tile = ty < TY;
  const int x = T.x0 + tx, y = T.y0 + ty;
  const bool inside = in_tile && (x < nx) && (y < ny);
  // solid-mask nodes (masked tiles only) take no part in the update
  const bool solid = MASKED && inside && D.mask && D.mask[y * nx + x] != 0;
  const bool active = inside && !solid;
  const int ri = (ty + hy) * RW + tx + 1;  // this slot in the halo region
  const bool wb = active && !py && y == 0, wt = active && !py && y == ny - 1;
  // an open column's node arrives completed (colbuf): no wall completion there
  const bool ocol = MASKED && MODE == kModeStep && active && open_column(D, x);
  const bool wcomp = (wb || wt) && !ocol;
  const int nring = 2 * hy * TX + 2 * TY;  // the halo ring without its corners

  // (1) first halo-ring node of this thread: issue its pull
  int ring_r = -1, rgx = 0, rgy = 0;
  R dr[9];
  if (threadIdx.x < nring) {
    int lx, ly;
    bool in_domain;
    if (t32) {
      ring_slot(threadIdx.x, kTileTX + 2, NT / kTileTX, hy, lx, ly);
      in_domain = region_node_once(lx, ly, T.x0, T.y0, hy, nx, ny, py, rgx, rgy);
    } else {
      ring_slot(threadIdx.x, RW, TY, hy, lx, ly);
      in_domain = region_node(lx, ly, T.x0, T.y0, hy, nx, ny, py, rgx, rgy);
    }
    if (in_domain) {
      ring_r = ly * RW + lx;
      if (MASKED && MODE == kModeStep && open_column(D, rgx)) {
        const R* cb = colbuf_node<R>(D, rgx, rgy);
#pragma unroll
        for (int i = 0; i < 9; ++i) dr[i] = cb[(size_t)i * 2 * ny];
      } else {
        int rm, rp;
        neighbour_rows(rgy, nx, ny, py, rm, rp);
        const int xm = rgx == 0 ? nx - 1 : rgx - 1, xp = rgx == nx - 1 ? 0 : rgx + 1;
        PopSource<R, MODE>::hydro(src, S, nx, rgy * nx + rgx, rgy * nx, rm, rp, rgx, xm, xp, dr);
      }
    }
  }

  // (2) own node: all 36 populations, force, history, wall slots
  R d[9], g[3][9], So[3] = {R(0), R(0), R(0)}, uxo = R(0), uyo = R(0), Fx = Fx0, Fy = Fy0;
  R post[3][3];  // own outgoing-to-wall post-collision slots (wall rows only)
  int k = 0;
  if (active) {
    k = y * nx + x;
    int rm, rp;
    neighbour_rows(y, nx, ny, py, rm, rp);
    const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
    const int rc = y * nx;
    if (ocol) {
      const R* cb = colbuf_node<R>(D, x, y);
      const int ld = 2 * ny;
#pragma unroll
      for (int i = 0; i < 9; ++i) d[i] = cb[(size_t)i * ld];
#pragma unroll
      for (int l = 0; l < 3; ++l)
#pragma unroll
        for (int i = 0; i < 9; ++i) g[l][i] = cb[(size_t)(9 + 9 * l + i) * ld];
    } else {
      PopSource<R, MODE>::hydro(src, S, nx, k, rc, rm, rp, x, xm, xp, d);
#pragma unroll
      for (int l = 0; l < 3; ++l)
        PopSource<R, MODE>::cde(src, l, S, nx, k, rc, rm, rp, x, xm, xp, g[l]);
    }
    if (ffield) {
      Fx = force[k];
      Fy = force[S + k];
    }
    if (MODE == kModeStep) {
      So[0] = hist[k];
      So[1] = hist[S + k];
      So[2] = hist[2 * S + k];
      uxo = hist[3 * S + k];
      uyo = hist[4 * S + k];
      if (FINAL) prefetch_prev_u(D, k, S);
      if (wcomp) {
        // bottom wall: H = {4, 7, 8}; top wall: H = {2, 5, 6}
        const int h0 = wb ? 4 : 2, h1 = wb ? 7 : 5, h2 = wb ? 8 : 6;
#pragma unroll
        for (int l = 0; l < 3; ++l) {
          const R* own = srcR + (size_t)(9 + 9 * l) * S + k;
          post[l][0] = own[h0 * S];
          post[l][1] = own[h1 * S];
          post[l][2] = own[h2 * S];
        }
      }
    }
  }

  // (3) ring node moments
  if (ring_r >= 0) {
    const int rk = rgy * nx + rgx;
    const R rFx = ffield ? force[rk] : Fx0;
    const R rFy = ffield ? force[S + rk] : Fy0;
    if (MODE == kModeStep && !py && (rgy == 0 || rgy == ny - 1) &&
        !(MASKED && open_column(D, rgx)))
      zou_he<R>(dr, rFx, rFy, rgy == 0);
    HydroM<R> m;
    hydro_moments<R>(dr, m);
    const R rho = R(1) + m.drho;
    s_rho[ring_r] = rho;
    const R irho = R(1) / rho;
    s_ux[ring_r] = (m.jx + R(0.5) * rFx) * irho;
    s_uy[ring_r] = (m.jy + R(0.5) * rFy) * irho;
  }

  // (4) own moments; conformation walls completed with the node's own u
  HydroM<R> hm;
  CdeM<R> cm[3];
  R rho = R(1), ux = R(0), uy = R(0);
  double wall_io[6] = {0, 0, 0, 0, 0, 0};
  if (active) {
    if (MODE == kModeStep && wcomp) zou_he<R>(d, Fx, Fy, wb);
    hydro_moments<R>(d, hm);
    rho = R(1) + hm.drho;
    const R irho_own = R(1) / rho;
    ux = (hm.jx + R(0.5) * Fx) * irho_own;
    uy = (hm.jy + R(0.5) * Fy) * irho_own;
    s_rho[ri] = rho;
    s_ux[ri] = ux;
    s_uy[ri] = uy;
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      if (MODE == kModeStep && wcomp) {
        const R delta = (l == 1) ? R(0) : R(1);
        cnebb<R>(g[l], post[l][0], post[l][1], post[l][2], delta, ux, uy, wb, wall_io[l],
                 wall_io[3 + l]);
      }
      cde_moments<R>(g[l], cm[l]);
    }
  } else if (in_tile && !inside) {
    // slot outside the domain (ragged tile): it may still be a periodic
    // neighbour of an active node, so fill it with the wrapped node
    const int gx = t32 ? wrap_once(x, nx) : x % nx;
    const int gy = py ? (t32 ? wrap_once(y, ny) : y % ny) : y;
    if (gy < ny) {
      R r, vx, vy;
      if constexpr (MASKED)
        region_rho_u<R, MODE>(D, src, force, ffield, Fx0, Fy0, S, nx, ny, py, gx, gy, r, vx, vy);
      else
        node_rho_u<R, MODE>(src, force, ffield, Fx0, Fy0, S, nx, ny, py, gx, gy, r, vx, vy);
      s_rho[ri] = r;
      s_ux[ri] = vx;
      s_uy[ri] = vy;
    }
  }

  // (5) remaining ring nodes (only when the ring outnumbers the threads)
  for (int q = threadIdx.x + blockDim.x; q < nring; q += blockDim.x) {
    int lx, ly, gx, gy;
    ring_slot(q, RW, TY, hy, lx, ly);
    if (!region_node(lx, ly, T.x0, T.y0, hy, nx, ny, py, gx, gy)) continue;
    R r, vx, vy;
    if constexpr (MASKED)
      region_rho_u<R, MODE>(D, src, force, ffield, Fx0, Fy0, S, nx, ny, py, gx, gy, r, vx, vy);
    else
      node_rho_u<R, MODE>(src, force, ffield, Fx0, Fy0, S, nx, ny, py, gx, gy, r, vx, vy);
    const int rr = ly * RW + lx;
    s_rho[rr] = r;
    s_ux[rr] = vx;
    s_uy[rr] = vy;
  }
  __syncthreads();

  // ---- phase B: gradients, source, collisions, stores ----------------------
  PartT<R> part[FINAL ? 14 : 1], plo[FINAL ? 12 : 1];
#pragma unroll
  for (int j = 0; j < (FINAL ? 14 : 1); ++j) part[j] = 0;
#pragma unroll
  for (int j = 0; j < (FINAL ? 12 : 1); ++j) plo[j] = 0;

  if (active) {
    // gradients: grad[g][b] = d_g u_b  (G00 = dx ux, G01 = dx uy, G10 = dy ux, G11 = dy uy)
    const R half = R(0.5);
    R G00 = half * (s_ux[ri + 1] - s_ux[ri - 1]);
    R G01 = half * (s_uy[ri + 1] - s_uy[ri - 1]);
    const R cxp = s_rho[ri + 1] * s_ux[ri + 1] * s_ux[ri + 1] * s_ux[ri + 1];
    const R cxm = s_rho[ri - 1] * s_ux[ri - 1] * s_ux[ri - 1] * s_ux[ri - 1];
    R dPx = half * (cxp - cxm);
    R G10, G11, dPy;
    // density gradient, only for the eq_p_G form of G~
    R dRx = (MASKED && D.gtilde) ? half * (s_rho[ri + 1] - s_rho[ri - 1]) : R(0), dRy = R(0);
    {
      // rows y-2..y+2 of this column (only those a wall row needs are read)
      const int a = wb ? ri : (wt ? ri - 2 * RW : ri), b = wb ? ri : (wt ? ri - RW : ri - RW);
      const int c = wb ? ri + RW : (wt ? ri : ri + RW), e = wb ? ri + 2 * RW : ri;
      y_gradients<R>(wb, wt, s_rho[a], s_ux[a], s_uy[a], s_rho[b], s_ux[b], s_uy[b], rho, ux,
                     uy, s_rho[c], s_ux[c], s_uy[c], s_rho[e], s_ux[e], s_uy[e], G10, G11, dPy);
      if (MASKED && D.gtilde) dRy = y_drho<R>(wb, wt, s_rho[a], s_rho[b], rho, s_rho[c], s_rho[e]);
    }
    if constexpr (MASKED) {
      // one-sided differences where an axis neighbour is solid; the values
      // two nodes away come straight from the pulled populations (L2)
      // a side is blocked by a solid node or, in an open channel, by the
      // end of the domain beyond the inlet / outlet column
      const uint8_t* __restrict__ M = D.mask;
      const int xp = x == nx - 1 ? 0 : x + 1, xm = x == 0 ? nx - 1 : x - 1;
      const bool sxp = (D.open_x && x == nx - 1) || (M && M[y * nx + xp] != 0);
      const bool sxm = (D.open_x && x == 0) || (M && M[y * nx + xm] != 0);
      if (sxp || sxm) {
        R gx0 = R(0), gx1 = R(0), gxc = R(0), gxr = R(0);
        if (!(sxp && sxm)) {
          const int t = sxp ? -1 : 1;
          const int i1 = t > 0 ? ri + 1 : ri - 1;
          const int x2 = (((x + 2 * t) % nx) + nx) % nx;
          const bool has2 = !(M && M[y * nx + x2] != 0);
          R r2 = R(1), u2x = R(0), u2y = R(0);
          if (has2)
            region_rho_u<R, MODE>(D, src, force, ffield, Fx0, Fy0, S, nx, ny, py, x2, y, r2,
                                  u2x, u2y);
          one_sided<R>(t, rho, ux, uy, s_rho[i1], s_ux[i1], s_uy[i1], has2, r2, u2x, u2y, 0, gx0,
                       gx1, gxc, gxr);
        }
        G00 = gx0;
        G01 = gx1;
        dPx = gxc;
        dRx = gxr;
      }
      if (!wb && !wt && M) {
        // rows next to a flat wall carry no mask, so y +- 1 lies in the domain
        const int yp = (py && y == ny - 1) ? 0 : y + 1, ym = (py && y == 0) ? ny - 1 : y - 1;
        const bool syp = M[yp * nx + x] != 0, sym = M[ym * nx + x] != 0;
        if (syp || sym) {
          R gy0 = R(0), gy1 = R(0), gyc = R(0), gyr = R(0);
          if (!(syp && sym)) {
            const int t = syp ? -1 : 1;
            const int i1 = t > 0 ? ri + RW : ri - RW;
            int y2 = y + 2 * t;
            if (py) y2 = ((y2 % ny) + ny) % ny;
            const bool has2 = y2 >= 0 && y2 < ny && M[y2 * nx + x] == 0;
            R r2 = R(1), u2x = R(0), u2y = R(0);
            if (has2)
              region_rho_u<R, MODE>(D, src, force, ffield, Fx0, Fy0, S, nx, ny, py, x, y2, r2,
                                    u2x, u2y);
            one_sided<R>(t, rho, ux, uy, s_rho[i1], s_ux[i1], s_uy[i1], has2, r2, u2x, u2y, 1,
                         gy0, gy1, gyc, gyr);
          }
          G10 = gy0;
          G11 = gy1;
          dPy = gyc;
          dRy = gyr;
        }
      }
    }
    if (FINAL) {
      if constexpr (sizeof(R) == 4) {
        if (wcomp) {
          // float32 pairs of the (float64) wall balances of a wall node
#pragma unroll
          for (int j = 0; j < 6; ++j) {
            const float hi = (float)wall_io[j];
            part[kWallIn + j] = hi;
            plo[kWallIn + j] = (float)(wall_io[j] - f2d_exact(hi));
          }
        }
      } else {
#pragma unroll
        for (int j = 0; j < 6; ++j) part[kWallIn + j] = wall_io[j];
      }
    }
    PartT<R> ux_prev = 0, uy_prev = 0;
    if (FINAL && MODE == kModeStep) {
      // prefetched into L2 above; read past L1 (nothing else touches these lines)
      ux_prev = (PartT<R>)__ldcg(D.fields + S + k);
      uy_prev = (PartT<R>)__ldcg(D.fields + 2 * S + k);
    }
    collide_node<R, MODE, FINAL, MASKED>(D, k, S, dst, hist, hm, cm, rho, ux, uy, G00, G01, G10,
                                         G11, dPx, dPy, dRx, dRy, Fx, Fy, So[0], So[1], So[2], uxo,
                                         uyo, ux_prev, uy_prev, part, plo);
  } else if (FINAL && solid) {
    // a solid node reports zero fields and adds nothing to the totals
    const int ks = y * nx + x;
#pragma unroll
    for (int j = 0; j < 6; ++j) D.fields[(size_t)j * S + ks] = 0.0;
  }

  if (FINAL) tile_partials<NT, PartT<R>>(D, T, part, plo, active, partials, s_red);
}

// One CTA of NT threads per tile (NT a multiple of 32, at least 32, with
// TX * TY <= NT for every tile of the launch).  The plain variant leaves
// masked tiles to the masked one (which runs over a separate list of just
// those tiles).
template <typename R, int MODE, bool FINAL, bool MASKED, int NT>
__global__ void __launch_bounds__(NT, MinBlocks<R, MASKED, NT>::value)
    step_kernel(const InstDev* __restrict__ insts, const TileDev* __restrict__ tiles,
                int parity, double* __restrict__ partials) {
  static_assert(NT % 32 == 0 && NT >= 32, "whole warps; the final-step reduction reads 14 lanes");
  constexpr int kRegion = region_max(NT);
  __shared__ R s_rho[kRegion];
  __shared__ R s_ux[kRegion];
  __shared__ R s_uy[kRegion];
  __shared__ double s_red[NT / 32][kPartial];
  const TileDev T = tiles[blockIdx.x];
  if (!MASKED && T.masked) return;
  process_tile<R, MODE, FINAL, MASKED, NT>(insts, T, parity, partials, s_rho, s_ux, s_uy, s_red);
}

// ---- float64 steps of tiny batches: one lattice per warp --------------------
//
// GB300 issues a float64 instruction only once every 64 cycles per warp, and
// a warp pays that for every instruction whatever the number of active
// lanes; four warps per SM saturate its float64 pipe.  A float64 batch too
// small to give every SM several warps is therefore bound by the float64
// instruction count of one thread's node, not by the number of nodes.  This
// variant spreads the update of each node over four warps: warp 0 carries
// the hydrodynamic lattice (pull, Zou-He, moments, rho and u, the gradients
// and the hydrodynamic collision), warp 1 + l the conformation lattice l
// (pull, CNEBB, moments, its component of Phi_ab and its collision); the
// warps meet in shared memory twice (rho, u; the three phi).  Every value is
// the same expression of the same operands as in process_tile, so the
// fields are bit-identical to those of the one-warp kernel.
//   Tiles of at most 32 nodes (TX * TY <= 32), plain tiles only (no mask, no
//   open column, Oldroyd-B with the eq_p_G_1 form of G~), time steps only
//   (the initialisation runs the one-warp kernel).
constexpr int kSplitThreads = 128;

template <bool FINAL>
__device__ __forceinline__ void process_tile_split(const InstDev* __restrict__ insts,
                                                   const TileDev T, int parity,
                                                   double* __restrict__ partials,
                                                   double* s_rho, double* s_ux, double* s_uy,
                                                   double (*s_phi)[32], double (*s_red)[kPartial]) {
  using R = double;
  constexpr int MODE = kModeStep;
  const InstDev& D = insts[T.inst];
  const int nx = D.nx, ny = D.ny, S = D.stride, TX = D.TX, TY = D.TY, hy = D.hy;
  const bool py = D.periodic_y != 0;
  const void* src = D.pop[parity];
  const R* __restrict__ srcR = (const R*)src;
  R* __restrict__ dst = (R*)D.pop[parity ^ 1];
  const R* __restrict__ force = (const R*)D.force;
  R* __restrict__ hist = (R*)D.hist;
  const bool ffield = D.force_field != 0;
  const R Fx0 = coef<R>(D, kCoefFx), Fy0 = coef<R>(D, kCoefFy);
  const int RW = TX + 2;
  const int role = threadIdx.x >> 5, lane = threadIdx.x & 31;  // 0 hydro, 1 + l lattice l
  const int tx = lane % TX, ty = lane / TX;
  const bool in_tile = ty < TY;
  const int x = T.x0 + tx, y = T.y0 + ty;
  const bool inside = in_tile && (x < nx) && (y < ny);
  const bool active = inside;
  const int ri = (ty + hy) * RW + tx + 1;
  const bool wb = active && !py && y == 0, wt = active && !py && y == ny - 1;
  const bool wcomp = wb || wt;
  const int nring = 2 * hy * TX + 2 * TY;

  // ---- phase A: pulls -------------------------------------------------------
  // the halo ring's hydrodynamic pulls go to the conformation warps (their
  // own float64 work is the lighter one)
  const int q = threadIdx.x - 32;
  int ring_r = -1, rgx = 0, rgy = 0;
  R dr[9];
  if (role > 0 && q < nring) {
    int lx, ly;
    ring_slot(q, RW, TY, hy, lx, ly);
    if (region_node(lx, ly, T.x0, T.y0, hy, nx, ny, py, rgx, rgy)) {
      ring_r = ly * RW + lx;
      int rm, rp;
      neighbour_rows(rgy, nx, ny, py, rm, rp);
      const int xm = rgx == 0 ? nx - 1 : rgx - 1, xp = rgx == nx - 1 ? 0 : rgx + 1;
      PopSource<R, MODE>::hydro(src, S, nx, rgy * nx + rgx, rgy * nx, rm, rp, rgx, xm, xp, dr);
    }
  }
  const int l = role - 1;
  R d[9], post[3] = {R(0), R(0), R(0)}, So = R(0), uxo = R(0), uyo = R(0), Fx = Fx0, Fy = Fy0;
  int k = 0;
  if (active) {
    k = y * nx + x;
    int rm, rp;
    neighbour_rows(y, nx, ny, py, rm, rp);
    const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
    if (role == 0) {
      PopSource<R, MODE>::hydro(src, S, nx, k, y * nx, rm, rp, x, xm, xp, d);
      if (FINAL) prefetch_prev_u(D, k, S);
    } else {
      PopSource<R, MODE>::cde(src, l, S, nx, k, y * nx, rm, rp, x, xm, xp, d);
      So = hist[(size_t)l * S + k];
      uxo = hist[3 * S + k];
      uyo = hist[4 * S + k];
      if (wcomp) {
        const int h0 = wb ? 4 : 2, h1 = wb ? 7 : 5, h2 = wb ? 8 : 6;
        const R* own = srcR + (size_t)(9 + 9 * l) * S + k;
        post[0] = own[h0 * S];
        post[1] = own[h1 * S];
        post[2] = own[h2 * S];
      }
    }
    if (ffield) {
      Fx = force[k];
      Fy = force[S + k];
    }
  }
  // ring moments (a ring longer than the three conformation warps, which the
  // tile widths of the one-warp CTAs never make, is finished by warp 0 below)
  if (ring_r >= 0) {
    const int rk = rgy * nx + rgx;
    const R rFx = ffield ? force[rk] : Fx0;
    const R rFy = ffield ? force[S + rk] : Fy0;
    if (!py && (rgy == 0 || rgy == ny - 1)) zou_he<R>(dr, rFx, rFy, rgy == 0);
    HydroM<R> m;
    hydro_moments<R>(dr, m);
    const R rho = R(1) + m.drho;
    s_rho[ring_r] = rho;
    const R irho = R(1) / rho;
    s_ux[ring_r] = (m.jx + R(0.5) * rFx) * irho;
    s_uy[ring_r] = (m.jy + R(0.5) * rFy) * irho;
  }
  for (int qq = kSplitThreads - 32 + threadIdx.x; role == 0 && qq < nring; qq += 32) {
    int lx, ly, gx, gy;
    ring_slot(qq, RW, TY, hy, lx, ly);
    if (!region_node(lx, ly, T.x0, T.y0, hy, nx, ny, py, gx, gy)) continue;
    R r, vx, vy;
    node_rho_u<R, MODE>(src, force, ffield, Fx0, Fy0, S, nx, ny, py, gx, gy, r, vx, vy);
    const int rr = ly * RW + lx;
    s_rho[rr] = r;
    s_ux[rr] = vx;
    s_uy[rr] = vy;
  }
  // own hydrodynamic moments (warp 0), and the wrapped nodes of a ragged tile
  HydroM<R> hm;
  if (role == 0) {
    if (active) {
      if (wcomp) zou_he<R>(d, Fx, Fy, wb);
      hydro_moments<R>(d, hm);
      const R rho = R(1) + hm.drho;
      const R irho_own = R(1) / rho;
      s_rho[ri] = rho;
      s_ux[ri] = (hm.jx + R(0.5) * Fx) * irho_own;
      s_uy[ri] = (hm.jy + R(0.5) * Fy) * irho_own;
    } else if (in_tile) {
      const int gx = x % nx;
      const int gy = py ? y % ny : y;
      if (gy < ny) {
        R r, vx, vy;
        node_rho_u<R, MODE>(src, force, ffield, Fx0, Fy0, S, nx, ny, py, gx, gy, r, vx, vy);
        s_rho[ri] = r;
        s_ux[ri] = vx;
        s_uy[ri] = vy;
      }
    }
  }
  __syncthreads();

  // ---- conformation walls with the node's own u, moments -----------------------
  R rho = R(1), ux = R(0), uy = R(0);
  if (active) {
    rho = s_rho[ri];
    ux = s_ux[ri];
    uy = s_uy[ri];
  }
  CdeM<R> cm;
  double wall_in = 0.0, wall_out = 0.0;
  if (role > 0 && active) {
    if (wcomp) {
      const R delta = (l == 1) ? R(0) : R(1);
      cnebb<R>(d, post[0], post[1], post[2], delta, ux, uy, wb, wall_in, wall_out);
    }
    cde_moments<R>(d, cm);
    s_phi[l][lane] = cm.dphi;
  }
  __syncthreads();

  // ---- phase B: gradients, source, this warp's collision, stores ---------------
  PartT<R> part[FINAL ? 14 : 1], plo[FINAL ? 12 : 1];
#pragma unroll
  for (int j = 0; j < (FINAL ? 14 : 1); ++j) part[j] = 0;
#pragma unroll
  for (int j = 0; j < (FINAL ? 12 : 1); ++j) plo[j] = 0;
  if (active) {
    const R half = R(0.5);
    const R G00 = half * (s_ux[ri + 1] - s_ux[ri - 1]);
    const R G01 = half * (s_uy[ri + 1] - s_uy[ri - 1]);
    R G10, G11, dPy;
    const int a = wb ? ri : (wt ? ri - 2 * RW : ri), b = wb ? ri : (wt ? ri - RW : ri - RW);
    const int c = wb ? ri + RW : (wt ? ri : ri + RW), e = wb ? ri + 2 * RW : ri;
    y_gradients<R>(wb, wt, s_rho[a], s_ux[a], s_uy[a], s_rho[b], s_ux[b], s_uy[b], rho, ux, uy,
                   s_rho[c], s_ux[c], s_uy[c], s_rho[e], s_ux[e], s_uy[e], G10, G11, dPy);
    R Axx, Axy, Ayy, Fxx, Fxy, Fyy;
    polymer_terms<R, false>(D, s_phi[0][lane], s_phi[1][lane], s_phi[2][lane], Axx, Axy, Ayy, Fxx,
                            Fxy, Fyy);
    if (role == 0) {
      const R cxp = s_rho[ri + 1] * s_ux[ri + 1] * s_ux[ri + 1] * s_ux[ri + 1];
      const R cxm = s_rho[ri - 1] * s_ux[ri - 1] * s_ux[ri - 1] * s_ux[ri - 1];
      const R dPx = half * (cxp - cxm);
      const R mpl = coef<R>(D, kCoefMupLam);
      const R txx = mpl * Fxx, txy = mpl * Fxy, tyy = mpl * Fyy;
      double ux_prev = 0.0, uy_prev = 0.0;
      if (FINAL) {
        ux_prev = D.fields[S + k];
        uy_prev = D.fields[2 * S + k];
      }
      collide_hydro<R>(D, k, S, dst, hm, rho, ux, uy, dPx, dPy, txx, txy, tyy, Fx, Fy);
      hist[3 * S + k] = ux;
      hist[4 * S + k] = uy;
      if (FINAL)
        final_node<R, MODE>(D, k, S, 0, hm.drho, rho, ux, uy, nullptr, ux_prev, uy_prev, part,
                            plo);
    } else {
      const R il = coef<R>(D, kCoefInvLam);
      const R sl = source_component<R>(l, Axx, Axy, Ayy, Fxx, Fxy, Fyy, il, G00, G01, G10, G11);
      collide_cde<R, false>(D, k, S, dst, l, cm, rho, ux, uy, sl, So, uxo, uyo, Fx, Fy, R(0),
                            R(0));
      hist[(size_t)l * S + k] = sl;
      if (FINAL) {
        const R dphi[3] = {s_phi[0][lane], s_phi[1][lane], s_phi[2][lane]};
        final_node<R, MODE>(D, k, S, role, R(0), rho, ux, uy, dphi, 0.0, 0.0, part, plo);
        part[kWallIn + l] = wall_in;
        part[kWallOut + l] = wall_out;
      }
    }
  }
  if (FINAL)
    tile_partials<kSplitThreads, double>(D, T, part, plo, active && role == 0, partials, s_red);
}

template <bool FINAL>
__global__ void __launch_bounds__(kSplitThreads, 4)
    step_kernel_split(const InstDev* __restrict__ insts, const TileDev* __restrict__ tiles,
                      int parity, double* __restrict__ partials) {
  constexpr int kRegion = region_max(32);
  __shared__ double s_rho[kRegion];
  __shared__ double s_ux[kRegion];
  __shared__ double s_uy[kRegion];
  __shared__ double s_phi[3][32];
  __shared__ double s_red[kSplitThreads / 32][kPartial];
  const TileDev T = tiles[blockIdx.x];
  if (T.masked) return;
  process_tile_split<FINAL>(insts, T, parity, partials, s_rho, s_ux, s_uy, s_phi, s_red);
}

}  // namespace lbve
