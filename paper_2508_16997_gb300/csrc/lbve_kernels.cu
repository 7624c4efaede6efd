// lbve_kernels.cu -- launchers of the step kernel, the deterministic float64
// reduction of per-tile partial records, and the force conversion kernel.
#include <cuda_runtime.h>

#include "lbve_internal.h"
#include "lbve_step.cuh"

namespace lbve {

template <typename R, int MODE, bool FINAL, bool MASKED, int NT>
static void launch_step_k(const InstDev* d_insts, const TileDev* d_tiles, int n_tiles, int parity,
                          double* d_partials, cudaStream_t st) {
  step_kernel<R, MODE, FINAL, MASKED, NT><<<n_tiles, NT, 0, st>>>(d_insts, d_tiles, parity,
                                                                  d_partials);
}

template <typename R, bool MASKED, int NT>
static int launch_step_t(const InstDev* d_insts, const TileDev* d_tiles, int n_tiles, int parity,
                         int mode, int flags, double* d_partials, cudaStream_t st) {
  if (n_tiles <= 0) return 0;
  const bool fin = (flags & kFinal) != 0;
  if (mode == kModeStep) {
    if (fin)
      launch_step_k<R, kModeStep, true, MASKED, NT>(d_insts, d_tiles, n_tiles, parity, d_partials,
                                                    st);
    else
      launch_step_k<R, kModeStep, false, MASKED, NT>(d_insts, d_tiles, n_tiles, parity,
                                                     d_partials, st);
  } else {
    launch_step_k<R, kModeInit, true, MASKED, NT>(d_insts, d_tiles, n_tiles, parity, d_partials,
                                                  st);
  }
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;  // the caller reads and clears it
}

template <typename R, int NT>
static int launch_step_m(const InstDev* d_insts, const TileDev* d_tiles, int n_tiles, int parity,
                         int mode, int flags, double* d_partials, cudaStream_t st, int masked) {
  return masked ? launch_step_t<R, true, NT>(d_insts, d_tiles, n_tiles, parity, mode, flags,
                                             d_partials, st)
                : launch_step_t<R, false, NT>(d_insts, d_tiles, n_tiles, parity, mode, flags,
                                              d_partials, st);
}

// Only the CTA sizes the host plans are instantiated; any other is refused.
int launch_step(int prec, int threads, const InstDev* d_insts, const TileDev* d_tiles,
                int n_tiles, int parity, int mode, int flags, double* d_partials, void* stream,
                int masked) {
  cudaStream_t st = (cudaStream_t)stream;
  if (prec == 0 && threads == kThreads64)
    return launch_step_m<double, kThreads64>(d_insts, d_tiles, n_tiles, parity, mode, flags,
                                             d_partials, st, masked);
  if (prec == 0 && threads == kThreads64Tiny) {
    // tiles of at most 32 nodes: the time steps of plain tiles spread each
    // node over four warps (one lattice each), the rest runs one warp a tile
    if (!masked && mode == kModeStep && n_tiles > 0) {
      if (flags & kFinal)
        step_kernel_split<true><<<n_tiles, kSplitThreads, 0, st>>>(d_insts, d_tiles, parity,
                                                                   d_partials);
      else
        step_kernel_split<false><<<n_tiles, kSplitThreads, 0, st>>>(d_insts, d_tiles, parity,
                                                                    d_partials);
      return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;  // the caller reads and clears it
    }
    return launch_step_m<double, kThreads64Tiny>(d_insts, d_tiles, n_tiles, parity, mode, flags,
                                                 d_partials, st, masked);
  }
  if (prec == 0 && threads == kThreads64Small)
    return launch_step_m<double, kThreads64Small>(d_insts, d_tiles, n_tiles, parity, mode, flags,
                                                  d_partials, st, masked);
  if (prec == 1 && threads == kThreads)
    return launch_step_m<float, kThreads>(d_insts, d_tiles, n_tiles, parity, mode, flags,
                                          d_partials, st, masked);
  if (prec == 2 && threads == kThreads && !masked)  // float32 pairs: plain tiles only
    return launch_step_t<df32, false, kThreads>(d_insts, d_tiles, n_tiles, parity, mode, flags,
                                                d_partials, st);
  return -1;
}

// One CTA per instance: sum (max for the residual) the partial records of the
// instance's tiles, and the wall-pass records of its mask walls, in a fixed
// order, so totals are bit-reproducible.  CTA b takes instance ids[b], or
// first_inst + b without a list.  Warp j of the 16 reduces total j: each lane
// runs over every 32nd record, then the warp folds its lanes by shuffles
// (no block-wide barrier: GB300 issues float64 additions slowly, so the
// sums are spread over warps instead of levels of a shared-memory tree).
constexpr int kReduceThreads = 32 * kTotals;
static_assert(kTotals == kDrag + 2, "one warp per total");
__global__ void __launch_bounds__(kReduceThreads) reduce_kernel(const InstDev* __restrict__ insts,
                                                                int first_inst,
                                                                const int32_t* __restrict__ ids,
                                                                const double* __restrict__ partials,
                                                                double* __restrict__ totals,
                                                                int32_t* __restrict__ flags) {
  const int inst = ids ? ids[blockIdx.x] : first_inst + blockIdx.x;
  const InstDev& D = insts[inst];
  const int j = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool is_max = j == kResid;
  double v = 0.0;
  if (j < kDrag)
    for (int q = D.slot_begin + lane; q < D.slot_end; q += 32) {
      const double p = partials[(size_t)q * kPartial + j];
      v = is_max ? fmax(v, p) : v + p;
    }
  // wall record layout: drag x, drag y, in x3, out x3
  const int r = (j >= kDrag) ? j - kDrag : (j >= kWallIn && j < kResid) ? 2 + (j - kWallIn) : -1;
  if (r >= 0)
    for (int q = lane; q < D.wall_cap; q += 32) v += D.wall_rec[(size_t)q * kWallRec + r];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double w = __shfl_xor_sync(0xffffffffu, v, o);
    v = is_max ? fmax(v, w) : v + w;
  }
  if (lane == 0) {
    totals[(size_t)inst * kTotals + j] = v;
    if (j == kNonFinite && v > 0.0) flags[inst] |= 1;
  }
}

int launch_reduce(const InstDev* d_insts, int first_inst, int n_insts, const double* d_partials,
                  double* d_totals, int32_t* d_flags, void* stream, const int32_t* d_ids) {
  if (n_insts <= 0) return 0;
  reduce_kernel<<<n_insts, kReduceThreads, 0, (cudaStream_t)stream>>>(d_insts, first_inst, d_ids,
                                                                      d_partials, d_totals,
                                                                      d_flags);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;  // the caller reads and clears it
}

// Staged inputs of a list of lbve_set_geometry calls, one grid row
// (blockIdx.y) per list entry j, instance ids[j]:
//   what[j] bit 0: a float64 body force is staged in pop[parity] ([2][stride]):
//                  checked and converted to the instance's precision into
//                  its force planes;
//   what[j] bit 1: float64 initial fields are staged in pop[parity ^ 1]
//                  ([6][stride]): checked; without it the default fields
//                  (rho = 1, u = 0, A = I) are written there.
// The checks test the float64 bit patterns as integers: every force
// component and initial field finite (exponent field not all ones), every
// initial density in (0, +inf).  A failure sets bit `bit` of flags[ids[j]],
// which clear_flags_kernel has zeroed.
template <typename R>
__device__ __forceinline__ void store_force(void* dst, size_t i, double v) {
  ((R*)dst)[i] = R(v);
}

__global__ void __launch_bounds__(256) geometry_inputs_kernel(const InstDev* __restrict__ insts,
                                                               const int32_t* __restrict__ ids,
                                                               const int32_t* __restrict__ what,
                                                               int parity,
                                                               int32_t* __restrict__ flags,
                                                               int bit) {
  const int j = blockIdx.y;
  const InstDev& D = insts[ids[j]];
  const int n = D.nx * D.ny, S = D.stride, w = what[j], prec = D.prec;
  const double* __restrict__ fstage = (const double*)D.pop[parity];
  double* __restrict__ stage = (double*)D.pop[parity ^ 1];
  bool bad = false;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (w & 1) {
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const double v = fstage[(size_t)c * S + i];
        bad |= ((__double_as_longlong(v) >> 52) & 0x7ff) == 0x7ff;
        if (prec == 0)
          store_force<double>(D.force, (size_t)c * S + i, v);
        else if (prec == 2)
          store_force<df32>(D.force, (size_t)c * S + i, v);
        else
          store_force<float>(D.force, (size_t)c * S + i, v);
      }
    }
    if (w & 2) {
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        const long long b = __double_as_longlong(stage[(size_t)c * S + i]);
        bad |= ((b >> 52) & 0x7ff) == 0x7ff;
      }
      const long long r = __double_as_longlong(stage[i]);
      bad |= !(r > 0 && r < 0x7ff0000000000000ll);
    } else {
      stage[i] = 1.0;
      stage[(size_t)S + i] = 0.0;
      stage[2 * (size_t)S + i] = 0.0;
      stage[3 * (size_t)S + i] = 1.0;
      stage[4 * (size_t)S + i] = 0.0;
      stage[5 * (size_t)S + i] = 1.0;
    }
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&flags[ids[j]], 1 << bit);
}

__global__ void clear_flags_kernel(const int32_t* __restrict__ ids, int n,
                                   int32_t* __restrict__ flags) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
    flags[ids[j]] = 0;
}

int launch_geometry_inputs(const InstDev* d_insts, const int32_t* d_ids, const int32_t* d_what,
                           int n_list, int max_nodes, int parity, int32_t* d_flags, int bit,
                           void* stream) {
  if (n_list <= 0) return 0;
  cudaStream_t st = (cudaStream_t)stream;
  clear_flags_kernel<<<(n_list + 255) / 256, 256, 0, st>>>(d_ids, n_list, d_flags);
  // about eight nodes per thread for the largest instance, at most 64 CTAs per entry
  int gx = (max_nodes + 2047) / 2048;
  gx = gx < 1 ? 1 : (gx > 64 ? 64 : gx);
  constexpr int kMaxRows = 65535;  // grid y limit
  for (int j0 = 0; j0 < n_list; j0 += kMaxRows) {
    const int rows = n_list - j0 < kMaxRows ? n_list - j0 : kMaxRows;
    geometry_inputs_kernel<<<dim3(gx, rows), 256, 0, st>>>(d_insts, d_ids + j0, d_what + j0, parity,
                                                           d_flags, bit);
  }
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;  // the caller reads and clears it
}

}  // namespace lbve
