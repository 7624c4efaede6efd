// lbve_adjoint.cu -- launchers of the adjoint passes (see lbve_adjoint.cuh).
#include <cuda_runtime.h>

#include "lbve_adjoint.cuh"
#include "lbve_internal.h"

namespace lbve {

template <typename R>
static AdjArgs<R> cast_args(const AdjArgsRaw& a) {
  AdjArgs<R> A;
  A.X = (const R*)a.X;
  A.init = a.init;
  A.force = (const R*)a.force;
  A.M = (R*)a.M;
  A.lam_next = (const R*)a.lam_next;
  A.lam_fields = a.lam_fields;
  A.lam_pulled = (R*)a.lam_pulled;
  A.lam_G = (R*)a.lam_G;
  A.lam_dir = (R*)a.lam_dir;
  A.lam_mh = (R*)a.lam_mh;
  A.lam_cur = (R*)a.lam_cur;
  A.dF = a.dF;
  A.mask = a.mask;
  A.widx = a.widx;
  A.walls = a.walls;
  A.dq = a.dq;
  A.drag_w[0] = a.drag_w[0];
  A.drag_w[1] = a.drag_w[1];
  A.final_pass = a.final_pass;
  return A;
}

// OPEN: the node passes' variant with an open channel's inlet and outlet
// columns (one-sided x-differences there in every mode, the column pass's
// completion in the step modes).
template <typename R, int MODE, bool OPEN>
static void run_pass(int pass, const InstDev* d, const AdjArgs<R>& A, int blocks, cudaStream_t st) {
  switch (pass) {
    case 0: adj_moments<R, MODE, OPEN><<<blocks, 256, 0, st>>>(d, A); break;
    case 1: adj_local<R, MODE, OPEN><<<blocks, 256, 0, st>>>(d, A); break;
    case 2: adj_gather<R, MODE, OPEN><<<blocks, 256, 0, st>>>(d, A); break;
    case 4: adj_column<R, MODE><<<blocks, 256, 0, st>>>(d, A); break;
    default: adj_pull<R><<<blocks, 256, 0, st>>>(d, A); break;
  }
}

template <typename R>
static void run_mode(int mode, int pass, bool open, const InstDev* d, const AdjArgs<R>& A,
                     int blocks, cudaStream_t st) {
  if (mode == kAdjStep) {
    if (open) run_pass<R, kAdjStep, true>(pass, d, A, blocks, st);
    else run_pass<R, kAdjStep, false>(pass, d, A, blocks, st);
  } else if (mode == kAdjFields) {
    if (open) run_pass<R, kAdjFields, true>(pass, d, A, blocks, st);
    else run_pass<R, kAdjFields, false>(pass, d, A, blocks, st);
  } else {
    if (open) run_pass<R, kAdjInit, true>(pass, d, A, blocks, st);
    else run_pass<R, kAdjInit, false>(pass, d, A, blocks, st);
  }
}

int launch_adjoint(int prec, int mode, int pass, const InstDev* d_desc, const AdjArgsRaw& a,
                   int n_nodes, void* stream) {
  const int blocks = (n_nodes + 255) / 256;
  if (blocks <= 0) return 0;
  cudaStream_t st = (cudaStream_t)stream;
  const bool open = a.open != 0;
  if (prec == 0) run_mode<double>(mode, pass, open, d_desc, cast_args<double>(a), blocks, st);
  else run_mode<float>(mode, pass, open, d_desc, cast_args<float>(a), blocks, st);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;  // the caller reads and clears it
}

}  // namespace lbve
