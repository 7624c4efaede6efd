// lbve_host.cu -- host side of the C ABI declared in include/lbve.h.
//
// Plans the workspace layout, derives the lattice coefficients in float64
// (Sec. 2.4-2.5 and the relaxation-time relations of Secs. 3.1-3.2), builds
// the tile tables and drives the kernels on the caller's stream.  It never
// allocates device memory: every buffer lives in the caller's workspace.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/lbve.h"
#include "lbve_internal.h"

using namespace lbve;

namespace {
thread_local std::string g_last_error;
}  // namespace

namespace lbve {
int set_error(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}
}  // namespace lbve

namespace {


int cuda_fail(cudaError_t e, const char* what) {
  return set_error(LBVE_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

constexpr size_t kAlign = 256;
constexpr int64_t kMaxNodes = int64_t(1) << 25;  // keeps 36 * stride in int32

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct Coeffs {
  double Uc, nu0, nus, mup, tau_s1, tau_s2, kappa, tau_p1, tau_p2, lambda;
};

// Sec. 2.4-2.5 and Secs. 3.1-3.2 (rho_0 = 1, dt = dx = 1, c_s^2 = 1/3).
Coeffs derive(const lbve_params& p) {
  Coeffs c;
  c.Uc = p.Ma * std::sqrt(1.0 / 3.0);              // eq_Mach
  c.nu0 = c.Uc * p.Lc / p.Re;                      // eqb5
  c.nus = p.beta * c.nu0;                          // eqb7
  c.mup = (1.0 - p.beta) * c.nu0;                  // mu_0 = mu_s + mu_p
  c.tau_s1 = 3.0 * c.nus + 0.5;                    // mu_s = rho cs2 (tau_s1 - 1/2)
  c.tau_s2 = p.Lambda_s / (c.tau_s1 - 0.5) + 0.5;  // Lambda_s relation
  c.kappa = c.nus / p.Sc;                          // eqb8
  c.tau_p1 = 3.0 * c.kappa + 0.5;                  // kappa = (tau_p1 - 1/2) cs2
  c.tau_p2 = p.Lambda_p / (c.tau_p1 - 0.5) + 0.5;  // tau_p2 relation
  c.lambda = p.Wi * p.Lc / c.Uc;                   // eqb6
  return c;
}

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

int validate(const lbve_params& p, int i) {
  if (p.nx < 1 || p.ny < 1) return set_error(LBVE_ERR_ARG, "instance %d: nx, ny must be >= 1", i);
  if (!p.periodic_y && p.ny < 3)
    return set_error(LBVE_ERR_ARG, "instance %d: a walled channel needs ny >= 3", i);
  if (int64_t(p.nx) * p.ny > kMaxNodes)
    return set_error(LBVE_ERR_ARG, "instance %d: more than %lld nodes", i, (long long)kMaxNodes);
  if (p.precision != LBVE_FP64 && p.precision != LBVE_FP32_DEV && p.precision != LBVE_DF32)
    return set_error(LBVE_ERR_ARG, "instance %d: unknown precision %d", i, p.precision);
  if (p.precision == LBVE_DF32 &&
      (p.max_wall_nodes != 0 || p.open_x != 0 || p.model != 0 || p.gtilde != 0))
    return set_error(LBVE_ERR_ARG,
                     "instance %d: LBVE_DF32 covers Oldroyd-B instances with flat walls or periodic "
                     "rows (no solid mask, open channel, FENE model or eq_p_G form)",
                     i);
  if (p.periodic_y != 0 && p.periodic_y != 1)
    return set_error(LBVE_ERR_ARG, "instance %d: periodic_y must be 0 or 1", i);
  if (!(std::isfinite(p.beta) && p.beta > 0.0 && p.beta <= 1.0))
    return set_error(LBVE_ERR_ARG, "instance %d: beta must be in (0, 1]", i);
  if (!finite_pos(p.Wi) || !finite_pos(p.Re) || !finite_pos(p.Sc) || !finite_pos(p.Ma) ||
      !finite_pos(p.Lc) || !finite_pos(p.Lambda_s) || !finite_pos(p.Lambda_p))
    return set_error(LBVE_ERR_ARG, "instance %d: Wi, Re, Sc, Ma, Lc, Lambda_s, Lambda_p must be > 0",
                i);
  if (!std::isfinite(p.Fx) || !std::isfinite(p.Fy))
    return set_error(LBVE_ERR_ARG, "instance %d: body force must be finite", i);
  if (p.model < 0 || p.model > 2)
    return set_error(LBVE_ERR_ARG, "instance %d: model must be 0 (Oldroyd-B), 1 (FENE-P) or 2 (FENE-CR)",
                i);
  if (p.model != 0 && !(std::isfinite(p.L2) && p.L2 > 2.0))
    return set_error(LBVE_ERR_ARG, "instance %d: a FENE model needs L2 > 2", i);
  if (p.gtilde != 0 && p.gtilde != 1)
    return set_error(LBVE_ERR_ARG, "instance %d: gtilde must be 0 or 1", i);
  if (p.open_x != 0 && p.open_x != 1)
    return set_error(LBVE_ERR_ARG, "instance %d: open_x must be 0 or 1", i);
  if (p.open_x && p.nx < 5)
    return set_error(LBVE_ERR_ARG, "instance %d: an open channel needs nx >= 5", i);
  if (p.max_wall_nodes < 0 || int64_t(p.max_wall_nodes) > int64_t(p.nx) * p.ny)
    return set_error(LBVE_ERR_ARG, "instance %d: max_wall_nodes must be in [0, nx*ny]", i);
  if (p.tile_tx != 0 &&
      (p.tile_tx < 1 || p.tile_tx > tile_tx_max(p.precision) || p.tile_tx > p.nx))
    return set_error(LBVE_ERR_ARG, "instance %d: tile_tx must be 0 or in [1, min(%d, nx)]", i,
                tile_tx_max(p.precision));
  const Coeffs c = derive(p);
  if (!(c.tau_s1 > 0.5) || !(c.tau_p1 > 0.5) || !std::isfinite(c.tau_s2) ||
      !std::isfinite(c.tau_p2) || !finite_pos(c.lambda))
    return set_error(LBVE_ERR_ARG, "instance %d: derived relaxation times are degenerate", i);
  return LBVE_OK;
}

// Tile lists, one per storage precision: 0 = float64, 1 = float32
// deviations, 2 = float32 pairs (the list index is the precision code).
constexpr int kLists = 3;

// Bytes of one stored value of a precision.
size_t elem_size(int precision) { return precision == LBVE_FP32_DEV ? 4 : 8; }

struct InstPlan {
  size_t off_pop[2], off_hist, off_force, off_fields, off_mask, off_inlet, off_colbuf;
  int col_begin;             // first open-column task of this instance in its list
  int wall_begin, wall_cap;  // wall-node records of this instance in its list
  int stride, TX, TY, hy, ntx, nty;
  int list;                  // tile list of this instance
  int tile_begin, ntiles;    // range in the list's tile table
  int slot_begin, nslots;    // partial-record slots
};

struct Plan {
  std::vector<InstPlan> inst;
  size_t off_insts, off_tiles[kLists], off_partials, off_totals, off_flags, off_geo, total;
  int ntiles[kLists], nslots;
  int cap_tiles[kLists];  // tile-table capacity: the most tiles any tile width gives
  int threads[kLists];    // CTA size of each list's step launches
  size_t off_mtiles[kLists], off_walls[kLists], off_wrec[kLists], off_cols[kLists];
  int wall_cap[kLists];   // wall-node records per list
  int ncols[kLists];      // open-column tasks per list
};

// Default tile width: 32 (one warp along x), or 8 for the one-warp float64
// CTAs, whose 8 x 4 tiles have a third of the halo ring of 32 x 1 tiles.
int default_tile_tx(const lbve_params& p, int threads = kThreads) {
  const int w = threads == kThreads64Tiny ? kTileTXTiny : kTileTX;
  return p.nx >= w ? w : p.nx;
}

int tile_width(const lbve_params& p, int threads) {
  return p.tile_tx > 0 ? p.tile_tx : default_tile_tx(p, threads);
}

// Tile of TX x (threads / TX) nodes for CTAs of `threads` threads.
void tile_shape(const lbve_params& p, int threads, int& TX, int& TY, int& hy) {
  TX = tile_width(p, threads);
  TY = threads / TX;
  hy = p.periodic_y ? 1 : 2;
}

int64_t tiles_for(const lbve_params& p, int TX, int threads) {
  const int TY = threads / TX;
  return int64_t((p.nx + TX - 1) / TX) * ((p.ny + TY - 1) / TY);
}

// Most tiles any admissible tile width and CTA size give for p: the
// workspace layout is sized by it, so the same workspace serves every tile
// width (and the CTA size the widths imply for the batch).
int64_t max_tiles(const lbve_params& p) {
  int64_t m = 0;
  for (int TX = 1; TX <= std::min(tile_tx_max(p.precision), p.nx); ++TX) {
    m = std::max(m, tiles_for(p, TX, threads_of(p.precision)));
    if (p.precision == LBVE_FP64 && TX <= kThreads64Small / 2)
      m = std::max(m, tiles_for(p, TX, kThreads64Small));
    if (p.precision == LBVE_FP64 && TX <= kThreads64Tiny / 2)
      m = std::max(m, tiles_for(p, TX, kThreads64Tiny));
  }
  return m;
}

// CTA size of the float64 list.  The FP64 pipe bounds the float64 step, so a
// batch whose 256-thread tiles would not give every SM one tile leaves SMs
// idle while the others work through 256 nodes each; 64-thread tiles spread
// the same nodes over four times as many CTAs, and one-warp tiles over eight
// times as many when even the 64-thread tiles number fewer than the SMs.
// Chosen from the parameters alone (the workspace plan needs no device): the
// smallest size whose larger neighbour would leave SMs without a tile, as
// long as no float64 instance asks for a tile wider than half the CTA.
int fp64_threads(const lbve_params* p, int n) {
  int64_t t256 = 0, t64 = 0;
  int maxtx = 0;
  bool any = false;
  for (int i = 0; i < n; ++i) {
    if (p[i].precision != LBVE_FP64) continue;
    if (p[i].tile_tx > kThreads64Small / 2) return kThreads64;
    any = true;
    maxtx = std::max(maxtx, (int)p[i].tile_tx);
    t256 += tiles_for(p[i], tile_width(p[i], kThreads64), kThreads64);
    t64 += tiles_for(p[i], tile_width(p[i], kThreads64Small), kThreads64Small);
  }
  if (!any || t256 >= kNumSMs) return kThreads64;
  if (maxtx > kThreads64Tiny / 2 || t64 >= kNumSMs) return kThreads64Small;
  return kThreads64Tiny;
}

Plan make_plan(const lbve_params* p, int n) {
  Plan pl;
  pl.inst.resize(n);
  size_t off = 0;
  for (int l = 0; l < kLists; ++l) pl.ntiles[l] = pl.cap_tiles[l] = pl.wall_cap[l] = pl.ncols[l] = 0;
  pl.threads[0] = fp64_threads(p, n);
  pl.threads[1] = kThreads;
  pl.threads[2] = kThreads;
  for (int i = 0; i < n; ++i) {
    InstPlan& q = pl.inst[i];
    const size_t es = elem_size(p[i].precision);
    const size_t nn = size_t(p[i].nx) * p[i].ny;
    q.stride = (int)align_up(nn, 64);
    const size_t plane = size_t(q.stride) * es;
    for (int b = 0; b < 2; ++b) {
      q.off_pop[b] = off;
      off = align_up(off + 36 * plane, kAlign);
    }
    q.off_hist = off;
    off = align_up(off + 5 * plane, kAlign);
    q.off_force = off;
    off = align_up(off + 2 * plane, kAlign);
    q.off_fields = off;
    off = align_up(off + 6 * size_t(q.stride) * 8, kAlign);
    q.off_mask = off;
    if (p[i].max_wall_nodes > 0) off = align_up(off + size_t(q.stride), kAlign);
    q.off_inlet = q.off_colbuf = off;
    if (p[i].open_x) {
      off = align_up(off + sizeof(double) * 5 * p[i].ny, kAlign);
      q.off_colbuf = off;
      off = align_up(off + 36 * 2 * size_t(p[i].ny) * es, kAlign);
    }
    q.list = p[i].precision;
    tile_shape(p[i], pl.threads[q.list], q.TX, q.TY, q.hy);
    q.wall_begin = pl.wall_cap[q.list];
    q.wall_cap = p[i].max_wall_nodes;
    pl.wall_cap[q.list] += q.wall_cap;
    q.col_begin = pl.ncols[q.list];
    if (p[i].open_x) pl.ncols[q.list] += 2 * p[i].ny;
    q.ntx = (p[i].nx + q.TX - 1) / q.TX;
    q.nty = (p[i].ny + q.TY - 1) / q.TY;
    q.tile_begin = pl.ntiles[q.list];
    q.ntiles = q.ntx * q.nty;
    pl.ntiles[q.list] += q.ntiles;
    pl.cap_tiles[q.list] += (int)max_tiles(p[i]);
  }
  // partial-record slots: [list 0 | list 1]
  pl.nslots = 0;
  for (int l = 0; l < kLists; ++l) pl.nslots += pl.ntiles[l];
  for (int i = 0; i < n; ++i) {
    InstPlan& q = pl.inst[i];
    int base = 0;
    for (int l = 0; l < q.list; ++l) base += pl.ntiles[l];
    q.slot_begin = base + q.tile_begin;
    q.nslots = q.ntiles;
  }
  pl.off_insts = off;
  off = align_up(off + sizeof(InstDev) * n, kAlign);
  for (int l = 0; l < kLists; ++l) {
    pl.off_tiles[l] = off;
    off = align_up(off + sizeof(TileDev) * std::max(pl.cap_tiles[l], 1), kAlign);
  }
  for (int l = 0; l < kLists; ++l) {
    pl.off_mtiles[l] = off;
    off = align_up(off + sizeof(TileDev) * std::max(pl.cap_tiles[l], 1), kAlign);
    pl.off_walls[l] = off;
    off = align_up(off + sizeof(WallDev) * std::max(pl.wall_cap[l], 1), kAlign);
    pl.off_wrec[l] = off;
    off = align_up(off + sizeof(double) * kWallRec * std::max(pl.wall_cap[l], 1), kAlign);
    pl.off_cols[l] = off;
    off = align_up(off + sizeof(ColTask) * std::max(pl.ncols[l], 1), kAlign);
  }
  pl.off_partials = off;
  int cap_all = 0;
  for (int l = 0; l < kLists; ++l) cap_all += pl.cap_tiles[l];
  off = align_up(off + sizeof(double) * kPartial * std::max(cap_all, 1), kAlign);
  pl.off_totals = off;
  off = align_up(off + sizeof(double) * kTotals * n, kAlign);
  pl.off_flags = off;
  off = align_up(off + sizeof(int32_t) * n, kAlign);
  pl.off_geo = off;  // list of a batched lbve_set_geometry: ids[n], what[n]
  off = align_up(off + sizeof(int32_t) * 2 * n, kAlign);
  pl.total = off;
  return pl;
}

}  // namespace

struct lbve_handle {
  int n = 0;
  std::vector<lbve_params> p;
  std::vector<Coeffs> c;
  Plan plan;
  char* ws = nullptr;
  cudaStream_t stream = nullptr;
  std::vector<InstDev> insts;
  InstDev* d_insts = nullptr;
  TileDev* d_tiles[kLists] = {};
  double* d_partials = nullptr;
  double* d_totals = nullptr;
  int32_t* d_flags = nullptr;
  int32_t* d_geo = nullptr;  // [2][n]: instance ids and staged inputs of a geometry call
  int parity = 0;
  std::vector<int64_t> t;
  std::vector<char> ready;
  // solid masks: host copies of the tile tables (their masked flags), the
  // masked-tile tables run by the masked kernel, and the wall-node records
  TileDev* d_mtiles[kLists] = {};
  WallDev* d_walls[kLists] = {};
  double* d_wrec[kLists] = {};
  std::vector<TileDev> tiles_h[kLists];
  int nmasked[kLists] = {};
  int nmasked_inst[kLists] = {};  // instances of the list that carry a mask
  std::vector<std::vector<TileDev>> mtiles_of;  // masked tiles of each instance
  std::vector<int> mbegin;                      // first entry of each in its masked table
  std::vector<std::vector<WallDev>> walls_of;   // wall-node records of each instance
  std::vector<std::vector<int32_t>> wall_index; // node -> record, per masked instance
  std::vector<uint64_t> geom_hash;              // mask + wall fractions, 0 = no mask
  std::vector<std::vector<uint8_t>> mask_h;     // host copy of each mask
  ColTask* d_cols[kLists] = {};  // open-column tasks per list
  int nopen_inst[kLists] = {};   // open channels per list
  std::vector<std::vector<double>> inlet_h;     // inlet profile of each open channel
  // CUDA graph of kGraphSteps non-final steps starting at parity 0, captured
  // on a private stream on first use and replayed on the caller's stream
  cudaStream_t cap_stream = nullptr;
  // masked tiles run on a forked stream beside the plain ones (disjoint
  // nodes, shared read-only source), joined before the step ends
  cudaStream_t side_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // chunked geometry set-up: the uploads of chunk c on the side stream, its
  // launches on the caller's stream once geo_ev[c] has passed
  static constexpr int kGeoChunks = 8;
  cudaEvent_t geo_ev[kGeoChunks] = {};
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  // per-launch timing of the plain step kernels (lbve_profile): two events
  // per launch, per tile list and per kind (0 non-final steps, 1 the final
  // step of a call), recorded on the caller's stream
  int prof_cap = 0;
  int prof_n[kLists][2] = {};
  std::vector<cudaEvent_t> prof_ev[kLists][2];
};

namespace {

constexpr int kGraphSteps = 32;  // even, so a replay leaves the parity unchanged

// Launch one time step of every tile list on stream st with the given parity.
// With masks the step forks: the side stream runs the wall pass (which
// completes the populations that wall nodes pull from solid nodes) and then
// the masked tiles, while the plain tiles, which never read what the wall
// pass writes, run on the caller's stream; the two join before the step ends.
int launch_one_step(lbve_handle* h, int parity, int flags, cudaStream_t st) {
  bool fork = false;  // any tile of the general variant
  for (int l = 0; l < kLists; ++l) fork = fork || h->nmasked[l] > 0;
  if (fork) {
    cudaError_t e = cudaEventRecord(h->ev_fork, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->side_stream, h->ev_fork, 0);
    if (e != cudaSuccess) return cuda_fail(e, "fork of the masked-tile stream");
    for (int l = 0; l < kLists; ++l) {
      const int prec = l;
      if (h->nmasked_inst[l] > 0 &&
          launch_wall(prec, h->d_insts, h->d_walls[l], h->d_wrec[l], h->plan.wall_cap[l], parity,
                      flags, h->side_stream))
        return cuda_fail(cudaGetLastError(), "wall pass launch");
      if (h->nopen_inst[l] > 0 &&
          launch_column(prec, h->d_insts, h->d_cols[l], h->plan.ncols[l], parity,
                        h->side_stream))
        return cuda_fail(cudaGetLastError(), "column pass launch");
    }
  }
  for (int l = 0; l < kLists; ++l) {
    const int prec = l;
    if (h->nmasked[l] > 0 &&
        launch_step(prec, h->plan.threads[l], h->d_insts, h->d_mtiles[l], h->nmasked[l], parity,
                    kModeStep, flags,
                    h->d_partials, h->side_stream, 1))
      return cuda_fail(cudaGetLastError(), "masked step kernel launch");
    if (h->plan.ntiles[l] <= 0) continue;
    const int kind = (flags & kFinal) ? 1 : 0;
    const bool timed = h->prof_cap > 0 && st == h->stream && h->prof_n[l][kind] < h->prof_cap;
    if (timed) {
      const cudaError_t e = cudaEventRecord(h->prof_ev[l][kind][2 * h->prof_n[l][kind]], st);
      if (e != cudaSuccess) return cuda_fail(e, "profile event");
    }
    if (launch_step(prec, h->plan.threads[l], h->d_insts, h->d_tiles[l], h->plan.ntiles[l],
                    parity, kModeStep, flags,
                    h->d_partials, st))
      return cuda_fail(cudaGetLastError(), "step kernel launch");
    if (timed) {
      const cudaError_t e = cudaEventRecord(h->prof_ev[l][kind][2 * h->prof_n[l][kind] + 1], st);
      if (e != cudaSuccess) return cuda_fail(e, "profile event");
      ++h->prof_n[l][kind];
    }
  }
  if (fork) {
    cudaError_t e = cudaEventRecord(h->ev_join, h->side_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, h->ev_join, 0);
    if (e != cudaSuccess) return cuda_fail(e, "join of the masked-tile stream");
  }
  return LBVE_OK;
}

int ensure_graph(lbve_handle* h) {
  if (h->graph_exec) return LBVE_OK;
  cudaError_t e = cudaSuccess;
  if (!h->cap_stream) e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(e, "graph capture start");
  int rc = LBVE_OK;
  for (int s = 0; s < kGraphSteps && rc == LBVE_OK; ++s) rc = launch_one_step(h, s & 1, 0, h->cap_stream);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(h->cap_stream, &g);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(e, "graph capture");
  e = cudaGraphInstantiate(&h->graph_exec, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    h->graph_exec = nullptr;
    return cuda_fail(e, "graph instantiation");
  }
  h->graph = g;
  return LBVE_OK;
}

// Drop the captured step graph (its launch configuration changed).
void drop_graph(lbve_handle* h) {
  if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
  if (h->graph) cudaGraphDestroy(h->graph);
  h->graph_exec = nullptr;
  h->graph = nullptr;
}

constexpr int kEx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
constexpr int kEy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

// FNV-1a over the mask and the wall links: identifies the geometry a saved
// state belongs to.
uint64_t geometry_hash(const std::vector<uint8_t>& m, const std::vector<WallDev>& walls) {
  uint64_t x = 1469598103934665603ull;
  auto mix = [&x](const void* p, size_t n) {
    const unsigned char* c = (const unsigned char*)p;
    for (size_t i = 0; i < n; ++i) {
      x ^= c[i];
      x *= 1099511628211ull;
    }
  };
  mix(m.data(), m.size());
  for (const WallDev& W : walls) {
    mix(&W.k, sizeof(W.k));
    mix(&W.umask, sizeof(W.umask));
    mix(W.q, sizeof(W.q));
  }
  return m.empty() ? 0 : (x | 1);
}

// Upload the wall-node records of instance i (unused capacity: inst = -1)
// and clear its final-step wall sums.
cudaError_t upload_walls(lbve_handle* h, int i) {
  const InstPlan& q = h->plan.inst[i];
  if (q.wall_cap <= 0) return cudaSuccess;
  std::vector<WallDev> blk(q.wall_cap);
  for (auto& W : blk) {
    std::memset(&W, 0, sizeof(W));
    W.inst = -1;
  }
  std::copy(h->walls_of[i].begin(), h->walls_of[i].end(), blk.begin());
  cudaError_t e = cudaMemcpyAsync(h->d_walls[q.list] + q.wall_begin, blk.data(),
                                  sizeof(WallDev) * q.wall_cap, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(h->d_wrec[q.list] + size_t(q.wall_begin) * kWallRec, 0,
                        sizeof(double) * kWallRec * q.wall_cap, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);  // blk is pageable and local
  return e;
}

// Hash of instance i's geometry: mask, wall links and, for an open channel,
// the inlet profile.
void update_geometry_hash(lbve_handle* h, int i) {
  uint64_t x = geometry_hash(h->mask_h[i], h->walls_of[i]);
  if (h->p[i].open_x) {
    const std::vector<double>& in = h->inlet_h[i];
    const unsigned char* c = (const unsigned char*)in.data();
    if (x == 0) x = 1469598103934665603ull;
    for (size_t b = 0; b < in.size() * sizeof(double); ++b) {
      x ^= c[b];
      x *= 1099511628211ull;
    }
    x |= 1;
  }
  h->geom_hash[i] = x;
}

// Flag the tiles of instance i that the masked kernel must run: every tile
// whose halo region (all TX x TY slots -- a ragged tile fills the slots past
// the edge with the wrapped nodes -- one column left and right, hy rows above
// and below), grown by one node, holds a solid node or a node of an open
// column.  Then no plain tile reads a slot the wall pass writes (solid nodes'
// slots, wall nodes' rest slots) or an open column's node, so plain tiles
// need not wait for the wall and column passes.  Rebuilds the list's
// masked-tile table and uploads both tables.
int flag_tiles(lbve_handle* h, int i) {
  const lbve_params& p = h->p[i];
  const InstPlan& q = h->plan.inst[i];
  const int nx = p.nx, ny = p.ny, l = q.list;
  const bool py = p.periodic_y != 0;
  const std::vector<uint8_t>& m = h->mask_h[i];
  auto flagged = [&](int x, int y) -> bool {
    const int xw = ((x % nx) + nx) % nx;
    if (py) y = ((y % ny) + ny) % ny;
    else if (y < 0 || y >= ny) return false;
    if (p.open_x && (xw == 0 || xw == nx - 1)) return true;
    return !m.empty() && m[size_t(y) * nx + xw] != 0;
  };
  // a model other than Oldroyd-B or the eq_p_G form of G~ runs every tile of
  // the instance in the general variant, keeping the plain one specialised
  const bool general = p.model != 0 || p.gtilde != 0;
  std::vector<TileDev>& T = h->tiles_h[l];
  std::vector<TileDev> mt;
  const bool any = !m.empty() || p.open_x || general;
  for (int j = q.tile_begin; j < q.tile_begin + q.ntiles; ++j) {
    TileDev& t = T[j];
    t.masked = general ? 1 : 0;
    const int xa = t.x0 - 2, xb = t.x0 + q.TX + 1;
    const int ya = t.y0 - q.hy - 1, yb = t.y0 + q.TY + q.hy;
    for (int y = ya; y <= yb && !t.masked && any; ++y)
      for (int x = xa; x <= xb && !t.masked; ++x)
        if (flagged(x, y)) t.masked = 1;
    if (t.masked) mt.push_back(t);
  }
  h->mtiles_of[i] = std::move(mt);
  std::vector<TileDev> table;
  for (int j = 0; j < h->n; ++j)
    if (h->plan.inst[j].list == l) {
      h->mbegin[j] = (int)table.size();
      table.insert(table.end(), h->mtiles_of[j].begin(), h->mtiles_of[j].end());
    }
  cudaError_t e = cudaMemcpyAsync(h->d_tiles[l] + q.tile_begin, T.data() + q.tile_begin,
                                  sizeof(TileDev) * q.ntiles, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess && !table.empty())
    e = cudaMemcpyAsync(h->d_mtiles[l], table.data(), sizeof(TileDev) * table.size(),
                        cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);  // table is pageable and local
  if (e != cudaSuccess) return cuda_fail(e, "tile table upload");
  h->nmasked[l] = (int)table.size();
  drop_graph(h);
  return LBVE_OK;
}

// Create the forked stream and its events (masks and open channels use them).
int ensure_side_stream(lbve_handle* h) {
  if (h->side_stream) return LBVE_OK;
  cudaError_t e = cudaStreamCreateWithFlags(&h->side_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming);
  if (e != cudaSuccess) return cuda_fail(e, "side stream creation");
  return LBVE_OK;
}

// Install (mask != null) or remove the solid mask of instance i: validate
// it, build the wall-node records (wall fraction 1/2), flag the tiles the
// masked kernel must run, rebuild the list's masked-tile table, upload.
int install_mask(lbve_handle* h, int i, const uint8_t* mask) {
  const lbve_params& p = h->p[i];
  const InstPlan& q = h->plan.inst[i];
  const int nx = p.nx, ny = p.ny, l = q.list;
  const bool py = p.periodic_y != 0;
  const size_t nn = size_t(nx) * ny;
  InstDev& D = h->insts[i];
  const bool had = D.mask != nullptr;
  std::vector<uint8_t> m;
  if (mask) {
    if (p.max_wall_nodes <= 0)
      return set_error(LBVE_ERR_GEOMETRY, "instance %d: max_wall_nodes is 0, so no mask fits", i);
    m.assign(nn, 0);
    size_t nsolid = 0;
    for (size_t k = 0; k < nn; ++k) nsolid += (m[k] = mask[k] ? 1 : 0);
    if (nsolid == nn) return set_error(LBVE_ERR_GEOMETRY, "instance %d: the mask leaves no fluid", i);
    if (nsolid == 0) m.clear();  // an empty mask is no mask
  }
  if (m.empty() && !had) return LBVE_OK;  // no mask before or after: nothing to change
  if (!m.empty()) {
    const int rc = ensure_side_stream(h);
    if (rc) return rc;
  }
  auto solid_at = [&](int x, int y) -> bool {
    if (m.empty()) return false;
    x = ((x % nx) + nx) % nx;
    if (py) y = ((y % ny) + ny) % ny;
    else if (y < 0 || y >= ny) return false;
    return m[size_t(y) * nx + x] != 0;
  };
  std::vector<WallDev> walls;
  std::vector<int32_t> index;
  if (!m.empty()) {
    if (!py)
      for (int x = 0; x < nx; ++x)
        for (int r = 0; r < 3; ++r)
          if (m[size_t(r) * nx + x] || m[size_t(ny - 1 - r) * nx + x])
            return set_error(LBVE_ERR_GEOMETRY,
                        "instance %d: rows 0-2 and ny-3..ny-1 of a walled domain must be fluid", i);
    if (p.open_x)
      for (int y = 0; y < ny; ++y)
        for (int r = 0; r < 3; ++r)
          if (m[size_t(y) * nx + r] || m[size_t(y) * nx + nx - 1 - r])
            return set_error(LBVE_ERR_GEOMETRY,
                        "instance %d: columns 0-2 and nx-3..nx-1 of an open channel must be fluid",
                        i);
    index.assign(nn, -1);
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const size_t k = size_t(y) * nx + x;
        if (m[k]) continue;
        int umask = 0, fmask = 0;
        for (int d = 1; d < 9; ++d) {
          if (!solid_at(x - kEx[d], y - kEy[d])) continue;
          if (solid_at(x + kEx[d], y + kEy[d]))
            return set_error(LBVE_ERR_GEOMETRY,
                        "instance %d: fluid node (%d, %d) has solid on both ends of link %d", i,
                        x, y, d);
          umask |= 1 << d;
          const int yf = y + kEy[d];
          if ((py || (yf >= 0 && yf < ny)) && !solid_at(x + kEx[d], yf)) fmask |= 1 << d;
        }
        if (!umask) continue;
        if ((int)walls.size() >= p.max_wall_nodes)
          return set_error(LBVE_ERR_GEOMETRY, "instance %d: more wall nodes than max_wall_nodes (%d)",
                      i, p.max_wall_nodes);
        WallDev W;
        std::memset(&W, 0, sizeof(W));
        W.inst = i;
        W.k = (int32_t)k;
        W.umask = umask;
        W.fmask = fmask;
        for (int d = 0; d < 8; ++d) W.q[d] = 0.5;
        index[k] = (int32_t)walls.size();
        walls.push_back(W);
      }
  }
  h->walls_of[i] = std::move(walls);
  h->wall_index[i] = std::move(index);
  cudaError_t e = cudaSuccess;
  if (!m.empty())
    e = cudaMemcpyAsync(h->ws + q.off_mask, m.data(), nn, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = upload_walls(h, i);  // synchronises: m is pageable and local
  if (e != cudaSuccess) return cuda_fail(e, "mask upload");
  D.mask = m.empty() ? nullptr : (const uint8_t*)(h->ws + q.off_mask);
  h->nmasked_inst[l] += (D.mask ? 1 : 0) - (had ? 1 : 0);
  h->mask_h[i] = std::move(m);
  update_geometry_hash(h, i);
  return flag_tiles(h, i);
}

}  // namespace

extern "C" {

const char* lbve_error_string(int code) {
  switch (code) {
    case LBVE_OK: return "ok";
    case LBVE_ERR_ARG: return "invalid argument";
    case LBVE_ERR_CUDA: return "CUDA error";
    case LBVE_ERR_NONFINITE: return "non-finite field";
    case LBVE_ERR_TIMEOUT: return "device wait timed out";
    case LBVE_ERR_GEOMETRY: return "unsupported or inconsistent geometry";
    case LBVE_ERR_WORKSPACE: return "workspace missing, too small or misaligned";
    case LBVE_ERR_STATE: return "call out of order";
    default: return "unknown error code";
  }
}

const char* lbve_last_error(void) { return g_last_error.c_str(); }

int lbve_workspace_bytes(const lbve_params* p, int32_t n, size_t* bytes) {
  if (!p || !bytes || n < 1) return set_error(LBVE_ERR_ARG, "null pointer or n_instances < 1");
  for (int i = 0; i < n; ++i) {
    const int rc = validate(p[i], i);
    if (rc) return rc;
  }
  *bytes = make_plan(p, n).total;
  return LBVE_OK;
}

int lbve_create(const lbve_params* p, int32_t n, void* d_workspace, size_t bytes,
                void* cuda_stream, lbve_handle** out) {
  if (!out) return set_error(LBVE_ERR_ARG, "out is null");
  *out = nullptr;
  size_t need = 0;
  int rc = lbve_workspace_bytes(p, n, &need);
  if (rc) return rc;
  if (!d_workspace || bytes < need)
    return set_error(LBVE_ERR_WORKSPACE, "workspace of %zu bytes given, %zu needed", bytes, need);
  if (reinterpret_cast<uintptr_t>(d_workspace) % kAlign)
    return set_error(LBVE_ERR_WORKSPACE, "workspace not %zu-byte aligned", kAlign);
  cudaPointerAttributes attr;
  cudaError_t e = cudaPointerGetAttributes(&attr, d_workspace);
  if (e != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
    cudaGetLastError();
    return set_error(LBVE_ERR_WORKSPACE, "workspace is not device memory");
  }

  lbve_handle* h = new lbve_handle();
  h->n = n;
  h->p.assign(p, p + n);
  h->plan = make_plan(p, n);
  h->ws = (char*)d_workspace;
  h->stream = (cudaStream_t)cuda_stream;
  h->t.assign(n, 0);
  h->ready.assign(n, 0);
  const Plan& pl = h->plan;
  h->d_insts = (InstDev*)(h->ws + pl.off_insts);
  for (int l = 0; l < kLists; ++l) h->d_tiles[l] = (TileDev*)(h->ws + pl.off_tiles[l]);
  for (int l = 0; l < kLists; ++l) {
    h->d_mtiles[l] = (TileDev*)(h->ws + pl.off_mtiles[l]);
    h->d_walls[l] = (WallDev*)(h->ws + pl.off_walls[l]);
    h->d_wrec[l] = (double*)(h->ws + pl.off_wrec[l]);
  }
  h->mtiles_of.assign(n, {});
  h->mbegin.assign(n, 0);
  h->walls_of.assign(n, {});
  h->wall_index.assign(n, {});
  h->geom_hash.assign(n, 0);
  h->mask_h.assign(n, {});
  h->inlet_h.assign(n, {});
  for (int l = 0; l < kLists; ++l) h->d_cols[l] = (ColTask*)(h->ws + pl.off_cols[l]);
  h->d_partials = (double*)(h->ws + pl.off_partials);
  h->d_totals = (double*)(h->ws + pl.off_totals);
  h->d_flags = (int32_t*)(h->ws + pl.off_flags);
  h->d_geo = (int32_t*)(h->ws + pl.off_geo);

  h->insts.resize(n);
  h->c.resize(n);
  std::vector<TileDev> tiles[kLists];
  for (int l = 0; l < kLists; ++l) tiles[l].resize(pl.ntiles[l]);
  for (int i = 0; i < n; ++i) {
    const InstPlan& q = pl.inst[i];
    const Coeffs c = derive(p[i]);
    h->c[i] = c;
    InstDev& D = h->insts[i];
    std::memset(&D, 0, sizeof(D));
    D.pop[0] = h->ws + q.off_pop[0];
    D.pop[1] = h->ws + q.off_pop[1];
    D.hist = h->ws + q.off_hist;
    D.force = h->ws + q.off_force;
    D.fields = (double*)(h->ws + q.off_fields);
    D.nx = p[i].nx;
    D.ny = p[i].ny;
    D.stride = q.stride;
    D.periodic_y = p[i].periodic_y;
    D.TX = q.TX;
    D.TY = q.TY;
    D.hy = q.hy;
    D.force_field = 0;
    D.slot_begin = q.slot_begin;
    D.slot_end = q.slot_begin + q.nslots;
    D.prec = p[i].precision;
    D.mask = nullptr;
    D.wall_rec = (double*)(h->ws + pl.off_wrec[q.list]) + size_t(q.wall_begin) * kWallRec;
    D.wall_cap = q.wall_cap;
    D.open_x = p[i].open_x;
    D.colbuf = p[i].open_x ? (void*)(h->ws + q.off_colbuf) : nullptr;
    D.inlet = p[i].open_x ? (const double*)(h->ws + q.off_inlet) : nullptr;
    D.inv_Uc = 1.0 / c.Uc;
    D.cd[kCoefFx] = p[i].Fx;
    D.cd[kCoefFy] = p[i].Fy;
    D.cd[kCoefCs1] = 1.0 - 1.0 / c.tau_s1;
    D.cd[kCoefCs2] = 1.0 - 1.0 / c.tau_s2;
    D.cd[kCoefHs1] = (c.tau_s1 - 0.5) / c.tau_s1;
    D.cd[kCoefWs1] = 1.0 / c.tau_s1;
    D.cd[kCoefEp1] = 2.0 - 1.0 / c.tau_p1;
    D.cd[kCoefCp2] = 1.0 - 1.0 / c.tau_p2;
    D.cd[kCoefHp1] = (c.tau_p1 - 0.5) / c.tau_p1;
    D.cd[kCoefInvLam] = 1.0 / c.lambda;
    D.cd[kCoefMupLam] = c.mup / c.lambda;
    D.cd[kCoefInvL2] = p[i].model != 0 ? 1.0 / p[i].L2 : 0.0;
    D.cd[kCoefAfene] = p[i].model == 1 ? 1.0 / (1.0 - 2.0 / p[i].L2) : 1.0;
    D.model = p[i].model;
    D.gtilde = p[i].gtilde;
    D.t32 = q.TX == kTileTX && (!p[i].periodic_y || p[i].ny >= q.TY + 2);
    for (int j = 0; j < kNumCoef; ++j) {
      D.cf[j] = (float)D.cd[j];
      D.cl[j] = (float)(D.cd[j] - (double)D.cf[j]);
    }
    int k = q.tile_begin;
    for (int ty = 0; ty < q.nty; ++ty)
      for (int tx = 0; tx < q.ntx; ++tx) {
        TileDev& T = tiles[q.list][k];
        T.inst = i;
        T.x0 = tx * q.TX;
        T.y0 = ty * q.TY;
        T.slot = q.slot_begin + (k - q.tile_begin);
        T.masked = 0;
        ++k;
      }
  }
  // unused wall-node records: inst = -1, zero wall sums
  std::vector<WallDev> no_walls[kLists];
  for (int l = 0; l < kLists; ++l) {
    no_walls[l].resize(pl.wall_cap[l]);
    for (auto& W : no_walls[l]) {
      std::memset(&W, 0, sizeof(W));
      W.inst = -1;
    }
  }
  // Synchronous copies from pageable host memory: the host vectors may go
  // out of scope as soon as the calls return.
  e = cudaMemcpyAsync(h->d_insts, h->insts.data(), sizeof(InstDev) * n, cudaMemcpyHostToDevice,
                      h->stream);
  for (int l = 0; l < kLists && e == cudaSuccess; ++l)
    if (!tiles[l].empty())
      e = cudaMemcpyAsync(h->d_tiles[l], tiles[l].data(), sizeof(TileDev) * tiles[l].size(),
                          cudaMemcpyHostToDevice, h->stream);
  for (int l = 0; l < kLists && e == cudaSuccess; ++l)
    if (pl.wall_cap[l] > 0) {
      e = cudaMemcpyAsync(h->d_walls[l], no_walls[l].data(), sizeof(WallDev) * pl.wall_cap[l],
                          cudaMemcpyHostToDevice, h->stream);
      if (e == cudaSuccess)
        e = cudaMemsetAsync(h->d_wrec[l], 0, sizeof(double) * kWallRec * pl.wall_cap[l],
                            h->stream);
    }
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d_flags, 0, sizeof(int32_t) * n, h->stream);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(h->d_totals, 0, sizeof(double) * kTotals * n, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    delete h;
    return cuda_fail(e, "lbve_create upload");
  }
  for (int l = 0; l < kLists; ++l) h->tiles_h[l] = std::move(tiles[l]);
  // open channels: column tasks, the default inlet (u = 0, A = I), tile flags
  std::vector<ColTask> cols[kLists];
  for (int l = 0; l < kLists; ++l) cols[l].resize(pl.ncols[l]);
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    if (!p[i].open_x) continue;
    const InstPlan& q = pl.inst[i];
    for (int side = 0; side < 2; ++side)
      for (int y = 0; y < p[i].ny; ++y)
        cols[q.list][q.col_begin + side * p[i].ny + y] = ColTask{i, y, side, 0};
    std::vector<double>& in = h->inlet_h[i];
    in.assign(5 * size_t(p[i].ny), 0.0);
    for (int y = 0; y < p[i].ny; ++y) in[2 * p[i].ny + y] = in[4 * p[i].ny + y] = 1.0;
    e = cudaMemcpyAsync(h->ws + q.off_inlet, in.data(), sizeof(double) * in.size(),
                        cudaMemcpyHostToDevice, h->stream);
    h->nopen_inst[q.list] += 1;
  }
  for (int l = 0; l < kLists && e == cudaSuccess; ++l)
    if (!cols[l].empty())
      e = cudaMemcpyAsync(h->d_cols[l], cols[l].data(), sizeof(ColTask) * cols[l].size(),
                          cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    delete h;
    return cuda_fail(e, "open-channel tables upload");
  }
  for (int i = 0; i < n; ++i) {
    if (!p[i].open_x && p[i].model == 0 && p[i].gtilde == 0) continue;
    if (p[i].open_x) update_geometry_hash(h, i);
    int rc2 = ensure_side_stream(h);
    if (rc2 == LBVE_OK) rc2 = flag_tiles(h, i);
    if (rc2) {
      lbve_destroy(h);
      return rc2;
    }
  }
  *out = h;
  return LBVE_OK;
}

// Host part of lbve_set_geometry for one instance: check and install the
// geometry, and start the uploads of the staged inputs (float64 force into
// pop[parity], float64 initial fields into pop[parity ^ 1]).  *what gets bit
// 0 for a staged force and bit 1 for staged fields.  From the first upload
// on, the instance is not ready until finish_geometry accepts it.
static int stage_geometry(lbve_handle* h, int32_t inst, const uint8_t* solid_mask,
                          const double* body_force, const double* init_fields, int32_t* what,
                          cudaStream_t cs) {
  *what = 0;
  {
    // the geometry is checked on the host before anything changes; the
    // values of the force and the initial fields on the device, after the
    // upload (init_geometry)
    const int rc = install_mask(h, inst, solid_mask);
    if (rc) return rc;
  }
  const lbve_params& p = h->p[inst];
  const size_t nn = size_t(p.nx) * p.ny;
  const size_t S = h->plan.inst[inst].stride;
  const int P = h->parity;
  InstDev& D = h->insts[inst];
  h->ready[inst] = 0;
  D.force_field = body_force ? 1 : 0;
  if (body_force) {
    const cudaError_t e = cudaMemcpy2DAsync(D.pop[P], S * 8, body_force, nn * 8, nn * 8, 2,
                                            cudaMemcpyHostToDevice, cs);
    if (e != cudaSuccess) return cuda_fail(e, "force upload");
    *what |= 1;
  }
  if (init_fields) {
    const cudaError_t e = cudaMemcpy2DAsync(D.pop[P ^ 1], S * 8, init_fields, nn * 8, nn * 8, 6,
                                            cudaMemcpyHostToDevice, cs);
    if (e != cudaSuccess) return cuda_fail(e, "initial field upload");
    *what |= 2;
  }
  return LBVE_OK;
}

// Device part for the staged list entries j < n (instance ids[j], inputs
// what[j]), a few launches for the whole list: the list and the descriptors
// are uploaded; one kernel checks the staged values, converts the forces and
// writes default fields; the equilibrium state of t = 0 is collided (one
// launch per precision when the list holds every instance of it); one
// reduction gives the totals.
static int init_geometry(lbve_handle* h, int32_t n, const int32_t* ids, const int32_t* what) {
  if (n <= 0) return LBVE_OK;
  std::vector<int32_t> geo(2 * (size_t)n);
  int max_nodes = 1;
  for (int32_t j = 0; j < n; ++j) {
    geo[j] = ids[j];
    geo[n + j] = what[j];
    max_nodes = std::max(max_nodes, h->p[ids[j]].nx * h->p[ids[j]].ny);
  }
  // pageable sources: the copies are staged before the calls return.  The
  // descriptors go up as one array when the list covers much of the handle,
  // else one by one (a single instance of a large batch moves 400 bytes)
  cudaError_t e = cudaMemcpyAsync(h->d_geo, geo.data(), sizeof(int32_t) * geo.size(),
                                  cudaMemcpyHostToDevice, h->stream);
  if ((size_t)n * 8 >= (size_t)h->n) {
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h->d_insts, h->insts.data(), sizeof(InstDev) * h->n,
                          cudaMemcpyHostToDevice, h->stream);
  } else {
    for (int32_t j = 0; j < n && e == cudaSuccess; ++j)
      e = cudaMemcpyAsync(h->d_insts + ids[j], &h->insts[ids[j]], sizeof(InstDev),
                          cudaMemcpyHostToDevice, h->stream);
  }
  if (e != cudaSuccess) return cuda_fail(e, "geometry list upload");
  const int P = h->parity;
  if (launch_geometry_inputs(h->d_insts, h->d_geo, h->d_geo + n, n, max_nodes, P, h->d_flags,
                             kFlagBadInput, h->stream))
    return cuda_fail(cudaGetLastError(), "input check launch");
  // collide the equilibrium state of t = 0: reads pop[P^1] (staging), writes
  // pop[P].  One launch per run of consecutive instances of one precision:
  // their tiles are contiguous in that precision's table
  for (int32_t j = 0; j < n;) {
    const int32_t first = ids[j];
    const int l = h->plan.inst[first].list;
    int32_t last = first, k = j + 1;
    while (k < n && ids[k] == last + 1 && h->plan.inst[ids[k]].list == l) last = ids[k++];
    const int t0 = h->plan.inst[first].tile_begin;
    const int t1 = h->plan.inst[last].tile_begin + h->plan.inst[last].ntiles;
    if (launch_step(l, h->plan.threads[l], h->d_insts, h->d_tiles[l] + t0, t1 - t0, P ^ 1,
                    kModeInit, kFinal, h->d_partials, h->stream))
      return cuda_fail(cudaGetLastError(), "init kernel launch");
    j = k;
  }
  for (int32_t j = 0; j < n; ++j) {
    const int32_t inst = ids[j];
    const InstPlan& q = h->plan.inst[inst];
    const int prec = h->p[inst].precision;
    if (!h->mtiles_of[inst].empty() &&
        launch_step(prec, h->plan.threads[q.list], h->d_insts,
                    h->d_mtiles[q.list] + h->mbegin[inst], (int)h->mtiles_of[inst].size(), P ^ 1,
                    kModeInit, kFinal, h->d_partials, h->stream, 1))
      return cuda_fail(cudaGetLastError(), "masked init kernel launch");
  }
  if (launch_reduce(h->d_insts, 0, n, h->d_partials, h->d_totals, h->d_flags, h->stream, h->d_geo))
    return cuda_fail(cudaGetLastError(), "reduce launch");
  return LBVE_OK;
}

// Synchronise once for the list entries ids[0..n-1] (the caller's host
// arrays are then free), read their input checks and mark the accepted
// instances ready at time 0.  Returns the error of the first rejected
// instance in list order.
static int finish_geometry(lbve_handle* h, int32_t n, const int32_t* ids) {
  std::vector<int32_t> flags(h->n, 0);
  cudaError_t e = cudaMemcpyAsync(flags.data(), h->d_flags, sizeof(int32_t) * h->n,
                                  cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "lbve_set_geometry");
  int rc = LBVE_OK;
  for (int32_t j = 0; j < n; ++j) {
    const int32_t inst = ids[j];
    if (flags[inst] & (1 << kFlagBadInput)) {
      if (rc == LBVE_OK)
        rc = set_error(LBVE_ERR_ARG,
                       "instance %d: a body force or initial field is not finite, or an initial "
                       "density is not > 0; the instance is left uninitialised",
                       inst);
      continue;
    }
    h->t[inst] = 0;
    h->ready[inst] = 1;
  }
  return rc;
}

int lbve_set_geometry(lbve_handle* h, int32_t inst, const uint8_t* solid_mask,
                      const double* body_force, const double* init_fields) {
  return lbve_set_geometry_many(h, 1, &inst, &solid_mask, &body_force, &init_fields);
}

int lbve_set_geometry_many(lbve_handle* h, int32_t n, const int32_t* insts,
                           const uint8_t* const* solid_masks, const double* const* body_forces,
                           const double* const* init_fields) {
  if (!h || n < 0 || (n > 0 && !insts)) return set_error(LBVE_ERR_ARG, "bad argument");
  std::vector<uint8_t> seen(h->n, 0);
  for (int32_t j = 0; j < n; ++j) {
    if (insts[j] < 0 || insts[j] >= h->n)
      return set_error(LBVE_ERR_ARG, "insts[%d] = %d is not an instance", j, insts[j]);
    if (seen[insts[j]]++)
      return set_error(LBVE_ERR_ARG, "instance %d is listed twice", insts[j]);
  }
  if (n == 0) return LBVE_OK;
  std::vector<int32_t> what(n, 0);
  // Lists of 16 or more instances go in up to kGeoChunks chunks: the uploads
  // on the side stream (after the caller's stream has reached this call),
  // each chunk's launches on the caller's stream after its uploads, so that
  // the launches of one chunk overlap the uploads of the next.
  const int nchunk = n >= 16 ? lbve_handle::kGeoChunks : 1;
  const int32_t per = (n + nchunk - 1) / nchunk;
  cudaStream_t cs = h->stream;
  if (nchunk > 1) {
    int rc = ensure_side_stream(h);
    cudaError_t e = cudaSuccess;
    for (int c = 0; c < nchunk && rc == LBVE_OK && e == cudaSuccess; ++c)
      if (!h->geo_ev[c]) e = cudaEventCreateWithFlags(&h->geo_ev[c], cudaEventDisableTiming);
    if (e == cudaSuccess && rc == LBVE_OK) e = cudaEventRecord(h->ev_fork, h->stream);
    if (e == cudaSuccess && rc == LBVE_OK) e = cudaStreamWaitEvent(h->side_stream, h->ev_fork, 0);
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "geometry upload stream");
    cs = h->side_stream;
  }
  int32_t staged = n;  // entries 0..staged-1 go through the device part
  int rc_stage = LBVE_OK, rc = LBVE_OK;
  char msg[512] = "";
  for (int32_t j0 = 0, c = 0; j0 < staged && rc == LBVE_OK; j0 += per, ++c) {
    const int32_t j1 = std::min(n, j0 + per);
    int32_t j = j0;
    for (; j < j1; ++j) {
      rc_stage = stage_geometry(h, insts[j], solid_masks ? solid_masks[j] : nullptr,
                                body_forces ? body_forces[j] : nullptr,
                                init_fields ? init_fields[j] : nullptr, &what[j], cs);
      if (rc_stage) {
        // entries before j are still initialised (and may report an earlier
        // error); entry j and the rest of the list are not set
        snprintf(msg, sizeof msg, "%s", lbve_last_error());
        staged = j;
        break;
      }
    }
    if (cs != h->stream) {
      cudaError_t e = cudaEventRecord(h->geo_ev[c], cs);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, h->geo_ev[c], 0);
      if (e != cudaSuccess) rc = cuda_fail(e, "geometry upload stream");
    }
    if (rc == LBVE_OK) rc = init_geometry(h, j - j0, insts + j0, what.data() + j0);
  }
  if (rc) {
    // what was enqueued finishes before the caller's arrays are released
    if (cs != h->stream) cudaStreamSynchronize(cs);
    cudaStreamSynchronize(h->stream);
    return rc;
  }
  rc = finish_geometry(h, staged, insts);
  if (rc) return rc;
  if (rc_stage) return set_error(rc_stage, "%s", msg);
  return LBVE_OK;
}

int lbve_step(lbve_handle* h, int64_t n_steps) {
  if (!h || n_steps < 0) return set_error(LBVE_ERR_ARG, "bad handle or negative step count");
  for (int i = 0; i < h->n; ++i)
    if (!h->ready[i]) return set_error(LBVE_ERR_STATE, "instance %d was never initialised", i);
  if (n_steps == 0) return LBVE_OK;
  int64_t left = n_steps - 1;  // non-final steps
  // non-final steps: whole graphs where possible (they start at parity 0);
  // while lbve_profile times launches, every step is launched directly
  if (h->prof_cap == 0 && left >= kGraphSteps + (h->parity ? 1 : 0)) {
    if (h->parity) {
      const int rc = launch_one_step(h, 1, 0, h->stream);
      if (rc) return rc;
      h->parity = 0;
      --left;
    }
    int rc = ensure_graph(h);
    if (rc) return rc;
    while (left >= kGraphSteps) {
      const cudaError_t e = cudaGraphLaunch(h->graph_exec, h->stream);
      if (e != cudaSuccess) return cuda_fail(e, "graph launch");
      left -= kGraphSteps;
    }
  }
  for (; left > 0; --left) {
    const int rc = launch_one_step(h, h->parity, 0, h->stream);
    if (rc) return rc;
    h->parity ^= 1;
  }
  // the final step also writes fields and partial records
  int rc = launch_one_step(h, h->parity, kFinal, h->stream);
  if (rc) return rc;
  h->parity ^= 1;
  if (launch_reduce(h->d_insts, 0, h->n, h->d_partials, h->d_totals, h->d_flags, h->stream))
    return cuda_fail(cudaGetLastError(), "reduce launch");
  for (int i = 0; i < h->n; ++i) h->t[i] += n_steps;
  return LBVE_OK;
}

int lbve_status(lbve_handle* h, int32_t* flags) {
  if (!h || !flags) return set_error(LBVE_ERR_ARG, "null argument");
  cudaError_t e = cudaMemcpyAsync(flags, h->d_flags, sizeof(int32_t) * h->n,
                                  cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "lbve_status");
  for (int i = 0; i < h->n; ++i)
    if (flags[i] & 1) return set_error(LBVE_ERR_NONFINITE, "instance %d has a non-finite field", i);
  return LBVE_OK;
}

int lbve_fields(lbve_handle* h, int32_t inst, double* out, int32_t on_device) {
  return lbve_fields_many(h, 1, &inst, &out, on_device);
}

int lbve_fields_many(lbve_handle* h, int32_t n, const int32_t* insts, double* const* outs,
                     int32_t on_device) {
  if (!h || n < 0 || (n > 0 && (!insts || !outs))) return set_error(LBVE_ERR_ARG, "bad argument");
  for (int32_t j = 0; j < n; ++j) {
    if (insts[j] < 0 || insts[j] >= h->n || !outs[j])
      return set_error(LBVE_ERR_ARG, "bad instance or output at list position %d", j);
    if (!h->ready[insts[j]])
      return set_error(LBVE_ERR_STATE, "instance %d was never initialised", insts[j]);
  }
  for (int32_t j = 0; j < n; ++j) {
    const int32_t inst = insts[j];
    const lbve_params& p = h->p[inst];
    const size_t nn = size_t(p.nx) * p.ny, S = h->plan.inst[inst].stride;
    const cudaError_t e =
        cudaMemcpy2DAsync(outs[j], nn * 8, h->insts[inst].fields, S * 8, nn * 8, 6,
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                          h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "lbve_fields");
  }
  if (!on_device && n > 0) {
    const cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "lbve_fields");
  }
  return LBVE_OK;
}

static int read_totals(lbve_handle* h, int32_t inst, double* rec) {
  if (!h || inst < 0 || inst >= h->n) return set_error(LBVE_ERR_ARG, "bad argument");
  if (!h->ready[inst]) return set_error(LBVE_ERR_STATE, "instance %d was never initialised", inst);
  cudaError_t e = cudaMemcpyAsync(rec, h->d_totals + (size_t)inst * kTotals,
                                  sizeof(double) * kTotals, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "totals readback");
  return LBVE_OK;
}

int lbve_totals(lbve_handle* h, int32_t inst, double out[LBVE_NTOTALS]) {
  if (!out) return set_error(LBVE_ERR_ARG, "out is null");
  double rec[kTotals];
  const int rc = read_totals(h, inst, rec);
  if (rc) return rc;
  for (int j = 0; j < 12; ++j) out[j] = rec[j];
  out[12] = rec[kDrag];
  out[13] = rec[kDrag + 1];
  return LBVE_OK;
}

int lbve_residual(lbve_handle* h, int32_t inst, double* out) {
  if (!out) return set_error(LBVE_ERR_ARG, "out is null");
  double rec[kTotals];
  const int rc = read_totals(h, inst, rec);
  if (rc) return rc;
  *out = rec[kResid];
  return LBVE_OK;
}

int lbve_time(lbve_handle* h, int32_t inst, int64_t* t) {
  if (!h || !t || inst < 0 || inst >= h->n) return set_error(LBVE_ERR_ARG, "bad argument");
  *t = h->t[inst];
  return LBVE_OK;
}

// ---- checkpoint / resume -------------------------------------------------
namespace {
constexpr uint32_t kStateMagic = 0x4556424cu;  // "LBVE"
constexpr uint32_t kStateVersion = 2;
struct StateHeader {
  uint32_t magic, version;
  int32_t n, reserved;
};
struct InstHeader {
  int64_t t;
  int32_t nx, ny, precision, periodic_y, force_field, ready;
  uint64_t geometry;  // hash of the solid mask and wall fractions, 0 = none
};
size_t inst_state_bytes(const lbve_params& p) {
  const size_t nn = size_t(p.nx) * p.ny, es = elem_size(p.precision);
  return sizeof(InstHeader) + (36 + 5 + 2) * nn * es + 6 * nn * 8;
}
}  // namespace

int lbve_state_bytes(lbve_handle* h, size_t* bytes) {
  if (!h || !bytes) return set_error(LBVE_ERR_ARG, "null argument");
  size_t b = sizeof(StateHeader);
  for (int i = 0; i < h->n; ++i) b += inst_state_bytes(h->p[i]);
  *bytes = b;
  return LBVE_OK;
}

int lbve_save(lbve_handle* h, void* host_buf, size_t bytes) {
  size_t need = 0;
  int rc = lbve_state_bytes(h, &need);
  if (rc) return rc;
  if (!host_buf || bytes < need) return set_error(LBVE_ERR_ARG, "state buffer of %zu bytes, %zu needed", bytes, need);
  char* out = (char*)host_buf;
  StateHeader H{kStateMagic, kStateVersion, h->n, 0};
  std::memcpy(out, &H, sizeof(H));
  out += sizeof(H);
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < h->n && e == cudaSuccess; ++i) {
    const lbve_params& p = h->p[i];
    const InstDev& D = h->insts[i];
    const size_t nn = size_t(p.nx) * p.ny, S = D.stride, es = elem_size(p.precision);
    InstHeader I{h->t[i], p.nx, p.ny, p.precision, p.periodic_y, D.force_field, h->ready[i],
                 h->geom_hash[i]};
    std::memcpy(out, &I, sizeof(I));
    out += sizeof(I);
    // current populations (36), history (5), force (2): planes of nn values
    e = cudaMemcpy2DAsync(out, nn * es, D.pop[h->parity], S * es, nn * es, 36,
                          cudaMemcpyDeviceToHost, h->stream);
    out += 36 * nn * es;
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(out, nn * es, D.hist, S * es, nn * es, 5, cudaMemcpyDeviceToHost,
                            h->stream);
    out += 5 * nn * es;
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(out, nn * es, D.force, S * es, nn * es, 2, cudaMemcpyDeviceToHost,
                            h->stream);
    out += 2 * nn * es;
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(out, nn * 8, D.fields, S * 8, nn * 8, 6, cudaMemcpyDeviceToHost,
                            h->stream);
    out += 6 * nn * 8;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "lbve_save");
  return LBVE_OK;
}

int lbve_load(lbve_handle* h, const void* host_buf, size_t bytes) {
  size_t need = 0;
  int rc = lbve_state_bytes(h, &need);
  if (rc) return rc;
  if (!host_buf || bytes < need) return set_error(LBVE_ERR_ARG, "state buffer of %zu bytes, %zu needed", bytes, need);
  const char* in = (const char*)host_buf;
  StateHeader H;
  std::memcpy(&H, in, sizeof(H));
  in += sizeof(H);
  if (H.magic != kStateMagic || H.version != kStateVersion || H.n != h->n)
    return set_error(LBVE_ERR_ARG, "state was not saved by lbve_save for this instance count");
  // validate every instance header before touching the device
  const char* scan = in;
  for (int i = 0; i < h->n; ++i) {
    InstHeader I;
    std::memcpy(&I, scan, sizeof(I));
    const lbve_params& p = h->p[i];
    if (I.nx != p.nx || I.ny != p.ny || I.precision != p.precision || I.periodic_y != p.periodic_y)
      return set_error(LBVE_ERR_ARG, "saved instance %d does not match this handle's parameters", i);
    if (I.geometry != h->geom_hash[i])
      return set_error(LBVE_ERR_GEOMETRY,
                  "saved instance %d was run on another solid mask (set it before loading)", i);
    scan += inst_state_bytes(p);
  }
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < h->n && e == cudaSuccess; ++i) {
    InstHeader I;
    std::memcpy(&I, in, sizeof(I));
    in += sizeof(I);
    const lbve_params& p = h->p[i];
    InstDev& D = h->insts[i];
    const size_t nn = size_t(p.nx) * p.ny, S = D.stride, es = elem_size(p.precision);
    e = cudaMemcpy2DAsync(D.pop[h->parity], S * es, in, nn * es, nn * es, 36,
                          cudaMemcpyHostToDevice, h->stream);
    in += 36 * nn * es;
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(D.hist, S * es, in, nn * es, nn * es, 5, cudaMemcpyHostToDevice,
                            h->stream);
    in += 5 * nn * es;
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(D.force, S * es, in, nn * es, nn * es, 2, cudaMemcpyHostToDevice,
                            h->stream);
    in += 2 * nn * es;
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(D.fields, S * 8, in, nn * 8, nn * 8, 6, cudaMemcpyHostToDevice,
                            h->stream);
    in += 6 * nn * 8;
    D.force_field = I.force_field;
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h->d_insts + i, &D, sizeof(InstDev), cudaMemcpyHostToDevice, h->stream);
    h->t[i] = I.t;
    h->ready[i] = (char)I.ready;
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d_flags, 0, sizeof(int32_t) * h->n, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "lbve_load");
  return LBVE_OK;
}

int lbve_set_inlet(lbve_handle* h, int32_t inst, const double* inlet) {
  if (!h || inst < 0 || inst >= h->n || !inlet) return set_error(LBVE_ERR_ARG, "bad handle, instance or pointer");
  const lbve_params& p = h->p[inst];
  if (!p.open_x) return set_error(LBVE_ERR_GEOMETRY, "instance %d is not an open channel", inst);
  const size_t cnt = 5 * size_t(p.ny);
  for (size_t k = 0; k < cnt; ++k)
    if (!std::isfinite(inlet[k])) return set_error(LBVE_ERR_ARG, "inlet profile not finite");
  std::vector<double>& in = h->inlet_h[inst];
  in.assign(inlet, inlet + cnt);
  cudaError_t e = cudaMemcpyAsync(h->ws + h->plan.inst[inst].off_inlet, in.data(),
                                  sizeof(double) * cnt, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "inlet upload");
  update_geometry_hash(h, inst);
  return LBVE_OK;
}

int lbve_set_wall_distances(lbve_handle* h, int32_t inst, int32_t n_links, const int32_t* node,
                            const int32_t* dir, const double* q) {
  if (!h || inst < 0 || inst >= h->n || n_links < 0 || (n_links > 0 && (!node || !dir || !q)))
    return set_error(LBVE_ERR_ARG, "bad handle, instance, count or pointer");
  if (!h->insts[inst].mask) return set_error(LBVE_ERR_GEOMETRY, "instance %d has no solid mask", inst);
  const lbve_params& p = h->p[inst];
  const int64_t nn = int64_t(p.nx) * p.ny;
  std::vector<WallDev>& W = h->walls_of[inst];
  const std::vector<int32_t>& idx = h->wall_index[inst];
  for (int32_t j = 0; j < n_links; ++j) {
    if (node[j] < 0 || node[j] >= nn || dir[j] < 1 || dir[j] > 8)
      return set_error(LBVE_ERR_ARG, "link %d: node or direction out of range", j);
    const int32_t r = idx[node[j]];
    if (r < 0 || !((W[r].umask >> dir[j]) & 1))
      return set_error(LBVE_ERR_GEOMETRY, "link %d (node %d, direction %d) is not a wall link", j,
                  node[j], dir[j]);
    if (!(q[j] > 0.0 && q[j] <= 1.0)) return set_error(LBVE_ERR_ARG, "link %d: q must be in (0, 1]", j);
  }
  for (int32_t j = 0; j < n_links; ++j) W[idx[node[j]]].q[dir[j] - 1] = q[j];
  const cudaError_t e = upload_walls(h, inst);
  if (e != cudaSuccess) return cuda_fail(e, "wall upload");
  update_geometry_hash(h, inst);
  return LBVE_OK;
}

static void release_profile(lbve_handle* h) {
  for (int l = 0; l < kLists; ++l)
    for (int f = 0; f < 2; ++f) {
      for (cudaEvent_t e : h->prof_ev[l][f])
        if (e) cudaEventDestroy(e);
      h->prof_ev[l][f].clear();
      h->prof_n[l][f] = 0;
    }
  h->prof_cap = 0;
}

int lbve_profile(lbve_handle* h, int32_t max_launches) {
  if (!h || max_launches < 0 || max_launches > (1 << 20))
    return set_error(LBVE_ERR_ARG, "bad handle or max_launches outside [0, 2^20]");
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(h->stream, &cs);
  if (e != cudaSuccess) return cuda_fail(e, "lbve_profile");
  if (cs != cudaStreamCaptureStatusNone)
    return set_error(LBVE_ERR_STATE, "lbve_profile: the stream is capturing");
  e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "lbve_profile");
  release_profile(h);
  if (max_launches == 0) return LBVE_OK;
  for (int l = 0; l < kLists; ++l) {
    if (h->plan.ntiles[l] <= 0) continue;
    for (int f = 0; f < 2; ++f) {
      h->prof_ev[l][f].resize(2 * (size_t)max_launches, nullptr);
      for (auto& ev : h->prof_ev[l][f]) {
        e = cudaEventCreate(&ev);
        if (e != cudaSuccess) {
          ev = nullptr;
          release_profile(h);
          return cuda_fail(e, "lbve_profile: event creation");
        }
      }
    }
  }
  h->prof_cap = max_launches;
  return LBVE_OK;
}

int lbve_profile_read(lbve_handle* h, int32_t precision, int32_t final_step, int32_t* launches,
                      double* ms_total, double* ms_min, double* ms_max) {
  if (!h || !launches || !ms_total || precision < 0 || precision >= kLists ||
      (final_step != 0 && final_step != 1))
    return set_error(LBVE_ERR_ARG, "bad handle, precision, final_step or null output");
  const int l = precision;
  *launches = 0;
  *ms_total = 0.0;
  double lo = 0.0, hi = 0.0;
  const int n = h->prof_cap > 0 ? h->prof_n[l][final_step] : 0;
  const std::vector<cudaEvent_t>& ev = h->prof_ev[l][final_step];
  if (n > 0) {
    cudaError_t e = cudaEventSynchronize(ev[2 * n - 1]);
    if (e != cudaSuccess) return cuda_fail(e, "lbve_profile_read");
    for (int j = 0; j < n; ++j) {
      float ms = 0.f;
      e = cudaEventElapsedTime(&ms, ev[2 * j], ev[2 * j + 1]);
      if (e != cudaSuccess) return cuda_fail(e, "lbve_profile_read");
      *ms_total += ms;
      lo = j == 0 ? ms : std::min(lo, (double)ms);
      hi = j == 0 ? ms : std::max(hi, (double)ms);
    }
  }
  *launches = n;
  if (ms_min) *ms_min = lo;
  if (ms_max) *ms_max = hi;
  return LBVE_OK;
}

void lbve_destroy(lbve_handle* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  release_profile(h);
  if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
  if (h->graph) cudaGraphDestroy(h->graph);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->side_stream) cudaStreamSynchronize(h->side_stream);
  if (h->side_stream) cudaStreamDestroy(h->side_stream);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  for (cudaEvent_t ev : h->geo_ev)
    if (ev) cudaEventDestroy(ev);
  delete h;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Tile-width autotuner.  The batch is timed as a whole (one launch per
// precision per step covers every instance, so widths interact only through
// the shared launch); instances are grouped into classes that admit the same
// candidate widths and have the same precision and wall layout, and one pass
// of coordinate descent over the classes keeps a width only when it beats the
// incumbent by more than kAutotuneGain.
namespace {

constexpr double kAutotuneGain = 0.01;
constexpr int kAutotuneRepeats = 2;  // the fastest of these timings counts

std::vector<int> width_candidates(const lbve_params& p) {
  std::vector<int> c;
  if (p.nx < 8) c.push_back(p.nx);
  for (int t = 8; t <= tile_tx_max(p.precision); t *= 2)
    if (t <= p.nx) c.push_back(t);
  return c;
}

// Milliseconds per step of trial_steps steps of the batch with tile widths
// q[i].tile_tx, from the rest state, on a handle built in the workspace.
int time_batch(const std::vector<lbve_params>& q, void* d_ws, size_t bytes, cudaStream_t st,
               int trial_steps, cudaEvent_t ev[2], double& ms_out) {
  ms_out = 1e300;
  for (int r = 0; r < kAutotuneRepeats; ++r) {
    lbve_handle* h = nullptr;
    int rc = lbve_create(q.data(), (int32_t)q.size(), d_ws, bytes, st, &h);
    if (rc) return rc;
    for (int i = 0; i < (int)q.size() && rc == LBVE_OK; ++i)
      rc = lbve_set_geometry(h, i, nullptr, nullptr, nullptr);
    if (rc == LBVE_OK) rc = lbve_step(h, trial_steps);  // warm-up, builds the step graph
    cudaError_t e = cudaSuccess;
    if (rc == LBVE_OK) {
      e = cudaEventRecord(ev[0], st);
      if (e == cudaSuccess && (rc = lbve_step(h, trial_steps)) == LBVE_OK) {
        e = cudaEventRecord(ev[1], st);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
        if (e == cudaSuccess) ms_out = std::min(ms_out, double(ms) / trial_steps);
      }
    }
    lbve_destroy(h);
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "autotune timing");
  }
  return LBVE_OK;
}

}  // namespace

extern "C" int lbve_autotune(const lbve_params* p, int32_t n, void* d_workspace, size_t bytes,
                             void* cuda_stream, int32_t trial_steps, int32_t* tile_tx_out) {
  if (!tile_tx_out) return set_error(LBVE_ERR_ARG, "tile_tx_out is null");
  if (trial_steps < 1 || trial_steps > 100000)
    return set_error(LBVE_ERR_ARG, "trial_steps must be in [1, 100000]");
  size_t need = 0;
  int rc = lbve_workspace_bytes(p, n, &need);
  if (rc) return rc;
  if (!d_workspace || bytes < need)
    return set_error(LBVE_ERR_WORKSPACE, "workspace of %zu bytes given, %zu needed", bytes, need);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(st, &cs);
  if (e != cudaSuccess) return cuda_fail(e, "stream query");
  if (cs != cudaStreamCaptureStatusNone)
    return set_error(LBVE_ERR_STATE, "lbve_autotune cannot run while the stream is being captured");

  std::vector<lbve_params> q(p, p + n);
  // the incumbent: every unset width at the default of the CTA size the
  // batch gets without tuning
  const int nt64 = fp64_threads(p, n);
  for (auto& x : q)
    x.tile_tx = x.tile_tx > 0 ? x.tile_tx
                              : default_tile_tx(x, x.precision == LBVE_FP64 ? nt64 : kThreads);
  // classes of instances with the same candidates, precision and walls
  std::vector<int> cls(n, -1);
  std::vector<std::vector<int>> cand_of;
  std::vector<std::vector<int>> members;
  for (int i = 0; i < n; ++i) {
    const std::vector<int> c = width_candidates(q[i]);
    for (size_t k = 0; k < cand_of.size() && cls[i] < 0; ++k) {
      const lbve_params& r = q[members[k][0]];
      if (cand_of[k] == c && r.precision == q[i].precision && r.periodic_y == q[i].periodic_y)
        cls[i] = (int)k;
    }
    if (cls[i] < 0) {
      cls[i] = (int)cand_of.size();
      cand_of.push_back(c);
      members.emplace_back();
    }
    members[cls[i]].push_back(i);
  }

  cudaEvent_t ev[2] = {nullptr, nullptr};
  e = cudaEventCreate(&ev[0]);
  if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
  if (e != cudaSuccess) {
    if (ev[0]) cudaEventDestroy(ev[0]);
    return cuda_fail(e, "event creation");
  }
  double best = 0.0;
  rc = time_batch(q, d_workspace, bytes, st, trial_steps, ev, best);
  for (size_t k = 0; k < cand_of.size() && rc == LBVE_OK; ++k) {
    if (cand_of[k].size() < 2) continue;
    const int incumbent = q[members[k][0]].tile_tx;
    int keep = incumbent;
    for (int c : cand_of[k]) {
      if (c == incumbent) continue;
      for (int i : members[k]) q[i].tile_tx = c;
      double ms = 0.0;
      rc = time_batch(q, d_workspace, bytes, st, trial_steps, ev, ms);
      if (rc) break;
      if (ms < best * (1.0 - kAutotuneGain)) {
        best = ms;
        keep = c;
      }
    }
    for (int i : members[k]) q[i].tile_tx = keep;
  }
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  if (rc) return rc;
  for (int i = 0; i < n; ++i) tile_tx_out[i] = q[i].tile_tx;
  return LBVE_OK;
}

// ---------------------------------------------------------------------------
// Adjoint: gradient of a loss on the final fields with respect to the
// per-node body force, by a hand-written discrete adjoint of every step
// (lbve_adjoint.cuh) with sqrt(T) checkpointing.
// ---------------------------------------------------------------------------
namespace {

struct AdjPlan {
  int64_t T, s, nck;             // steps, checkpoint interval, checkpoints
  size_t state_bytes;            // one stored state: 41 planes
  size_t off_desc, off_tiles, off_partials, off_fields, off_stage, off_ck, off_seg, off_lam[2],
      off_pulled, off_G, off_dir, off_mh, off_M, off_zero, total;
  // solid masks: the raw-state scratch the wall pass completes, the wall
  // records and final-step records, each node's record, the masked tiles
  int nwall, nmtiles;
  size_t off_scratch, off_walls, off_wrec, off_widx, off_mtiles;
  size_t off_cols;  // open channels: the column tasks of the instance (2 ny)
};

// The square-root checkpoint interval: ceil(sqrt(T)).
int64_t sqrt_interval(int64_t T) {
  int64_t s = 1;
  while (s * s < T) ++s;
  return s;
}

// Workspace plan of the adjoint for T steps with checkpoints every `interval`
// steps (0: the square-root interval).
AdjPlan make_adj_plan(const lbve_params& p, const InstPlan& q, int64_t T, int nwall = 0,
                      int nmtiles = 0, int64_t interval = 0) {
  AdjPlan a;
  a.nwall = nwall;
  a.nmtiles = nmtiles;
  a.T = T;
  a.s = interval > 0 ? interval : sqrt_interval(T);
  a.nck = (T + a.s - 1) / a.s;
  const size_t es = elem_size(p.precision);
  const size_t plane = size_t(q.stride) * es;
  a.state_bytes = 41 * plane;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + std::max<size_t>(bytes, 1), kAlign);
    return o;
  };
  a.off_desc = take(sizeof(InstDev));
  a.off_tiles = take(sizeof(TileDev) * q.ntiles);
  a.off_partials = take(sizeof(double) * kPartial * q.ntiles);
  a.off_fields = take(sizeof(double) * 6 * q.stride);
  a.off_stage = take(sizeof(double) * 6 * q.stride);
  a.off_ck = take(a.state_bytes * a.nck);
  a.off_seg = take(a.state_bytes * (a.s + 1));
  a.off_lam[0] = take(a.state_bytes);
  a.off_lam[1] = take(a.state_bytes);
  a.off_pulled = take(36 * plane);
  a.off_G = take(6 * plane);
  a.off_dir = take(3 * plane);
  a.off_mh = take(8 * plane);
  a.off_M = take(3 * plane);
  a.off_zero = take(sizeof(double) * 6 * q.stride);
  a.off_scratch = a.off_walls = a.off_wrec = a.off_widx = a.off_mtiles = a.off_cols = off;
  if (nwall > 0) {
    a.off_scratch = take(36 * plane);
    a.off_walls = take(sizeof(WallDev) * nwall);
    a.off_wrec = take(sizeof(double) * kWallRec * nwall);
    a.off_widx = take(sizeof(int32_t) * q.stride);
  }
  if (nmtiles > 0) a.off_mtiles = take(sizeof(TileDev) * nmtiles);
  if (p.open_x) a.off_cols = take(sizeof(ColTask) * 2 * size_t(p.ny));
  a.total = off;
  return a;
}

}  // namespace

extern "C" int lbve_adjoint_workspace_bytes(lbve_handle* h, int32_t inst, int64_t n_steps,
                                            size_t* bytes) {
  if (!h || !bytes || inst < 0 || inst >= h->n || n_steps < 1)
    return set_error(LBVE_ERR_ARG, "bad handle, instance, step count or output pointer");
  *bytes = make_adj_plan(h->p[inst], h->plan.inst[inst], n_steps, (int)h->walls_of[inst].size(),
                         (int)h->mtiles_of[inst].size())
               .total;
  return LBVE_OK;
}

extern "C" int lbve_adjoint_workspace_bytes_interval(lbve_handle* h, int32_t inst,
                                                     int64_t n_steps, int64_t interval,
                                                     size_t* bytes) {
  if (!h || !bytes || inst < 0 || inst >= h->n || n_steps < 1 || interval < 1 ||
      interval > n_steps)
    return set_error(LBVE_ERR_ARG, "bad handle, instance, step count, interval or output pointer");
  *bytes = make_adj_plan(h->p[inst], h->plan.inst[inst], n_steps, (int)h->walls_of[inst].size(),
                         (int)h->mtiles_of[inst].size(), interval)
               .total;
  return LBVE_OK;
}

extern "C" int lbve_adjoint_step_ex(lbve_handle* h, int32_t inst, const double* init_fields,
                                    const double* d_dL_dfields, const double* dL_ddrag,
                                    int64_t n_steps, void* d_ws, size_t bytes,
                                    double* d_dL_dforce, double* d_dL_dq) {
  if (!h || inst < 0 || inst >= h->n || !d_dL_dforce || n_steps < 1)
    return set_error(LBVE_ERR_ARG, "bad handle, instance, pointer or step count");
  if (!d_dL_dfields && !dL_ddrag) return set_error(LBVE_ERR_ARG, "no loss: dL/dfields and dL/ddrag are null");
  if (!h->ready[inst]) return set_error(LBVE_ERR_STATE, "instance %d was never initialised", inst);
  if (h->p[inst].model != 0 || h->p[inst].gtilde != 0)
    return set_error(LBVE_ERR_ARG, "the adjoint covers Oldroyd-B with eq_p_G_1 only (instance %d)",
                inst);
  if (h->p[inst].precision == LBVE_DF32)
    return set_error(LBVE_ERR_ARG,
                     "the adjoint covers LBVE_FP64 and LBVE_FP32_DEV instances (instance %d)", inst);
  const bool masked = h->insts[inst].mask != nullptr;
  const bool open = h->p[inst].open_x != 0;
  if (!masked && (dL_ddrag || d_dL_dq))
    return set_error(LBVE_ERR_GEOMETRY, "drag and wall-fraction gradients need a solid mask");
  if (dL_ddrag && !(std::isfinite(dL_ddrag[0]) && std::isfinite(dL_ddrag[1])))
    return set_error(LBVE_ERR_ARG, "dL/ddrag not finite");
  const lbve_params& p = h->p[inst];
  const InstPlan& q = h->plan.inst[inst];
  const std::vector<WallDev>& walls_h = h->walls_of[inst];
  const std::vector<TileDev>& mtiles_h = h->mtiles_of[inst];
  // the shortest checkpoint interval whose plan fits the workspace given
  // (the square-root interval needs the least)
  // masked tiles: those of a mask and of an open channel's columns
  const int nw = masked ? (int)walls_h.size() : 0;
  const int nm = (masked || open) ? (int)mtiles_h.size() : 0;
  const int64_t s_max = sqrt_interval(n_steps);
  AdjPlan a = make_adj_plan(p, q, n_steps, nw, nm, s_max);
  for (int64_t s = 1; s < s_max; ++s) {
    const AdjPlan b = make_adj_plan(p, q, n_steps, nw, nm, s);
    if (b.total <= bytes) {
      a = b;
      break;
    }
  }
  if (!d_ws || bytes < a.total)
    return set_error(LBVE_ERR_WORKSPACE, "adjoint workspace of %zu bytes given, %zu needed", bytes,
                a.total);
  if (reinterpret_cast<uintptr_t>(d_ws) % kAlign)
    return set_error(LBVE_ERR_WORKSPACE, "adjoint workspace not %zu-byte aligned", kAlign);
  char* ws = (char*)d_ws;
  cudaStream_t st = h->stream;
  const int prec = p.precision;
  const size_t nn = size_t(p.nx) * p.ny, S = q.stride;
  const size_t es = elem_size(prec);
  const size_t plane = S * es;
  cudaError_t e = cudaSuccess;

  // single-instance descriptor and tile table (instance index 0)
  InstDev D = h->insts[inst];
  D.fields = (double*)(ws + a.off_fields);
  D.slot_begin = 0;
  D.slot_end = q.ntiles;
  std::vector<TileDev> tiles(q.ntiles);
  std::vector<TileDev> mtiles;
  for (int ty = 0, k = 0; ty < q.nty; ++ty)
    for (int tx = 0; tx < q.ntx; ++tx, ++k) {
      // the handle's masked flags of this instance's tiles (same order)
      const int mk = (masked || open) ? h->tiles_h[q.list][q.tile_begin + k].masked : 0;
      tiles[k] = TileDev{0, tx * q.TX, ty * q.TY, k, mk};
      if (mk) mtiles.push_back(tiles[k]);
    }
  InstDev* d_desc = (InstDev*)(ws + a.off_desc);
  TileDev* d_tiles = (TileDev*)(ws + a.off_tiles);
  double* d_partials = (double*)(ws + a.off_partials);
  e = cudaMemcpyAsync(d_tiles, tiles.data(), sizeof(TileDev) * q.ntiles, cudaMemcpyHostToDevice,
                      st);
  if (e != cudaSuccess) return cuda_fail(e, "adjoint tile upload");
  // solid mask: the instance's wall records as instance 0, each node's record
  TileDev* d_mtiles = (TileDev*)(ws + a.off_mtiles);
  WallDev* d_walls = (WallDev*)(ws + a.off_walls);
  int32_t* d_widx = (int32_t*)(ws + a.off_widx);
  char* scratch = ws + a.off_scratch;
  std::vector<WallDev> wcopy;
  std::vector<int32_t> widx;
  if (open) {
    // the column pass of instance 0 (the inlet profile is the instance's)
    std::vector<ColTask> cols(2 * size_t(p.ny));
    for (int side = 0; side < 2; ++side)
      for (int y = 0; y < p.ny; ++y) cols[side * p.ny + y] = ColTask{0, y, side, 0};
    e = cudaMemcpyAsync(ws + a.off_cols, cols.data(), sizeof(ColTask) * cols.size(),
                        cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "adjoint column tasks");
    if (!mtiles.empty() && !masked) {
      e = cudaMemcpyAsync(ws + a.off_mtiles, mtiles.data(), sizeof(TileDev) * mtiles.size(),
                          cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) return cuda_fail(e, "adjoint masked tiles");
    }
  }
  if (masked) {
    wcopy = walls_h;
    widx.assign(q.stride, -1);
    for (size_t r = 0; r < wcopy.size(); ++r) {
      wcopy[r].inst = 0;
      widx[wcopy[r].k] = (int32_t)r;
    }
    if (!wcopy.empty())
      e = cudaMemcpyAsync(d_walls, wcopy.data(), sizeof(WallDev) * wcopy.size(),
                          cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_widx, widx.data(), sizeof(int32_t) * widx.size(),
                          cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !mtiles.empty())
      e = cudaMemcpyAsync(d_mtiles, mtiles.data(), sizeof(TileDev) * mtiles.size(),
                          cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "adjoint mask tables");
  }
  const int nmt = (int)mtiles.size();
  auto launch_tiles = [&](int mode, int flags) -> bool {
    const int nt = h->plan.threads[q.list];
    if (launch_step(prec, nt, d_desc, d_tiles, q.ntiles, 0, mode, flags, d_partials, st))
      return false;
    if (nmt > 0 &&
        launch_step(prec, nt, d_desc, d_mtiles, nmt, 0, mode, flags, d_partials, st, 1))
      return false;
    return true;
  };
  auto set_desc = [&](void* pop0, void* pop1, void* hist) -> cudaError_t {
    D.pop[0] = pop0;
    D.pop[1] = pop1;
    D.hist = hist;
    // ordered on the stream; a pageable source is staged before the call
    // returns, so D may change right after
    return cudaMemcpyAsync(d_desc, &D, sizeof(InstDev), cudaMemcpyHostToDevice, st);
  };
  auto state = [&](char* base) { return base; };
  auto hist_of = [&](char* st_) { return st_ + 36 * plane; };
  char* ck = ws + a.off_ck;
  char* seg = ws + a.off_seg;

  // staged initial fields (float64 [6][S])
  double* stage = (double*)(ws + a.off_stage);
  if (init_fields) {
    e = cudaMemcpy2DAsync(stage, S * 8, init_fields, nn * 8, nn * 8, 6, cudaMemcpyHostToDevice,
                          st);
  } else {
    std::vector<double> def(6 * nn, 0.0);
    for (size_t k = 0; k < nn; ++k) def[k] = def[3 * nn + k] = def[5 * nn + k] = 1.0;
    e = cudaMemcpy2DAsync(stage, S * 8, def.data(), nn * 8, nn * 8, 6, cudaMemcpyHostToDevice,
                          st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "adjoint initial-field upload");
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "adjoint set-up");

  // one forward step from state `from` into state `to` (history copied, then
  // updated in place).  With a mask the wall pass completes a scratch copy of
  // `from`, so stored states stay raw (the reverse passes redo the completion).
  auto fwd = [&](char* from, char* to) -> int {
    cudaError_t ee = cudaMemcpyAsync(hist_of(to), hist_of(from), 5 * plane,
                                     cudaMemcpyDeviceToDevice, st);
    if (ee != cudaSuccess) return cuda_fail(ee, "adjoint history copy");
    char* src = state(from);
    if (masked) {
      ee = cudaMemcpyAsync(scratch, state(from), 36 * plane, cudaMemcpyDeviceToDevice, st);
      if (ee != cudaSuccess) return cuda_fail(ee, "adjoint scratch copy");
      src = scratch;
    }
    if ((ee = set_desc(src, state(to), hist_of(to))) != cudaSuccess)
      return cuda_fail(ee, "adjoint descriptor");
    if (masked && !wcopy.empty() &&
        launch_wall(prec, d_desc, d_walls, (double*)(ws + a.off_wrec), (int)wcopy.size(), 0, 0,
                    st))
      return cuda_fail(cudaGetLastError(), "adjoint wall pass");
    if (open && launch_column(prec, d_desc, (const ColTask*)(ws + a.off_cols), 2 * p.ny, 0, st))
      return cuda_fail(cudaGetLastError(), "adjoint column pass");
    if (!launch_tiles(kModeStep, 0)) return cuda_fail(cudaGetLastError(), "adjoint forward step");
    return LBVE_OK;
  };

  // ---- forward sweep: X_0 from the initial fields, checkpoints every s steps ----
  if ((e = set_desc(stage, state(ck), hist_of(ck))) != cudaSuccess)
    return cuda_fail(e, "adjoint descriptor");
  if (!launch_tiles(kModeInit, kFinal)) return cuda_fail(cudaGetLastError(), "adjoint init step");
  for (int64_t j = 1; j < a.nck; ++j) {
    // X_{j s} from X_{(j-1) s}: s steps through two rolling buffers of the segment area
    char* cur = ck + (j - 1) * a.state_bytes;
    for (int64_t m = 0; m < a.s; ++m) {
      char* nxt = (m == a.s - 1) ? ck + j * a.state_bytes : seg + (m % 2) * a.state_bytes;
      const int rc = fwd(cur, nxt);
      if (rc) return rc;
      cur = nxt;
    }
  }

  // ---- reverse sweep ----
  AdjArgsRaw A;
  std::memset(&A, 0, sizeof(A));
  A.init = stage;
  A.force = D.force_field ? D.force : nullptr;
  A.M = ws + a.off_M;
  A.lam_pulled = ws + a.off_pulled;
  A.lam_G = ws + a.off_G;
  A.lam_dir = ws + a.off_dir;
  A.lam_mh = ws + a.off_mh;
  A.dF = d_dL_dforce;
  if ((e = cudaMemsetAsync(d_dL_dforce, 0, sizeof(double) * 2 * nn, st)) != cudaSuccess)
    return cuda_fail(e, "gradient reset");
  if (masked) {
    A.mask = h->insts[inst].mask;
    A.widx = d_widx;
    A.walls = d_walls;
  }
  if (d_dL_dq) {
    A.dq = d_dL_dq;
    if ((e = cudaMemsetAsync(d_dL_dq, 0, sizeof(double) * 8 * nn, st)) != cudaSuccess)
      return cuda_fail(e, "gradient reset");
  }
  if (dL_ddrag) {
    A.drag_w[0] = dL_ddrag[0];
    A.drag_w[1] = dL_ddrag[1];
  }
  A.open = open ? 1 : 0;
  // without a field loss the final pass reads zeros
  const double* fields_seed = d_dL_dfields;
  if (!fields_seed) {
    fields_seed = (const double*)(ws + a.off_zero);
    if ((e = cudaMemsetAsync(ws + a.off_zero, 0, sizeof(double) * 6 * S, st)) != cudaSuccess)
      return cuda_fail(e, "adjoint seed");
  }
  char* lam[2] = {ws + a.off_lam[0], ws + a.off_lam[1]};
  int li = 0;  // lam[li] holds lambda of the most recent (later) state
  const int n_nodes = (int)nn;
  auto pass = [&](int mode, int which) -> int {
    if (launch_adjoint(prec, mode, which, d_desc, A, n_nodes, st))
      return cuda_fail(cudaGetLastError(), "adjoint pass launch");
    return LBVE_OK;
  };
  bool first = true;  // the last state carries the loss
  for (int64_t j = a.nck - 1; j >= 0; --j) {
    const int64_t m0 = j * a.s, m1 = std::min<int64_t>((j + 1) * a.s, a.T);  // states m0..m1-1
    // recompute the segment's states into seg[0 .. m1-m0-1] (with interval 1
    // every state is a checkpoint and is read in place)
    if (a.s > 1) {
      e = cudaMemcpyAsync(seg, ck + j * a.state_bytes, a.state_bytes, cudaMemcpyDeviceToDevice,
                          st);
      if (e != cudaSuccess) return cuda_fail(e, "adjoint checkpoint copy");
    }
    for (int64_t m = m0 + 1; m < m1; ++m) {
      const int rc = fwd(seg + (m - 1 - m0) * a.state_bytes, seg + (m - m0) * a.state_bytes);
      if (rc) return rc;
    }
    for (int64_t m = m1 - 1; m >= m0; --m) {
      char* X = a.s > 1 ? seg + (m - m0) * a.state_bytes : ck + j * a.state_bytes;
      if ((e = set_desc(state(X), state(X), hist_of(X))) != cudaSuccess)
        return cuda_fail(e, "adjoint descriptor");
      A.X = X;
      A.lam_cur = lam[li ^ 1];
      int mode;
      if (first) {
        mode = kAdjFields;
        A.lam_next = nullptr;
        A.lam_fields = fields_seed;
        A.final_pass = 1;
        first = false;
      } else {
        mode = kAdjStep;
        A.lam_next = lam[li];
        A.lam_fields = nullptr;
        A.final_pass = 0;
      }
      int rc = pass(mode, 0);
      if (!rc) rc = pass(mode, 1);
      if (!rc) rc = pass(mode, 2);
      if (!rc && open && launch_adjoint(prec, mode, 4, d_desc, A, 2 * p.ny, st))
        rc = cuda_fail(cudaGetLastError(), "adjoint column reverse launch");
      if (!rc) rc = pass(mode, 3);
      if (rc) return rc;
      li ^= 1;
    }
  }
  // the initial collision (X_0 from the equilibrium of the initial fields)
  if ((e = set_desc(stage, ck, hist_of(ck))) != cudaSuccess)
    return cuda_fail(e, "adjoint descriptor");
  A.X = nullptr;
  A.lam_next = lam[li];
  A.lam_fields = nullptr;
  A.lam_cur = lam[li ^ 1];
  A.final_pass = 0;
  int rc = pass(kAdjInit, 0);
  if (!rc) rc = pass(kAdjInit, 1);
  if (!rc) rc = pass(kAdjInit, 2);
  if (rc) return rc;
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "lbve_adjoint_step");
  return LBVE_OK;
}

extern "C" int lbve_adjoint_step(lbve_handle* h, int32_t inst, const double* init_fields,
                                 const double* d_dL_dfields, int64_t n_steps, void* d_ws,
                                 size_t bytes, double* d_dL_dforce) {
  if (!d_dL_dfields) return set_error(LBVE_ERR_ARG, "d_dL_dfields is null");
  return lbve_adjoint_step_ex(h, inst, init_fields, d_dL_dfields, nullptr, n_steps, d_ws, bytes,
                              d_dL_dforce, nullptr);
}
