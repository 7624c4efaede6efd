// lbve_internal.h -- layout shared by the host code and the CUDA kernels of
// liblbve (not part of the public ABI).
#pragma once
#include <cstdint>

namespace lbve {

// Record a one-line detail of an error for lbve_last_error() on the calling
// thread and return code (every entry point reports its errors this way).
int set_error(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));

// Threads per CTA of the step kernel, per storage precision.  Float32: 96
// (32 x 3 tiles) measured fastest on GB300 among 64..256; seven such CTAs per
// SM give 21 warps in seven independent load / barrier / compute phases.
// Float64 (bound by the FP64 pipe): 256 (32 x 8 tiles), two per SM.  A
// float64 batch too small to give every SM one such tile runs 64-thread CTAs
// (32 x 2 tiles, eight per SM, the same registers per thread) instead: each
// SM's FP64 pipe then has a quarter of the nodes to work through.
#ifndef LBVE_THREADS
#define LBVE_THREADS 96
#endif
#ifndef LBVE_THREADS_FP64
#define LBVE_THREADS_FP64 256
#endif
#ifndef LBVE_THREADS_FP64_SMALL
#define LBVE_THREADS_FP64_SMALL 64
#endif
// Float64 batches too small to give every SM one 64-thread tile run one-warp
// CTAs (default tiles 8 x 4): one tile per SM spreads the FP64 work of a few
// thousand nodes over up to all 152 SMs.
#ifndef LBVE_THREADS_FP64_TINY
#define LBVE_THREADS_FP64_TINY 32
#endif
#ifndef LBVE_TILE_TX
#define LBVE_TILE_TX 32
#endif
constexpr int kThreads = LBVE_THREADS;          // float32 step kernel
constexpr int kThreads64 = LBVE_THREADS_FP64;   // float64 step kernel
constexpr int kThreads64Small = LBVE_THREADS_FP64_SMALL;  // float64, small batches
constexpr int kThreads64Tiny = LBVE_THREADS_FP64_TINY;    // float64, tiny batches
constexpr int kTileTXTiny = 8;  // default tile width of the one-warp float64 CTAs
constexpr int kNumSMs = 152;  // GB300; sizes the small-batch choice only
constexpr int kTileTX = LBVE_TILE_TX;   // default tile width (nodes along x) for nx >= kTileTX
// threads per CTA (for float64, the size of all but small batches) and the
// widest tile a caller may ask for, by precision (0 = float64, 1 = float32
// deviations, 2 = float32 pairs, as LBVE_FP64 / LBVE_FP32_DEV / LBVE_DF32)
__host__ __device__ constexpr int threads_of(int prec) { return prec == 0 ? kThreads64 : kThreads; }
__host__ __device__ constexpr int tile_tx_max(int prec) { return threads_of(prec) / 2; }
// Halo region of a tile: (TX+2)(TY+2*hy) <= (TX+2)(T/TX+4) = T + 4 TX + 2 T/TX
// + 8 for T threads, which is convex in TX and equals 3 (T + 4) at both ends
// of 1 <= TX <= T/2 (TY = T/TX, hy <= 2).
__host__ __device__ constexpr int region_max(int threads) { return 3 * (threads + 4); }
constexpr int kPartial = 16;      // doubles per tile partial record
constexpr int kTotals = 16;       // doubles per instance totals record

// Partial / totals record slots.
enum : int {
  kSumRho = 0, kSumJx = 1, kSumJy = 2, kSumPhi = 3,  // 3..5
  kWallIn = 6,                                        // 6..8
  kWallOut = 9,                                       // 9..11
  kResid = 12, kNonFinite = 13,
  kDrag = 14                                          // 14..15 (totals only)
};

// Kernel flags.
enum : int { kFinal = 1 };

// Coefficient slots of InstDev::cd / InstDev::cf.
enum : int {
  kCoefFx = 0, kCoefFy,
  kCoefCs1,     // 1 - 1/tau_s1
  kCoefCs2,     // 1 - 1/tau_s2
  kCoefHs1,     // 1 - 1/(2 tau_s1)
  kCoefWs1,     // 1/tau_s1
  kCoefEp1,     // 2 - 1/tau_p1, so that 1 - 1/tau_p1 = ep - 1
  kCoefCp2,     // 1 - 1/tau_p2
  kCoefHp1,     // 1 - 1/(2 tau_p1)
  kCoefInvLam,  // 1/lambda
  kCoefMupLam,  // mu_p/lambda
  kCoefInvL2,   // 1/L^2 of the FENE models (0 for Oldroyd-B)
  kCoefAfene,   // a = 1/(1 - 2/L^2) of FENE-P
  kNumCoef
};

// Everything a CTA needs about its instance.  Pointers are device addresses
// inside the caller's workspace.  Coefficients are derived in float64 on
// the host (Sec. 3.1-3.2 relaxation-time relations) and rounded once.
// Layout: 16-byte aligned, the fields the step kernel reads first (buffers,
// geometry, flags, float32 coefficients) in the leading 16-byte groups, so
// that each CTA's prologue loads them as a few 16-byte vectors.
struct alignas(16) InstDev {
  void* pop[2];        // [36][stride] post-collision populations, ping-pong
  void* hist;          // [5][stride]  S_xx, S_xy, S_yy, ux, uy of the last step
  void* force;         // [2][stride]  per-node body force (if force_field)
  int32_t nx, ny, stride, periodic_y;
  int32_t TX, TY, hy, force_field;
  int32_t t32;                   // tiles are kTileTX wide and rows wrap at most once
                                 // inside a tile's halo region (plain tiles specialise)
  int32_t open_x;                // inlet column x = 0, outlet x = nx - 1
  int32_t model, gtilde;         // constitutive model (0 Oldroyd-B, 1 FENE-P, 2 FENE-CR);
                                 // G~ form (0 eq_p_G_1, 1 eq_p_G)
  int32_t slot_begin, slot_end;  // partial-record slots of this instance
  int32_t prec, wall_cap;        // wall_cap: wall-node records of this instance
  // Collision coefficients rounded once to float32 (cf), their float64
  // values (cd) and the low parts of the LBVE_DF32 pairs (cl = cd - cf), so
  // that no kernel converts precision per node.
  float cf[16];
  double* fields;                // [6][stride]  rho, ux, uy, Axx, Axy, Ayy (float64)
  const uint8_t* mask;           // [stride] 1 = solid node, or null (no mask)
  double* wall_rec;              // [wall_cap][kWallRec] final-step wall sums
  void* colbuf;                  // [36][2 ny] completed populations of the two open
                                 // columns (inlet rows, then outlet rows), deviations
  const double* inlet;           // [5][ny] u_x, u_y, A_xx, A_xy, A_yy at the inlet
  double inv_Uc;
  double cd[16];
  float cl[16];
};
static_assert(sizeof(InstDev) % 16 == 0, "descriptor size");

// One tile of one instance: {instance, x0, y0, partial slot, masked}.
// masked: the tile holds a solid node or a node with a solid neighbour along
// x or y; such tiles are run by the masked variant of the step kernel.
// Padded to 32 bytes and aligned to 16, so that a CTA reads its entry with
// vector loads.
struct alignas(16) TileDev {
  int32_t inst, x0, y0, slot, masked, pad0, pad1, pad2;
};

// One fluid node next to the solid mask (the compact link list of the wall
// pass).  inst < 0 marks an unused record.
//   umask bit i: link i is a wall link (node k - e_i is solid)
//   fmask bit i: node k + e_i is fluid (second operand of the interpolation)
//   q[i-1]:      wall fraction of link i, in (0, 1]
struct WallDev {
  int32_t inst, k, umask, fmask;
  double q[8];
};
constexpr int kWallRec = 8;  // drag x, drag y, wall in x3, wall out x3

// One node of an open column: {instance, row, side (0 inlet, 1 outlet)}.
struct ColTask {
  int32_t inst, y, side, pad;
};

// Launchers implemented in lbve_kernels.cu (templated over float/double).
enum : int { kModeStep = 0, kModeInit = 1 };

// threads: CTA size of the tiles (kThreads for float32; kThreads64,
// kThreads64Small or kThreads64Tiny for float64).  masked = 0 runs the plain kernel (which
// skips masked tiles), 1 the masked variant.
int launch_step(int prec, int threads, const InstDev* d_insts, const TileDev* d_tiles,
                int n_tiles, int parity, int mode, int flags, double* d_partials, void* stream,
                int masked = 0);
// Wall pass before a step: completes the populations of the wall links of
// n_walls records in the buffer pop[parity]; on the final step it writes one
// kWallRec record per wall node to d_rec (lbve_wall.cu).
int launch_wall(int prec, const InstDev* d_insts, const WallDev* d_walls, double* d_rec,
                int n_walls, int parity, int flags, void* stream);
// Column pass before a step: the completed populations of the open columns'
// nodes (n_tasks of them) into each instance's colbuf (lbve_wall.cu).
int launch_column(int prec, const InstDev* d_insts, const ColTask* d_tasks, int n_tasks,
                  int parity, void* stream);
// Adjoint pass modes: a normal step, the final fields (the loss), the initial collision.
enum : int { kAdjStep = 0, kAdjFields = 1, kAdjInit = 2 };

// Untyped pointers of one adjoint pass (see AdjArgs in lbve_adjoint.cuh).
struct AdjArgsRaw {
  const void* X;
  const double* init;
  const void* force;
  void* M;
  const void* lam_next;
  const double* lam_fields;
  void* lam_pulled;
  void* lam_G;
  void* lam_dir;
  void* lam_mh;
  void* lam_cur;
  double* dF;
  // solid masks (null without one): the mask, each node's wall record (-1 if
  // none), the records (instance index 0), dL/dq [8][n] (or null), and the
  // weights of the final step's force on the solid in the loss
  const uint8_t* mask;
  const int32_t* widx;
  const WallDev* walls;
  double* dq;
  double drag_w[2];
  int final_pass;
  int open;  // open channel: the node passes are the variants with the open columns
};
// pass: 0 moments, 1 local reverse, 2 gather, 3 reverse pull, 4 reverse of an
// open channel's column pass (n_nodes = 2 ny: one thread per open-column
// node); mode: kAdjStep, kAdjFields, kAdjInit (lbve_adjoint.cuh).
int launch_adjoint(int prec, int mode, int pass, const InstDev* d_desc, const AdjArgsRaw& a,
                   int n_nodes, void* stream);
// Totals of n_insts instances: ids[0..n_insts-1] (device), or first_inst..
// first_inst + n_insts - 1 when d_ids is null.
int launch_reduce(const InstDev* d_insts, int first_inst, int n_insts, const double* d_partials,
                  double* d_totals, int32_t* d_flags, void* stream,
                  const int32_t* d_ids = nullptr);
// Staged inputs of the list entries j < n_list (instance d_ids[j], d_what[j]
// bit 0 force staged in pop[parity], bit 1 initial fields staged in
// pop[parity ^ 1]): zero the instances' flags, check the staged values (bit
// `bit` of the flag on failure), convert the force to the instance's
// precision, write default fields where none are staged.  max_nodes: the
// largest nx * ny of the list.
int launch_geometry_inputs(const InstDev* d_insts, const int32_t* d_ids, const int32_t* d_what,
                           int n_list, int max_nodes, int parity, int32_t* d_flags, int bit,
                           void* stream);
constexpr int kFlagBadInput = 1;  // status bit of a rejected lbve_set_geometry

}  // namespace lbve
