// Internal types and device helpers shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstdio>
#include <mutex>
#include <string>
#include <vector>

#include "formopt_gb300.h"

// ----------------------------------------------------------------------------- host side
struct fo_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  size_t budget = 0;        // 0 = unlimited
  size_t in_use = 0;
  int num_sms = 0;
  std::string err;
  std::vector<fo_mesh *> meshes;
  std::vector<fo_problem *> problems;
  // pinned host staging for scalar read-backs
  double *h_scalars = nullptr;
  // per-phase timing of fo_opt_step
  int timing = 0;
  cudaEvent_t ev[8] = {};
  // with timing on: device time of the last persistent multigrid solve launch alone
  cudaEvent_t ev_solve[2] = {};
  double last_solve_ms = 0.0;
  // persistent launches take at most 1/grid_share of the co-resident block slots
  int grid_share = 1;
};

// Structured Kuhn grid: everything a kernel needs to enumerate nodes and elements.
struct Grid {
  int dim;
  int n[3];              // cells per axis (1 for unused axes)
  long long nn[3];       // nodes per axis
  long long stride[3];   // node id strides
  long long cstride[3];  // cell id strides
  long long num_nodes, num_cells, num_elems;
  double lo[3], hi[3];
  double h[3];           // cell spacing (hi - lo) / n
  double inv_h[3];
  double vol_e;          // measure of every simplex: prod h / d!
  double facet_area[3];  // measure of a boundary facet on a face normal to axis a
};

struct fo_umesh;
struct fo_mesh {
  fo_ctx *ctx;
  Grid g;                       // general meshes: dim, num_nodes, num_elems and the box only
  fo_umesh *um = nullptr;       // non-null for a mesh given as arrays (fo_mesh_from_arrays)
  int32_t *d_cells = nullptr;   // [N_T][d+1]
  double *d_coords = nullptr;   // [N_n][d]
  double h_diam = 0;
};

// Krylov scratch kept per problem (sized for the largest system it solves).
struct Scratch {
  void *buf = nullptr;
  size_t bytes = 0;
};

// Task-parallel batch of screened Helmholtz instances on one mesh.  Fields are
// instance-minor with the instance count padded to nip = 32, 64 or 128: the value
// of instance i at node a sits at a * nip + i, so a warp that owns a node reads each
// field's row with coalesced loads (lane l holds instances l, l + 32, ...).  Padding
// instances have k = 1, omega = 0 and a zero source, hence a zero solution.
struct fo_batch {
  int n_inst = 0, nip = 0;
  std::vector<int> lane_of;                 // caller's instance i lives in lane lane_of[i]
  std::vector<double> h_k, h_omega;         // per lane
  double *kk = nullptr, *w2 = nullptr;      // [nip] k_i and omega_i^2
  double *f = nullptr;                      // [N_n][nip] nodal sources
  double *B = nullptr;                      // [N_n][nip] loads F_i (0 on Dirichlet nodes)
  double *U = nullptr, *P = nullptr;        // [N_n][nip] states and explicit adjoints
  double *WK = nullptr, *WM = nullptr;      // [N_n][S] stiffness (A-weighted) / mass stencils
  float *WK32 = nullptr, *WM32 = nullptr;   // the same in FP32
  double *dinv = nullptr;                   // [N_n][nip] Jacobi inverse diagonal
  float *dinv32 = nullptr;
  int *inst_iters = nullptr;                // [nip] last solve: active iterations
  double *inst_res = nullptr;               // [nip] last solve: final relative residual
  int tuned_ts[2] = {0, 0}, tuned_block[2] = {0, 0}, tuned_bpsm[2] = {0, 0};   // per precision (FO_FP64, FO_MIXED)
  double tuned_us[2] = {0, 0};
  struct fo_bmg *mg = nullptr;              // multigrid hierarchy of the batched operator
};

// Geometric multigrid hierarchy of a problem's state operator (fo_mg.cu): level 0 is the
// problem's grid, level l halves every axis of level l-1.
#define MG_MAX_LEVELS 10
struct fo_mg {
  int L = 0, npn = 1, blk = 1;             // components per node, stencil entries per slot
  bool own0 = false;                       // level 0's FP32 rows, diagonal, mask owned here
  long long built_epoch = -1;
  Grid g[MG_MAX_LEVELS];
  float *b[MG_MAX_LEVELS] = {}, *z0[MG_MAX_LEVELS] = {}, *z1[MG_MAX_LEVELS] = {}, *t[MG_MAX_LEVELS] = {};
  double *coef[MG_MAX_LEVELS] = {}, *W64[MG_MAX_LEVELS] = {}, *dinv64[MG_MAX_LEVELS] = {};
  float *W32[MG_MAX_LEVELS] = {}, *dinv32[MG_MAX_LEVELS] = {};
  __nv_bfloat16 *Wh[MG_MAX_LEVELS] = {};   // BF16 copies of the grid-run levels' rows (on request)
  int Lg = 0;                              // levels >= Lg run in one block (set by the upload)
  int rows_bf16 = 0;                       // the uploaded table points the grid levels at Wh
  uint8_t *dir[MG_MAX_LEVELS] = {};
  int nd = 0;                              // coarsest level's unknowns when solved directly
  float *ainv = nullptr;                   // [nd][nd] its inverse (FP32)
  double *adense = nullptr;                // nd > MG_DIRECT_MAX: the FP64 matrix the whole grid
                                           // inverts ([nd][nd], then 16 doubles: barrier, status)
  void *dev = nullptr;                     // device copy of the level table
  std::vector<unsigned char> host;         // its host image (kept alive for the async copy)
};

// Inverse-elasticity model (fo_inverse.cu): the second states, their adjoints, the measurement
// extensions (n_cases x N_dof each) and the operator with the whole boundary clamped.
struct fo_inv {
  double *v = nullptr, *q = nullptr, *g = nullptr, *r = nullptr;   // r: one N_dof work vector
  double *W = nullptr, *dinv = nullptr;      // rows with every boundary DOF clamped (FP64)
  float *W32 = nullptr, *dinv32 = nullptr;
  uint8_t *dirb = nullptr, *none = nullptr;  // boundary mask per DOF; an all-zero mask
  uint8_t *gamma1 = nullptr;                 // per node: bit (2 axis + side) of the Gamma1 faces it is on
  long long rows_epoch = -1;                 // coefficient epoch of W
  fo_mg *mgb = nullptr;                      // multigrid hierarchy of the boundary-clamped operator
  std::vector<std::pair<void **, size_t>> allocs;
};

struct fo_problem {
  fo_ctx *ctx;
  fo_mesh *mesh;
  fo_model_desc desc;
  int ncomp = 1;                 // state components per node
  long long ndof = 0;            // state DOFs
  double lame_lambda = 0, lame_mu = 0;
  // device fields
  double *phi = nullptr;         // N_n
  double *coef = nullptr;        // N_T  (A_e, times k for Helmholtz)
  float *coef32 = nullptr;       // N_T
  uint8_t *chi = nullptr;        // N_T
  double *chif = nullptr;        // N_T material fraction (1 / 0 for the one-point rule)
  uint8_t *regmask = nullptr;    // N_T bit j: the element lies in constraint region j
  int ncases = 1;                // load cases (u, p, load hold ncases blocks of N_dof)
  int nvol = 0;                  // region constraints (0: the single |Omega| / V, if any)
  uint8_t *omega0 = nullptr;     // N_T
  uint8_t *dir = nullptr;        // N_dof state Dirichlet mask
  uint8_t *vdir = nullptr;       // N_n velocity Dirichlet mask (H^1_0)
  double *f = nullptr;           // N_n nodal source (heat / Helmholtz), the initial Newton
                                 // guess (logistic: a model without a source), or null
  double *load = nullptr;        // N_dof
  double *u = nullptr;           // N_dof
  double *p = nullptr;           // N_dof
  double *rhs = nullptr;         // d * N_n
  double *theta = nullptr;       // d * N_n
  double *dinv_state = nullptr;  // N_dof
  float *dinv_state32 = nullptr; // N_dof
  double *dinv_vel = nullptr;    // d * N_n
  double *Wst = nullptr;         // state operator rows, stencil form [S][ncomp^2][N_n]
  float *Wst32 = nullptr;        // the same in FP32
  double *Wvel = nullptr;        // velocity operator rows, [S][d][N_n] (component diagonal)
  double *L = nullptr, *R = nullptr;   // transport stencils [S][N_n]
  double *dinvL = nullptr;       // N_n
  double *red = nullptr;         // reduction partials
  unsigned *bar = nullptr;       // grid barrier counter
  int *dev_status = nullptr;     // device error word + solver outputs
  Scratch scratch;
  bool coef_valid = false, u_valid = false, rhs_valid = false, theta_valid = false;
  int newton_steps = 0;          // Newton steps of the last logistic state solve
  fo_inv *inv = nullptr;         // inverse-elasticity data (desc.inverse)
  bool transport_valid = false;
  double transport_dt = 0, transport_h = 0;
  int transport_smooth = 0;
  double last_lambda = 0;
  fo_batch *batch = nullptr;     // non-null for a task-parallel batch (FO_HELMHOLTZ)
  fo_mg *mg = nullptr;           // state multigrid hierarchy, built on the first multigrid solve
  fo_mg *mgv = nullptr;          // velocity multigrid hierarchy (the form is fixed: built once)
  long long coef_epoch = 0;      // incremented by every coefficient update
};

// status helpers
void fo_note_launch(int n);   // count kernel launches made by the library
fo_status fo_fail(fo_ctx *ctx, fo_status st, const char *fmt, ...);
fo_status fo_cuda_check(fo_ctx *ctx, cudaError_t e, const char *what);
fo_status fo_alloc(fo_ctx *ctx, void **p, size_t bytes);
void fo_free(fo_ctx *ctx, void *p, size_t bytes);

#define FO_CU(ctx, call)                                                   \
  do {                                                                     \
    cudaError_t _e = (call);                                               \
    if (_e != cudaSuccess) return fo_cuda_check((ctx), _e, #call);         \
  } while (0)
#define FO_TRY(call)                       \
  do {                                     \
    fo_status _s = (call);                 \
    if (_s != FO_OK) return _s;            \
  } while (0)

// device status words (prob->dev_status[...])
enum { DS_ERR = 0, DS_ITERS = 1, DS_APPLIES = 2, DS_FLAG = 3, DS_COUNT = 8 };
enum { DEV_OK = 0, DEV_TIMEOUT = 1, DEV_NAN = 2, DEV_NOCONV = 3 };

// ----------------------------------------------------------------------------- device side
#define FO_BLOCK 256
#define FO_RED_DOUBLES (1 << 17)   // per-problem reduction buffer (partials + solver outputs)

// Kuhn permutation pi_l of simplex p (lexicographic order of the axis permutations).
template <int D>
__host__ __device__ __forceinline__ int kperm(int p, int l) {
  if (D == 2) return (p == 0) ? l : 1 - l;
  // 012, 021, 102, 120, 201, 210
  switch (p) {
    case 0: return l;
    case 1: return l == 0 ? 0 : (l == 1 ? 2 : 1);
    case 2: return l == 0 ? 1 : (l == 1 ? 0 : 2);
    case 3: return l == 0 ? 1 : (l == 1 ? 2 : 0);
    case 4: return l == 0 ? 2 : (l == 1 ? 0 : 1);
    default: return l == 0 ? 2 : (l == 1 ? 1 : 0);
  }
}
template <int D> struct KP { static constexpr int P = (D == 2) ? 2 : 6; };

__device__ __forceinline__ void node_ijk(const Grid &g, long long a, int idx[3]) {
  if (g.num_nodes <= 0xffffffffLL) {   // 32-bit division (every grid below 2^32 nodes)
    const unsigned ua = (unsigned)a, n0 = (unsigned)g.nn[0], n1 = (unsigned)g.nn[1];
    const unsigned t = ua / n0;
    idx[0] = (int)(ua - t * n0);
    idx[1] = (int)(t % n1);
    idx[2] = (int)(t / n1);
    return;
  }
  idx[0] = (int)(a % g.nn[0]);
  long long t = a / g.nn[0];
  idx[1] = (int)(t % g.nn[1]);
  idx[2] = (int)(t / g.nn[1]);
}

// Element (p, m) of node `a` at grid index idx: node is vertex m of simplex p whose cell
// corner is idx - sum_{l<m} e_{pi_l}.  Returns false when that cell lies outside the grid.
// On success writes the element id and the vertex node ids v[0..D].
template <int D>
__device__ __forceinline__ bool kuhn_elem(const Grid &g, const int idx[3], long long a, int p, int m,
                                          long long &elem, long long v[D + 1]) {
  int c[3] = {idx[0], idx[1], idx[2]};
#pragma unroll
  for (int l = 0; l < D; ++l)
    if (l < m) c[kperm<D>(p, l)] -= 1;
#pragma unroll
  for (int k = 0; k < D; ++k)
    if (c[k] < 0 || c[k] >= g.n[k]) return false;
  long long cell = c[0] + g.cstride[1] * c[1] + (D == 3 ? g.cstride[2] * c[2] : 0);
  elem = (long long)KP<D>::P * cell + p;
  long long base = c[0] + g.stride[1] * c[1] + (D == 3 ? g.stride[2] * c[2] : 0);
  v[0] = base;
#pragma unroll
  for (int l = 0; l < D; ++l) v[l + 1] = v[l] + g.stride[kperm<D>(p, l)];
  (void)a;
  return true;
}

// Stencil slot of the neighbour at offset delta (each component in {-1, 0, 1}); Kuhn
// neighbours have delta in {0,1}^D or -{0,1}^D.  Slot order: 0 = self, then positive
// offsets by bitmask 1..2^D-1, then negative offsets by bitmask.
template <int D>
__device__ __forceinline__ int stencil_slot(const int delta[3]) {
  int pos = 0, neg = 0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    if (delta[k] > 0) pos |= 1 << k;
    if (delta[k] < 0) neg |= 1 << k;
  }
  if (pos == 0 && neg == 0) return 0;
  if (neg == 0) return pos;
  return (1 << D) - 1 + neg;
}
// Stencil slots of a node (itself and its Kuhn neighbours); stored operator rows keep the first
// SH of them (the node's own slot and its positive-direction neighbours, slot_offset below):
// the operators stored by rows are symmetric, so a negative-direction block is the transpose of
// the neighbour's block in the opposite slot.
template <int D> struct ST {
  static constexpr int S = (D == 2) ? 7 : 15;
  static constexpr int SH = 1 << D;
};
inline int fo_row_slots(int dim) { return dim == 2 ? 4 : 8; }

template <int D>
__device__ __forceinline__ void slot_offset(int s, int delta[3]) {
  delta[0] = delta[1] = delta[2] = 0;
  if (s == 0) return;
  int sign = 1, mask = s;
  if (s >= (1 << D)) { sign = -1; mask = s - ((1 << D) - 1); }
#pragma unroll
  for (int k = 0; k < D; ++k)
    if (mask & (1 << k)) delta[k] = sign;
}

// ---- bounded grid barrier --------------------------------------------------------------
// One counter; block 0 adds 2^31 - (G - 1), every other block adds 1, so the top bit flips
// exactly when all G blocks have arrived.  The counter must hold 0 at launch and the grid
// must be co-resident (cooperative launch).  A wait longer than `limit_ns` sets the error
// word to DEV_TIMEOUT and returns false.  The error word is read only by a block that is
// already waiting long (after 1024 polls), so a released barrier costs no extra round trip:
// a block that timed out stops arriving, and every other block then leaves its next wait
// early through the error word, or by its own time limit.
__device__ __forceinline__ unsigned fo_ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned fo_atom_add_release(unsigned *p, unsigned v) {
  unsigned old;
  asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ unsigned long long fo_globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

struct GridBar {
  unsigned *count;
  int *err;
  unsigned long long limit_ns;
};

// Thread 0's part of the barrier: arrive, then wait (bounded).  Returns 0 on a time-out.
__device__ __forceinline__ int grid_arrive_wait(const GridBar &b) {
  unsigned inc = (blockIdx.x == 0) ? (0x80000000u - (gridDim.x - 1)) : 1u;
  // arrival with release semantics (the block's writes, ordered before it by the block
  // barrier before the call, become visible to every block that acquires the released
  // count); polling with acquire loads orders the other blocks' writes before this block's reads
  unsigned old;
  asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(b.count), "r"(inc) : "memory");
  int ok = 1;
  unsigned long long t0 = 0;
  unsigned spins = 0;
  while (((old ^ fo_ld_acquire(b.count)) & 0x80000000u) == 0) {
    if (++spins == 1024) t0 = fo_globaltimer();
    if (spins > 1024 && (spins & 255) == 0) {
      __nanosleep(64);
      if (*(volatile int *)b.err == DEV_TIMEOUT) {   // another block gave up
        ok = 0;
        break;
      }
      if (fo_globaltimer() - t0 > b.limit_ns) {
        atomicExch(b.err, DEV_TIMEOUT);
        ok = 0;
        break;
      }
    }
  }
  return ok;
}

__device__ __forceinline__ bool grid_sync(const GridBar &b) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) s_ok = grid_arrive_wait(b);
  __syncthreads();
  return s_ok != 0;
}

// The barrier with block-local work `side` done by thread 32 while thread 0 waits for the
// grid (work that only this block reads after the barrier, such as small serial FP64 chains
// on shared-memory data).  With a single warp, thread 0 does it before arriving.
template <class F>
__device__ __forceinline__ bool grid_sync_side(const GridBar &b, F side) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    if (blockDim.x <= 32) side();
    s_ok = grid_arrive_wait(b);
  } else if (threadIdx.x == 32) {
    side();
  }
  __syncthreads();
  return s_ok != 0;
}

// ---- deterministic reductions -----------------------------------------------------------
// Warp reduce-scatter of C values (slots 0..C-1 of v) at exchange distance O and below.  At
// each distance a lane keeps one half of its values (the upper half when its lane bit O is
// set), sends the other half to its partner and adds the partner's copy of the half it kept:
// ceil(C/2) FP64 adds per level instead of C for a plain shuffle tree, which matters where
// the FP64 pipe is narrow.  An odd middle slot is kept by both partners (a + b and b + a:
// the same bits).  src(p, lane) is the value that slot p holds after all levels.
template <int NR, int C, int O>
struct WarpScatter {
  static constexpr int HC = (C + 1) / 2;
  using Next = WarpScatter<NR, HC, O / 2>;
  static constexpr int CF = Next::CF;   // slots left after all levels
  static __device__ __forceinline__ void run(double (&v)[NR], int lane) {
    const bool up = (lane & O) != 0;
#pragma unroll
    for (int i = 0; i < C - HC; ++i) {
      const double send = up ? v[i] : v[i + HC];
      const double keep = up ? v[i + HC] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, O);
    }
    if (C & 1) v[HC - 1] += __shfl_xor_sync(0xffffffffu, v[HC - 1], O);
    Next::run(v, lane);
  }
  static __device__ __forceinline__ int src(int p, int lane) {
    const int q = Next::src(p, lane);   // the slot of this level's output
    return (q < C - HC && (lane & O)) ? q + HC : q;
  }
};
template <int NR, int C>
struct WarpScatter<NR, C, 0> {
  static constexpr int CF = C;
  static __device__ __forceinline__ void run(double (&)[NR], int) {}
  static __device__ __forceinline__ int src(int p, int) { return p; }
};

// Block sum of NR values (fixed exchange pattern, fixed warp order); result valid in thread 0.
template <int NR>
__device__ __forceinline__ void block_sum(double (&v)[NR], double *smem /* [32*NR] */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  using WS = WarpScatter<NR, NR, 16>;
  WS::run(v, lane);
  __syncthreads();
  // every lane holding a value writes it; lanes that hold the same value hold the same bits
#pragma unroll
  for (int k = 0; k < WS::CF; ++k) smem[warp * NR + WS::src(k, lane)] = v[k];
  __syncthreads();
  // value j is finished by warp j mod nw (the values proceed in parallel); its result goes
  // to smem[j], a slot only that warp reads
  int top = 1;
  while (top < nw) top <<= 1;
  for (int j = warp; j < NR; j += nw) {
    double t = (lane < nw) ? smem[lane * NR + j] : 0.0;
    for (int o = top >> 1; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0) smem[j] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0)
#pragma unroll
    for (int j = 0; j < NR; ++j) v[j] = smem[j];
}

// Sum of the per-block partials [G][NR] in a fixed order; every block gets the same bits.
// Values are spread over the warps; each lane issues its partial loads in independent
// batches of four before adding them (a fixed order), so a reduction costs about one L2
// round trip instead of one per partial.  Result broadcast through smem_out[NR].
template <int NR>
__device__ __forceinline__ void grid_total(const double *partials, double *smem_out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int G = (int)gridDim.x;
  for (int j = warp; j < NR; j += nw) {
    double t = 0.0;
    int b = lane;
    for (; b + 96 < G; b += 128) {
      const double x0 = __ldcg(partials + (size_t)b * NR + j);
      const double x1 = __ldcg(partials + (size_t)(b + 32) * NR + j);
      const double x2 = __ldcg(partials + (size_t)(b + 64) * NR + j);
      const double x3 = __ldcg(partials + (size_t)(b + 96) * NR + j);
      t += x0;
      t += x1;
      t += x2;
      t += x3;
    }
    for (; b < G; b += 32) t += __ldcg(partials + (size_t)b * NR + j);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0) smem_out[j] = t;
  }
  __syncthreads();
}

// Block-sum the NR values, publish the block partial, wait for the grid, and sum all
// partials in a fixed order into stot.  Consecutive reductions alternate between two
// partial buffers: a block that races ahead to the next reduction cannot overwrite a
// partial that a slower block is still summing (it passed the barrier in between).
template <int NR>
__device__ __forceinline__ bool reduce_grid(double (&v)[NR], double *sred, double *stot, double *partials, int &rk,
                                            const GridBar &bar) {
  block_sum<NR>(v, sred);
  double *part = partials + (size_t)(rk & 1) * gridDim.x * NR;
  if (threadIdx.x == 0)
#pragma unroll
    for (int j = 0; j < NR; ++j) part[(size_t)blockIdx.x * NR + j] = v[j];
  if (!grid_sync(bar)) return false;
  grid_total<NR>(part, stot);
  ++rk;
  return true;
}

// ---- exact cut-cell fraction -----------------------------------------------------------
// |e cap {phi < 0}| / |e| for the P1 phi with vertex values v[0..D] (a vertex with phi = 0 is
// on the outer side).  Closed forms by the number of negative vertices, with a_i = -v_i on the
// negative side and c_j = v_j on the other; each is written as a ratio of sums of positive
// terms, so no difference of nearly equal numbers occurs:
//   one negative:     a^D / prod_j (a + c_j);
//   one non-negative: 1 - c^D / prod_i (c + a_i), expanded: 2D (c (a1 + a2) + a1 a2) / prod,
//                     3D (c^2 (a1+a2+a3) + c (a1 a2 + a1 a3 + a2 a3) + a1 a2 a3) / prod;
//   3D two and two:   the divided difference of min(x, 0)^3 over the vertex values, expanded
//                     into the positive-term ratio `num / den` below (a, b negative; c, e not).
template <int D>
__device__ __forceinline__ double cut_fraction(const double *v) {
  double a[4], c[4];
  int na = 0, nc = 0;
#pragma unroll
  for (int i = 0; i <= D; ++i) {
    if (v[i] < 0.0) a[na++] = -v[i];
    else c[nc++] = v[i];
  }
  if (na == 0) return 0.0;
  if (nc == 0) return 1.0;
  if (D == 2) {
    if (na == 1) return a[0] * a[0] / ((a[0] + c[0]) * (a[0] + c[1]));
    return (c[0] * (a[0] + a[1]) + a[0] * a[1]) / ((c[0] + a[0]) * (c[0] + a[1]));
  }
  if (na == 1) return a[0] * a[0] * a[0] / ((a[0] + c[0]) * (a[0] + c[1]) * (a[0] + c[2]));
  if (nc == 1) {
    const double s1 = a[0] + a[1] + a[2], s2 = a[0] * a[1] + a[0] * a[2] + a[1] * a[2], s3 = a[0] * a[1] * a[2];
    return (c[0] * c[0] * s1 + c[0] * s2 + s3) / ((c[0] + a[0]) * (c[0] + a[1]) * (c[0] + a[2]));
  }
  const double A = a[0], B = a[1], C = c[0], E = c[1];
  const double num = C * A * A * E + C * A * A * B + E * A * A * B + C * E * A * B + A * A * B * B + C * A * B * B +
                     E * A * B * B + C * E * B * B;
  return num / ((A + E) * (B + E) * (A + C) * (B + C));
}

// ---- host launch helpers ------------------------------------------------------------------
inline int fo_blocks_for(long long n, int block = FO_BLOCK, int cap = 1 << 20) {
  long long b = (n + block - 1) / block;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (int)b;
}

// internal entry points implemented across translation units
fo_status fo_launch_coefficients(fo_problem *p);
// several load cases and constraints (fo_fem.cu)
fo_status fo_launch_functionals_on(fo_problem *p, const double *u, const double *load, double *J, double *vol);
fo_status fo_launch_shape_rhs_ex(fo_problem *p, const double *u, const double *f, double lambda, const double *w,
                                 double inv_V, int add);
fo_status fo_region_volumes(fo_problem *p, const double *vol, double *out);
fo_status fo_region_weight(fo_problem *p, int j, double *w);
// task-parallel batch (fo_batch.cu)
fo_status fo_batch_create(fo_problem *p, const fo_model_desc *desc);
void fo_batch_destroy(fo_problem *p);
fo_status fo_batch_prepare(fo_problem *p);     // stencils and Jacobi diagonal from A_e
fo_status fo_batch_state(fo_problem *p, bool adjoint, const fo_solve_opts *o, fo_solve_stats *st);
fo_status fo_batch_functionals(fo_problem *p, double *J, double *vol, double *J_inst);
fo_status fo_batch_shape_rhs(fo_problem *p, double lambda);
fo_status fo_batch_apply(fo_problem *p, const double *x, double *y, bool fp32);
// inverse elasticity (fo_inverse.cu)
fo_status fo_inverse_create(fo_problem *p, const fo_model_desc *desc);
void fo_inverse_destroy(fo_problem *p);
fo_status fo_inverse_states(fo_problem *p, const fo_solve_opts *o, fo_solve_stats *st);
fo_status fo_inverse_adjoints(fo_problem *p, const fo_solve_opts *o, fo_solve_stats *st);
fo_status fo_inverse_cost(fo_problem *p, double *J);
fo_status fo_inverse_shape(fo_problem *p);
fo_status fo_launch_scalar_stencil(fo_ctx *ctx, const Grid &g, const double *coef, const uint8_t *dir, double *W,
                                   float *W32, double *di, float *di32);
// logistic population model (fo_logistic.cu)
fo_status fo_logistic_state(fo_problem *p, const fo_solve_opts *o, fo_solve_stats *st, int *steps_out);
fo_status fo_logistic_adjoint(fo_problem *p, const fo_solve_opts *o, fo_solve_stats *st);
fo_status fo_launch_logistic_shape(fo_problem *p, double lambda, const double *chif, double inv_V, int add);
// multigrid (fo_mg.cu)
fo_status fo_state_pcg_mg(fo_problem *p, const double *b, double *x, const fo_solve_opts *o, fo_solve_stats *st);
void fo_mg_destroy(fo_problem *p);
void fo_mg_release(fo_ctx *ctx, fo_mg *&mg);
size_t fo_mg_bytes(int dim, const int n[3], int npn, int blk, bool own0, bool bf16 = false);
bool fo_mg_applicable(const Grid &g0, int npn, bool general = true);
int fo_mg_plan(const Grid &g0, Grid *g, int max_levels, long long stop_unknowns = 0, int npn = 1, bool general = false);
void fo_mg_restrict(fo_ctx *ctx, const Grid &gc, const Grid &gf, int npn, const double *coef_f, const uint8_t *dir_f,
                    double *coef_c, uint8_t *dir_c);
// batched multigrid (fo_batch_mg.cu) and the batch stencil builder it shares (fo_batch.cu)
void fo_launch_batch_stencil(cudaStream_t s, const Grid &g, const double *coef, const uint8_t *dir, double *WK,
                             double *WM, float *WK32, float *WM32);
fo_status fo_batch_state_mg(fo_problem *p, const double *B, double bscale, double *X, const fo_solve_opts *o, int warm,
                            fo_solve_stats *st);
void fo_bmg_destroy(fo_problem *p);
fo_status fo_batch_read(fo_problem *p, fo_solve_stats *st, const fo_solve_opts *o);   // stats of the last batched solve
fo_status fo_velocity_pcg_mg(fo_problem *p, const fo_solve_opts *o, double *Btt, fo_solve_stats *st);
fo_status fo_launch_velocity_stencil_on(fo_problem *p, const Grid &g, const double *mcoef, const uint8_t *dofmask,
                                        double *W, float *W32, double *dinv, float *dinv32);
// State rows of several grids in one launch (the coarse levels of a hierarchy).
struct StencilLevels {
  int n = 0;
  Grid g[MG_MAX_LEVELS];
  const double *coef[MG_MAX_LEVELS];
  const uint8_t *dir[MG_MAX_LEVELS];
  double *W[MG_MAX_LEVELS];
  float *W32[MG_MAX_LEVELS];
  double *di[MG_MAX_LEVELS];
  float *di32[MG_MAX_LEVELS];
  int first_block[MG_MAX_LEVELS + 1];
};
fo_status fo_launch_stencil_levels(fo_problem *p, const StencilLevels &L);
fo_status fo_launch_stencil_on(fo_problem *p, const Grid &g, const double *coef, const uint8_t *dir, double *W,
                               float *W32, double *dinv, float *dinv32);
fo_status fo_launch_loads(fo_problem *p);
fo_status fo_launch_masks(fo_problem *p);
fo_status fo_launch_state_diag(fo_problem *p);
fo_status fo_launch_velocity_diag(fo_problem *p);
fo_status fo_launch_state_apply(fo_problem *p, const double *x, double *y, bool mask_input);
fo_status fo_launch_state_apply32(fo_problem *p, const double *x, double *y);
fo_status fo_launch_velocity_apply(fo_problem *p, const double *x, double *y);
fo_status fo_launch_functionals(fo_problem *p, double *J, double *vol);
fo_status fo_launch_shape_rhs(fo_problem *p, double lambda);
fo_status fo_launch_mesh_build(fo_mesh *m);
bool fo_grid_make(int dim, const int n[3], const double lo[3], const double hi[3], Grid &g);
size_t fo_problem_footprint(int dim, const int n[3], int kind, int state_vecs, int vel_vecs, int n_bumps);
fo_status fo_launch_phi_bumps(fo_problem *p, int count, const double *centers, double width, double offset);
fo_status fo_launch_initial_level(fo_problem *p, int count, const double *centers, const double *radii,
                                  double factor, int ord);
fo_status fo_state_pcg(fo_problem *p, const double *b, double *x, const fo_solve_opts *o, fo_solve_stats *st);
fo_status fo_velocity_pcg(fo_problem *p, const fo_solve_opts *o, double *Btt, fo_solve_stats *st);
fo_status fo_launch_transport_assemble(fo_problem *p, double dt, double h, int smooth);
fo_status fo_launch_stencil_apply(fo_problem *p, const double *S, const double *x, double *y);
fo_status fo_transport_run(fo_problem *p, int nsteps, const fo_solve_opts *o, fo_solve_stats *st);
fo_status fo_reinit_run(fo_problem *p, int nsteps, double dt, double h, const fo_solve_opts *o,
                        fo_solve_stats *st);
fo_status fo_scratch(fo_problem *p, size_t bytes, void **out);
int fo_persistent_block(const fo_problem *p, long long n);
fo_status fo_cooperative_grid(fo_problem *p, const void *kernel, int block, size_t smem, long long work,
                              int requested, int *grid);
// Kernel attributes are process-wide, while the library may run one context per host thread
// (the request server's executors).  A launch whose dynamic shared memory depends on the
// problem (the multigrid solve's staged levels, the coarsest-level inverse) holds this lock
// from raising the kernel's limit through its occupancy query to the launch, and limits only
// rise (fo_smem_limit, called with the lock held): another thread can then neither lower the
// limit below a launch's request nor change it between a grid's sizing and its launch.
std::mutex &fo_launch_mutex();
fo_status fo_smem_limit(fo_ctx *ctx, const void *kernel, size_t bytes);
