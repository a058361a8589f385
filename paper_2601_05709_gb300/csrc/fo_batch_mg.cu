// Batched geometric multigrid for the task-parallel batch (Sec. 5.3): every screened
// Helmholtz instance -div(A k_i grad u_i) + omega_i^2 u_i = f_i is solved by FP64 conjugate
// gradients preconditioned by one FP32 V-cycle of its own operator, all instances and all
// levels in one persistent cooperative launch.
//
// Hierarchy: the grids of the single-problem multigrid (every axis halved while even).  On a
// coarse grid the stiffness is K_A with children-mean element coefficients and the mass is
// the coarse consistent mass, which is exactly P^T M P since the P1 spaces of the nested Kuhn
// grids are nested; both come from the batch stencil builder.  The rows are stored once for
// all instances, FP32, slot-major, in difference form:
//   SK[0][a] = row sum R_K,  SK[s][a] = off-diagonal weight of slot s,  SK[S][a] = diagonal,
// and likewise SM for the mass, so instance i's row and Jacobi diagonal are formed in
// registers from its two scalars (k_i, w_i = omega_i^2):
//   (A_i z)(a) = (k_i R_K + w_i R_M) z(a) + sum_{s>=1} (k_i WK_s + w_i WM_s) (z(nb_s) - z(a)),
//   D_i(a)     = k_i DK(a) + w_i DM(a).
// Transfers and smoother as in the single-problem V-cycle: P1 interpolation along Kuhn edges,
// R = P^T, damped Jacobi with nu sweeps before and after (one on the finest level), nuc on the
// coarsest level.  Fields
// are instance-minor [N_l][nip]: a warp owns a node and lane l holds instances l, l + 32, ...,
// so a neighbour row is one coalesced 128-byte load per 32 instances and the stencil rows are
// read once for all of them.  The coarse levels (at most BMG_INST_NODES nodes) run one instance
// per block, the instance's vectors in shared memory and a thread per node, with block barriers
// only.
//
// Outer loop: one FP64 CG recurrence per instance on the FP64 stencils of the fine grid,
// stopping instance i when ||b_i - A_i x_i||_2 (recurrence) <= rtol ||b_i||_2; a converged
// instance is frozen (step length zero) and the launch ends when every instance has
// converged.  Reductions are per instance, deterministic and independent of timing: per-warp
// values, a fixed warp order in a block, then every column summed over the blocks by one warp
// in a fixed order.  An instance's arithmetic never mixes with another's and every rounding
// step is spelled out (explicit fma / _rn intrinsics, so the compiler's contraction cannot
// differ between the 32-, 64- and 128-lane kernels): its result does not depend on the rest
// of the batch (for a fixed launch shape).
#include <cmath>
#include <cstring>
#include <algorithm>
#include <vector>

#include "fo_internal.cuh"
#include "fo_ops.cuh"

#define BMG_WARPS 8              // warps per block
#define BMG_INST_NODES 1100      // levels of at most this many nodes run one instance per block
#define BMG_DIRECT_MAX 64        // coarsest levels of at most this many nodes are solved exactly

struct BmgLevel {
  Grid g;
  const float *SK, *SM;   // [S + 1][N] rows in difference form (slot 0 row sum, slot S diagonal)
  const uint8_t *dir;     // [N] Dirichlet mask
  float *b, *z[2], *t;    // [N][nip] right-hand side, iterate (ping-pong), residual
};

struct BmgDev {
  int L, Lg;              // levels; levels >= Lg run one instance per block in shared memory
  int nu0, nu, nuc;       // smoothing sweeps on level 0, on the other levels, on the coarsest
  int nd;                 // > 0: the coarsest level (nd nodes) is solved with the instance's
  const float *ainv;      // inverse of its operator, ainv[i][nd][nd], where direct[i] is set
  const int *direct;
  float omega;
  BmgLevel lv[MG_MAX_LEVELS];
};

struct BmgCg {
  const double *WK, *WM;     // fine FP64 rows, node-major [N][S] (slot 0 = the node itself)
  const double *kk, *w2;     // [nip] k_i, omega_i^2
  const double *B;           // loads [N][nip]; the right-hand side is bscale * B
  double bscale;
  double *X, *r, *p[2], *s;  // [N][nip]; the directions double-buffered (gathered at neighbours)
  double *partials;          // [2 nip][G]
  double *totals;            // [2 nip]
  int *status;
  GridBar bar;
  int *inst_iters;
  double *inst_res;
  double rtol2;
  int maxit, warm;
  // mixed-precision refinement: inner CG vectors [N][nip]; the correction d accumulates in
  // FP64 (an FP32 copy would carry rounding noise that A amplifies by its largest eigenvalue)
  double *d64;
  float *q32[2], *s32;
  double inner_rtol2;
  int inner_maxit;
};

// ------------------------------------------------------------------ instance scalars
// A lane's instances' k_i and omega_i^2 in FP32 (the V-cycle's arithmetic).
template <int D, int NJ>
struct BmgOps {
  struct Coef {
    float k[NJ], w[NJ];
  };
};

// ------------------------------------------------------------------ tiled grid passes
// Levels run by the whole grid are swept tile by tile: a block stages with cp.async (many
// independent 16-byte copies in flight, zero-filled outside the grid) the rows it needs --
// the iterate on the tile's halo box, its own right-hand sides and stencil rows -- and then
// forms its own nodes' rows from shared memory, a warp per node and a lane per instance.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(valid ? 16 : 0) : "memory");
}
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(valid ? 8 : 0) : "memory");
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem), "r"(valid ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// A tile of TX x TY (x TZ) own nodes and its halo box, one node wider on every side (every
// Kuhn neighbour is within one step per axis).  Own dimensions are even, so that the coarse
// nodes the halo interpolates from form a (T/2 + 2)-wide box.
template <int D, int TX_, int TY_, int TZ_>
struct Tile {
  static constexpr int TX = TX_, TY = TY_, TZ = D == 3 ? TZ_ : 1;
  static constexpr int HX = TX + 2, HY = TY + 2, HZ = D == 3 ? TZ + 2 : 1;
  static constexpr int NH = HX * HY * HZ, NT = TX * TY * TZ;
  static_assert(TX % 2 == 0 && TY % 2 == 0 && (D == 2 || TZ % 2 == 0), "even tiles");
  __host__ __device__ static long long count(const Grid &g) {
    return ((g.nn[0] + TX - 1) / TX) * ((g.nn[1] + TY - 1) / TY) * (D == 3 ? (g.nn[2] + TZ - 1) / TZ : 1);
  }
  __device__ static void origin(const Grid &g, long long t, int o[3]) {
    const long long ntx = (g.nn[0] + TX - 1) / TX, nty = (g.nn[1] + TY - 1) / TY;
    o[0] = (int)(t % ntx) * TX;
    const long long r = t / ntx;
    o[1] = (int)(r % nty) * TY;
    o[2] = D == 3 ? (int)(r / nty) * TZ : 0;
  }
  // node of halo slot h (-1 outside the grid)
  __device__ static long long halo_node(const Grid &g, const int o[3], int h) {
    const int hx = h % HX, hy = (h / HX) % HY, hz = h / (HX * HY);
    const int x = o[0] - 1 + hx, y = o[1] - 1 + hy, z = D == 3 ? o[2] - 1 + hz : 0;
    if (x < 0 || x >= g.nn[0] || y < 0 || y >= g.nn[1]) return -1;
    if (D == 3 && (z < 0 || z >= g.nn[2])) return -1;
    return x + g.stride[1] * y + (D == 3 ? g.stride[2] * z : 0);
  }
  // node of own slot t (-1 outside the grid) and its halo slot
  __device__ static long long own_node(const Grid &g, const int o[3], int t, int &hs) {
    const int tx = t % TX, ty = (t / TX) % TY, tz = t / (TX * TY);
    hs = (tx + 1) + HX * (ty + 1) + (D == 3 ? HX * HY * (tz + 1) : 0);
    const int x = o[0] + tx, y = o[1] + ty, z = o[2] + tz;
    if (x >= g.nn[0] || y >= g.nn[1] || (D == 3 && z >= g.nn[2])) return -1;
    return x + g.stride[1] * y + (D == 3 ? g.stride[2] * z : 0);
  }
  __device__ static int slot_shift(int s) {
    int dl[3];
    slot_offset<D>(s, dl);
    return dl[0] + HX * dl[1] + (D == 3 ? HX * HY * dl[2] : 0);
  }
};

// Tile shapes per dimension and instance slab count: FP32 stencil passes, restriction (coarse
// tile), FP64 operator passes, FP32 operator pass of the refinement's inner CG.  The 32- and 64-lane kernels share shapes, so an instance's
// reductions run in the same order in both.
template <int D, int NJ>
struct BmgTiles;
template <> struct BmgTiles<2, 1> { using T32 = Tile<2, 16, 8, 1>; using TR = Tile<2, 8, 4, 1>; using T64 = Tile<2, 16, 4, 1>; using TA = T32; };
template <> struct BmgTiles<2, 2> { using T32 = Tile<2, 16, 8, 1>; using TR = Tile<2, 8, 4, 1>; using T64 = Tile<2, 16, 4, 1>; using TA = T32; };
template <> struct BmgTiles<2, 4> { using T32 = Tile<2, 8, 4, 1>; using TR = Tile<2, 8, 2, 1>; using T64 = Tile<2, 8, 2, 1>; using TA = T32; };
template <> struct BmgTiles<3, 1> { using T32 = Tile<3, 4, 4, 4>; using TR = Tile<3, 4, 2, 2>; using T64 = Tile<3, 4, 2, 2>; using TA = T64; };
template <> struct BmgTiles<3, 2> { using T32 = Tile<3, 4, 4, 4>; using TR = Tile<3, 4, 2, 2>; using T64 = Tile<3, 4, 2, 2>; using TA = T64; };
template <> struct BmgTiles<3, 4> { using T32 = Tile<3, 4, 2, 2>; using TR = Tile<3, 2, 2, 2>; using T64 = Tile<3, 2, 2, 2>; using TA = T64; };

template <int D, int NJ>
struct BmgTiled {
  using TL = typename BmgTiles<D, NJ>::T32;
  using TR = typename BmgTiles<D, NJ>::TR;
  using T6 = typename BmgTiles<D, NJ>::T64;
  using TA = typename BmgTiles<D, NJ>::TA;
  using Coef = typename BmgOps<D, NJ>::Coef;
  static constexpr int S = ST<D>::S, NIP = 32 * NJ;
  static constexpr int CH32 = NIP * 4 / 16, CH64 = NIP * 8 / 16;   // 16-byte chunks per row
  // coarse box behind a T32 halo; fine box behind a coarse TR tile
  static constexpr int CHX = TL::TX / 2 + 2, CHY = TL::TY / 2 + 2, CHZ = D == 3 ? TL::TZ / 2 + 2 : 1;
  static constexpr int NC = CHX * CHY * CHZ;
  static constexpr int FRX = 2 * TR::TX + 1, FRY = 2 * TR::TY + 1, FRZ = D == 3 ? 2 * TR::TZ + 1 : 1;
  static constexpr int NFR = FRX * FRY * FRZ;
  static constexpr size_t smem_stencil =
      4 * ((size_t)TL::NH * NIP + (size_t)TL::NT * NIP + (size_t)NC * NIP + 2 * (S + 1) * (size_t)TL::NT) + TL::NH;
  static constexpr size_t smem_restrict = 4 * ((size_t)NFR * NIP + 2 * (size_t)TR::NT) + TR::NT;
  static constexpr size_t smem_apply = 12 * (size_t)T6::NH * NIP + 16 * (size_t)S * T6::NT;
  static constexpr size_t smem_reduce = 8 * ((size_t)BMG_WARPS * 2 * NIP + 2 * NIP);
  static constexpr size_t smem_apply32 = 8 * (size_t)TA::NH * NIP + 8 * (size_t)(S + 1) * TA::NT;
  static constexpr size_t smem_resid64 = 8 * ((size_t)T6::NH * NIP + (size_t)T6::NT * NIP + 2 * (size_t)S * T6::NT);
  static constexpr size_t cmax(size_t a, size_t b) { return a > b ? a : b; }
  static constexpr size_t smem =
      (cmax(cmax(cmax(smem_stencil, smem_restrict), cmax(smem_apply, smem_reduce)), cmax(smem_apply32, smem_resid64)) +
       15) / 16 * 16;

  // MODE 0: z_out = z_in + omega D^{-1} (b - A z_in).  MODE 1: the same after adding the
  // prolongated coarse correction P z_c to z_in on the fly (prolongation and first post-sweep
  // in one pass; the corrected iterate is never stored).  MODE 2: t = b - A z_in.
  // dot (MODE 0/1, when given): += (b, z_out) of the own nodes, FP32 over a warp's nodes of a
  // tile and FP64 across tiles (on level 0 of the refinement's inner CG b is its residual).
  template <int MODE>
  static __device__ void stencil_pass(const BmgLevel &L, const float *zin, float *out, float omega, const Coef &cf,
                                      const BmgLevel *C, const float *zc, unsigned char *smem, int lane,
                                      double *dot = nullptr) {
    const Grid &g = L.g;
    const long long N = g.num_nodes;
    float *sz = reinterpret_cast<float *>(smem);
    float *sb = sz + TL::NH * NIP;
    float *sc = sb + TL::NT * NIP;
    float *swK = sc + NC * NIP;
    float *swM = swK + (S + 1) * TL::NT;
    unsigned char *sdir = reinterpret_cast<unsigned char *>(swM + (S + 1) * TL::NT);
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const long long ntile = TL::count(g);
    for (long long tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
      int o[3];
      TL::origin(g, tile, o);
      __syncthreads();   // the previous tile's shared data is consumed
      for (int c = threadIdx.x; c < TL::NH * CH32; c += blockDim.x) {
        const int h = c / CH32, k = c - h * CH32;
        const long long nb = TL::halo_node(g, o, h);
        cp_async16(sz + h * NIP + 4 * k, zin + (nb < 0 ? 0 : nb * NIP) + 4 * k, nb >= 0);
      }
      for (int c = threadIdx.x; c < TL::NT * CH32; c += blockDim.x) {
        const int t = c / CH32, k = c - t * CH32;
        int hs;
        const long long a = TL::own_node(g, o, t, hs);
        cp_async16(sb + t * NIP + 4 * k, L.b + (a < 0 ? 0 : a * NIP) + 4 * k, a >= 0);
      }
      for (int c = threadIdx.x; c < (S + 1) * TL::NT; c += blockDim.x) {
        const int s = c / TL::NT, t = c - s * TL::NT;
        int hs;
        const long long a = TL::own_node(g, o, t, hs);
        const long long off = a < 0 ? 0 : (long long)s * N + a;
        cp_async4(swK + c, L.SK + off, a >= 0);
        cp_async4(swM + c, L.SM + off, a >= 0);
      }
      const int co[3] = {o[0] / 2 - 1, o[1] / 2 - 1, D == 3 ? o[2] / 2 - 1 : 0};
      if (MODE == 1) {
        const Grid &gc = C->g;
        for (int c = threadIdx.x; c < NC * CH32; c += blockDim.x) {
          const int q = c / CH32, k = c - q * CH32;
          const int x = co[0] + q % CHX, y = co[1] + (q / CHX) % CHY, z = co[2] + q / (CHX * CHY);
          const bool in = x >= 0 && x < gc.nn[0] && y >= 0 && y < gc.nn[1] && (D == 2 || (z >= 0 && z < gc.nn[2]));
          const long long cn = in ? x + gc.stride[1] * y + (D == 3 ? gc.stride[2] * z : 0) : 0;
          cp_async16(sc + q * NIP + 4 * k, zc + cn * NIP + 4 * k, in);
        }
        for (int h = threadIdx.x; h < TL::NH; h += blockDim.x) {
          const long long nb = TL::halo_node(g, o, h);
          sdir[h] = nb < 0 ? 1 : L.dir[nb];
        }
      }
      cp_async_wait_all();
      __syncthreads();
      if (MODE == 1) {   // halo iterate += P z_c (Dirichlet nodes and nodes outside untouched)
        for (int h = warp; h < TL::NH; h += nw) {
          if (sdir[h]) continue;
          const int f[3] = {o[0] - 1 + h % TL::HX, o[1] - 1 + (h / TL::HX) % TL::HY,
                            D == 3 ? o[2] - 1 + h / (TL::HX * TL::HY) : 0};
          const int cst[3] = {1, CHX, CHX * CHY};
          int q1 = 0, q2 = 0;
          bool mid = false;
#pragma unroll
          for (int k = 0; k < D; ++k) {
            const int bit = f[k] & 1;
            mid |= bit != 0;
            q1 += ((f[k] - bit) / 2 - co[k]) * cst[k];
            q2 += ((f[k] + bit) / 2 - co[k]) * cst[k];
          }
#pragma unroll
          for (int j = 0; j < NJ; ++j) {
            const int i = lane + 32 * j;
            const float v = mid ? __fmul_rn(0.5f, __fadd_rn(sc[q1 * NIP + i], sc[q2 * NIP + i])) : sc[q1 * NIP + i];
            sz[h * NIP + i] = __fadd_rn(sz[h * NIP + i], v);
          }
        }
        __syncthreads();
      }
      float df[NJ];
#pragma unroll
      for (int j = 0; j < NJ; ++j) df[j] = 0.f;
      for (int t = warp; t < TL::NT; t += nw) {
        int hs;
        const long long a = TL::own_node(g, o, t, hs);
        if (a < 0) continue;
        const float rk = swK[t], rm = swM[t], dk = swK[S * TL::NT + t], dm = swM[S * TL::NT + t];
        float za[NJ], az[NJ];
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
          za[j] = sz[hs * NIP + lane + 32 * j];
          az[j] = __fmul_rn(fmaf(cf.k[j], rk, __fmul_rn(cf.w[j], rm)), za[j]);
        }
#pragma unroll
        for (int s = 1; s < S; ++s) {
          const float wk = swK[s * TL::NT + t], wm = swM[s * TL::NT + t];
          if (wk == 0.f && wm == 0.f) continue;
          const int hn = hs + TL::slot_shift(s);
#pragma unroll
          for (int j = 0; j < NJ; ++j)
            az[j] = fmaf(fmaf(cf.k[j], wk, __fmul_rn(cf.w[j], wm)), __fsub_rn(sz[hn * NIP + lane + 32 * j], za[j]),
                         az[j]);
        }
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
          const int i = lane + 32 * j;
          const float bq = sb[t * NIP + i];
          if (MODE == 2) {
            out[a * NIP + i] = __fsub_rn(bq, az[j]);
          } else {
            const float dg = fmaf(cf.k[j], dk, __fmul_rn(cf.w[j], dm));
            const float zn = __fadd_rn(za[j], __fdiv_rn(__fmul_rn(omega, __fsub_rn(bq, az[j])), dg));
            out[a * NIP + i] = zn;
            if (dot) df[j] = fmaf(bq, zn, df[j]);
          }
        }
      }
      if (dot)
#pragma unroll
        for (int j = 0; j < NJ; ++j) dot[j] += (double)df[j];
    }
  }

  // coarse b = P^T t (zero on coarse Dirichlet nodes) and the coarse level's first sweep
  static __device__ void restrict_pass(const BmgLevel &F, const BmgLevel &C, float omega, const Coef &cf,
                                       unsigned char *smem, int lane) {
    const Grid &gc = C.g, &gf = F.g;
    const long long Nc = gc.num_nodes;
    float *st = reinterpret_cast<float *>(smem);
    float *sdk = st + NFR * NIP;
    float *sdm = sdk + TR::NT;
    unsigned char *sdc = reinterpret_cast<unsigned char *>(sdm + TR::NT);
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const long long ntile = TR::count(gc);
    for (long long tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
      int co[3];
      TR::origin(gc, tile, co);
      __syncthreads();
      const int fo[3] = {2 * co[0] - 1, 2 * co[1] - 1, D == 3 ? 2 * co[2] - 1 : 0};
      for (int c = threadIdx.x; c < NFR * CH32; c += blockDim.x) {
        const int q = c / CH32, k = c - q * CH32;
        const int x = fo[0] + q % FRX, y = fo[1] + (q / FRX) % FRY, z = fo[2] + q / (FRX * FRY);
        const bool in = x >= 0 && x < gf.nn[0] && y >= 0 && y < gf.nn[1] && (D == 2 || (z >= 0 && z < gf.nn[2]));
        const long long fn = in ? x + gf.stride[1] * y + (D == 3 ? gf.stride[2] * z : 0) : 0;
        cp_async16(st + q * NIP + 4 * k, F.t + fn * NIP + 4 * k, in);
      }
      for (int t = threadIdx.x; t < TR::NT; t += blockDim.x) {
        int hs;
        const long long cn = TR::own_node(gc, co, t, hs);
        sdk[t] = cn < 0 ? 1.f : C.SK[S * Nc + cn];
        sdm[t] = cn < 0 ? 0.f : C.SM[S * Nc + cn];
        sdc[t] = cn < 0 ? 1 : C.dir[cn];
      }
      cp_async_wait_all();
      __syncthreads();
      for (int t = warp; t < TR::NT; t += nw) {
        int hs;
        const long long cn = TR::own_node(gc, co, t, hs);
        if (cn < 0) continue;
        const int tx = t % TR::TX, ty = (t / TR::TX) % TR::TY, tz = t / (TR::TX * TR::TY);
        const int q0 = (2 * tx + 1) + FRX * (2 * ty + 1) + (D == 3 ? FRX * FRY * (2 * tz + 1) : 0);
        float v[NJ];
#pragma unroll
        for (int j = 0; j < NJ; ++j) v[j] = st[q0 * NIP + lane + 32 * j];
#pragma unroll
        for (int s = 1; s < S; ++s) {
          int dl[3];
          slot_offset<D>(s, dl);
          const int q = q0 + dl[0] + FRX * dl[1] + (D == 3 ? FRX * FRY * dl[2] : 0);
#pragma unroll
          for (int j = 0; j < NJ; ++j) v[j] = fmaf(0.5f, st[q * NIP + lane + 32 * j], v[j]);
        }
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
          const long long qq = cn * NIP + lane + 32 * j;
          const float bk = sdc[t] ? 0.f : v[j];
          C.b[qq] = bk;
          C.z[0][qq] = __fdiv_rn(__fmul_rn(omega, bk), fmaf(cf.k[j], sdk[t], __fmul_rn(cf.w[j], sdm[t])));
        }
      }
    }
  }

  // p_new = z + beta p_old (formed on the halo in shared memory), s = A p_new in FP64 from the
  // plain node-major FP64 rows; writes p_new and s of the own nodes; dot += (p_new, s).
  static __device__ void apply_pass(const Grid &g, const double *WK, const double *WM, const double *pold,
                                    const float *z, double *pnew, double *sout, const double (&beta)[NJ],
                                    const double (&kk)[NJ], const double (&w2)[NJ], double (&dot)[NJ],
                                    unsigned char *smem, int lane) {
    double *sp = reinterpret_cast<double *>(smem);
    float *szz = reinterpret_cast<float *>(sp + T6::NH * NIP);
    double *swK = reinterpret_cast<double *>(szz + T6::NH * NIP);
    double *swM = swK + S * T6::NT;
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const long long ntile = T6::count(g);
    for (long long tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
      int o[3];
      T6::origin(g, tile, o);
      __syncthreads();
      for (int c = threadIdx.x; c < T6::NH * CH64; c += blockDim.x) {
        const int h = c / CH64, k = c - h * CH64;
        const long long nb = T6::halo_node(g, o, h);
        cp_async16(sp + h * NIP + 2 * k, pold + (nb < 0 ? 0 : nb * NIP) + 2 * k, nb >= 0);
      }
      for (int c = threadIdx.x; c < T6::NH * CH32; c += blockDim.x) {
        const int h = c / CH32, k = c - h * CH32;
        const long long nb = T6::halo_node(g, o, h);
        cp_async16(szz + h * NIP + 4 * k, z + (nb < 0 ? 0 : nb * NIP) + 4 * k, nb >= 0);
      }
      for (int c = threadIdx.x; c < S * T6::NT; c += blockDim.x) {
        const int t = c / S, s = c - t * S;
        int hs;
        const long long a = T6::own_node(g, o, t, hs);
        const long long off = a < 0 ? 0 : a * S + s;
        cp_async8(swK + c, WK + off, a >= 0);
        cp_async8(swM + c, WM + off, a >= 0);
      }
      cp_async_wait_all();
      __syncthreads();
      for (int h = warp; h < T6::NH; h += nw)
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
          const int q = h * NIP + lane + 32 * j;
          sp[q] = fma(beta[j], sp[q], (double)szz[q]);
        }
      __syncthreads();
      for (int t = warp; t < T6::NT; t += nw) {
        int hs;
        const long long a = T6::own_node(g, o, t, hs);
        if (a < 0) continue;
        double yk[NJ], ym[NJ];
#pragma unroll
        for (int j = 0; j < NJ; ++j) yk[j] = ym[j] = 0.0;
#pragma unroll
        for (int s = 0; s < S; ++s) {
          const double wk = swK[t * S + s], wm = swM[t * S + s];
          if (s > 0 && wk == 0.0 && wm == 0.0) continue;
          const int hn = hs + T6::slot_shift(s);
#pragma unroll
          for (int j = 0; j < NJ; ++j) {
            const double xv = sp[hn * NIP + lane + 32 * j];
            yk[j] = fma(wk, xv, yk[j]);
            ym[j] = fma(wm, xv, ym[j]);
          }
        }
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
          const int i = lane + 32 * j;
          const double y = fma(kk[j], yk[j], __dmul_rn(w2[j], ym[j]));
          const double pv = sp[hs * NIP + i];
          pnew[a * NIP + i] = pv;
          sout[a * NIP + i] = y;
          dot[j] = fma(pv, y, dot[j]);
        }
      }
    }
  }

  // Inner CG of the refinement (FP32): q_new = z + beta q_old (on the halo in shared memory),
  // s = A_i q_new with the level's FP32 difference-form rows; writes q_new and s of the own
  // nodes; dot += (q_new, s) (FP32 over a warp's nodes of a tile, FP64 across tiles).
  static __device__ void apply32_pass(const BmgLevel &L, const float *qold, const float *z, float *qnew, float *sout,
                                      const float (&beta)[NJ], const Coef &cf, double (&dot)[NJ], unsigned char *smem,
                                      int lane) {
    const Grid &g = L.g;
    const long long N = g.num_nodes;
    float *sq = reinterpret_cast<float *>(smem);
    float *szz = sq + TA::NH * NIP;
    float *swK = szz + TA::NH * NIP;
    float *swM = swK + (S + 1) * TA::NT;
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const long long ntile = TA::count(g);
    for (long long tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
      int o[3];
      TA::origin(g, tile, o);
      __syncthreads();
      for (int c = threadIdx.x; c < TA::NH * CH32; c += blockDim.x) {
        const int h = c / CH32, k = c - h * CH32;
        const long long nb = TA::halo_node(g, o, h);
        const long long off = (nb < 0 ? 0 : nb * NIP) + 4 * k;
        cp_async16(sq + h * NIP + 4 * k, qold + off, nb >= 0);
        cp_async16(szz + h * NIP + 4 * k, z + off, nb >= 0);
      }
      for (int c = threadIdx.x; c < (S + 1) * TA::NT; c += blockDim.x) {
        const int s = c / TA::NT, t = c - s * TA::NT;
        int hs;
        const long long a = TA::own_node(g, o, t, hs);
        const long long off = a < 0 ? 0 : (long long)s * N + a;
        cp_async4(swK + c, L.SK + off, a >= 0);
        cp_async4(swM + c, L.SM + off, a >= 0);
      }
      cp_async_wait_all();
      __syncthreads();
      for (int h = warp; h < TA::NH; h += nw)
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
          const int q = h * NIP + lane + 32 * j;
          sq[q] = fmaf(beta[j], sq[q], szz[q]);
        }
      __syncthreads();
      float df[NJ];
#pragma unroll
      for (int j = 0; j < NJ; ++j) df[j] = 0.f;
      for (int t = warp; t < TA::NT; t += nw) {
        int hs;
        const long long a = TA::own_node(g, o, t, hs);
        if (a < 0) continue;
        const float rk = swK[t], rm = swM[t];
        float pa[NJ], y[NJ];
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
          pa[j] = sq[hs * NIP + lane + 32 * j];
          y[j] = __fmul_rn(fmaf(cf.k[j], rk, __fmul_rn(cf.w[j], rm)), pa[j]);
        }
#pragma unroll
        for (int s = 1; s < S; ++s) {
          const float wk = swK[s * TA::NT + t], wm = swM[s * TA::NT + t];
          if (wk == 0.f && wm == 0.f) continue;
          const int hn = hs + TA::slot_shift(s);
#pragma unroll
          for (int j = 0; j < NJ; ++j)
            y[j] = fmaf(fmaf(cf.k[j], wk, __fmul_rn(cf.w[j], wm)), __fsub_rn(sq[hn * NIP + lane + 32 * j], pa[j]), y[j]);
        }
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
          const int i = lane + 32 * j;
          qnew[a * NIP + i] = pa[j];
          sout[a * NIP + i] = y[j];
          df[j] = fmaf(pa[j], y[j], df[j]);
        }
      }
#pragma unroll
      for (int j = 0; j < NJ; ++j) dot[j] += (double)df[j];
    }
  }

  // r = bscale B - A_i X in FP64 from the plain node-major FP64 rows (X = 0 when !use_x);
  // rr += ||r||^2, bb += ||bscale B||^2.
  static __device__ void residual64_pass(const Grid &g, const double *WK, const double *WM, const double *X, bool use_x,
                                         const double *B, double bscale, double *r64, const double (&kk)[NJ],
                                         const double (&w2)[NJ], double (&rr)[NJ], double (&bb)[NJ],
                                         unsigned char *smem, int lane) {
    double *sx = reinterpret_cast<double *>(smem);
    double *sB = sx + T6::NH * NIP;
    double *swK = sB + T6::NT * NIP;
    double *swM = swK + S * T6::NT;
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const long long ntile = T6::count(g);
    for (long long tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
      int o[3];
      T6::origin(g, tile, o);
      __syncthreads();
      if (use_x)
        for (int c = threadIdx.x; c < T6::NH * CH64; c += blockDim.x) {
          const int h = c / CH64, k = c - h * CH64;
          const long long nb = T6::halo_node(g, o, h);
          cp_async16(sx + h * NIP + 2 * k, X + (nb < 0 ? 0 : nb * NIP) + 2 * k, nb >= 0);
        }
      for (int c = threadIdx.x; c < T6::NT * CH64; c += blockDim.x) {
        const int t = c / CH64, k = c - t * CH64;
        int hs;
        const long long a = T6::own_node(g, o, t, hs);
        cp_async16(sB + t * NIP + 2 * k, B + (a < 0 ? 0 : a * NIP) + 2 * k, a >= 0);
      }
      if (use_x)
        for (int c = threadIdx.x; c < S * T6::NT; c += blockDim.x) {
          const int t = c / S, s = c - t * S;
          int hs;
          const long long a = T6::own_node(g, o, t, hs);
          const long long off = a < 0 ? 0 : a * S + s;
          cp_async8(swK + c, WK + off, a >= 0);
          cp_async8(swM + c, WM + off, a >= 0);
        }
      cp_async_wait_all();
      __syncthreads();
      for (int t = warp; t < T6::NT; t += nw) {
        int hs;
        const long long a = T6::own_node(g, o, t, hs);
        if (a < 0) continue;
        double ax[NJ];
#pragma unroll
        for (int j = 0; j < NJ; ++j) ax[j] = 0.0;
        if (use_x) {
          double yk[NJ], ym[NJ];
#pragma unroll
          for (int j = 0; j < NJ; ++j) yk[j] = ym[j] = 0.0;
#pragma unroll
          for (int s = 0; s < S; ++s) {
            const double wk = swK[t * S + s], wm = swM[t * S + s];
            if (s > 0 && wk == 0.0 && wm == 0.0) continue;
            const int hn = hs + T6::slot_shift(s);
#pragma unroll
            for (int j = 0; j < NJ; ++j) {
              const double xv = sx[hn * NIP + lane + 32 * j];
              yk[j] = fma(wk, xv, yk[j]);
              ym[j] = fma(wm, xv, ym[j]);
            }
          }
#pragma unroll
          for (int j = 0; j < NJ; ++j) ax[j] = fma(kk[j], yk[j], __dmul_rn(w2[j], ym[j]));
        }
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
          const int i = lane + 32 * j;
          const double bq = __dmul_rn(bscale, sB[t * NIP + i]);
          const double r = __dsub_rn(bq, ax[j]);
          r64[a * NIP + i] = r;
          rr[j] = fma(r, r, rr[j]);
          bb[j] = fma(bq, bq, bb[j]);
        }
      }
    }
  }
};

// Buffer index of each level's final iterate after a V-cycle (fixed by the sweep counts).
__host__ __device__ inline int bmg_nu(const BmgDev &mg, int l) { return l == 0 ? mg.nu0 : mg.nu; }
__host__ __device__ inline void bmg_final_buffers(const BmgDev &mg, int *zc) {
  for (int l = 0; l < mg.L; ++l) {
    const int nu = bmg_nu(mg, l);
    const int sweeps = (l == mg.L - 1) ? mg.nuc : nu;
    int c = (sweeps - 1) & 1;
    if (l < mg.L - 1) c = (c + nu) & 1;
    zc[l] = c;
  }
}

// Levels >= from, one instance per block (instances blockIdx.x, blockIdx.x + G, ...): the
// instance's vectors of these levels live in shared memory (b, z0, z1, t of every level), a
// thread per node; the rows are read through L1.  Starts from b_from and z_from[0] in global
// memory and writes level `from`'s final iterate back to z_from[zc[from]].
template <int D>
__device__ void bmg_inst_cycle(const BmgDev &mg, const double *kk, const double *w2, int nip, int from, float *sm) {
  constexpr int S = ST<D>::S;
  const float omega = mg.omega;
  auto vec = [&](int l, int q) {   // q: 0 b, 1 z0, 2 z1, 3 t
    long long off = 0;
    for (int m = from; m < l; ++m) off += 4 * mg.lv[m].g.num_nodes;
    return sm + off + q * mg.lv[l].g.num_nodes;
  };
  auto row = [&](int l, long long a, const float *z, float ki, float wi, float &za, float &az, float &dg) {
    const BmgLevel &L = mg.lv[l];
    const long long N = L.g.num_nodes;
    int idx[3];
    node_ijk(L.g, a, idx);
    const float rk = L.SK[a], rm = L.SM[a], dk = L.SK[S * N + a], dm = L.SM[S * N + a];
    za = z[a];
    az = __fmul_rn(fmaf(ki, rk, __fmul_rn(wi, rm)), za);
    dg = fmaf(ki, dk, __fmul_rn(wi, dm));
#pragma unroll
    for (int s = 1; s < S; ++s) {
      const long long nb = slot_node<D>(L.g, idx, a, s);
      if (nb < 0) continue;
      const float wk = L.SK[s * N + a], wm = L.SM[s * N + a];
      if (wk == 0.f && wm == 0.f) continue;
      az = fmaf(fmaf(ki, wk, __fmul_rn(wi, wm)), __fsub_rn(z[nb], za), az);
    }
  };
  const int NIP = nip;
  for (int inst = blockIdx.x; inst < nip; inst += gridDim.x) {
    const float ki = (float)kk[inst], wi = (float)w2[inst];
    __syncthreads();   // shared memory free
    {
      const BmgLevel &L = mg.lv[from];
      float *b = vec(from, 0), *z0 = vec(from, 1);
      for (long long a = threadIdx.x; a < L.g.num_nodes; a += blockDim.x) {
        b[a] = L.b[a * NIP + inst];
        z0[a] = L.z[0][a * NIP + inst];
      }
    }
    int zl[MG_MAX_LEVELS];
    for (int l = from; l < mg.L; ++l) {
      const long long N = mg.lv[l].g.num_nodes;
      const bool coarsest = l == mg.L - 1;
      const int sweeps = coarsest ? mg.nuc : bmg_nu(mg, l);
      float *b = vec(l, 0);
      int c = 0;
      if (coarsest && mg.nd > 0 && mg.direct[inst]) {   // exact solve, into the sweeps' last buffer
        c = (sweeps - 1) & 1;
        __syncthreads();
        const float *A = mg.ainv + (size_t)inst * mg.nd * mg.nd;
        float *zo = vec(l, 1 + c);
        for (int a = threadIdx.x; a < mg.nd; a += blockDim.x) {
          float acc = 0.f;
          for (int k = 0; k < mg.nd; ++k) acc = fmaf(A[a * mg.nd + k], b[k], acc);
          zo[a] = acc;
        }
        zl[l] = c;
        break;
      }
      for (int j = 1; j < sweeps; ++j) {
        __syncthreads();
        const float *zi = vec(l, 1 + c);
        float *zo = vec(l, 2 - c);
        for (long long a = threadIdx.x; a < N; a += blockDim.x) {
          float za, az, dg;
          row(l, a, zi, ki, wi, za, az, dg);
          zo[a] = __fadd_rn(za, __fdiv_rn(__fmul_rn(omega, __fsub_rn(b[a], az)), dg));
        }
        c ^= 1;
      }
      zl[l] = c;
      if (coarsest) break;
      __syncthreads();
      {
        const float *zi = vec(l, 1 + c);
        float *t = vec(l, 3);
        for (long long a = threadIdx.x; a < N; a += blockDim.x) {
          float za, az, dg;
          row(l, a, zi, ki, wi, za, az, dg);
          t[a] = __fsub_rn(b[a], az);
        }
      }
      __syncthreads();
      {   // restriction to level l + 1 and its first sweep from zero
        const BmgLevel &F = mg.lv[l], &Cl = mg.lv[l + 1];
        const long long Nc = Cl.g.num_nodes;
        const float *t = vec(l, 3);
        float *bc = vec(l + 1, 0), *zc0 = vec(l + 1, 1);
        for (long long cn = threadIdx.x; cn < Nc; cn += blockDim.x) {
          int ic[3];
          node_ijk(Cl.g, cn, ic);
          int ifn[3] = {2 * ic[0], 2 * ic[1], D == 3 ? 2 * ic[2] : 0};
          const long long f0 = ifn[0] + F.g.stride[1] * ifn[1] + (D == 3 ? F.g.stride[2] * ifn[2] : 0);
          float v = t[f0];
#pragma unroll
          for (int s = 1; s < S; ++s) {
            const long long nb = slot_node<D>(F.g, ifn, f0, s);
            if (nb >= 0) v = fmaf(0.5f, t[nb], v);
          }
          const float bk = Cl.dir[cn] ? 0.f : v;
          bc[cn] = bk;
          zc0[cn] = __fdiv_rn(__fmul_rn(omega, bk), fmaf(ki, Cl.SK[S * Nc + cn], __fmul_rn(wi, Cl.SM[S * Nc + cn])));
        }
      }
    }
    for (int l = mg.L - 2; l >= from; --l) {
      const BmgLevel &F = mg.lv[l], &Cl = mg.lv[l + 1];
      const long long N = F.g.num_nodes;
      __syncthreads();
      {   // z_l += P z_{l+1}
        float *zf = vec(l, 1 + zl[l]);
        const float *zcv = vec(l + 1, 1 + zl[l + 1]);
        for (long long a = threadIdx.x; a < N; a += blockDim.x) {
          if (F.dir[a]) continue;
          int idx[3];
          node_ijk(F.g, a, idx);
          long long c1 = 0, c2 = 0;
          bool mid = false;
#pragma unroll
          for (int k = 0; k < D; ++k) {
            const int bit = idx[k] & 1;
            mid |= bit != 0;
            c1 += (long long)((idx[k] - bit) / 2) * Cl.g.stride[k];
            c2 += (long long)((idx[k] + bit) / 2) * Cl.g.stride[k];
          }
          const float v = mid ? __fmul_rn(0.5f, __fadd_rn(zcv[c1], zcv[c2])) : zcv[c1];
          zf[a] = __fadd_rn(zf[a], v);
        }
      }
      int c = zl[l];
      float *b = vec(l, 0);
      for (int j = 0; j < bmg_nu(mg, l); ++j) {
        __syncthreads();
        const float *zi = vec(l, 1 + c);
        float *zo = vec(l, 2 - c);
        for (long long a = threadIdx.x; a < N; a += blockDim.x) {
          float za, az, dg;
          row(l, a, zi, ki, wi, za, az, dg);
          zo[a] = __fadd_rn(za, __fdiv_rn(__fmul_rn(omega, __fsub_rn(b[a], az)), dg));
        }
        c ^= 1;
      }
      zl[l] = c;
    }
    __syncthreads();
    {
      const BmgLevel &L = mg.lv[from];
      const float *zf = vec(from, 1 + zl[from]);
      float *dst = L.z[zl[from]];
      for (long long a = threadIdx.x; a < L.g.num_nodes; a += blockDim.x) dst[a * NIP + inst] = zf[a];
    }
  }
}

// One V-cycle from level 0, whose b and first sweep were written before a grid barrier.
// Level 0's result ends in z[zc[0]], written by the warp that owns each node's tile slot (no
// barrier after the last sweep: the caller's next pass reads it only after one).
// gdot (when given and level 0 is swept by the grid): += (b_0, z_0) over the own nodes, formed
// in the last sweep on level 0.
template <int D, int NJ>
__device__ bool bmg_vcycle(const BmgDev &mg, const typename BmgOps<D, NJ>::Coef &cf, const double *kk,
                           const double *w2, int *zc, const GridBar &bar, unsigned char *smem, int lane,
                           double *gdot = nullptr) {
  using TP = BmgTiled<D, NJ>;
  const int Lg = mg.Lg;
  if (Lg == 0) {
    bmg_inst_cycle<D>(mg, kk, w2, 32 * NJ, 0, reinterpret_cast<float *>(smem));
    return grid_sync(bar);
  }
  for (int l = 0; l < Lg; ++l) {
    const BmgLevel &L = mg.lv[l];
    const bool coarsest = l == mg.L - 1;
    const int sweeps = coarsest ? mg.nuc : bmg_nu(mg, l);
    int c = 0;
    for (int j = 1; j < sweeps; ++j) {
      TP::template stencil_pass<0>(L, L.z[c], L.z[c ^ 1], mg.omega, cf, nullptr, nullptr, smem, lane);
      c ^= 1;
      if (!grid_sync(bar)) return false;
    }
    zc[l] = c;
    if (coarsest) break;
    TP::template stencil_pass<2>(L, L.z[c], L.t, mg.omega, cf, nullptr, nullptr, smem, lane);
    if (!grid_sync(bar)) return false;
    TP::restrict_pass(L, mg.lv[l + 1], mg.omega, cf, smem, lane);
    if (!grid_sync(bar)) return false;
  }
  if (Lg < mg.L) {
    bmg_inst_cycle<D>(mg, kk, w2, 32 * NJ, Lg, reinterpret_cast<float *>(smem));
    if (!grid_sync(bar)) return false;
  }
  for (int l = (Lg < mg.L - 1 ? Lg : mg.L - 1) - 1; l >= 0; --l) {
    const BmgLevel &L = mg.lv[l];
    const BmgLevel &C = mg.lv[l + 1];
    int c = zc[l];
    for (int j = 0; j < bmg_nu(mg, l); ++j) {
      double *dot = (l == 0 && j + 1 == bmg_nu(mg, l)) ? gdot : nullptr;
      if (j == 0) TP::template stencil_pass<1>(L, L.z[c], L.z[c ^ 1], mg.omega, cf, &C, C.z[zc[l + 1]], smem, lane, dot);
      else TP::template stencil_pass<0>(L, L.z[c], L.z[c ^ 1], mg.omega, cf, nullptr, nullptr, smem, lane, dot);
      c ^= 1;
      if (l > 0 || j + 1 < bmg_nu(mg, l))
        if (!grid_sync(bar)) return false;
    }
    zc[l] = c;
  }
  return true;
}

// Per-instance sums of NCOL columns over the grid into tot[c * NIP + i] (same bits in every
// block).  part: BMG_WARPS * NCOL * NIP doubles of shared memory.
template <int NCOL, int NJ>
__device__ bool bmg_allreduce(const BmgCg &C, const double (&v)[NCOL][NJ], double *part, double *tot) {
  constexpr int NIP = 32 * NJ;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int G = (int)gridDim.x;
  __syncthreads();   // the scratch may still be read by the previous pass or reduction
#pragma unroll
  for (int c = 0; c < NCOL; ++c)
#pragma unroll
    for (int j = 0; j < NJ; ++j) part[(warp * NCOL + c) * NIP + lane + 32 * j] = v[c][j];
  __syncthreads();
  for (int t = threadIdx.x; t < NCOL * NIP; t += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += part[w * NCOL * NIP + t];
    __stcg(C.partials + (size_t)t * G + blockIdx.x, s);
  }
  if (!grid_sync(C.bar)) return false;
  const int gw = blockIdx.x * nw + warp, nwt = G * nw;
  for (int col = gw; col < NCOL * NIP; col += nwt) {
    const double *src = C.partials + (size_t)col * G;
    double t = 0.0;
    for (int b = lane; b < G; b += 32) t += __ldcg(src + b);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0) __stcg(C.totals + col, t);
  }
  if (!grid_sync(C.bar)) return false;
  for (int t = threadIdx.x; t < NCOL * NIP; t += blockDim.x) tot[t] = __ldcg(C.totals + t);
  __syncthreads();
  return true;
}

template <int D, int NJ>
__global__ void __launch_bounds__(32 * BMG_WARPS, 2) k_bmg_pcg(const BmgDev *mgp, BmgCg C) {
  constexpr int S = ST<D>::S, NIP = 32 * NJ;
  using O = BmgOps<D, NJ>;
  using TP = BmgTiled<D, NJ>;
  extern __shared__ __align__(16) unsigned char bmg_smem[];
  __shared__ BmgDev mg;
  double *part = reinterpret_cast<double *>(bmg_smem);   // reduction scratch between passes
  double *tot = part + BMG_WARPS * 2 * NIP;
  {
    const int *src = reinterpret_cast<const int *>(mgp);
    int *dst = reinterpret_cast<int *>(&mg);
    for (int i = threadIdx.x; i < (int)(sizeof(BmgDev) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const long long first = blockIdx.x * (long long)nw + warp, step = (long long)gridDim.x * nw;
  const BmgLevel &L0 = mg.lv[0];
  const Grid &g = L0.g;
  const long long N = g.num_nodes;
  double kk[NJ], w2[NJ];
  typename O::Coef cf;
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    kk[j] = C.kk[lane + 32 * j];
    w2[j] = C.w2[lane + 32 * j];
    cf.k[j] = (float)kk[j];
    cf.w[j] = (float)w2[j];
  }
  int zc[MG_MAX_LEVELS];
  bmg_final_buffers(mg, zc);
  const int zfin = zc[0];
  const float omega = mg.omega;

  double bb[NJ], rr[NJ], gam[NJ];
  bool done[NJ];
  int its[NJ];
  bool nan_seen = false;
  // r = b - A x; p = 0; level-0 right-hand side and first sweep; ||b||^2, ||r||^2 (once per
  // solve: warp per node)
  {
    double v[2][NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) v[0][j] = v[1][j] = 0.0;
    for (long long a = first; a < N; a += step) {
      int idx[3];
      node_ijk(g, a, idx);
      double ax[NJ];
#pragma unroll
      for (int j = 0; j < NJ; ++j) ax[j] = 0.0;
      if (C.warm) {
        double yk[NJ], ym[NJ];
#pragma unroll
        for (int j = 0; j < NJ; ++j) yk[j] = ym[j] = 0.0;
#pragma unroll
        for (int s = 0; s < S; ++s) {
          const long long nb = slot_node<D>(g, idx, a, s);
          if (nb < 0) continue;
          const double wk = C.WK[a * S + s], wm = C.WM[a * S + s];
#pragma unroll
          for (int j = 0; j < NJ; ++j) {
            const double xv = C.X[nb * NIP + lane + 32 * j];
            yk[j] = fma(wk, xv, yk[j]);
            ym[j] = fma(wm, xv, ym[j]);
          }
        }
#pragma unroll
        for (int j = 0; j < NJ; ++j) ax[j] = fma(kk[j], yk[j], __dmul_rn(w2[j], ym[j]));
      }
      const float dk = L0.SK[S * N + a], dm = L0.SM[S * N + a];
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const long long q = a * NIP + lane + 32 * j;
        const double bq = C.bscale * C.B[q];
        const double r0 = bq - ax[j];
        C.r[q] = r0;
        C.p[0][q] = 0.0;
        const float bf = (float)r0;
        L0.b[q] = bf;
        L0.z[0][q] = __fdiv_rn(__fmul_rn(omega, bf), fmaf(cf.k[j], dk, __fmul_rn(cf.w[j], dm)));
        v[0][j] = fma(bq, bq, v[0][j]);
        v[1][j] = fma(r0, r0, v[1][j]);
      }
    }
    if (!bmg_allreduce<2, NJ>(C, v, part, tot)) return;
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      bb[j] = tot[lane + 32 * j];
      rr[j] = tot[NIP + lane + 32 * j];
      done[j] = rr[j] <= C.rtol2 * bb[j];
      its[j] = 0;
      gam[j] = 0.0;
    }
    if (!C.warm)   // X = 0 (after every block has read X for the residual: none did)
      for (long long a = first; a < N; a += step)
#pragma unroll
        for (int j = 0; j < NJ; ++j) C.X[a * NIP + lane + 32 * j] = 0.0;
  }
  int it = 0, cur = 0;
  for (;;) {
    bool all = true;
#pragma unroll
    for (int j = 0; j < NJ; ++j) all = all && done[j];
    all = __all_sync(0xffffffffu, all);
    if (all || it >= C.maxit) break;
    if (!bmg_vcycle<D, NJ>(mg, cf, C.kk, C.w2, zc, C.bar, bmg_smem, lane)) return;
    const float *z = L0.z[zfin];
    // gamma = (r, z), in the tile order of the last sweep (each z read by the thread that
    // wrote it: no barrier needed), four nodes at a time
    double v1[1][NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) v1[0][j] = 0.0;
    {
      using TL = typename TP::TL;
      const long long ntile = TL::count(g);
      for (long long tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
        int o[3];
        TL::origin(g, tile, o);
        for (int t0 = warp; t0 < TL::NT; t0 += 4 * nw) {
          double rv[4][NJ];
          float zv[4][NJ];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            int hs;
            const int t = t0 + u * nw;
            long long a = t < TL::NT ? TL::own_node(g, o, t, hs) : -1;
#pragma unroll
            for (int j = 0; j < NJ; ++j) {
              const long long q = (a < 0 ? 0 : a) * NIP + lane + 32 * j;
              rv[u][j] = a < 0 ? 0.0 : C.r[q];
              zv[u][j] = a < 0 ? 0.f : z[q];
            }
          }
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int j = 0; j < NJ; ++j) v1[0][j] = fma(rv[u][j], (double)zv[u][j], v1[0][j]);
        }
      }
    }
    if (!bmg_allreduce<1, NJ>(C, v1, part, tot)) return;
    double beta[NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const double gn = tot[lane + 32 * j];
      beta[j] = (it > 0 && gam[j] > 0.0) ? gn / gam[j] : 0.0;
      gam[j] = gn;
    }
    // p_new = z + beta p_old, s = A p_new, (p_new, s)
#pragma unroll
    for (int j = 0; j < NJ; ++j) v1[0][j] = 0.0;
    TP::apply_pass(g, C.WK, C.WM, C.p[cur], z, C.p[cur ^ 1], C.s, beta, kk, w2, v1[0], bmg_smem, lane);
    cur ^= 1;
    if (!bmg_allreduce<1, NJ>(C, v1, part, tot)) return;
    double alpha[NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const double sig = tot[lane + 32 * j];
      alpha[j] = 0.0;
      if (!done[j]) {
        if (sig > 0.0 && gam[j] > 0.0) alpha[j] = gam[j] / sig;
        else done[j] = true;   // exact zero residual, or definiteness lost in rounding: stop here
      }
    }
    // x += alpha p; r -= alpha s; next level-0 right-hand side and first sweep; ||r||^2
#pragma unroll
    for (int j = 0; j < NJ; ++j) v1[0][j] = 0.0;
    const double *pc = C.p[cur];
    for (long long a0 = first; a0 < N; a0 += 2 * step) {
      double xv[2][NJ], pv[2][NJ], rv[2][NJ], sv[2][NJ];
      float dk[2], dm[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const long long a = a0 + u * step, ac = a < N ? a : 0;
        dk[u] = L0.SK[S * N + ac];
        dm[u] = L0.SM[S * N + ac];
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
          const long long q = ac * NIP + lane + 32 * j;
          xv[u][j] = C.X[q];
          pv[u][j] = pc[q];
          rv[u][j] = C.r[q];
          sv[u][j] = C.s[q];
        }
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const long long a = a0 + u * step;
        if (a >= N) continue;
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
          const long long q = a * NIP + lane + 32 * j;
          C.X[q] = fma(alpha[j], pv[u][j], xv[u][j]);
          const double r1 = fma(-alpha[j], sv[u][j], rv[u][j]);
          C.r[q] = r1;
          const float bf = (float)r1;
          L0.b[q] = bf;
          L0.z[0][q] = __fdiv_rn(__fmul_rn(omega, bf), fmaf(cf.k[j], dk[u], __fmul_rn(cf.w[j], dm[u])));
          v1[0][j] = fma(r1, r1, v1[0][j]);
        }
      }
    }
    if (!bmg_allreduce<1, NJ>(C, v1, part, tot)) return;
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      if (done[j]) continue;
      its[j] += 1;
      rr[j] = tot[lane + 32 * j];
      if (rr[j] != rr[j]) {
        nan_seen = true;
        done[j] = true;
      } else if (rr[j] <= C.rtol2 * bb[j]) {
        done[j] = true;
      }
    }
    ++it;
  }
  bool conv = true;
#pragma unroll
  for (int j = 0; j < NJ; ++j) conv = conv && rr[j] <= C.rtol2 * bb[j];
  conv = __all_sync(0xffffffffu, conv);
  nan_seen = __any_sync(0xffffffffu, nan_seen);
  if (blockIdx.x == 0 && warp == 0) {
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const int i = lane + 32 * j;
      C.inst_iters[i] = its[j];
      C.inst_res[i] = bb[j] > 0.0 ? sqrt(rr[j] / bb[j]) : sqrt(rr[j]);
    }
    if (lane == 0) {
      C.status[DS_ITERS] = it;
      C.status[DS_APPLIES] = it;
      C.status[DS_FLAG] = 0;
      if (nan_seen) atomicCAS(C.status + DS_ERR, DEV_OK, DEV_NAN);
      else if (!conv) atomicCAS(C.status + DS_ERR, DEV_OK, DEV_NOCONV);
    }
  }
}

// Mixed precision: FP64 iterative refinement around an FP32 conjugate-gradient solve, the
// same V-cycle as preconditioner.  Each refinement step forms the true residual
// r = b - A x in FP64, hands r / ||r|| (per instance) to the FP32 CG, which runs until its
// recursive residual is below inner_rtol (or inner_maxit), and adds ||r|| d to x in FP64.
// Only the residual pass and the update of x use FP64 arithmetic; an iteration of the inner
// CG moves FP32 vectors only.  An instance stops when its true residual meets rtol, or when a
// refinement step fails to halve it (the residual has reached the rounding floor of its FP64
// evaluation; the solve then reports non-convergence with the residual reached).
template <int D, int NJ>
__global__ void __launch_bounds__(32 * BMG_WARPS, 2) k_bmg_ir(const BmgDev *mgp, BmgCg C) {
  constexpr int S = ST<D>::S, NIP = 32 * NJ;
  using O = BmgOps<D, NJ>;
  using TP = BmgTiled<D, NJ>;
  extern __shared__ __align__(16) unsigned char bmg_smem[];
  __shared__ BmgDev mg;
  double *part = reinterpret_cast<double *>(bmg_smem);
  double *tot = part + BMG_WARPS * 2 * NIP;
  {
    const int *src = reinterpret_cast<const int *>(mgp);
    int *dst = reinterpret_cast<int *>(&mg);
    for (int i = threadIdx.x; i < (int)(sizeof(BmgDev) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const long long first = blockIdx.x * (long long)nw + warp, step = (long long)gridDim.x * nw;
  const BmgLevel &L0 = mg.lv[0];
  const Grid &g = L0.g;
  const long long N = g.num_nodes;
  double kk[NJ], w2[NJ];
  typename O::Coef cf;
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    kk[j] = C.kk[lane + 32 * j];
    w2[j] = C.w2[lane + 32 * j];
    cf.k[j] = (float)kk[j];
    cf.w[j] = (float)w2[j];
  }
  int zc[MG_MAX_LEVELS];
  bmg_final_buffers(mg, zc);
  const int zfin = zc[0];
  const float omega = mg.omega;
  float *r32 = L0.b;   // the inner residual is the V-cycle's level-0 right-hand side

  double bb[NJ], rr[NJ];
  int its[NJ];
  bool nan_seen = false;
  {
    double v[2][NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) v[0][j] = v[1][j] = 0.0;
    TP::residual64_pass(g, C.WK, C.WM, C.X, C.warm != 0, C.B, C.bscale, C.r, kk, w2, v[1], v[0], bmg_smem, lane);
    if (!C.warm)
      for (long long a = first; a < N; a += step)
#pragma unroll
        for (int j = 0; j < NJ; ++j) C.X[a * NIP + lane + 32 * j] = 0.0;
    if (!bmg_allreduce<2, NJ>(C, v, part, tot)) return;
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      bb[j] = tot[lane + 32 * j];
      rr[j] = tot[NIP + lane + 32 * j];
      its[j] = 0;
    }
  }
  int total = 0, outer = 0;
  bool stalled[NJ];
  double rr_prev[NJ];
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    stalled[j] = false;
    rr_prev[j] = INFINITY;
  }
  for (;;) {
    bool act[NJ], any = false;
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      if (rr[j] != rr[j]) nan_seen = true;
      // a step that did not halve the true residual has reached the FP64 floor of b - A x
      if (rr[j] > 0.25 * rr_prev[j]) stalled[j] = true;
      act[j] = !stalled[j] && rr[j] == rr[j] && rr[j] > C.rtol2 * bb[j];
      any = any || act[j];
    }
    if (!__any_sync(0xffffffffu, any) || total >= C.maxit) break;
    double scale[NJ];
    float inv[NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      scale[j] = act[j] ? sqrt(rr[j]) : 0.0;
      inv[j] = act[j] ? (float)(1.0 / scale[j]) : 0.f;
    }
    // inner start: r32 = r / ||r||, d = 0, q = 0, level-0 first sweep
    for (long long a = first; a < N; a += step) {
      const float dk = L0.SK[S * N + a], dm = L0.SM[S * N + a];
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const long long q = a * NIP + lane + 32 * j;
        const float rf = __fmul_rn((float)C.r[q], inv[j]);
        r32[q] = rf;
        L0.z[0][q] = __fdiv_rn(__fmul_rn(omega, rf), fmaf(cf.k[j], dk, __fmul_rn(cf.w[j], dm)));
        C.d64[q] = 0.0;
        C.q32[0][q] = 0.f;
      }
    }
    if (!grid_sync(C.bar)) return;
    bool idone[NJ];
    double gam[NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      idone[j] = !act[j];
      gam[j] = 0.0;
    }
    int cur = 0;
    for (int ii = 0;; ++ii) {
      bool all = true;
#pragma unroll
      for (int j = 0; j < NJ; ++j) all = all && idone[j];
      if (__all_sync(0xffffffffu, all) || ii >= C.inner_maxit || total >= C.maxit) break;
      // gamma = (r32, z): formed by the V-cycle's last sweep on level 0 (r32 is that level's
      // right-hand side), or, when level 0 runs per instance, by a pass in the tile order of
      // the last sweep (own values, no barrier needed)
      double v1[1][NJ];
#pragma unroll
      for (int j = 0; j < NJ; ++j) v1[0][j] = 0.0;
      if (!bmg_vcycle<D, NJ>(mg, cf, C.kk, C.w2, zc, C.bar, bmg_smem, lane, mg.Lg > 0 ? v1[0] : nullptr)) return;
      const float *z = L0.z[zfin];
      if (mg.Lg == 0) {
        using TL = typename TP::TL;
        const long long ntile = TL::count(g);
        for (long long tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
          int o[3];
          TL::origin(g, tile, o);
          float df[NJ];
#pragma unroll
          for (int j = 0; j < NJ; ++j) df[j] = 0.f;
          for (int t0 = warp; t0 < TL::NT; t0 += 4 * nw) {
            float rv[4][NJ], zv[4][NJ];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              int hs;
              const int t = t0 + u * nw;
              const long long a = t < TL::NT ? TL::own_node(g, o, t, hs) : -1;
#pragma unroll
              for (int j = 0; j < NJ; ++j) {
                const long long q = (a < 0 ? 0 : a) * NIP + lane + 32 * j;
                rv[u][j] = a < 0 ? 0.f : r32[q];
                zv[u][j] = a < 0 ? 0.f : z[q];
              }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
              for (int j = 0; j < NJ; ++j) df[j] = fmaf(rv[u][j], zv[u][j], df[j]);
          }
#pragma unroll
          for (int j = 0; j < NJ; ++j) v1[0][j] += (double)df[j];
        }
      }
      if (!bmg_allreduce<1, NJ>(C, v1, part, tot)) return;
      float beta[NJ];
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const double gn = tot[lane + 32 * j];
        beta[j] = (ii > 0 && gam[j] > 0.0) ? (float)(gn / gam[j]) : 0.f;
        gam[j] = gn;
      }
#pragma unroll
      for (int j = 0; j < NJ; ++j) v1[0][j] = 0.0;
      TP::apply32_pass(L0, C.q32[cur], z, C.q32[cur ^ 1], C.s32, beta, cf, v1[0], bmg_smem, lane);
      cur ^= 1;
      if (!bmg_allreduce<1, NJ>(C, v1, part, tot)) return;
      float alpha[NJ];
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const double sig = tot[lane + 32 * j];
        alpha[j] = 0.f;
        if (!idone[j]) {
          if (sig > 0.0 && gam[j] > 0.0) alpha[j] = (float)(gam[j] / sig);
          else idone[j] = true;
        }
      }
      // d += alpha q; r32 -= alpha s; level-0 first sweep; ||r32||^2
#pragma unroll
      for (int j = 0; j < NJ; ++j) v1[0][j] = 0.0;
      const float *qc = C.q32[cur];
      for (long long a0 = first; a0 < N; a0 += 4 * step) {
        double dv[4][NJ];
        float pv[4][NJ], rv[4][NJ], sv[4][NJ], dk[4], dm[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const long long a = a0 + u * step, ac = a < N ? a : 0;
          dk[u] = L0.SK[S * N + ac];
          dm[u] = L0.SM[S * N + ac];
#pragma unroll
          for (int j = 0; j < NJ; ++j) {
            const long long q = ac * NIP + lane + 32 * j;
            dv[u][j] = C.d64[q];
            pv[u][j] = qc[q];
            rv[u][j] = r32[q];
            sv[u][j] = C.s32[q];
          }
        }
        float rf[NJ];
#pragma unroll
        for (int j = 0; j < NJ; ++j) rf[j] = 0.f;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const long long a = a0 + u * step;
          if (a >= N) continue;
#pragma unroll
          for (int j = 0; j < NJ; ++j) {
            const long long q = a * NIP + lane + 32 * j;
            C.d64[q] = fma((double)alpha[j], (double)pv[u][j], dv[u][j]);
            const float r1 = fmaf(-alpha[j], sv[u][j], rv[u][j]);
            r32[q] = r1;
            L0.z[0][q] = __fdiv_rn(__fmul_rn(omega, r1), fmaf(cf.k[j], dk[u], __fmul_rn(cf.w[j], dm[u])));
            rf[j] = fmaf(r1, r1, rf[j]);
          }
        }
#pragma unroll
        for (int j = 0; j < NJ; ++j) v1[0][j] += (double)rf[j];
      }
      if (!bmg_allreduce<1, NJ>(C, v1, part, tot)) return;
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        if (idone[j]) continue;
        its[j] += 1;
        const double r2 = tot[lane + 32 * j];
        if (!(r2 > C.inner_rtol2)) idone[j] = true;   // met, or NaN (caught by the FP64 residual)
      }
      ++total;
    }
    // x += ||r|| d (FP64), then the true residual
    for (long long a = first; a < N; a += step)
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const long long q = a * NIP + lane + 32 * j;
        C.X[q] = fma(scale[j], C.d64[q], C.X[q]);
      }
    if (!grid_sync(C.bar)) return;
    double v[2][NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) v[0][j] = v[1][j] = 0.0;
    TP::residual64_pass(g, C.WK, C.WM, C.X, true, C.B, C.bscale, C.r, kk, w2, v[1], v[0], bmg_smem, lane);
    if (!bmg_allreduce<2, NJ>(C, v, part, tot)) return;
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      if (act[j]) rr_prev[j] = rr[j];
      rr[j] = tot[NIP + lane + 32 * j];
    }
    ++outer;
  }
  bool conv = true;
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    conv = conv && rr[j] <= C.rtol2 * bb[j];
    nan_seen = nan_seen || rr[j] != rr[j];
  }
  conv = __all_sync(0xffffffffu, conv);
  nan_seen = __any_sync(0xffffffffu, nan_seen);
  if (blockIdx.x == 0 && warp == 0) {
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const int i = lane + 32 * j;
      C.inst_iters[i] = its[j];
      C.inst_res[i] = bb[j] > 0.0 ? sqrt(rr[j] / bb[j]) : sqrt(rr[j]);
    }
    if (lane == 0) {
      C.status[DS_ITERS] = total;
      C.status[DS_APPLIES] = total + outer + 1;
      C.status[DS_FLAG] = outer;
      if (nan_seen) atomicCAS(C.status + DS_ERR, DEV_OK, DEV_NAN);
      else if (!conv) atomicCAS(C.status + DS_ERR, DEV_OK, DEV_NOCONV);
    }
  }
}

// Difference-form FP32 rows (slot-major, slot S the diagonal) from plain node-major FP64 rows
// whose Dirichlet columns are already zero.
__global__ void k_bmg_rows(long long N, int S, const double *WK, const double *WM, float *SK, float *SM) {
  for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < N; a += (long long)gridDim.x * blockDim.x) {
    double rk = 0.0, rm = 0.0;
    for (int s = 0; s < S; ++s) {
      rk += WK[a * S + s];
      rm += WM[a * S + s];
    }
    SK[a] = (float)rk;
    SM[a] = (float)rm;
    for (int s = 1; s < S; ++s) {
      SK[s * N + a] = (float)WK[a * S + s];
      SM[s * N + a] = (float)WM[a * S + s];
    }
    SK[(long long)S * N + a] = (float)WK[a * S];
    SM[(long long)S * N + a] = (float)WM[a * S];
  }
}

// Inverse of instance i's operator k_i K + omega_i^2 M on the coarsest level (nd nodes, at most
// BMG_DIRECT_MAX), one block per instance: the dense matrix from the level's plain FP64 rows
// (Dirichlet rows identity, their columns eliminated), inverted in place in shared memory by
// Gauss-Jordan elimination without pivoting (symmetric positive definite), stored in FP32.
template <int D>
__global__ void k_bmg_coarse_inverse(Grid g, const double *WK, const double *WM, const double *kk, const double *w2,
                                     int nd, float *ainv, int *direct) {
  constexpr int S = ST<D>::S;
  __shared__ double A[BMG_DIRECT_MAX * BMG_DIRECT_MAX];
  __shared__ double piv, dmax;
  __shared__ int ok;
  const int inst = blockIdx.x;
  const double k = kk[inst], w = w2[inst];
  for (int q = threadIdx.x; q < nd * nd; q += blockDim.x) A[q] = 0.0;
  __syncthreads();
  for (long long a = threadIdx.x; a < nd; a += blockDim.x) {
    int idx[3];
    node_ijk(g, a, idx);
    for (int s = 0; s < S; ++s) {
      const long long nb = slot_node<D>(g, idx, a, s);
      if (nb < 0) continue;
      A[a * nd + nb] += fma(k, WK[a * S + s], w * WM[a * S + s]);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    dmax = 0.0;
    for (int a = 0; a < nd; ++a) dmax = fmax(dmax, fabs(A[a * nd + a]));
    ok = 1;
  }
  for (int p = 0; p < nd; ++p) {
    __syncthreads();
    if (threadIdx.x == 0) {
      // a pivot that is not clearly positive (a singular instance: no Dirichlet node and
      // omega = 0) leaves the instance to the Jacobi sweeps
      const double d = A[p * nd + p];
      if (!(d > 1e-10 * dmax)) ok = 0;
      piv = ok ? 1.0 / d : 0.0;
    }
    __syncthreads();
    const double q = piv;
    for (int e = threadIdx.x; e < nd * nd; e += blockDim.x) {
      const int i = e / nd, j = e - i * nd;
      if (i != p && j != p) A[e] -= A[i * nd + p] * A[p * nd + j] * q;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nd; e += blockDim.x)
      if (e != p) {
        A[p * nd + e] *= q;
        A[e * nd + p] *= -q;
      }
    if (threadIdx.x == 0) A[p * nd + p] = q;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nd * nd; e += blockDim.x) ainv[(size_t)inst * nd * nd + e] = ok ? (float)A[e] : 0.f;
  if (threadIdx.x == 0) direct[inst] = ok;
}

// ===================================================================================== host
struct fo_bmg {
  int L = 0, nip = 0, grid_cap = 0, per_sm = 0;
  int Lg0 = 0;                // first level run one instance per block (from the size limits)
  // schedule chosen by fo_batch_mg_autotune per precision (index 1: FO_MIXED; tuned = 0: the
  // defaults: grid_cap blocks, one finest-level sweep, per-instance levels from Lg0)
  int tuned[2] = {0, 0}, t_bpsm[2] = {0, 0}, t_nu0[2] = {1, 1}, t_lgshift[2] = {0, 0};
  int up_pi = -1;             // precision index of the uploaded level table (-1: none)
  long long built_epoch = -1;
  Grid g[MG_MAX_LEVELS];
  double *coef[MG_MAX_LEVELS] = {}, *WK[MG_MAX_LEVELS] = {}, *WM[MG_MAX_LEVELS] = {};
  uint8_t *dir[MG_MAX_LEVELS] = {};
  float *SK[MG_MAX_LEVELS] = {}, *SM[MG_MAX_LEVELS] = {};
  float *b[MG_MAX_LEVELS] = {}, *z0[MG_MAX_LEVELS] = {}, *z1[MG_MAX_LEVELS] = {}, *t[MG_MAX_LEVELS] = {};
  double *r = nullptr, *p0 = nullptr, *p1 = nullptr, *s = nullptr, *partials = nullptr;
  double *d64 = nullptr;
  float *q0 = nullptr, *q1 = nullptr, *s32 = nullptr;
  int nd = 0;                 // coarsest nodes when it is solved exactly
  float *ainv = nullptr;      // [nip][nd][nd]
  int *direct = nullptr;      // [nip]
  void *dev = nullptr;
  std::vector<unsigned char> host;
  std::vector<std::pair<void **, size_t>> allocs;
};

void fo_bmg_destroy(fo_problem *p) {
  if (!p->batch || !p->batch->mg) return;
  fo_bmg *mg = p->batch->mg;
  for (auto &e : mg->allocs) fo_free(p->ctx, *e.first, e.second);
  delete mg;
  p->batch->mg = nullptr;
}

struct BmgKernel {
  void (*fn)(const BmgDev *, BmgCg) = nullptr;
  size_t smem = 0;
};
template <int D, int NJ>
static BmgKernel bmg_entry(bool mixed) {
  BmgKernel k;
  k.fn = mixed ? k_bmg_ir<D, NJ> : k_bmg_pcg<D, NJ>;
  k.smem = BmgTiled<D, NJ>::smem;
  return k;
}
// FP64 CG (mixed = false) or FP64 refinement around an FP32 CG (mixed = true)
static BmgKernel bmg_kernel(int dim, int nj, bool mixed) {
  if (dim == 2)
    return nj == 1 ? bmg_entry<2, 1>(mixed) : (nj == 2 ? bmg_entry<2, 2>(mixed) : bmg_entry<2, 4>(mixed));
  return nj == 1 ? bmg_entry<3, 1>(mixed) : (nj == 2 ? bmg_entry<3, 2>(mixed) : bmg_entry<3, 4>(mixed));
}

static fo_status bmg_alloc(fo_problem *p) {
  fo_ctx *ctx = p->ctx;
  fo_batch *bt = p->batch;
  fo_bmg *mg = new fo_bmg();
  bt->mg = mg;
  mg->nip = bt->nip;
  mg->L = fo_mg_plan(p->mesh->g, mg->g, MG_MAX_LEVELS);
  const int S = p->mesh->g.dim == 2 ? 7 : 15;
  const size_t nip = (size_t)bt->nip;
  int per_sm = 1 << 30;
  for (int mixed = 0; mixed < 2; ++mixed) {   // one grid that both solvers can hold co-resident
    const BmgKernel k = bmg_kernel(p->mesh->g.dim, bt->nip / 32, mixed != 0);
    int v = 0;
    FO_CU(ctx, cudaFuncSetAttribute((const void *)k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem));
    FO_CU(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, (const void *)k.fn, 32 * BMG_WARPS, k.smem));
    per_sm = std::min(per_sm, v);
  }
  if (per_sm < 1) return fo_fail(ctx, FO_ECUDA, "batched multigrid kernel does not fit on an SM");
  mg->per_sm = per_sm;
  mg->grid_cap = std::min(per_sm * ctx->num_sms, 4096);
  auto add = [&](void **ptr, size_t bytes) { mg->allocs.push_back({ptr, bytes}); };
  for (int l = 0; l < mg->L; ++l) {
    const size_t N = (size_t)mg->g[l].num_nodes;
    if (l > 0) {
      add((void **)&mg->coef[l], sizeof(double) * mg->g[l].num_elems);
      add((void **)&mg->dir[l], N);
      add((void **)&mg->WK[l], sizeof(double) * S * N);
      add((void **)&mg->WM[l], sizeof(double) * S * N);
    }
    add((void **)&mg->SK[l], sizeof(float) * (S + 1) * N);
    add((void **)&mg->SM[l], sizeof(float) * (S + 1) * N);
    add((void **)&mg->b[l], sizeof(float) * N * nip);
    add((void **)&mg->z0[l], sizeof(float) * N * nip);
    add((void **)&mg->z1[l], sizeof(float) * N * nip);
    add((void **)&mg->t[l], sizeof(float) * N * nip);
  }
  const size_t n0 = (size_t)mg->g[0].num_nodes * nip;
  add((void **)&mg->r, sizeof(double) * n0);
  add((void **)&mg->p0, sizeof(double) * n0);
  add((void **)&mg->p1, sizeof(double) * n0);
  add((void **)&mg->d64, sizeof(double) * n0);
  add((void **)&mg->q0, sizeof(float) * n0);
  add((void **)&mg->q1, sizeof(float) * n0);
  add((void **)&mg->s32, sizeof(float) * n0);
  add((void **)&mg->s, sizeof(double) * n0);
  add((void **)&mg->partials, sizeof(double) * (2 * nip * (size_t)mg->grid_cap + 2 * nip));
  if (mg->L >= 2 && mg->g[mg->L - 1].num_nodes <= BMG_DIRECT_MAX) {
    mg->nd = (int)mg->g[mg->L - 1].num_nodes;
    add((void **)&mg->ainv, sizeof(float) * nip * mg->nd * mg->nd);
    add((void **)&mg->direct, sizeof(int) * nip);
  }
  add(&mg->dev, sizeof(BmgDev));
  for (auto &e : mg->allocs) FO_TRY(fo_alloc(ctx, e.first, e.second));
  return FO_OK;
}

// The level table with the current schedule: one sweep before and after the coarse correction
// on the finest level (its passes carry nearly all the traffic; 104 instead of 100 iterations
// on the 64-instance 512x512 batch, 13 % less time per solve) unless tuned otherwise, two on
// the coarser ones; per-instance levels from Lg0, or one level later when tuned so.
static fo_status bmg_upload(fo_problem *p, int pi) {
  fo_ctx *ctx = p->ctx;
  fo_batch *bt = p->batch;
  fo_bmg *mg = bt->mg;
  BmgDev h;
  memset(&h, 0, sizeof h);
  h.L = mg->L;
  h.Lg = mg->Lg0;
  if (mg->tuned[pi] && mg->t_lgshift[pi] > 0 && mg->Lg0 + mg->t_lgshift[pi] < mg->L) h.Lg = mg->Lg0 + mg->t_lgshift[pi];
  h.nu0 = mg->tuned[pi] ? mg->t_nu0[pi] : 1;
  h.nu = 2;
  h.nuc = 16;
  h.omega = 0.8f;
  if (mg->nd > 0 && h.Lg < h.L) {
    h.nd = mg->nd;
    h.ainv = mg->ainv;
    h.direct = mg->direct;
  }
  for (int l = 0; l < mg->L; ++l) {
    BmgLevel &d = h.lv[l];
    d.g = mg->g[l];
    d.SK = mg->SK[l];
    d.SM = mg->SM[l];
    d.dir = l == 0 ? p->dir : mg->dir[l];
    d.b = mg->b[l];
    d.z[0] = mg->z0[l];
    d.z[1] = mg->z1[l];
    d.t = mg->t[l];
  }
  mg->host.resize(sizeof(BmgDev));
  memcpy(mg->host.data(), &h, sizeof(BmgDev));
  FO_CU(ctx, cudaMemcpyAsync(mg->dev, mg->host.data(), sizeof(BmgDev), cudaMemcpyHostToDevice, ctx->stream));
  FO_CU(ctx, cudaGetLastError());
  mg->up_pi = pi;
  return FO_OK;
}

// Rows of every level from the current coefficients (the batch's fine FP64 rows are rebuilt
// by every coefficient update; coarse levels from children-mean coefficients).
static fo_status bmg_prepare(fo_problem *p) {
  fo_ctx *ctx = p->ctx;
  fo_batch *bt = p->batch;
  if (!bt->mg) FO_TRY(bmg_alloc(p));
  fo_bmg *mg = bt->mg;
  if (mg->built_epoch == p->coef_epoch) return FO_OK;
  cudaStream_t s = ctx->stream;
  const int S = mg->g[0].dim == 2 ? 7 : 15;
  for (int l = 0; l < mg->L; ++l) {
    const double *WK = bt->WK, *WM = bt->WM;
    if (l > 0) {
      fo_mg_restrict(ctx, mg->g[l], mg->g[l - 1], 1, l == 1 ? p->coef : mg->coef[l - 1], l == 1 ? p->dir : mg->dir[l - 1],
                     mg->coef[l], mg->dir[l]);
      fo_launch_batch_stencil(s, mg->g[l], mg->coef[l], mg->dir[l], mg->WK[l], mg->WM[l], nullptr, nullptr);
      WK = mg->WK[l];
      WM = mg->WM[l];
    }
    k_bmg_rows<<<fo_blocks_for(mg->g[l].num_nodes, FO_BLOCK, 65536), FO_BLOCK, 0, s>>>(mg->g[l].num_nodes, S, WK, WM,
                                                                                      mg->SK[l], mg->SM[l]);
    fo_note_launch(1);
  }
  // levels from Lg down run one instance per block in shared memory: small enough, and their
  // vectors (b, z0, z1, t of every such level) fit in the kernel's dynamic shared memory
  mg->Lg0 = mg->L;
  {
    const size_t cap = bmg_kernel(mg->g[0].dim, bt->nip / 32, false).smem;
    for (int l = 0; l < mg->L; ++l) {
      size_t need = 0;
      for (int m = l; m < mg->L; ++m) need += 16 * (size_t)mg->g[m].num_nodes;
      if (mg->g[l].num_nodes <= BMG_INST_NODES && need <= cap) {
        mg->Lg0 = l;
        break;
      }
    }
  }
  if (mg->nd > 0 && mg->Lg0 < mg->L) {   // the coarsest level runs in the per-instance cycle
    const int L1 = mg->L - 1;
    const double *WK = L1 == 0 ? bt->WK : mg->WK[L1], *WM = L1 == 0 ? bt->WM : mg->WM[L1];
    if (mg->g[0].dim == 2)
      k_bmg_coarse_inverse<2><<<bt->nip, 256, 0, s>>>(mg->g[L1], WK, WM, bt->kk, bt->w2, mg->nd, mg->ainv, mg->direct);
    else
      k_bmg_coarse_inverse<3><<<bt->nip, 256, 0, s>>>(mg->g[L1], WK, WM, bt->kk, bt->w2, mg->nd, mg->ainv, mg->direct);
    fo_note_launch(1);
  }
  mg->up_pi = -1;   // the level table is uploaded by the solve, for its precision
  mg->built_epoch = p->coef_epoch;
  return FO_OK;
}

fo_status fo_batch_state_mg(fo_problem *p, const double *B, double bscale, double *X, const fo_solve_opts *o, int warm,
                            fo_solve_stats *st) {
  fo_ctx *ctx = p->ctx;
  fo_batch *bt = p->batch;
  FO_TRY(bmg_prepare(p));
  fo_bmg *mg = bt->mg;
  const Grid &g = p->mesh->g;
  const int nip = bt->nip;
  const int pi = o->precision == FO_MIXED ? 1 : 0;
  if (mg->up_pi != pi) FO_TRY(bmg_upload(p, pi));
  long long grid = o->grid_blocks > 0 ? o->grid_blocks
                                      : (mg->tuned[pi] ? (long long)mg->t_bpsm[pi] * ctx->num_sms : mg->grid_cap);
  grid = std::min(grid, (long long)mg->grid_cap);
  grid = std::min(grid, (g.num_nodes + BMG_WARPS - 1) / BMG_WARPS);
  grid = std::max(grid, 1LL);
  BmgCg C{};
  C.WK = bt->WK;
  C.WM = bt->WM;
  C.kk = bt->kk;
  C.w2 = bt->w2;
  C.B = B;
  C.bscale = bscale;
  C.X = X;
  C.r = mg->r;
  C.p[0] = mg->p0;
  C.p[1] = mg->p1;
  C.s = mg->s;
  C.partials = mg->partials;
  C.totals = mg->partials + (size_t)2 * nip * grid;
  C.status = p->dev_status;
  C.bar = GridBar{p->bar, p->dev_status + DS_ERR, 2000000000ull};
  C.inst_iters = bt->inst_iters;
  C.inst_res = bt->inst_res;
  C.rtol2 = o->rtol * o->rtol;
  C.maxit = o->maxit;
  C.warm = warm;
  C.d64 = mg->d64;
  C.q32[0] = mg->q0;
  C.q32[1] = mg->q1;
  C.s32 = mg->s32;
  C.inner_rtol2 = o->inner_rtol * o->inner_rtol;
  C.inner_maxit = std::max(o->inner_maxit, 1);
  const BmgDev *dev = (const BmgDev *)mg->dev;
  FO_CU(ctx, cudaMemsetAsync(p->bar, 0, 64, ctx->stream));
  FO_CU(ctx, cudaMemsetAsync(p->dev_status, 0, sizeof(int) * DS_COUNT, ctx->stream));
  void *argv[] = {(void *)&dev, (void *)&C};
  const BmgKernel k = bmg_kernel(g.dim, nip / 32, o->precision == FO_MIXED);
  FO_CU(ctx, cudaFuncSetAttribute((const void *)k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem));
  FO_CU(ctx, cudaLaunchCooperativeKernel((const void *)k.fn, (int)grid, 32 * BMG_WARPS, argv, k.smem, ctx->stream));
  fo_note_launch(1);
  FO_CU(ctx, cudaGetLastError());
  fo_solve_stats s;
  memset(&s, 0, sizeof s);
  fo_status r = fo_batch_read(p, &s, o);
  if (st) *st = s;
  return r;
}

// FP32-pass tile of the batched multigrid kernels for a dimension and batch width.
template <int D, int NJ>
static void bmg_tile_of(int tile[3]) {
  using TL = typename BmgTiles<D, NJ>::T32;
  tile[0] = TL::TX;
  tile[1] = TL::TY;
  tile[2] = TL::TZ;
}

// Schedule autotuner of the batched multigrid: every candidate (blocks per SM from 1 to the
// kernel's co-residency limit, one or two smoothing sweeps on the finest level, per-instance
// levels from the size limit or one level later) solves the batch's current system from zero to
// rtol into a scratch solution, timed with CUDA events on the context stream; the fastest one
// that converges is kept (a schedule changes the iteration count, not the accuracy: every
// candidate stops on the same FP64 residual test).
extern "C" fo_status fo_batch_mg_autotune(fo_problem *p, int precision, double rtol, fo_mg_tune_result *out) {
  if (!p || (precision != FO_FP64 && precision != FO_MIXED) || !(rtol > 0)) return FO_EINVAL;
  if (!p->batch) return fo_fail(p->ctx, FO_EINVAL, "not a batch problem");
  fo_ctx *ctx = p->ctx;
  fo_batch *bt = p->batch;
  const Grid &g = p->mesh->g;
  if (!fo_mg_applicable(g, 1, false))
    return fo_fail(ctx, FO_EINVAL, "the batched multigrid needs a grid that halves");
  if (!p->coef_valid) FO_TRY(fo_coefficients(p));
  FO_TRY(bmg_prepare(p));
  fo_bmg *mg = bt->mg;
  const size_t nx = (size_t)g.num_nodes * bt->nip;
  double *X;
  FO_TRY(fo_alloc(ctx, (void **)&X, sizeof(double) * nx));
  fo_solve_opts o;
  fo_solve_opts_default(&o);
  o.precision = precision;
  o.precond = FO_PC_MG;
  o.rtol = rtol;
  o.maxit = 5000;
  o.inner_rtol = 1e-3;
  o.inner_maxit = 1000;
  cudaEvent_t e0, e1;
  FO_CU(ctx, cudaEventCreate(&e0));
  FO_CU(ctx, cudaEventCreate(&e1));
  const int shifts = (mg->Lg0 + 1 < mg->L) ? 2 : 1;
  int best_b = 0, best_nu = 1, best_sh = 0, best_it = 0, cand = 0;
  double best = INFINITY;
  fo_status st = FO_OK;
  for (int b = 1; b <= mg->per_sm && st == FO_OK; ++b)
    for (int nu = 1; nu <= 2 && st == FO_OK; ++nu)
      for (int sh = 0; sh < shifts && st == FO_OK; ++sh) {
        const int pi = precision == FO_MIXED ? 1 : 0;
        mg->tuned[pi] = 1;
        mg->t_bpsm[pi] = b;
        mg->t_nu0[pi] = nu;
        mg->t_lgshift[pi] = sh;
        mg->up_pi = -1;   // the solve uploads the candidate's table
        float ms = 0.f;
        fo_solve_stats s;
        bool conv = true;
        for (int rep = 0; rep < 2 && st == FO_OK && conv; ++rep) {   // the first run warms the caches
          FO_CU(ctx, cudaMemsetAsync(X, 0, sizeof(double) * nx, ctx->stream));
          FO_CU(ctx, cudaEventRecord(e0, ctx->stream));
          const fo_status r = fo_batch_state_mg(p, bt->B, 1.0, X, &o, 0, &s);
          FO_CU(ctx, cudaEventRecord(e1, ctx->stream));
          if (r == FO_ENOCONV) conv = false;               // this schedule does not converge
          else st = r;
        }
        if (st != FO_OK) break;
        if (!conv) continue;
        FO_CU(ctx, cudaEventSynchronize(e1));
        FO_CU(ctx, cudaEventElapsedTime(&ms, e0, e1));
        ++cand;
        if (ms < best) {
          best = ms;
          best_b = b;
          best_nu = nu;
          best_sh = sh;
          best_it = s.iterations;
        }
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  fo_free(ctx, X, sizeof(double) * nx);
  if (st == FO_OK && cand == 0) st = fo_fail(ctx, FO_ENOCONV, "no schedule of the batched multigrid converged");
  const int pi = precision == FO_MIXED ? 1 : 0;
  mg->up_pi = -1;
  if (st != FO_OK) {
    mg->tuned[pi] = 0;
    return st;
  }
  mg->tuned[pi] = 1;
  mg->t_bpsm[pi] = best_b;
  mg->t_nu0[pi] = best_nu;
  mg->t_lgshift[pi] = best_sh;
  if (out) {
    memset(out, 0, sizeof *out);
    out->blocks_per_sm = best_b;
    out->nu0 = best_nu;
    out->inst_levels = mg->L - std::min(mg->Lg0 + best_sh, mg->L);
    out->ms = best;
    out->iterations = best_it;
    out->candidates = cand;
    const int nj = bt->nip / 32;
    if (g.dim == 2) nj == 1 ? bmg_tile_of<2, 1>(out->tile) : (nj == 2 ? bmg_tile_of<2, 2>(out->tile) : bmg_tile_of<2, 4>(out->tile));
    else nj == 1 ? bmg_tile_of<3, 1>(out->tile) : (nj == 2 ? bmg_tile_of<3, 2>(out->tile) : bmg_tile_of<3, 4>(out->tile));
  }
  return FO_OK;
}
