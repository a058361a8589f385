// Geometric multigrid preconditioner for the state solve: an FP64 conjugate-gradient loop whose
// preconditioner is one FP32 V-cycle, all in one persistent cooperative launch.
//
// The Kuhn triangulation is nested under uniform refinement (each simplex of the grid with
// n/2 cells per axis is the union of 2^d simplices of the grid with n cells), so the P1 spaces
// are nested.  The coarse operators are rediscretisations: the P1 operator of the coarse grid
// with each coarse element's coefficient the mean of its 2^d fine children's.  That is the
// Galerkin product P^T A P of a piecewise-constant A (the coarse hat gradients are constant
// on a coarse simplex, whose children have equal measure) and of the mass and penalty terms,
// except next to Dirichlet nodes, where P skips the fine Dirichlet DOFs.  Coarse rows are
// built by the same stencil builder as the fine ones, from the restricted coefficients.  P is P1
// interpolation along the Kuhn edges: a fine node with index parities b in {0,1}^d takes the
// mean of the coarse nodes (i - b)/2 and (i + b)/2; the restriction is P^T.  Smoother: damped
// Jacobi, nu1 = nu2 sweeps; coarsest level: an exact solve with its precomputed inverse when
// it has at most MG_DIRECT_MAX unknowns, else nuc sweeps.  Levels of at most MG_BLOCK_DOFS
// unknowns are run by block 0 alone with block barriers only (a grid barrier per sweep would
// dominate their tiny work); the rest by the whole grid with grid barriers.
//
// The V-cycle is a fixed linear map (same sweeps and damping every call), symmetric up to
// FP32 rounding, so plain PCG applies; the CG residual, directions and dot products are FP64
// and the CG stops on ||b - A x||_2 (recurrence) <= rtol ||b||_2.
#pragma once
#include <cmath>
#include <cstring>
#include <algorithm>
#include <mutex>
#include <vector>

#include "fo_internal.cuh"
#include "fo_ops.cuh"

#define MG_BLOCK_DOFS 2048
#define MG_STAGE_MAX_BYTES (180 * 1024)   // shared memory block 0 may take for its levels
#define MG_DIRECT_MAX 64                  // coarsest levels of at most this many unknowns are
                                          // solved with a precomputed inverse (built by one block)
#define MG_DIRECT_GRID_MAX 400            // a coarsest level the hierarchy cannot coarsen below
                                          // MG_DIRECT_MAX gets one too up to this size (built by the
                                          // whole grid; its inverse stays in global memory)

struct MgLevelDev {
  Grid g;
  const float *W;       // difference-form stencil rows [S][BLK][N]
  const __nv_bfloat16 *Wh;   // non-null: the same rows rounded to BF16, which the sweeps and
                             // residuals of this (grid-run) level read instead of W
  const float *dinv;    // [N * NPN]
  const uint8_t *dir;   // [N * NPN]
  float *b, *z[2], *t;  // right-hand side, iterate (ping-pong), residual
};

struct MgDev {
  int L, Lg;            // levels; levels >= Lg run in block 0 alone
  float omega;          // damping of the coarsest level's sweeps
  float om[2];          // damping of the two smoothing sweeps: om[0] then om[1] before the coarse
                        // correction, om[1] then om[0] after it (the V-cycle stays symmetric)
  int nu, nuc;
  int nd;               // > 0: the coarsest level is solved with its inverse ainv [nd][nd]
  const float *ainv;
  MgLevelDev lv[MG_MAX_LEVELS];
};

// Arguments of the CG loop.  V is the type of its vectors and of the fine operator's rows:
// double for the FP64 CG, float for the inner CG of the mixed solve (FP64 refinement around an
// FP32 CG); its dot products and scalars are FP64 either way.
template <class V>
struct MgCgT {
  const V *W;           // fine stencil rows
  const V *b;           // right-hand side (zero on Dirichlet DOFs)
  V *x;                 // solution (start value when warm)
  V *r, *p[2], *s, *z;
  double *partials, *out;
  int *status;
  GridBar bar;
  double rtol2;
  int maxit, warm;
  int stage;            // block 0 keeps the levels it runs alone in shared memory
};
using MgCg = MgCgT<double>;

// ------------------------------------------------------------------ level operations
// Level pairs: a coarse grid either halves every axis of the fine one (nested: the existing
// Kuhn refinement relation) or, where an axis does not halve, has ceil(n/2) cells per axis over
// the same box (non-nested).  Then P is P1 interpolation of the coarse field at the fine nodes:
// a fine node at coarse coordinate s = i n_c / n_f per axis lies in coarse cell floor(s) with
// local coordinates t = frac(s) (exact in integers: the remainder of i n_c / n_f), in the Kuhn
// simplex whose axis order sorts t descending (ties by axis index), with barycentric weights
// 1 - t_(0), t_(0) - t_(1), ..., t_(d-1) on the path vertices; R = P^T.
__host__ __device__ __forceinline__ bool mg_nested(const Grid &F, const Grid &C) {
  for (int k = 0; k < F.dim; ++k)
    if (F.n[k] != 2 * C.n[k]) return false;
  return true;
}

template <int D>
__device__ __forceinline__ void mg_interp(const Grid &F, const Grid &C, const int ifn[3], long long vert[D + 1],
                                          float w[D + 1]) {
  // 32-bit integer arithmetic: node indices and cell counts per axis stay below 2^15 on any grid
  // that fits the device, so i n_c and the cross products below stay below 2^30 (64-bit
  // divisions are emulated and cost far more)
  int cc[3] = {0, 0, 0}, ax[3] = {0, 1, 2};
  int rem[3] = {0, 0, 0};
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const int num = ifn[k] * C.n[k];
    cc[k] = num / F.n[k];
    rem[k] = num - cc[k] * F.n[k];
  }
  // axes by t_k = rem_k / n_f,k descending (cross-multiplied: exact), ties by axis index
#pragma unroll
  for (int i = 1; i < D; ++i)
    for (int j = i; j > 0; --j) {
      const int a = ax[j], b = ax[j - 1];
      if (rem[a] * F.n[b] > rem[b] * F.n[a]) {
        ax[j] = b;
        ax[j - 1] = a;
      } else {
        break;
      }
    }
  double t[3];
#pragma unroll
  for (int m = 0; m < D; ++m) t[m] = (double)rem[ax[m]] / (double)F.n[ax[m]];
  long long v = cc[0] + C.stride[1] * cc[1] + (D == 3 ? C.stride[2] * cc[2] : 0);
  vert[0] = v;
  w[0] = (float)(1.0 - t[0]);
#pragma unroll
  for (int m = 0; m < D; ++m) {
    const double wm = (m + 1 < D) ? t[m] - t[m + 1] : t[m];
    v += C.stride[ax[m]];
    vert[m + 1] = wm > 0.0 ? v : -1;   // a zero weight may point past the grid
    w[m + 1] = (float)wm;
  }
}

template <int D, int NPN, bool FULL>
struct MgOps {
  using Op = StencilOp<D, NPN, FULL, float>;
  using OpH = StencilOp<D, NPN, FULL, float, __nv_bfloat16>;
  static __device__ __forceinline__ Op op(const MgLevelDev &L) {
    Op o;
    o.g = L.g;
    o.W = L.W;
    return o;
  }
  static __device__ __forceinline__ OpH oph(const MgLevelDev &L) {
    OpH o;
    o.g = L.g;
    o.W = L.Wh;
    return o;
  }
  // one damped Jacobi sweep z_out = z_in + omega D^{-1} (b - A z_in) over nodes [first, N) step
  template <class O>
  static __device__ __forceinline__ void sweep_with(const O &o, const MgLevelDev &L, const float *zin, float *zout,
                                                    float omega, long long first, long long step) {
    for (long long a = first; a < L.g.num_nodes; a += step) {
      int idx[3];
      node_ijk(L.g, a, idx);
      float az[NPN];
      o.row(a, idx, VecX<float>{zin}, az);
#pragma unroll
      for (int c = 0; c < NPN; ++c) {
        const long long k = a * NPN + c;
        zout[k] = zin[k] + omega * L.dinv[k] * (L.b[k] - az[c]);
      }
    }
  }
  static __device__ void sweep(const MgLevelDev &L, const float *zin, float *zout, float omega, long long first,
                               long long step) {
    if (L.Wh) sweep_with(oph(L), L, zin, zout, omega, first, step);
    else sweep_with(op(L), L, zin, zout, omega, first, step);
  }
  template <class O>
  static __device__ __forceinline__ void residual_with(const O &o, const MgLevelDev &L, const float *z,
                                                       long long first, long long step) {
    for (long long a = first; a < L.g.num_nodes; a += step) {
      int idx[3];
      node_ijk(L.g, a, idx);
      float az[NPN];
      o.row(a, idx, VecX<float>{z}, az);
#pragma unroll
      for (int c = 0; c < NPN; ++c) L.t[a * NPN + c] = L.b[a * NPN + c] - az[c];
    }
  }
  static __device__ void residual(const MgLevelDev &L, const float *z, long long first, long long step) {
    if (L.Wh) residual_with(oph(L), L, z, first, step);
    else residual_with(op(L), L, z, first, step);
  }
  // the gather of restrict_ between non-nested grids, out of line: the nested transfers are the
  // hot path, and the general ones (integer point location per fine node) would otherwise
  // be inlined into every caller of the persistent kernel
  static __device__ __noinline__ void restrict_general(const MgLevelDev &F, const MgLevelDev &C, float omega,
                                                       long long first, long long step) {
    for (long long c = first; c < C.g.num_nodes; c += step) {
      int ic[3];
      node_ijk(C.g, c, ic);
      int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const long long nf = F.g.n[k], ncs = C.g.n[k];
        // the coarse hat of c lives on coarse coordinates (c - 1, c + 1) along each axis
        lo[k] = ic[k] == 0 ? 0 : (int)(((long long)(ic[k] - 1) * nf + ncs - 1) / ncs);
        hi[k] = (int)std::min(nf, ((long long)(ic[k] + 1) * nf) / ncs);
      }
      float v[NPN];
#pragma unroll
      for (int j = 0; j < NPN; ++j) v[j] = 0.f;
      for (int i2 = lo[2]; i2 <= (D == 3 ? hi[2] : 0); ++i2)
        for (int i1 = lo[1]; i1 <= hi[1]; ++i1)
          for (int i0 = lo[0]; i0 <= hi[0]; ++i0) {
            const int ifn[3] = {i0, i1, i2};
            long long vert[D + 1];
            float w[D + 1];
            mg_interp<D>(F.g, C.g, ifn, vert, w);
            float wc = 0.f;
#pragma unroll
            for (int m = 0; m <= D; ++m)
              if (vert[m] == c) wc = w[m];
            if (wc == 0.f) continue;
            const long long f = i0 + F.g.stride[1] * i1 + (D == 3 ? F.g.stride[2] * i2 : 0);
#pragma unroll
            for (int j = 0; j < NPN; ++j) v[j] = fmaf(wc, F.t[f * NPN + j], v[j]);
          }
#pragma unroll
      for (int j = 0; j < NPN; ++j) {
        const long long k = c * NPN + j;
        const float bk = C.dir[k] ? 0.f : v[j];
        C.b[k] = bk;
        C.z[0][k] = omega * C.dinv[k] * bk;
      }
    }
  }
  // coarse b = P^T t (fine residual), and the coarse level's first sweep from zero
  static __device__ void restrict_(const MgLevelDev &F, const MgLevelDev &C, float omega, long long first,
                                   long long step) {
    if (!mg_nested(F.g, C.g)) {   // gather over the fine nodes whose interpolation uses c
      restrict_general(F, C, omega, first, step);
      return;
    }
    for (long long c = first; c < C.g.num_nodes; c += step) {
      int ic[3];
      node_ijk(C.g, c, ic);
      int ifn[3] = {2 * ic[0], D >= 2 ? 2 * ic[1] : 0, D == 3 ? 2 * ic[2] : 0};
      const long long f0 = ifn[0] + F.g.stride[1] * ifn[1] + (D == 3 ? F.g.stride[2] * ifn[2] : 0);
      float v[NPN];
#pragma unroll
      for (int j = 0; j < NPN; ++j) v[j] = F.t[f0 * NPN + j];
#pragma unroll
      for (int s = 1; s < ST<D>::S; ++s) {
        const long long nb = slot_node<D>(F.g, ifn, f0, s);
        if (nb < 0) continue;
#pragma unroll
        for (int j = 0; j < NPN; ++j) v[j] += 0.5f * F.t[nb * NPN + j];
      }
#pragma unroll
      for (int j = 0; j < NPN; ++j) {
        const long long k = c * NPN + j;
        const float bk = C.dir[k] ? 0.f : v[j];
        C.b[k] = bk;
        C.z[0][k] = omega * C.dinv[k] * bk;
      }
    }
  }
  // P between non-nested grids (P1 interpolation of the coarse field at each fine node), out of
  // line like restrict_general
  static __device__ __noinline__ void prolong_general(const MgLevelDev &F, float *zf, const MgLevelDev &C,
                                                      const float *zc, long long first, long long step) {
    for (long long a = first; a < F.g.num_nodes; a += step) {
      int idx[3];
      node_ijk(F.g, a, idx);
      long long vert[D + 1];
      float w[D + 1];
      mg_interp<D>(F.g, C.g, idx, vert, w);
#pragma unroll
      for (int j = 0; j < NPN; ++j) {
        const long long k = a * NPN + j;
        if (F.dir[k]) continue;
        float v = 0.f;
#pragma unroll
        for (int m = 0; m <= D; ++m)
          if (vert[m] >= 0) v = fmaf(w[m], zc[vert[m] * NPN + j], v);
        zf[k] += v;
      }
    }
  }
  // fine z += P (coarse z)
  static __device__ void prolong(const MgLevelDev &F, float *zf, const MgLevelDev &C, const float *zc,
                                 long long first, long long step) {
    if (!mg_nested(F.g, C.g)) {
      prolong_general(F, zf, C, zc, first, step);
      return;
    }
    for (long long a = first; a < F.g.num_nodes; a += step) {
      int idx[3];
      node_ijk(F.g, a, idx);
      long long c1 = 0, c2 = 0;
      bool mid = false;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const int bit = idx[k] & 1;
        mid |= bit != 0;
        c1 += (long long)((idx[k] - bit) / 2) * C.g.stride[k];
        c2 += (long long)((idx[k] + bit) / 2) * C.g.stride[k];
      }
#pragma unroll
      for (int j = 0; j < NPN; ++j) {
        const long long k = a * NPN + j;
        if (F.dir[k]) continue;
        const float v = mid ? 0.5f * (zc[c1 * NPN + j] + zc[c2 * NPN + j]) : zc[c1 * NPN + j];
        zf[k] += v;
      }
    }
  }
};

// The V-cycle on levels l >= from, in block 0 alone (block barriers), starting from b_from and
// z_from[0] (its first sweep from zero already taken).  zc[l]: buffer holding level l's iterate.
template <int D, int NPN, bool FULL>
__device__ void mg_block_cycle(const MgDev &mg, int from, int *zc) {
  using M = MgOps<D, NPN, FULL>;
  const long long t = threadIdx.x, st = blockDim.x;
  for (int l = from; l < mg.L; ++l) {
    const MgLevelDev &L = mg.lv[l];
    const int sweeps = (l == mg.L - 1) ? mg.nuc : mg.nu;
    int c = 0;
    if (l == mg.L - 1 && mg.nd > 0) {   // exact coarse solve, into the sweeps' final buffer
      c = (sweeps - 1) & 1;
      __syncthreads();
      for (long long i = t; i < mg.nd; i += st) {   // z_i = sum_k (A^-1)_ki b_k (A^-1 symmetric:
        float acc = 0.f;                               // a warp's loads of one k are contiguous)
        for (int k = 0; k < mg.nd; ++k) acc = fmaf(mg.ainv[(long long)k * mg.nd + i], L.b[k], acc);
        L.z[c][i] = acc;
      }
      zc[l] = c;
      break;
    }
    for (int j = 1; j < sweeps; ++j) {
      __syncthreads();
      M::sweep(L, L.z[c], L.z[c ^ 1], l == mg.L - 1 ? mg.omega : mg.om[j & 1], t, st);
      c ^= 1;
    }
    zc[l] = c;
    if (l == mg.L - 1) break;
    __syncthreads();
    M::residual(L, L.z[c], t, st);
    __syncthreads();
    M::restrict_(L, mg.lv[l + 1], l + 1 == mg.L - 1 ? mg.omega : mg.om[0], t, st);
  }
  for (int l = mg.L - 2; l >= from; --l) {
    const MgLevelDev &L = mg.lv[l];
    __syncthreads();
    M::prolong(L, L.z[zc[l]], mg.lv[l + 1], mg.lv[l + 1].z[zc[l + 1]], t, st);
    int c = zc[l];
    for (int j = 0; j < mg.nu; ++j) {
      __syncthreads();
      M::sweep(L, L.z[c], L.z[c ^ 1], mg.om[1 - (j & 1)], t, st);
      c ^= 1;
    }
    zc[l] = c;
  }
  __syncthreads();
}

// Shared-memory copy of the levels >= Lg that block 0 runs alone: their FP32 rows, inverse
// diagonals and Dirichlet masks (constant during a solve: copied once per launch) and their
// vectors b, z[2], t.  Bytes needed (each array 16-byte aligned): see mg_stage_bytes.
template <int D, int NPN, bool FULL>
__host__ __device__ inline size_t mg_stage_layout(const MgDev &mg, MgDev *out, unsigned char *base) {
  constexpr int S = ST<D>::SH, BLK = FULL ? NPN * NPN : NPN;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    unsigned char *p = base ? base + off : nullptr;
    off += (bytes + 15) / 16 * 16;
    return p;
  };
  if (mg.nd > 0 && mg.nd <= MG_DIRECT_MAX) {   // a larger inverse stays in global memory (L2)
    float *a = (float *)take(sizeof(float) * (size_t)mg.nd * mg.nd);
    if (out) out->ainv = a;
  }
  for (int l = mg.Lg; l < mg.L; ++l) {
    const size_t n = (size_t)mg.lv[l].g.num_nodes;
    float *W = (float *)take(sizeof(float) * S * BLK * n);
    float *dinv = (float *)take(sizeof(float) * NPN * n);
    float *b = (float *)take(sizeof(float) * NPN * n);
    float *z0 = (float *)take(sizeof(float) * NPN * n);
    float *z1 = (float *)take(sizeof(float) * NPN * n);
    float *t = (float *)take(sizeof(float) * NPN * n);
    uint8_t *dir = (uint8_t *)take(NPN * n);
    if (out) {
      MgLevelDev &d = out->lv[l];
      d.W = W;
      d.dinv = dinv;
      d.dir = dir;
      d.b = b;
      d.z[0] = z0;
      d.z[1] = z1;
      d.t = t;
    }
  }
  return off;
}

// Block 0: the staged view mgs of mg (levels >= Lg in shared memory, constants copied).
template <int D, int NPN, bool FULL>
__device__ void mg_stage(const MgDev &mg, MgDev &mgs, unsigned char *smem) {
  constexpr int S = ST<D>::SH, BLK = FULL ? NPN * NPN : NPN;
  {
    const int *src = reinterpret_cast<const int *>(&mg);
    int *dst = reinterpret_cast<int *>(&mgs);
    for (int i = threadIdx.x; i < (int)(sizeof(MgDev) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) mg_stage_layout<D, NPN, FULL>(mg, &mgs, smem);
  __syncthreads();
  if (mg.nd > 0 && mg.nd <= MG_DIRECT_MAX)
    for (int k = threadIdx.x; k < mg.nd * mg.nd; k += blockDim.x) const_cast<float *>(mgs.ainv)[k] = mg.ainv[k];
  for (int l = mg.Lg; l < mg.L; ++l) {
    const long long n = mg.lv[l].g.num_nodes;
    const MgLevelDev &G = mg.lv[l];
    MgLevelDev &Sm = mgs.lv[l];
    float *W = const_cast<float *>(Sm.W), *dinv = const_cast<float *>(Sm.dinv);
    uint8_t *dir = const_cast<uint8_t *>(Sm.dir);
    for (long long k = threadIdx.x; k < (long long)S * BLK * n; k += blockDim.x) W[k] = G.W[k];
    for (long long k = threadIdx.x; k < NPN * n; k += blockDim.x) {
      dinv[k] = G.dinv[k];
      dir[k] = G.dir[k];
    }
  }
  __syncthreads();
}

// The block cycle on the staged view: level `from`'s b and first sweep come from (and its
// final iterate goes back to) global memory, where the grid passes read and write them.
template <int D, int NPN, bool FULL>
__device__ void mg_block_cycle_staged(const MgDev &mg, const MgDev &mgs, int from, int *zc) {
  const MgLevelDev &G = mg.lv[from], &Sm = mgs.lv[from];
  const long long n = G.g.num_nodes * NPN;
  for (long long k = threadIdx.x; k < n; k += blockDim.x) {
    Sm.b[k] = G.b[k];
    Sm.z[0][k] = G.z[0][k];
  }
  __syncthreads();
  mg_block_cycle<D, NPN, FULL>(mgs, from, zc);
  const float *zs = Sm.z[zc[from]];
  float *zg = G.z[zc[from]];
  for (long long k = threadIdx.x; k < n; k += blockDim.x) zg[k] = zs[k];
}

// The V-cycle from level 0, whose b and first sweep were written by the caller before a grid
// barrier.  Returns false if a grid barrier failed; level 0's result is in z[zc[0]].
template <int D, int NPN, bool FULL>
__device__ bool mg_vcycle(const MgDev &mg, const MgDev &mgs, bool staged, int *zc, const GridBar &bar) {
  using M = MgOps<D, NPN, FULL>;
  const long long first = blockIdx.x * (long long)blockDim.x + threadIdx.x, step = (long long)gridDim.x * blockDim.x;
  const int Lg = mg.Lg;
  if (Lg == 0) {   // everything is small: block 0 runs the whole cycle
    if (blockIdx.x == 0) {
      if (staged) mg_block_cycle_staged<D, NPN, FULL>(mg, mgs, 0, zc);
      else mg_block_cycle<D, NPN, FULL>(mg, 0, zc);
    }
    return grid_sync(bar);
  }
  for (int l = 0; l < Lg; ++l) {
    const MgLevelDev &L = mg.lv[l];
    const bool coarsest = l == mg.L - 1;
    const int sweeps = coarsest ? mg.nuc : mg.nu;
    int c = 0;
    for (int j = 1; j < sweeps; ++j) {
      M::sweep(L, L.z[c], L.z[c ^ 1], coarsest ? mg.omega : mg.om[j & 1], first, step);
      c ^= 1;
      if (!grid_sync(bar)) return false;
    }
    zc[l] = c;
    if (coarsest) break;
    M::residual(L, L.z[c], first, step);
    if (!grid_sync(bar)) return false;
    M::restrict_(L, mg.lv[l + 1], l + 1 == mg.L - 1 ? mg.omega : mg.om[0], first, step);
    if (!grid_sync(bar)) return false;
  }
  if (Lg < mg.L) {   // the other blocks know the block-run levels' final buffers (fixed)
    if (blockIdx.x == 0) {
      if (staged) mg_block_cycle_staged<D, NPN, FULL>(mg, mgs, Lg, zc);
      else mg_block_cycle<D, NPN, FULL>(mg, Lg, zc);
    }
    if (!grid_sync(bar)) return false;
  }
  for (int l = std::min(Lg, mg.L - 1) - 1; l >= 0; --l) {
    const MgLevelDev &L = mg.lv[l];
    M::prolong(L, L.z[zc[l]], mg.lv[l + 1], mg.lv[l + 1].z[zc[l + 1]], first, step);
    if (!grid_sync(bar)) return false;
    int c = zc[l];
    for (int j = 0; j < mg.nu; ++j) {
      M::sweep(L, L.z[c], L.z[c ^ 1], mg.om[1 - (j & 1)], first, step);
      c ^= 1;
      if (l > 0 || j + 1 < mg.nu)
        if (!grid_sync(bar)) return false;
    }
    zc[l] = c;
  }
  return true;
}

// Buffer index of each level's final iterate after a V-cycle: fixed by the sweep counts, so
// every block knows it without communication.
__host__ __device__ inline void mg_final_buffers(int L, int Lg, int nu, int nuc, int *zc) {
  for (int l = 0; l < L; ++l) {
    const int sweeps = (l == L - 1) ? nuc : nu;
    int c = (sweeps - 1) & 1;                      // after the down sweeps
    if (l < L - 1) c = (c + nu) & 1;               // after the post sweeps
    zc[l] = c;
  }
  (void)Lg;
}

// NC independent systems share the loop: NC = 1 for a coupled system (scalar, or elastic
// blocks), NC = NPN for the component-decoupled velocity form (one CG recurrence per
// component, DOF k belonging to system k % NC); the loop stops when the summed residual meets
// rtol.  Ends with the dot product b . x (for B(theta, theta) of the velocity solve).
template <int D, int NPN, bool FULL, int NC, class V = double>
__global__ void __launch_bounds__(FO_BLOCK, D == 2 ? 1 : 2) k_pcg_mg(const MgDev *mgp, MgCgT<V> C) {
  extern __shared__ __align__(16) unsigned char mg_dsmem[];
  __shared__ MgDev mg;
  __shared__ MgDev mgs;   // block 0's view with the block-run levels in shared memory
  __shared__ double sred[32 * 3 * NC];
  __shared__ double stot[3 * NC];
  __shared__ double scal[NC];   // a step's quotients, formed once per block by thread 0
  {
    const int *src = reinterpret_cast<const int *>(mgp);
    int *dst = reinterpret_cast<int *>(&mg);
    for (int i = threadIdx.x; i < (int)(sizeof(MgDev) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  const bool staged = C.stage != 0 && mg.Lg < mg.L;
  if (staged && blockIdx.x == 0) mg_stage<D, NPN, FULL>(mg, mgs, mg_dsmem);
  const MgLevelDev &L0 = mg.lv[0];
  const Grid &g = L0.g;
  const long long N = g.num_nodes;
  const long long first = blockIdx.x * (long long)blockDim.x + threadIdx.x, step = (long long)gridDim.x * blockDim.x;
  StencilOp<D, NPN, FULL, V> A;
  A.g = g;
  A.W = C.W;
  int rk = 0, zc[MG_MAX_LEVELS];
  mg_final_buffers(mg.L, mg.Lg, mg.nu, mg.nuc, zc);
  const int zfin = zc[0];
  auto sys = [](int c) { return NC == 1 ? 0 : c; };
  double gam[NC], bb[NC], rho[NC], beta[NC];
  int it = 0, cur = 0;
  double rr = 0.0, bbt = 0.0;

  // r = b - A x;  level-0 right-hand side and first sweep;  ||b||^2
  {
    double v[3 * NC];
#pragma unroll
    for (int j = 0; j < 3 * NC; ++j) v[j] = 0.0;
    for (long long a = first; a < N; a += step) {
      int idx[3];
      node_ijk(g, a, idx);
      V ax[NPN];
      if (C.warm) A.row(a, idx, VecX<V>{C.x}, ax);
#pragma unroll
      for (int c = 0; c < NPN; ++c) {
        const long long k = a * NPN + c;
        if (!C.warm) {
          C.x[k] = V(0);
          ax[c] = V(0);
        }
        const V rk0 = C.b[k] - ax[c];
        C.r[k] = rk0;
        C.p[0][k] = V(0);
        const float bf = (float)rk0;
        L0.b[k] = bf;
        L0.z[0][k] = (mg.L == 1 ? mg.omega : mg.om[0]) * L0.dinv[k] * bf;
        v[NC + sys(c)] += (double)C.b[k] * (double)C.b[k];
      }
    }
    if (!grid_sync(C.bar)) return;
    if (!mg_vcycle<D, NPN, FULL>(mg, mgs, staged, zc, C.bar)) return;
    // z = M r; gamma_c = (r, z)_c; rho_c = (r, r)_c
    for (long long a = first; a < N; a += step)
#pragma unroll
      for (int c = 0; c < NPN; ++c) {
        const long long k = a * NPN + c;
        const V zk = (V)L0.z[zfin][k];
        C.z[k] = zk;
        v[sys(c)] += (double)C.r[k] * (double)zk;
        v[2 * NC + sys(c)] += (double)C.r[k] * (double)C.r[k];
      }
    if (!reduce_grid<3 * NC>(v, sred, stot, C.partials, rk, C.bar)) return;
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      gam[q] = stot[q];
      bb[q] = stot[NC + q];
      rho[q] = stot[2 * NC + q];
      beta[q] = 0.0;
      rr += rho[q];
      bbt += bb[q];
    }
  }
  for (;;) {
    bool live = false;
#pragma unroll
    for (int q = 0; q < NC; ++q) live = live || gam[q] > 0.0;
    if (!(rr > C.rtol2 * bbt) || it >= C.maxit || !live) break;
    // p = z + beta p_old (formed at neighbours on the fly); s = A p; (p, s)_c
    double ps[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) ps[q] = 0.0;
    const V *po = C.p[cur];
    V *pn = C.p[cur ^ 1];
    CombX<V, NC> pv{C.z, po, {}};
#pragma unroll
    for (int q = 0; q < NC; ++q) pv.beta[q] = (V)beta[q];
    for (long long a = first; a < N; a += step) {
      int idx[3];
      node_ijk(g, a, idx);
      V ap[NPN];
      A.row(a, idx, pv, ap);
#pragma unroll
      for (int c = 0; c < NPN; ++c) {
        const long long k = a * NPN + c;
        const V pk = C.z[k] + pv.beta[sys(c)] * po[k];
        pn[k] = pk;
        C.s[k] = ap[c];
        ps[sys(c)] += (double)pk * (double)ap[c];
      }
    }
    if (!reduce_grid<NC>(ps, sred, stot, C.partials, rk, C.bar)) return;
    if (threadIdx.x == 0)
#pragma unroll
      for (int q = 0; q < NC; ++q) scal[q] = gam[q] > 0.0 ? gam[q] / stot[q] : 0.0;
    __syncthreads();
    double alpha[NC];
    bool ok = true;
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      alpha[q] = scal[q];
      ok = ok && (gam[q] <= 0.0 || stot[q] > 0.0);
    }
    if (!ok) break;   // lost positive definiteness in rounding: stop with x as is
    cur ^= 1;
    // x += alpha p; r -= alpha s; level-0 right-hand side and first sweep
    for (long long a = first; a < N; a += step)
#pragma unroll
      for (int c = 0; c < NPN; ++c) {
        const long long k = a * NPN + c;
        C.x[k] += (V)alpha[sys(c)] * pn[k];
        const V rk1 = C.r[k] - (V)alpha[sys(c)] * C.s[k];
        C.r[k] = rk1;
        const float bf = (float)rk1;
        L0.b[k] = bf;
        L0.z[0][k] = (mg.L == 1 ? mg.omega : mg.om[0]) * L0.dinv[k] * bf;
      }
    if (!grid_sync(C.bar)) return;
    if (!mg_vcycle<D, NPN, FULL>(mg, mgs, staged, zc, C.bar)) return;
    double w[2 * NC];
#pragma unroll
    for (int j = 0; j < 2 * NC; ++j) w[j] = 0.0;
    for (long long a = first; a < N; a += step)
#pragma unroll
      for (int c = 0; c < NPN; ++c) {
        const long long k = a * NPN + c;
        const V zk = (V)L0.z[zfin][k];
        C.z[k] = zk;
        w[sys(c)] += (double)C.r[k] * (double)zk;
        w[NC + sys(c)] += (double)C.r[k] * (double)C.r[k];
      }
    if (!reduce_grid<2 * NC>(w, sred, stot, C.partials, rk, C.bar)) return;
    if (threadIdx.x == 0)
#pragma unroll
      for (int q = 0; q < NC; ++q) scal[q] = gam[q] > 0.0 ? stot[q] / gam[q] : 0.0;
    __syncthreads();
    rr = 0.0;
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      beta[q] = scal[q];
      gam[q] = stot[q];
      rho[q] = stot[NC + q];
      rr += rho[q];
    }
    ++it;
  }
  // b . x
  double bx[1] = {0.0};
  for (long long a = first; a < N; a += step)
#pragma unroll
    for (int c = 0; c < NPN; ++c) bx[0] += (double)C.b[a * NPN + c] * (double)C.x[a * NPN + c];
  if (!reduce_grid<1>(bx, sred, stot, C.partials, rk, C.bar)) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    C.out[0] = rr;
    C.out[1] = bbt;
    C.out[2] = stot[0];
    C.status[DS_ITERS] = it;
    if (rr > C.rtol2 * bbt && it >= C.maxit) atomicCAS(C.status + DS_ERR, DEV_OK, DEV_NOCONV);
  }
}

// ------------------------------------------------------------------------------ launch
// One persistent launch of the CG loop with the arguments C (vectors bound by the caller).
template <int D, int NPN, bool FULL, int NC, class V>
fo_status mg_launch(fo_problem *p, fo_mg *mg, MgCgT<V> C, const fo_solve_opts *o, double rtol, int maxit,
                           int warm, fo_solve_stats *st, double *bx) {
  fo_ctx *ctx = p->ctx;
  C.partials = p->red;
  C.out = p->red + (FO_RED_DOUBLES - 64);
  C.status = p->dev_status;
  C.bar = GridBar{p->bar, p->dev_status + DS_ERR, 2000000000ull};
  C.rtol2 = rtol * rtol;
  C.maxit = maxit;
  C.warm = warm;
  auto kern = k_pcg_mg<D, NPN, FULL, NC, V>;
  int grid;
  std::unique_lock<std::mutex> lk(fo_launch_mutex());
  FO_TRY(fo_cooperative_grid(p, (const void *)kern, FO_BLOCK, 0, p->mesh->g.num_nodes, o->grid_blocks, &grid));
  // Block 0 keeps the levels it runs alone in shared memory when they fit and the launch
  // keeps its grid (the extra shared memory per block may lower the co-resident count).
  size_t smem = 0;
  {
    const MgDev *h = reinterpret_cast<const MgDev *>(mg->host.data());
    const size_t bytes = h->Lg < h->L ? mg_stage_layout<D, NPN, FULL>(*h, nullptr, nullptr) : 0;
    if (bytes > 0 && bytes <= MG_STAGE_MAX_BYTES) {
      FO_TRY(fo_smem_limit(ctx, (const void *)kern, bytes));
      int g1 = 0;
      FO_TRY(fo_cooperative_grid(p, (const void *)kern, FO_BLOCK, bytes, p->mesh->g.num_nodes, o->grid_blocks, &g1));
      if (g1 == grid) smem = bytes;
    }
  }
  C.stage = smem > 0;
  const MgDev *mgp = (const MgDev *)mg->dev;
  void *argv[] = {(void *)&mgp, (void *)&C};
  FO_CU(ctx, cudaMemsetAsync(p->bar, 0, 64, ctx->stream));
  FO_CU(ctx, cudaMemsetAsync(p->dev_status, 0, sizeof(int) * DS_COUNT, ctx->stream));
  const bool tm = ctx->timing != 0 && ctx->ev_solve[0] != nullptr;
  if (tm) FO_CU(ctx, cudaEventRecord(ctx->ev_solve[0], ctx->stream));
  FO_CU(ctx, cudaLaunchCooperativeKernel((const void *)kern, grid, FO_BLOCK, argv, smem, ctx->stream));
  fo_note_launch(1);
  FO_CU(ctx, cudaGetLastError());
  lk.unlock();
  if (tm) FO_CU(ctx, cudaEventRecord(ctx->ev_solve[1], ctx->stream));
  FO_CU(ctx, cudaMemcpyAsync(ctx->h_scalars, C.out, 3 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  FO_CU(ctx, cudaMemcpyAsync(ctx->h_scalars + 32, p->dev_status, sizeof(int) * DS_COUNT, cudaMemcpyDeviceToHost,
                             ctx->stream));
  FO_CU(ctx, cudaStreamSynchronize(ctx->stream));
  if (tm) {
    float ms = 0.f;
    FO_CU(ctx, cudaEventElapsedTime(&ms, ctx->ev_solve[0], ctx->ev_solve[1]));
    ctx->last_solve_ms += ms;
  }
  const int *hs = (const int *)(ctx->h_scalars + 32);
  if (st) {
    memset(st, 0, sizeof *st);
    st->iterations = hs[DS_ITERS];
    st->operator_applies = hs[DS_ITERS] + 1 + (warm ? 1 : 0);
    st->outer_iterations = 1;
    st->rel_residual = ctx->h_scalars[1] > 0 ? std::sqrt(ctx->h_scalars[0] / ctx->h_scalars[1]) : 0.0;
  }
  if (bx) *bx = ctx->h_scalars[2];
  if (hs[DS_ERR] == DEV_TIMEOUT) return fo_fail(ctx, FO_ETIMEOUT, "grid barrier timed out in the multigrid PCG");
  if (!std::isfinite(ctx->h_scalars[0])) return fo_fail(ctx, FO_ENAN, "NaN in the multigrid PCG");
  if (hs[DS_ERR] == DEV_NOCONV) return fo_fail(ctx, FO_ENOCONV, "multigrid PCG reached maxit=%d", maxit);
  return FO_OK;
}

// The launch is instantiated in one translation unit per dimension and vector type
// (fo_mg_k2d.cu, fo_mg_k2f.cu, fo_mg_k3d.cu, fo_mg_k3v.cu, fo_mg_k3f.cu), so that they compile in
// parallel.
#define FO_MG_INSTANCES(X)                                                                     \
  X(2, 1, true, 1, double) X(2, 2, true, 1, double) X(2, 2, false, 2, double)                  \
  X(2, 1, true, 1, float) X(2, 2, true, 1, float)                                              \
  X(3, 1, true, 1, double) X(3, 3, true, 1, double) X(3, 3, false, 3, double)                  \
  X(3, 1, true, 1, float) X(3, 3, true, 1, float)
#define FO_MG_LAUNCH_SIG(D, NPN, FULL, NC, V)                                                    \
  fo_status mg_launch<D, NPN, FULL, NC, V>(fo_problem *, fo_mg *, MgCgT<V>, const fo_solve_opts *, double, int, \
                                           int, fo_solve_stats *, double *)
#define FO_MG_EXTERN(D, NPN, FULL, NC, V) extern template FO_MG_LAUNCH_SIG(D, NPN, FULL, NC, V);
#define FO_MG_DEFINE(D, NPN, FULL, NC, V) template FO_MG_LAUNCH_SIG(D, NPN, FULL, NC, V);
