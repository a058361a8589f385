// Geometric multigrid preconditioner for the state solve: an FP64 conjugate-gradient loop whose
// preconditioner is one FP32 V-cycle, all in one persistent cooperative launch.
//
// The Kuhn triangulation is nested under uniform refinement (each simplex of the grid with
// n/2 cells per axis is the union of 2^d simplices of the grid with n cells), so the P1 spaces
// are nested and the Galerkin coarse operator P^T A P is exactly the P1 operator of the coarse
// grid with each coarse element's coefficient the mean of its 2^d fine children's (A is
// piecewise constant; the mass terms have constant coefficients).  Coarse rows are therefore
// built by the same stencil builder as the fine ones, from restricted coefficients.  P is P1
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
#include <cmath>
#include <cstring>
#include <algorithm>
#include <vector>

#include "fo_internal.cuh"
#include "fo_ops.cuh"

#define MG_BLOCK_DOFS 2048
#define MG_STAGE_MAX_BYTES (180 * 1024)   // shared memory block 0 may take for its levels
#define MG_DIRECT_MAX 64                  // coarsest levels of at most this many unknowns are
                                          // solved with a precomputed inverse

struct MgLevelDev {
  Grid g;
  const float *W;       // difference-form stencil rows [S][BLK][N]
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
  int cc[3] = {0, 0, 0}, ax[3] = {0, 1, 2};
  long long rem[3] = {0, 0, 0};
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const long long num = (long long)ifn[k] * C.n[k];
    cc[k] = (int)(num / F.n[k]);
    rem[k] = num % F.n[k];
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
  static __device__ __forceinline__ Op op(const MgLevelDev &L) {
    Op o;
    o.g = L.g;
    o.W = L.W;
    return o;
  }
  // one damped Jacobi sweep z_out = z_in + omega D^{-1} (b - A z_in) over nodes [first, N) step
  static __device__ void sweep(const MgLevelDev &L, const float *zin, float *zout, float omega, long long first,
                               long long step) {
    const Op o = op(L);
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
  static __device__ void residual(const MgLevelDev &L, const float *z, long long first, long long step) {
    const Op o = op(L);
    for (long long a = first; a < L.g.num_nodes; a += step) {
      int idx[3];
      node_ijk(L.g, a, idx);
      float az[NPN];
      o.row(a, idx, VecX<float>{z}, az);
#pragma unroll
      for (int c = 0; c < NPN; ++c) L.t[a * NPN + c] = L.b[a * NPN + c] - az[c];
    }
  }
  // coarse b = P^T t (fine residual), and the coarse level's first sweep from zero
  static __device__ void restrict_(const MgLevelDev &F, const MgLevelDev &C, float omega, long long first,
                                   long long step) {
    if (!mg_nested(F.g, C.g)) {   // gather over the fine nodes whose interpolation uses c
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
  // fine z += P (coarse z)
  static __device__ void prolong(const MgLevelDev &F, float *zf, const MgLevelDev &C, const float *zc,
                                 long long first, long long step) {
    if (!mg_nested(F.g, C.g)) {
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
      for (long long i = t; i < mg.nd; i += st) {
        const float *row = mg.ainv + i * mg.nd;
        float acc = 0.f;
        for (int k = 0; k < mg.nd; ++k) acc = fmaf(row[k], L.b[k], acc);
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
  constexpr int S = ST<D>::S, BLK = FULL ? NPN * NPN : NPN;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    unsigned char *p = base ? base + off : nullptr;
    off += (bytes + 15) / 16 * 16;
    return p;
  };
  if (mg.nd > 0) {
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
  constexpr int S = ST<D>::S, BLK = FULL ? NPN * NPN : NPN;
  {
    const int *src = reinterpret_cast<const int *>(&mg);
    int *dst = reinterpret_cast<int *>(&mgs);
    for (int i = threadIdx.x; i < (int)(sizeof(MgDev) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) mg_stage_layout<D, NPN, FULL>(mg, &mgs, smem);
  __syncthreads();
  if (mg.nd > 0)
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

// ===================================================================================== host
template <int D>
__global__ void k_mg_restrict_coef(Grid gc, Grid gf, const double *coef_f, double *coef_c) {
  constexpr int P = KP<D>::P;
  for (long long ec = blockIdx.x * (long long)blockDim.x + threadIdx.x; ec < gc.num_elems;
       ec += (long long)gridDim.x * blockDim.x) {
    const long long cell = ec / P;
    const int pc = (int)(ec % P);
    int ci[3];
    ci[0] = (int)(cell % gc.n[0]);
    const long long t = cell / gc.n[0];
    ci[1] = (int)(t % gc.n[1]);
    ci[2] = (int)(t / gc.n[1]);
    double sum = 0.0;
    for (int o = 0; o < (1 << D); ++o) {
      int fi[3] = {2 * ci[0] + (o & 1), 2 * ci[1] + ((o >> 1) & 1), D == 3 ? 2 * ci[2] + ((o >> 2) & 1) : 0};
      const long long fcell = fi[0] + gf.cstride[1] * fi[1] + (D == 3 ? gf.cstride[2] * fi[2] : 0);
      for (int pf = 0; pf < P; ++pf) {
        // the coarse simplex holding fine simplex pf of the fine cell at offset o: axes sorted
        // by offset (descending), ties in the fine simplex's own axis order
        int order[3], n = 0;
        for (int ob = 1; ob >= 0; --ob)
          for (int l = 0; l < D; ++l) {
            const int ax = kperm<D>(pf, l);
            if (((o >> ax) & 1) == ob) order[n++] = ax;
          }
        int q = -1;
        for (int cand = 0; cand < P && q < 0; ++cand) {
          bool same = true;
          for (int l = 0; l < D; ++l) same = same && kperm<D>(cand, l) == order[l];
          if (same) q = cand;
        }
        if (q == pc) sum += coef_f[(long long)P * fcell + pf];
      }
    }
    coef_c[ec] = sum / (double)(1 << D);
  }
}

// Non-nested pair: the coarse element's coefficient is the mean over the fine elements whose
// centroid lies in it (in integer coordinates: exact), or, should none, the coefficient of the
// fine element holding the coarse element's centroid.  A Kuhn simplex's centroid has local
// coordinate (D - j) / (D + 1) along axis pi_j.
template <int D>
__device__ __forceinline__ int mg_simplex_of(const long long rem[3], const long long den[3]) {
  int ax[3] = {0, 1, 2};
  for (int i = 1; i < D; ++i)
    for (int j = i; j > 0; --j) {
      const int a = ax[j], b = ax[j - 1];
      if (rem[a] * den[b] > rem[b] * den[a]) {
        ax[j] = b;
        ax[j - 1] = a;
      } else {
        break;
      }
    }
  for (int cand = 0; cand < KP<D>::P; ++cand) {
    bool same = true;
    for (int l = 0; l < D; ++l) same = same && kperm<D>(cand, l) == ax[l];
    if (same) return cand;
  }
  return 0;
}

template <int D>
__global__ void k_mg_restrict_coef_general(Grid gc, Grid gf, const double *coef_f, double *coef_c) {
  constexpr int P = KP<D>::P;
  for (long long ec = blockIdx.x * (long long)blockDim.x + threadIdx.x; ec < gc.num_elems;
       ec += (long long)gridDim.x * blockDim.x) {
    const long long cellc = ec / P;
    const int pc = (int)(ec % P);
    int ci[3];
    ci[0] = (int)(cellc % gc.n[0]);
    long long tt = cellc / gc.n[0];
    ci[1] = (int)(tt % gc.n[1]);
    ci[2] = (int)(tt / gc.n[1]);
    int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int k = 0; k < D; ++k) {
      lo[k] = (int)(((long long)ci[k] * gf.n[k]) / gc.n[k]);
      hi[k] = (int)std::min<long long>(gf.n[k] - 1, ((long long)(ci[k] + 1) * gf.n[k] + gc.n[k] - 1) / gc.n[k] - 1);
    }
    double sum = 0.0;
    int cnt = 0;
    for (int i2 = lo[2]; i2 <= (D == 3 ? hi[2] : 0); ++i2)
      for (int i1 = lo[1]; i1 <= hi[1]; ++i1)
        for (int i0 = lo[0]; i0 <= hi[0]; ++i0) {
          const int fi[3] = {i0, i1, i2};
          const long long fcell = i0 + gf.cstride[1] * i1 + (D == 3 ? gf.cstride[2] * i2 : 0);
          for (int pf = 0; pf < P; ++pf) {
            long long rem[3] = {0, 0, 0}, den[3] = {1, 1, 1};
            bool in = true;
            for (int j = 0; j < D; ++j) {
              const int k = kperm<D>(pf, j);
              const long long num = ((long long)fi[k] * (D + 1) + (D - j)) * gc.n[k];
              den[k] = (long long)gf.n[k] * (D + 1);
              in = in && num / den[k] == ci[k];
              rem[k] = num % den[k];
            }
            if (in && mg_simplex_of<D>(rem, den) == pc) {
              sum += coef_f[(long long)P * fcell + pf];
              ++cnt;
            }
          }
        }
    if (cnt == 0) {   // the fine element holding the coarse centroid
      int fi[3] = {0, 0, 0};
      long long rem[3] = {0, 0, 0}, den[3] = {1, 1, 1};
      for (int j = 0; j < D; ++j) {
        const int k = kperm<D>(pc, j);
        const long long num = ((long long)ci[k] * (D + 1) + (D - j)) * gf.n[k];
        den[k] = (long long)gc.n[k] * (D + 1);
        fi[k] = (int)std::min<long long>(gf.n[k] - 1, num / den[k]);
        rem[k] = num % den[k];
      }
      const long long fcell = fi[0] + gf.cstride[1] * fi[1] + (D == 3 ? gf.cstride[2] * fi[2] : 0);
      sum = coef_f[(long long)P * fcell + mg_simplex_of<D>(rem, den)];
      cnt = 1;
    }
    coef_c[ec] = sum / (double)cnt;
  }
}

// Non-nested pair: a coarse node takes the Dirichlet flags of the fine node nearest to it
// (boundary nodes map to boundary nodes of the same faces).
__global__ void k_mg_coarse_dir_general(Grid gc, Grid gf, int npn, const uint8_t *dir_f, uint8_t *dir_c) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < gc.num_nodes;
       c += (long long)gridDim.x * blockDim.x) {
    int ic[3];
    node_ijk(gc, c, ic);
    long long f = 0;
    for (int k = 0; k < gc.dim; ++k) {
      const long long i = (2LL * ic[k] * gf.n[k] + gc.n[k]) / (2LL * gc.n[k]);   // round(ic n_f / n_c)
      f += i * gf.stride[k];
    }
    for (int j = 0; j < npn; ++j) dir_c[c * npn + j] = dir_f[f * npn + j];
  }
}

__global__ void k_mg_coarse_dir(Grid gc, Grid gf, int npn, const uint8_t *dir_f, uint8_t *dir_c) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < gc.num_nodes;
       c += (long long)gridDim.x * blockDim.x) {
    int ic[3];
    node_ijk(gc, c, ic);
    const long long f = 2LL * ic[0] + gf.stride[1] * 2LL * ic[1] + (gc.dim == 3 ? gf.stride[2] * 2LL * ic[2] : 0);
    for (int j = 0; j < npn; ++j) dir_c[c * npn + j] = dir_f[f * npn + j];
  }
}

// Inverse of the coarsest level's operator, for the exact coarse solve.  One block: the dense
// n x n matrix (n = nodes x components <= MG_DIRECT_MAX) is assembled in shared memory from
// the level's FP64 difference-form rows -- A[(a,c),(a,k)] = R_ck - sum_s W_s,ck and
// A[(a,c),(nb_s,k)] = W_s,ck, a thread per node -- and inverted in place by Gauss-Jordan
// elimination without pivoting (the matrix is symmetric positive definite: Dirichlet rows are
// identity rows and their columns eliminated), in FP64; the inverse is stored in FP32.
template <int D, int NPN, bool FULL>
__global__ void k_mg_coarse_inverse(Grid g, const double *W, int n, float *ainv) {
  constexpr int S = ST<D>::S, BLK = FULL ? NPN * NPN : NPN;
  extern __shared__ __align__(16) double A[];   // [n][n]
  __shared__ double piv;
  const long long N = g.num_nodes;
  for (int k = threadIdx.x; k < n * n; k += blockDim.x) A[k] = 0.0;
  __syncthreads();
  for (long long a = threadIdx.x; a < N; a += blockDim.x) {   // rows of node a only
    int idx[3];
    node_ijk(g, a, idx);
    for (int c = 0; c < NPN; ++c)
      for (int k = 0; k < NPN; ++k) {
        if (!FULL && k != c) continue;
        const int e = FULL ? c * NPN + k : c;
        const long long r = a * NPN + c;
        double diag = W[(long long)e * N + a];
        for (int s = 1; s < S; ++s) {
          const long long nb = slot_node<D>(g, idx, a, s);
          if (nb < 0) continue;
          const double w = W[((long long)s * BLK + e) * N + a];
          diag -= w;
          A[r * n + nb * NPN + k] += w;
        }
        A[r * n + a * NPN + k] += diag;
      }
  }
  for (int p = 0; p < n; ++p) {
    __syncthreads();
    if (threadIdx.x == 0) piv = 1.0 / A[p * n + p];
    __syncthreads();
    const double q = piv;
    for (int k = threadIdx.x; k < n * n; k += blockDim.x) {   // outside row and column p
      const int i = k / n, j = k - i * n;
      if (i != p && j != p) A[k] -= A[i * n + p] * A[p * n + j] * q;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < n; k += blockDim.x)
      if (k != p) {
        A[p * n + k] *= q;
        A[k * n + p] *= -q;
      }
    if (threadIdx.x == 0) A[p * n + p] = q;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < n * n; k += blockDim.x) ainv[k] = (float)A[k];
}

static fo_status mg_build_inverse(fo_ctx *ctx, fo_mg *mg) {
  if (mg->nd == 0) return FO_OK;
  const Grid &gc = mg->g[mg->L - 1];
  const double *W = mg->W64[mg->L - 1];
  cudaStream_t s = ctx->stream;
  const size_t smem = sizeof(double) * mg->nd * mg->nd;
  auto run = [&](auto kern) -> fo_status {
    std::lock_guard<std::mutex> lk(fo_launch_mutex());
    FO_TRY(fo_smem_limit(ctx, (const void *)kern, smem));
    kern<<<1, 256, smem, s>>>(gc, W, mg->nd, mg->ainv);
    fo_note_launch(1);
    FO_CU(ctx, cudaGetLastError());
    return FO_OK;
  };
  if (gc.dim == 2) {
    if (mg->npn == 1) return run(k_mg_coarse_inverse<2, 1, true>);
    if (mg->blk == 4) return run(k_mg_coarse_inverse<2, 2, true>);
    return run(k_mg_coarse_inverse<2, 2, false>);
  }
  if (mg->npn == 1) return run(k_mg_coarse_inverse<3, 1, true>);
  if (mg->blk == 9) return run(k_mg_coarse_inverse<3, 3, true>);
  return run(k_mg_coarse_inverse<3, 3, false>);
}

// The single-problem hierarchy ends at the first level small enough to be solved directly.
static int mg_plan_single(const Grid &g0, Grid *g, int npn) {
  return fo_mg_plan(g0, g, MG_MAX_LEVELS, MG_DIRECT_MAX, npn, true);
}

static int mg_direct_unknowns(const Grid *g, int L, int npn) {
  if (L < 2) return 0;
  const long long n = g[L - 1].num_nodes * npn;
  return n <= MG_DIRECT_MAX ? (int)n : 0;
}


// ------------------------------------------------------------------------- hierarchies
// Levels: halve every axis while all are even and the coarse grid keeps >= 2 cells per axis;
// with stop_unknowns > 0, also stop at the first level of at most that many unknowns (npn per
// node).
int fo_mg_plan(const Grid &g0, Grid *g, int max_levels, long long stop_unknowns, int npn, bool general) {
  g[0] = g0;
  int L = 1;
  while (L < max_levels) {
    const Grid &f = g[L - 1];
    if (stop_unknowns > 0 && f.num_nodes * npn <= stop_unknowns) break;
    int n[3] = {1, 1, 1};
    bool ok = true, even = true;
    for (int a = 0; a < f.dim; ++a) even = even && f.n[a] % 2 == 0 && f.n[a] / 2 >= 2;
    for (int a = 0; a < f.dim; ++a) {
      // halve while every axis halves; otherwise (general) ceil(n/2) cells per axis
      n[a] = even ? f.n[a] / 2 : (f.n[a] + 1) / 2;
      if (!even && (!general || f.n[a] < 3)) ok = false;
    }
    if (!ok) break;
    if (!fo_grid_make(f.dim, n, f.lo, f.hi, g[L])) break;
    ++L;
  }
  return L;
}

// Byte sizes of level l's arrays, in the order b, z0, z1, t, coef, W64, W32, dinv64, dinv32, dir
// (coarse levels own all; level 0 owns coef, W32, dinv32 and dir only when own0).
static void mg_sizes(const Grid &g, int npn, int blk, bool coarse, bool own0, size_t sz[10]) {
  const size_t N = (size_t)g.num_nodes, S = g.dim == 2 ? 7 : 15;
  for (int i = 0; i < 4; ++i) sz[i] = sizeof(float) * N * npn;
  sz[4] = (coarse || own0) ? sizeof(double) * g.num_elems : 0;
  sz[5] = coarse ? sizeof(double) * S * blk * N : 0;
  sz[6] = (coarse || own0) ? sizeof(float) * S * blk * N : 0;
  sz[7] = coarse ? sizeof(double) * N * npn : 0;
  sz[8] = (coarse || own0) ? sizeof(float) * N * npn : 0;
  sz[9] = (coarse || own0) ? N * npn : 0;
}

static void **mg_slot(fo_mg *mg, int l, int i) {
  switch (i) {
    case 0: return (void **)&mg->b[l];
    case 1: return (void **)&mg->z0[l];
    case 2: return (void **)&mg->z1[l];
    case 3: return (void **)&mg->t[l];
    case 4: return (void **)&mg->coef[l];
    case 5: return (void **)&mg->W64[l];
    case 6: return (void **)&mg->W32[l];
    case 7: return (void **)&mg->dinv64[l];
    case 8: return (void **)&mg->dinv32[l];
    default: return (void **)&mg->dir[l];
  }
}

static void mg_release(fo_ctx *ctx, fo_mg *&mg) {
  if (!mg) return;
  for (int l = 0; l < mg->L; ++l) {
    size_t sz[10];
    mg_sizes(mg->g[l], mg->npn, mg->blk, l > 0, mg->own0, sz);
    for (int i = 0; i < 10; ++i)
      if (sz[i]) fo_free(ctx, *mg_slot(mg, l, i), sz[i]);
  }
  if (mg->nd > 0) {
    fo_free(ctx, mg->ainv, sizeof(float) * mg->nd * mg->nd);
  }
  fo_free(ctx, mg->dev, sizeof(MgDev));
  delete mg;
  mg = nullptr;
}

void fo_mg_destroy(fo_problem *p) {
  mg_release(p->ctx, p->mg);
  mg_release(p->ctx, p->mgv);
}

// Multigrid pays when the hierarchy reaches a small coarsest level.  Single problems coarsen
// any grid (non-nested levels where an axis does not halve); the batched multigrid needs nested
// levels (general = false), so grids not divisible by enough powers of two keep its Jacobi
// solver.
#define MG_COARSEST_MAX_DOFS 8192
bool fo_mg_applicable(const Grid &g0, int npn, bool general) {
  Grid g[MG_MAX_LEVELS];
  const int L = fo_mg_plan(g0, g, MG_MAX_LEVELS, MG_DIRECT_MAX, npn, general);
  return L >= 2 && g[L - 1].num_nodes * npn <= MG_COARSEST_MAX_DOFS;
}

size_t fo_mg_bytes(int dim, const int n[3], int npn, int blk, bool own0) {
  Grid g0;
  const double lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1};
  if (!fo_grid_make(dim, n, lo, hi, g0)) return 0;
  Grid g[MG_MAX_LEVELS];
  const int L = mg_plan_single(g0, g, npn);
  size_t b = sizeof(MgDev);
  for (int l = 0; l < L; ++l) {
    size_t sz[10];
    mg_sizes(g[l], npn, blk, l > 0, own0, sz);
    for (int i = 0; i < 10; ++i) b += sz[i];
  }
  const size_t nd = (size_t)mg_direct_unknowns(g, L, npn);
  return b + nd * nd * sizeof(float);
}

static fo_status mg_alloc(fo_ctx *ctx, fo_mg *&out, const Grid &g0, int npn, int blk, bool own0) {
  fo_mg *mg = new fo_mg();
  out = mg;
  mg->npn = npn;
  mg->blk = blk;
  mg->own0 = own0;
  mg->L = mg_plan_single(g0, mg->g, npn);
  for (int l = 0; l < mg->L; ++l) {
    size_t sz[10];
    mg_sizes(mg->g[l], npn, blk, l > 0, own0, sz);
    for (int i = 0; i < 10; ++i)
      if (sz[i]) FO_TRY(fo_alloc(ctx, mg_slot(mg, l, i), sz[i]));
  }
  mg->nd = mg_direct_unknowns(mg->g, mg->L, npn);
  if (mg->nd > 0) {
    FO_TRY(fo_alloc(ctx, (void **)&mg->ainv, sizeof(float) * mg->nd * mg->nd));
  }
  FO_TRY(fo_alloc(ctx, (void **)&mg->dev, sizeof(MgDev)));
  return FO_OK;
}

// Level table to the device; level 0's FP32 rows, FP32 inverse diagonal and Dirichlet mask.
static fo_status mg_upload(fo_ctx *ctx, fo_mg *mg, const float *W0, const float *dinv0, const uint8_t *dir0,
                           float omega) {
  MgDev h;
  memset(&h, 0, sizeof h);
  h.L = mg->L;
  h.Lg = mg->L;
  for (int l = 0; l < mg->L; ++l)
    if ((long long)mg->g[l].num_nodes * mg->npn <= MG_BLOCK_DOFS) {
      h.Lg = l;
      break;
    }
  h.omega = omega;
  h.om[0] = omega;
  h.om[1] = omega;
  h.nu = 2;
  h.nuc = 16;
  h.nd = mg->nd;
  h.ainv = mg->ainv;
  for (int l = 0; l < mg->L; ++l) {
    MgLevelDev &d = h.lv[l];
    d.g = mg->g[l];
    d.W = l == 0 ? W0 : mg->W32[l];
    d.dinv = l == 0 ? dinv0 : mg->dinv32[l];
    d.dir = l == 0 ? dir0 : mg->dir[l];
    d.b = mg->b[l];
    d.z[0] = mg->z0[l];
    d.z[1] = mg->z1[l];
    d.t = mg->t[l];
  }
  mg->host.resize(sizeof(MgDev));
  memcpy(mg->host.data(), &h, sizeof(MgDev));
  FO_CU(ctx, cudaMemcpyAsync(mg->dev, mg->host.data(), sizeof(MgDev), cudaMemcpyHostToDevice, ctx->stream));
  FO_CU(ctx, cudaGetLastError());
  return FO_OK;
}

// Coarse per-element coefficient (children means) and per-DOF Dirichlet mask of grid gc from
// those of the grid gf it halves.
void fo_mg_restrict(fo_ctx *ctx, const Grid &gc, const Grid &gf, int npn, const double *coef_f, const uint8_t *dir_f,
                    double *coef_c, uint8_t *dir_c) {
  cudaStream_t s = ctx->stream;
  const int blocks = fo_blocks_for(gc.num_elems, FO_BLOCK, 65536);
  if (!mg_nested(gf, gc)) {
    if (gc.dim == 2) k_mg_restrict_coef_general<2><<<blocks, FO_BLOCK, 0, s>>>(gc, gf, coef_f, coef_c);
    else k_mg_restrict_coef_general<3><<<blocks, FO_BLOCK, 0, s>>>(gc, gf, coef_f, coef_c);
    k_mg_coarse_dir_general<<<fo_blocks_for(gc.num_nodes, FO_BLOCK, 65536), FO_BLOCK, 0, s>>>(gc, gf, npn, dir_f,
                                                                                              dir_c);
    fo_note_launch(2);
    return;
  }
  if (gc.dim == 2) k_mg_restrict_coef<2><<<blocks, FO_BLOCK, 0, s>>>(gc, gf, coef_f, coef_c);
  else k_mg_restrict_coef<3><<<blocks, FO_BLOCK, 0, s>>>(gc, gf, coef_f, coef_c);
  k_mg_coarse_dir<<<fo_blocks_for(gc.num_nodes, FO_BLOCK, 65536), FO_BLOCK, 0, s>>>(gc, gf, npn, dir_f, dir_c);
  fo_note_launch(2);
}

// restrict a per-element coefficient and the per-DOF Dirichlet mask from level l-1 to level l
static void mg_restrict_level(fo_ctx *ctx, fo_mg *mg, int l, const double *coef_f, const uint8_t *dir_f) {
  fo_mg_restrict(ctx, mg->g[l], mg->g[l - 1], mg->npn, coef_f, dir_f, mg->coef[l], mg->dir[l]);
}

// State hierarchy: rebuilt after every coefficient update (coarse coefficients are the
// children means of the current A_e).
static fo_status mg_prepare_state(fo_problem *p) {
  fo_ctx *ctx = p->ctx;
  if (!p->mg) {
    FO_TRY(mg_alloc(ctx, p->mg, p->mesh->g, p->ncomp, p->ncomp * p->ncomp, false));
    p->mg->built_epoch = -1;
  }
  fo_mg *mg = p->mg;
  if (mg->built_epoch == p->coef_epoch) return FO_OK;
  for (int l = 1; l < mg->L; ++l) {
    mg_restrict_level(ctx, mg, l, l == 1 ? p->coef : mg->coef[l - 1], l == 1 ? p->dir : mg->dir[l - 1]);
    FO_TRY(fo_launch_stencil_on(p, mg->g[l], mg->coef[l], mg->dir[l], mg->W64[l], mg->W32[l], mg->dinv64[l],
                                mg->dinv32[l]));
  }
  FO_TRY(mg_build_inverse(ctx, mg));
  FO_TRY(mg_upload(ctx, mg, p->Wst32, p->dinv_state32, p->dir, p->ncomp == 1 ? 0.8f : 0.6f));
  mg->built_epoch = p->coef_epoch;
  return FO_OK;
}

__global__ void k_vel_mass_coef(long long ne, const uint8_t *omega0, double alpha, double gamma0, double *mc) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ne; e += (long long)gridDim.x * blockDim.x)
    mc[e] = alpha + (omega0[e] ? gamma0 : 0.0);
}
__global__ void k_vel_dof_mask(long long nn, int d, const uint8_t *vdir, int on, uint8_t *mask) {
  for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < nn; a += (long long)gridDim.x * blockDim.x)
    for (int c = 0; c < d; ++c) mask[a * d + c] = on && vdir[a];
}
// -b on the velocity DOFs, zero on H^1_0 rows
__global__ void k_vel_rhs(long long nn, int d, const double *b, const uint8_t *mask, double *out) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nn * d; k += (long long)gridDim.x * blockDim.x)
    out[k] = mask[k] ? 0.0 : -b[k];
}

// Velocity hierarchy: the form does not depend on phi, so it is built once.  Level 0's rows
// are the problem's velocity rows; coarse levels carry the children mean of the mass-type
// coefficient alpha + gamma_0 chi_Omega0 and the same normal penalty on their faces.
static fo_status mg_prepare_velocity(fo_problem *p) {
  if (p->mgv) return FO_OK;
  fo_ctx *ctx = p->ctx;
  const Grid &g0 = p->mesh->g;
  const int d = g0.dim;
  FO_TRY(mg_alloc(ctx, p->mgv, g0, d, d, true));
  fo_mg *mg = p->mgv;
  cudaStream_t s = ctx->stream;
  const double al = p->desc.alpha_mass, ga0 = p->desc.omega0_weight;
  k_vel_mass_coef<<<fo_blocks_for(g0.num_elems, FO_BLOCK, 65536), FO_BLOCK, 0, s>>>(g0.num_elems, p->omega0, al, ga0,
                                                                                   mg->coef[0]);
  k_vel_dof_mask<<<fo_blocks_for(g0.num_nodes, FO_BLOCK, 65536), FO_BLOCK, 0, s>>>(
      g0.num_nodes, d, p->vdir, p->desc.velocity_dirichlet ? 1 : 0, mg->dir[0]);
  fo_note_launch(2);
  // level 0 again with FP32 copies (same rows as the problem's FP64 ones)
  FO_TRY(fo_launch_velocity_stencil_on(p, g0, mg->coef[0], mg->dir[0], p->Wvel, mg->W32[0], p->dinv_vel,
                                       mg->dinv32[0]));
  for (int l = 1; l < mg->L; ++l) {
    mg_restrict_level(ctx, mg, l, mg->coef[l - 1], mg->dir[l - 1]);
    FO_TRY(fo_launch_velocity_stencil_on(p, mg->g[l], mg->coef[l], mg->dir[l], mg->W64[l], mg->W32[l], mg->dinv64[l],
                                         mg->dinv32[l]));
  }
  FO_TRY(mg_build_inverse(ctx, mg));
  FO_TRY(mg_upload(ctx, mg, mg->W32[0], mg->dinv32[0], mg->dir[0], 0.8f));
  return FO_OK;
}

// ------------------------------------------------------------------------------ solves
// One persistent launch of the CG loop with the arguments C (vectors bound by the caller).
template <int D, int NPN, bool FULL, int NC, class V>
static fo_status mg_launch(fo_problem *p, fo_mg *mg, MgCgT<V> C, const fo_solve_opts *o, double rtol, int maxit,
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

template <int D, int NPN, bool FULL, int NC>
static fo_status mg_run(fo_problem *p, fo_mg *mg, const double *W64, const double *b, double *x, long long n,
                        const fo_solve_opts *o, fo_solve_stats *st, double *bx) {
  double *buf;
  FO_TRY(fo_scratch(p, sizeof(double) * 6 * n, (void **)&buf));
  MgCg C{};
  C.W = W64;
  C.b = b;
  C.x = x;
  C.r = buf;
  C.p[0] = buf + n;
  C.p[1] = buf + 2 * n;
  C.s = buf + 3 * n;
  C.z = buf + 4 * n;
  return mg_launch<D, NPN, FULL, NC, double>(p, mg, C, o, o->rtol, o->maxit, o->warm_start, st, bx);
}

// ---- mixed: FP64 iterative refinement around the FP32 multigrid CG
// r = b - A x with the FP64 rows; ||r||^2 and ||b||^2 as per-block partials
__global__ void k_mg_ir_residual(const double *b, const double *ax, double *r, long long n, double *partials) {
  __shared__ double sm[64];
  double v[2] = {0, 0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double ri = b[i] - ax[i];
    r[i] = ri;
    v[0] += ri * ri;
    v[1] += b[i] * b[i];
  }
  block_sum<2>(v, sm);
  if (threadIdx.x == 0) {
    partials[blockIdx.x * 2] = v[0];
    partials[blockIdx.x * 2 + 1] = v[1];
  }
}
// the two sums in a fixed order (deterministic)
__global__ void k_mg_ir_total(const double *partials, int nblocks, double *out) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (w >= 2) return;
  double t = 0;
  for (int b = lane; b < nblocks; b += 32) t += partials[(size_t)b * 2 + w];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  if (lane == 0) out[w] = t;
}
// the inner right-hand side: the residual scaled to unit norm, in FP32
__global__ void k_mg_ir_scale(const double *r, double inv, float *b32, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b32[i] = (float)(r[i] * inv);
}
// x += scale * d (the correction accumulated in FP64)
__global__ void k_mg_ir_update(double *x, const float *d, double scale, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] = fma(scale, (double)d[i], x[i]);
}

// Each refinement step forms the true residual r = b - A x in FP64, solves A d = r / ||r|| with
// the FP32 CG (FP32 rows and vectors, FP64 dot products) preconditioned by the same FP32
// V-cycle to the relative reduction inner_rtol, and adds ||r|| d to x in FP64.  It stops when
// ||r|| <= rtol ||b||, or when two consecutive steps fail to halve ||r|| (the FP64 residual's
// own rounding floor is reached).
template <int D, int NPN>
static fo_status mg_state_mixed(fo_problem *p, const double *b, double *x, const fo_solve_opts *o, fo_solve_stats *st) {
  fo_ctx *ctx = p->ctx;
  const long long n = p->ndof;
  double *buf;
  FO_TRY(fo_scratch(p, sizeof(double) * 2 * n + sizeof(float) * 7 * n + 256, (void **)&buf));
  double *r64 = buf, *ax64 = buf + n;
  float *f = reinterpret_cast<float *>(buf + 2 * n);
  MgCgT<float> C{};
  C.W = p->Wst32;
  C.b = f;
  C.x = f + n;
  C.r = f + 2 * n;
  C.p[0] = f + 3 * n;
  C.p[1] = f + 4 * n;
  C.s = f + 5 * n;
  C.z = f + 6 * n;
  const int blocks = fo_blocks_for(n, FO_BLOCK, 1024);
  double *sums = p->red + (FO_RED_DOUBLES - 128);
  if (!o->warm_start) FO_CU(ctx, cudaMemsetAsync(x, 0, sizeof(double) * n, ctx->stream));
  fo_solve_stats s;
  memset(&s, 0, sizeof s);
  double bnorm2 = -1, prev_rn2 = INFINITY, prev2_rn2 = INFINITY;
  const int max_outer = 60;
  for (int outer = 0;; ++outer) {
    FO_TRY(fo_launch_state_apply(p, x, ax64, true));
    k_mg_ir_residual<<<blocks, FO_BLOCK, 0, ctx->stream>>>(b, ax64, r64, n, p->red);
    k_mg_ir_total<<<1, 64, 0, ctx->stream>>>(p->red, blocks, sums);
    fo_note_launch(2);
    FO_CU(ctx, cudaGetLastError());
    FO_CU(ctx, cudaMemcpyAsync(ctx->h_scalars, sums, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    FO_CU(ctx, cudaStreamSynchronize(ctx->stream));
    const double rn2 = ctx->h_scalars[0];
    if (bnorm2 < 0) bnorm2 = ctx->h_scalars[1];
    s.operator_applies += 1;
    s.rel_residual = bnorm2 > 0 ? std::sqrt(rn2 / bnorm2) : 0.0;
    if (!std::isfinite(rn2)) return fo_fail(ctx, FO_ENAN, "NaN in the refinement residual");
    if (rn2 <= o->rtol * o->rtol * bnorm2 || bnorm2 == 0 || rn2 == 0) break;
    if (outer >= 2 && rn2 > 0.25 * prev_rn2 && prev_rn2 > 0.25 * prev2_rn2) break;
    prev2_rn2 = prev_rn2;
    prev_rn2 = rn2;
    if (outer >= max_outer || s.iterations >= o->maxit) {
      if (st) *st = s;
      return fo_fail(ctx, FO_ENOCONV, "iterative refinement stalled at %.3e", s.rel_residual);
    }
    const double rn = std::sqrt(rn2);
    k_mg_ir_scale<<<blocks, FO_BLOCK, 0, ctx->stream>>>(r64, 1.0 / rn, f, n);
    fo_note_launch(1);
    fo_solve_stats in;
    const fo_status r = mg_launch<D, NPN, true, 1, float>(p, p->mg, C, o, o->inner_rtol, o->inner_maxit, 0, &in,
                                                          nullptr);
    if (r != FO_OK && r != FO_ENOCONV) return r;   // an inner cap only ends that step
    s.iterations += in.iterations;
    s.operator_applies += in.operator_applies;
    s.outer_iterations = outer + 1;
    k_mg_ir_update<<<blocks, FO_BLOCK, 0, ctx->stream>>>(x, C.x, rn, n);
    fo_note_launch(1);
    FO_CU(ctx, cudaGetLastError());
  }
  if (st) *st = s;
  return FO_OK;
}

fo_status fo_state_pcg_mg(fo_problem *p, const double *b, double *x, const fo_solve_opts *o, fo_solve_stats *st) {
  FO_TRY(mg_prepare_state(p));
  const int d = p->mesh->g.dim;
  const long long n = p->ndof;
  if (o->precision == FO_MIXED) {
    if (p->desc.kind == FO_ELASTIC) return d == 2 ? mg_state_mixed<2, 2>(p, b, x, o, st) : mg_state_mixed<3, 3>(p, b, x, o, st);
    return d == 2 ? mg_state_mixed<2, 1>(p, b, x, o, st) : mg_state_mixed<3, 1>(p, b, x, o, st);
  }
  if (p->desc.kind == FO_ELASTIC)
    return d == 2 ? mg_run<2, 2, true, 1>(p, p->mg, p->Wst, b, x, n, o, st, nullptr)
                  : mg_run<3, 3, true, 1>(p, p->mg, p->Wst, b, x, n, o, st, nullptr);
  return d == 2 ? mg_run<2, 1, true, 1>(p, p->mg, p->Wst, b, x, n, o, st, nullptr)
                : mg_run<3, 1, true, 1>(p, p->mg, p->Wst, b, x, n, o, st, nullptr);
}

// Velocity solve B theta = -b with multigrid: the d component systems share one launch.
fo_status fo_velocity_pcg_mg(fo_problem *p, const fo_solve_opts *o, double *Btt, fo_solve_stats *st) {
  FO_TRY(mg_prepare_velocity(p));
  const Grid &g = p->mesh->g;
  const int d = g.dim;
  const long long n = (long long)d * g.num_nodes;
  double *rhs;
  FO_TRY(fo_scratch(p, sizeof(double) * 7 * n, (void **)&rhs));
  rhs += 6 * n;   // after the solver's six vectors
  k_vel_rhs<<<fo_blocks_for(n, FO_BLOCK, 65536), FO_BLOCK, 0, p->ctx->stream>>>(g.num_nodes, d, p->rhs, p->mgv->dir[0],
                                                                               rhs);
  fo_note_launch(1);
  double bx = 0.0;
  fo_status r = d == 2 ? mg_run<2, 2, false, 2>(p, p->mgv, p->Wvel, rhs, p->theta, n, o, st, &bx)
                       : mg_run<3, 3, false, 3>(p, p->mgv, p->Wvel, rhs, p->theta, n, o, st, &bx);
  if (Btt) *Btt = bx;   // B(theta, theta) = -b . theta
  return r;
}
