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
// R = P^T, damped Jacobi with nu sweeps before and after, nuc on the coarsest level.  Fields
// are instance-minor [N_l][nip]: a warp owns a node and lane l holds instances l, l + 32, ...,
// so a neighbour row is one coalesced 128-byte load per 32 instances and the stencil rows are
// read once for all of them.  Levels of at most BMG_BLOCK_NODES nodes run in block 0 alone.
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
#define BMG_BLOCK_NODES 96       // levels of at most this many nodes run in block 0 alone

struct BmgLevel {
  Grid g;
  const float *SK, *SM;   // [S + 1][N] rows in difference form (slot 0 row sum, slot S diagonal)
  const uint8_t *dir;     // [N] Dirichlet mask
  float *b, *z[2], *t;    // [N][nip] right-hand side, iterate (ping-pong), residual
};

struct BmgDev {
  int L, Lg;              // levels; levels >= Lg run in block 0 alone
  int nu, nuc;
  float omega;
  BmgLevel lv[MG_MAX_LEVELS];
};

struct BmgCg {
  const double *WK, *WM;     // fine FP64 rows, node-major [N][S] (slot 0 = the node itself)
  const double *kk, *w2;     // [nip] k_i, omega_i^2
  const double *B;           // loads [N][nip]; the right-hand side is bscale * B
  double bscale;
  double *X, *r, *p, *s;     // [N][nip]
  double *partials;          // [2 nip][G]
  double *totals;            // [2 nip]
  int *status;
  GridBar bar;
  int *inst_iters;
  double *inst_res;
  double rtol2;
  int maxit, warm;
};

// ------------------------------------------------------------------ level operations
template <int D, int NJ>
struct BmgOps {
  static constexpr int S = ST<D>::S, NIP = 32 * NJ;
  struct Coef {
    float k[NJ], w[NJ];
  };
  // (A_i z)(a), D_i(a) and z(a) for the lane's instances
  static __device__ __forceinline__ void row(const BmgLevel &L, long long a, const int *idx, const float *z,
                                             const Coef &c, int lane, float (&za)[NJ], float (&az)[NJ],
                                             float (&dg)[NJ]) {
    const long long N = L.g.num_nodes;
    const float rk = L.SK[a], rm = L.SM[a], dk = L.SK[S * N + a], dm = L.SM[S * N + a];
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      za[j] = z[a * NIP + lane + 32 * j];
      az[j] = __fmul_rn(fmaf(c.k[j], rk, __fmul_rn(c.w[j], rm)), za[j]);
      dg[j] = fmaf(c.k[j], dk, __fmul_rn(c.w[j], dm));
    }
#pragma unroll
    for (int s = 1; s < S; ++s) {
      const long long nb = slot_node<D>(L.g, idx, a, s);
      if (nb < 0) continue;
      const float wk = L.SK[s * N + a], wm = L.SM[s * N + a];
      if (wk == 0.f && wm == 0.f) continue;   // eliminated Dirichlet column (warp-uniform)
#pragma unroll
      for (int j = 0; j < NJ; ++j)
        az[j] = fmaf(fmaf(c.k[j], wk, __fmul_rn(c.w[j], wm)), __fsub_rn(z[nb * NIP + lane + 32 * j], za[j]), az[j]);
    }
  }
  // z_out = z_in + omega D^{-1} (b - A z_in) on nodes first, first + step, ...
  static __device__ void sweep(const BmgLevel &L, const float *zin, float *zout, float omega, const Coef &c,
                               long long first, long long step, int lane) {
    for (long long a = first; a < L.g.num_nodes; a += step) {
      int idx[3];
      node_ijk(L.g, a, idx);
      float za[NJ], az[NJ], dg[NJ];
      row(L, a, idx, zin, c, lane, za, az, dg);
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const long long q = a * NIP + lane + 32 * j;
        zout[q] = __fadd_rn(za[j], __fdiv_rn(__fmul_rn(omega, __fsub_rn(L.b[q], az[j])), dg[j]));
      }
    }
  }
  static __device__ void residual(const BmgLevel &L, const float *z, const Coef &c, long long first, long long step,
                                  int lane) {
    for (long long a = first; a < L.g.num_nodes; a += step) {
      int idx[3];
      node_ijk(L.g, a, idx);
      float za[NJ], az[NJ], dg[NJ];
      row(L, a, idx, z, c, lane, za, az, dg);
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const long long q = a * NIP + lane + 32 * j;
        L.t[q] = L.b[q] - az[j];
      }
    }
  }
  // coarse b = P^T t (fine residual; zero on coarse Dirichlet nodes) and the coarse level's
  // first sweep from zero
  static __device__ void restrict_(const BmgLevel &F, const BmgLevel &C, float omega, const Coef &c, long long first,
                                   long long step, int lane) {
    const long long Nc = C.g.num_nodes;
    for (long long cn = first; cn < Nc; cn += step) {
      int ic[3];
      node_ijk(C.g, cn, ic);
      int ifn[3] = {2 * ic[0], D >= 2 ? 2 * ic[1] : 0, D == 3 ? 2 * ic[2] : 0};
      const long long f0 = ifn[0] + F.g.stride[1] * ifn[1] + (D == 3 ? F.g.stride[2] * ifn[2] : 0);
      float v[NJ];
#pragma unroll
      for (int j = 0; j < NJ; ++j) v[j] = F.t[f0 * NIP + lane + 32 * j];
#pragma unroll
      for (int s = 1; s < S; ++s) {
        const long long nb = slot_node<D>(F.g, ifn, f0, s);
        if (nb < 0) continue;
#pragma unroll
        for (int j = 0; j < NJ; ++j) v[j] = fmaf(0.5f, F.t[nb * NIP + lane + 32 * j], v[j]);
      }
      const bool dirc = C.dir[cn] != 0;
      const float dk = C.SK[S * Nc + cn], dm = C.SM[S * Nc + cn];
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const long long q = cn * NIP + lane + 32 * j;
        const float bk = dirc ? 0.f : v[j];
        C.b[q] = bk;
        C.z[0][q] = __fdiv_rn(__fmul_rn(omega, bk), fmaf(c.k[j], dk, __fmul_rn(c.w[j], dm)));
      }
    }
  }
  // fine z += P (coarse z), Dirichlet nodes untouched
  static __device__ void prolong(const BmgLevel &F, float *zf, const BmgLevel &C, const float *zc, long long first,
                                 long long step, int lane) {
    for (long long a = first; a < F.g.num_nodes; a += step) {
      if (F.dir[a]) continue;
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
      for (int j = 0; j < NJ; ++j) {
        const int i = lane + 32 * j;
        const float v = mid ? __fmul_rn(0.5f, __fadd_rn(zc[c1 * NIP + i], zc[c2 * NIP + i])) : zc[c1 * NIP + i];
        zf[a * NIP + i] = __fadd_rn(zf[a * NIP + i], v);
      }
    }
  }
};

// Buffer index of each level's final iterate after a V-cycle (fixed by the sweep counts).
__host__ __device__ inline void bmg_final_buffers(int L, int nu, int nuc, int *zc) {
  for (int l = 0; l < L; ++l) {
    const int sweeps = (l == L - 1) ? nuc : nu;
    int c = (sweeps - 1) & 1;
    if (l < L - 1) c = (c + nu) & 1;
    zc[l] = c;
  }
}

// Levels >= from in block 0 alone (block barriers), from b_from and z_from[0] (first sweep
// taken).
template <int D, int NJ>
__device__ void bmg_block_cycle(const BmgDev &mg, const typename BmgOps<D, NJ>::Coef &cf, int from, int *zc,
                                int lane) {
  using O = BmgOps<D, NJ>;
  const long long w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int l = from; l < mg.L; ++l) {
    const BmgLevel &L = mg.lv[l];
    const int sweeps = (l == mg.L - 1) ? mg.nuc : mg.nu;
    int c = 0;
    for (int j = 1; j < sweeps; ++j) {
      __syncthreads();
      O::sweep(L, L.z[c], L.z[c ^ 1], mg.omega, cf, w, nw, lane);
      c ^= 1;
    }
    zc[l] = c;
    if (l == mg.L - 1) break;
    __syncthreads();
    O::residual(L, L.z[c], cf, w, nw, lane);
    __syncthreads();
    O::restrict_(L, mg.lv[l + 1], mg.omega, cf, w, nw, lane);
  }
  for (int l = mg.L - 2; l >= from; --l) {
    const BmgLevel &L = mg.lv[l];
    __syncthreads();
    O::prolong(L, L.z[zc[l]], mg.lv[l + 1], mg.lv[l + 1].z[zc[l + 1]], w, nw, lane);
    int c = zc[l];
    for (int j = 0; j < mg.nu; ++j) {
      __syncthreads();
      O::sweep(L, L.z[c], L.z[c ^ 1], mg.omega, cf, w, nw, lane);
      c ^= 1;
    }
    zc[l] = c;
  }
  __syncthreads();
}

// One V-cycle from level 0, whose b and first sweep were written before a grid barrier.
// Level 0's result ends in z[zc[0]], written by the warp that owns each node (no barrier
// after the last sweep: the caller reads own nodes first).
template <int D, int NJ>
__device__ bool bmg_vcycle(const BmgDev &mg, const typename BmgOps<D, NJ>::Coef &cf, int *zc, const GridBar &bar,
                           int lane) {
  using O = BmgOps<D, NJ>;
  const long long nw = blockDim.x >> 5;
  const long long first = blockIdx.x * nw + (threadIdx.x >> 5), step = (long long)gridDim.x * nw;
  const int Lg = mg.Lg;
  if (Lg == 0) {
    if (blockIdx.x == 0) bmg_block_cycle<D, NJ>(mg, cf, 0, zc, lane);
    return grid_sync(bar);
  }
  for (int l = 0; l < Lg; ++l) {
    const BmgLevel &L = mg.lv[l];
    const bool coarsest = l == mg.L - 1;
    const int sweeps = coarsest ? mg.nuc : mg.nu;
    int c = 0;
    for (int j = 1; j < sweeps; ++j) {
      O::sweep(L, L.z[c], L.z[c ^ 1], mg.omega, cf, first, step, lane);
      c ^= 1;
      if (!grid_sync(bar)) return false;
    }
    zc[l] = c;
    if (coarsest) break;
    O::residual(L, L.z[c], cf, first, step, lane);
    if (!grid_sync(bar)) return false;
    O::restrict_(L, mg.lv[l + 1], mg.omega, cf, first, step, lane);
    if (!grid_sync(bar)) return false;
  }
  if (Lg < mg.L) {
    if (blockIdx.x == 0) bmg_block_cycle<D, NJ>(mg, cf, Lg, zc, lane);
    if (!grid_sync(bar)) return false;
  }
  for (int l = std::min(Lg, mg.L - 1) - 1; l >= 0; --l) {
    const BmgLevel &L = mg.lv[l];
    O::prolong(L, L.z[zc[l]], mg.lv[l + 1], mg.lv[l + 1].z[zc[l + 1]], first, step, lane);
    if (!grid_sync(bar)) return false;
    int c = zc[l];
    for (int j = 0; j < mg.nu; ++j) {
      O::sweep(L, L.z[c], L.z[c ^ 1], mg.omega, cf, first, step, lane);
      c ^= 1;
      if (l > 0 || j + 1 < mg.nu)
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
  __shared__ BmgDev mg;
  __shared__ double part[BMG_WARPS * 2 * NIP];
  __shared__ double tot[2 * NIP];
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
  bmg_final_buffers(mg.L, mg.nu, mg.nuc, zc);
  const int zfin = zc[0];
  const float omega = mg.omega;

  // y = A_i x at node a in FP64 (plain-form rows)
  auto apply64 = [&](long long a, const int *idx, const double *x, double (&y)[NJ]) {
    double yk[NJ], ym[NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) yk[j] = ym[j] = 0.0;
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const long long nb = slot_node<D>(g, idx, a, s);
      if (nb < 0) continue;
      const double wk = C.WK[a * S + s], wm = C.WM[a * S + s];
      if (s > 0 && wk == 0.0 && wm == 0.0) continue;
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const double xv = x[nb * NIP + lane + 32 * j];
        yk[j] = fma(wk, xv, yk[j]);
        ym[j] = fma(wm, xv, ym[j]);
      }
    }
#pragma unroll
    for (int j = 0; j < NJ; ++j) y[j] = fma(kk[j], yk[j], __dmul_rn(w2[j], ym[j]));
  };

  double bb[NJ], rr[NJ], gam[NJ];
  bool done[NJ];
  int its[NJ];
  bool nan_seen = false;
  // r = b - A x; p = 0; level-0 right-hand side and first sweep; ||b||^2, ||r||^2
  {
    double v[2][NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) v[0][j] = v[1][j] = 0.0;
    for (long long a = first; a < N; a += step) {
      int idx[3];
      node_ijk(g, a, idx);
      double ax[NJ];
      if (C.warm) apply64(a, idx, C.X, ax);
      const float dk = L0.SK[S * N + a], dm = L0.SM[S * N + a];
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const long long q = a * NIP + lane + 32 * j;
        const double bq = C.bscale * C.B[q];
        if (!C.warm) {
          C.X[q] = 0.0;
          ax[j] = 0.0;
        }
        const double r0 = bq - ax[j];
        C.r[q] = r0;
        C.p[q] = 0.0;
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
  }
  int it = 0;
  for (;;) {
    bool all = true;
#pragma unroll
    for (int j = 0; j < NJ; ++j) all = all && done[j];
    all = __all_sync(0xffffffffu, all);
    if (all || it >= C.maxit) break;
    if (!bmg_vcycle<D, NJ>(mg, cf, zc, C.bar, lane)) return;
    const float *z = L0.z[zfin];
    // gamma = (r, z)
    double v1[1][NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) v1[0][j] = 0.0;
    for (long long a = first; a < N; a += step)
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const long long q = a * NIP + lane + 32 * j;
        v1[0][j] = fma(C.r[q], (double)z[q], v1[0][j]);
      }
    if (!bmg_allreduce<1, NJ>(C, v1, part, tot)) return;
    double beta[NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const double gn = tot[lane + 32 * j];
      beta[j] = (it > 0 && gam[j] > 0.0) ? gn / gam[j] : 0.0;
      gam[j] = gn;
    }
    // p = z + beta p
    for (long long a = first; a < N; a += step)
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const long long q = a * NIP + lane + 32 * j;
        C.p[q] = fma(beta[j], C.p[q], (double)z[q]);
      }
    if (!grid_sync(C.bar)) return;
    // s = A p; (p, s)
#pragma unroll
    for (int j = 0; j < NJ; ++j) v1[0][j] = 0.0;
    for (long long a = first; a < N; a += step) {
      int idx[3];
      node_ijk(g, a, idx);
      double sv[NJ];
      apply64(a, idx, C.p, sv);
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const long long q = a * NIP + lane + 32 * j;
        C.s[q] = sv[j];
        v1[0][j] = fma(C.p[q], sv[j], v1[0][j]);
      }
    }
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
    for (long long a = first; a < N; a += step) {
      const float dk = L0.SK[S * N + a], dm = L0.SM[S * N + a];
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const long long q = a * NIP + lane + 32 * j;
        C.X[q] = fma(alpha[j], C.p[q], C.X[q]);
        const double r1 = fma(-alpha[j], C.s[q], C.r[q]);
        C.r[q] = r1;
        const float bf = (float)r1;
        L0.b[q] = bf;
        L0.z[0][q] = __fdiv_rn(__fmul_rn(omega, bf), fmaf(cf.k[j], dk, __fmul_rn(cf.w[j], dm)));
        v1[0][j] = fma(r1, r1, v1[0][j]);
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

// ===================================================================================== host
struct fo_bmg {
  int L = 0, nip = 0, grid_cap = 0;
  long long built_epoch = -1;
  Grid g[MG_MAX_LEVELS];
  double *coef[MG_MAX_LEVELS] = {}, *WK[MG_MAX_LEVELS] = {}, *WM[MG_MAX_LEVELS] = {};
  uint8_t *dir[MG_MAX_LEVELS] = {};
  float *SK[MG_MAX_LEVELS] = {}, *SM[MG_MAX_LEVELS] = {};
  float *b[MG_MAX_LEVELS] = {}, *z0[MG_MAX_LEVELS] = {}, *z1[MG_MAX_LEVELS] = {}, *t[MG_MAX_LEVELS] = {};
  double *r = nullptr, *p = nullptr, *s = nullptr, *partials = nullptr;
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

using BmgKernel = void (*)(const BmgDev *, BmgCg);
static BmgKernel bmg_kernel(int dim, int nj) {
  if (dim == 2) return nj == 1 ? k_bmg_pcg<2, 1> : (nj == 2 ? k_bmg_pcg<2, 2> : k_bmg_pcg<2, 4>);
  return nj == 1 ? k_bmg_pcg<3, 1> : (nj == 2 ? k_bmg_pcg<3, 2> : k_bmg_pcg<3, 4>);
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
  int per_sm = 0;
  FO_CU(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)bmg_kernel(p->mesh->g.dim, bt->nip / 32),
                                                          32 * BMG_WARPS, 0));
  if (per_sm < 1) return fo_fail(ctx, FO_ECUDA, "batched multigrid kernel does not fit on an SM");
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
  add((void **)&mg->p, sizeof(double) * n0);
  add((void **)&mg->s, sizeof(double) * n0);
  add((void **)&mg->partials, sizeof(double) * (2 * nip * (size_t)mg->grid_cap + 2 * nip));
  add(&mg->dev, sizeof(BmgDev));
  for (auto &e : mg->allocs) FO_TRY(fo_alloc(ctx, e.first, e.second));
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
  BmgDev h;
  memset(&h, 0, sizeof h);
  h.L = mg->L;
  h.Lg = mg->L;
  for (int l = 0; l < mg->L; ++l)
    if (mg->g[l].num_nodes <= BMG_BLOCK_NODES) {
      h.Lg = l;
      break;
    }
  h.nu = 2;
  h.nuc = 16;
  h.omega = 0.8f;
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
  FO_CU(ctx, cudaMemcpyAsync(mg->dev, mg->host.data(), sizeof(BmgDev), cudaMemcpyHostToDevice, s));
  FO_CU(ctx, cudaGetLastError());
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
  long long grid = o->grid_blocks > 0 ? o->grid_blocks : mg->grid_cap;
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
  C.p = mg->p;
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
  const BmgDev *dev = (const BmgDev *)mg->dev;
  FO_CU(ctx, cudaMemsetAsync(p->bar, 0, 64, ctx->stream));
  FO_CU(ctx, cudaMemsetAsync(p->dev_status, 0, sizeof(int) * DS_COUNT, ctx->stream));
  void *argv[] = {(void *)&dev, (void *)&C};
  FO_CU(ctx, cudaLaunchCooperativeKernel((const void *)bmg_kernel(g.dim, nip / 32), (int)grid, 32 * BMG_WARPS, argv, 0,
                                         ctx->stream));
  fo_note_launch(1);
  FO_CU(ctx, cudaGetLastError());
  fo_solve_stats s;
  memset(&s, 0, sizeof s);
  fo_status r = fo_batch_read(p, &s, o);
  if (st) *st = s;
  return r;
}
