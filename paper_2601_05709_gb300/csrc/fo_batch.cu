// Task-parallel batch (Sec. 5.3): a family of screened Helmholtz state problems that share
// the mesh, phi and A_e, solved together on one GPU.
//
// Instance i:  -div(A k_i grad u_i) + omega_i^2 u_i = f_i,  J_i = int f_i u_i,  p_i = -u_i.
// On the Kuhn grid the operator of every instance is one node stencil up to two scalars,
//   (K_i x)(a) = k_i sum_s WK[a][s] x(nb_s) + omega_i^2 sum_s WM[a][s] x(nb_s),
// WK the A-weighted P1 stiffness stencil and WM the consistent-mass stencil of node a
// (Dirichlet columns zeroed; a Dirichlet row keeps WK[a][0] = 1 only, so u_i = 0 there).
// The stencils are built once per coefficient update.  Fields are instance-minor
// (x[a * nip + i]); a warp owns a node and lane l holds instances l, l + 32, ..., so each
// neighbour row is one coalesced 128-byte load per 32 instances and the stencil weights are
// read once for all instances.
//
// The solver is one persistent cooperative kernel per batched solve.
//  * FO_MIXED: FP64 iterative refinement -- residual b - K x and solution x in FP64 -- around
//    an inner Chronopoulos-Gear PCG (the single-reduction recurrence of fo_krylov.cu) whose
//    vectors, stencils and arithmetic are FP32.  Its dot products are FP32 products summed
//    in FP32 over at most DOT_CHUNK nodes per lane and in FP64 from there up.
//  * FO_FP64: the same kernel with FP64 inner vectors, stopping on ||b - K x||_2.
// Each instance has its own recurrence scalars; an instance that has converged is frozen
// (step length zero) while the others continue, and the launch ends when all have.
// Reductions are deterministic and do not depend on timing: per-warp values (one lane per
// instance), a fixed warp order within a block, then each column summed over the blocks
// by one warp in a fixed order; a reduction costs two grid barriers.
#include <cmath>
#include <cstring>
#include <algorithm>
#include <type_traits>
#include <vector>

#include "fo_internal.cuh"
#include "fo_ops.cuh"

#define BATCH_MAX_WARPS 8     // threads per block <= 256
#define DOT_CHUNK 16          // nodes per lane summed in FP32 before an FP64 accumulation

// ------------------------------------------------------------------------ stencils
// WK, WM of node a from the simplices (p, m) around it: in simplex p the node is path vertex
// m, coupled in the stiffness only to its path neighbours m -+ 1 (grad lambda_m is sparse on
// the Kuhn simplex) and in the mass to every vertex with |e| (1 + delta) / ((D+1)(D+2)).
template <int D>
__global__ void k_batch_stencil(Grid g, const double *coef, const uint8_t *dir, double *WK, double *WM,
                                float *WK32, float *WM32) {
  constexpr int S = ST<D>::S;
  double sk[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) sk[k] = g.vol_e * g.inv_h[k] * g.inv_h[k];
  const double mref = g.vol_e / ((D + 1) * (D + 2));
  for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < g.num_nodes;
       a += (long long)gridDim.x * blockDim.x) {
    int idx[3];
    node_ijk(g, a, idx);
    double wk[S], wm[S];
#pragma unroll
    for (int s = 0; s < S; ++s) wk[s] = wm[s] = 0.0;
    if (dir[a]) {
      wk[0] = 1.0;
    } else {
#pragma unroll
      for (int p = 0; p < KP<D>::P; ++p)
#pragma unroll
        for (int m = 0; m <= D; ++m) {
          long long e;
          if (!elem_of<D>(g, idx, p, m, e)) continue;
          const double Ae = coef[e];
          if (m >= 1) {
            const double c = Ae * sk[kperm<D>(p, m - 1)];
            wk[0] += c;
            wk[rel_slot<D>(p, m, m - 1)] -= c;
          }
          if (m < D) {
            const double c = Ae * sk[kperm<D>(p, m)];
            wk[0] += c;
            wk[rel_slot<D>(p, m, m + 1)] -= c;
          }
          wm[0] += mref;
#pragma unroll
          for (int l = 0; l <= D; ++l) wm[rel_slot<D>(p, m, l)] += mref;
        }
#pragma unroll
      for (int s = 1; s < S; ++s) {
        const long long nb = slot_node<D>(g, idx, a, s);
        if (nb < 0 || dir[nb]) wk[s] = wm[s] = 0.0;
      }
    }
#pragma unroll
    for (int s = 0; s < S; ++s) {
      WK[a * S + s] = wk[s];
      WM[a * S + s] = wm[s];
      if (WK32) {
        WK32[a * S + s] = (float)wk[s];
        WM32[a * S + s] = (float)wm[s];
      }
    }
  }
}

__global__ void k_batch_dinv(long long n, int S, int nip, const double *WK, const double *WM, const double *kk,
                             const double *w2, double *dinv, float *dinv32) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n * nip;
       t += (long long)gridDim.x * blockDim.x) {
    const long long a = t / nip;
    const int i = (int)(t - a * nip);
    const double v = 1.0 / (kk[i] * WK[a * S] + w2[i] * WM[a * S]);
    dinv[t] = v;
    dinv32[t] = (float)v;
  }
}

// Loads F_i(a) = int f_i psi_a with f_i the P1 interpolant: sum over the simplices of a of
// |e| / ((D+1)(D+2)) (f_i(a) + sum_l f_i(v_l)); zero on Dirichlet nodes.
template <int D>
__global__ void k_batch_load(Grid g, const uint8_t *dir, int nip, const double *f, double *B) {
  const double mref = g.vol_e / ((D + 1) * (D + 2));
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < g.num_nodes * nip;
       t += (long long)gridDim.x * blockDim.x) {
    const long long a = t / nip;
    const int i = (int)(t - a * nip);
    if (dir[a]) {
      B[t] = 0.0;
      continue;
    }
    int idx[3];
    node_ijk(g, a, idx);
    double acc = 0.0;
#pragma unroll
    for (int p = 0; p < KP<D>::P; ++p)
#pragma unroll
      for (int m = 0; m <= D; ++m) {
        long long e;
        if (!elem_of<D>(g, idx, p, m, e)) continue;
        double s = f[t];
#pragma unroll
        for (int l = 0; l <= D; ++l) s += f[slot_node<D>(g, idx, a, rel_slot<D>(p, m, l)) * nip + i];
        acc += mref * s;
      }
    B[t] = acc;
  }
}

// y = K_i x for every instance (parity tests): warp per node, weights in W.
template <int D, int NJ, typename W>
__global__ void k_batch_apply(Grid g, const W *WK, const W *WM, const double *kk, const double *w2, const double *x,
                              double *y) {
  constexpr int S = ST<D>::S, NIP = 32 * NJ;
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (long long a = blockIdx.x * (long long)nw + (threadIdx.x >> 5); a < g.num_nodes; a += (long long)gridDim.x * nw) {
    int idx[3];
    node_ijk(g, a, idx);
    W yk[NJ], ym[NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) yk[j] = ym[j] = W(0);
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const long long nb = slot_node<D>(g, idx, a, s);
      if (nb < 0) continue;
      const W wk = WK[a * S + s], wm = WM[a * S + s];
      if (s > 0 && wk == W(0) && wm == W(0)) continue;
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const W xv = (W)x[nb * NIP + lane + 32 * j];
        yk[j] = fma(wk, xv, yk[j]);
        ym[j] = fma(wm, xv, ym[j]);
      }
    }
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const int i = lane + 32 * j;
      y[a * NIP + i] = (double)fma((W)kk[i], yk[j], (W)w2[i] * ym[j]);
    }
  }
}

// ------------------------------------------------------------------------ solver
// Node tiles of the batched sweep (nodes per tile along x, y, z); the autotuner picks one.
template <int D, int TS>
struct BatchTile;
template <> struct BatchTile<2, 0> { static constexpr int TX = 16, TY = 8, TZ = 1; };
template <> struct BatchTile<2, 1> { static constexpr int TX = 32, TY = 8, TZ = 1; };
template <> struct BatchTile<3, 0> { static constexpr int TX = 4, TY = 4, TZ = 2; };
template <> struct BatchTile<3, 1> { static constexpr int TX = 8, TY = 4, TZ = 4; };

template <typename T>
struct BatchVecs {
  T *x, *p;
  T *r[2], *w[2], *s[2];
  const T *dinv, *WK, *WM;
};

struct BatchArgs {
  Grid g;
  const double *B;
  double bscale;             // the system's right-hand side is bscale * B
  double *X;                 // FP64 solution [N_n][nip]
  const double *WK, *WM;     // FP64 stencils (refinement residual)
  const double *kk, *w2;     // [nip]
  double *partials;          // [3 nip][G]
  double *totals;            // [3 nip]
  int *status;
  GridBar bar;
  int *inst_iters;
  double *inst_res;
  double rtol2, inner_rtol2;
  int maxit, inner_maxit, warm;
};

template <int NIP>
struct BatchShared {
  double tot[3 * NIP];
  double alpha[NIP], beta[NIP], gam[NIP], gref[NIP], bn2[NIP], rn2p[NIP], rn2pp[NIP], res[NIP];
  int act[NIP], done[NIP], iters[NIP], upd[NIP], kloc[NIP];
};

// Sum NCOL columns of per-instance values over the whole grid; totals land in sh.tot
// (column c of instance i at c * NIP + i), the same bits in every block.  part: shared
// scratch of BATCH_MAX_WARPS * NCOL * NIP doubles.
template <int NCOL, int NJ>
__device__ bool batch_allreduce(const BatchArgs &A, const double (&v)[NCOL][NJ], double *part,
                                BatchShared<32 * NJ> &sh) {
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
    __stcg(A.partials + (size_t)t * G + blockIdx.x, s);
  }
  if (!grid_sync(A.bar)) return false;
  const int gw = blockIdx.x * nw + warp, nwt = G * nw;
  for (int col = gw; col < NCOL * NIP; col += nwt) {
    const double *src = A.partials + (size_t)col * G;
    double t = 0.0;
    int b = lane;
    for (; b + 96 < G; b += 128) {
      const double x0 = __ldcg(src + b), x1 = __ldcg(src + b + 32), x2 = __ldcg(src + b + 64),
                   x3 = __ldcg(src + b + 96);
      t += x0;
      t += x1;
      t += x2;
      t += x3;
    }
    for (; b < G; b += 32) t += __ldcg(src + b);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0) __stcg(A.totals + col, t);
  }
  if (!grid_sync(A.bar)) return false;
  for (int t = threadIdx.x; t < NCOL * NIP; t += blockDim.x) sh.tot[t] = __ldcg(A.totals + t);
  __syncthreads();
  return true;
}

// The persistent batched solver.  An inner iteration walks the grid tile by tile:
//   stage 1 -- every node of the tile's halo box: s_{k-1} = w_{k-1} + b s_{k-2},
//              r_k = r_{k-1} - a s_{k-1}, u_k = D^{-1} r_k into shared memory; on the tile's
//              own nodes also p_{k-1} = u_{k-1} + b p_{k-2}, x_k = x_{k-1} + a p_{k-1}, and
//              r_k, s_{k-1} are stored;
//   stage 2 -- own nodes: w_k = K u_k from the shared-memory stencil, stored.
// u_k of a node is formed by the same expression in every tile that holds it, so the halo
// copies agree bit for bit with the owner's.  r, w and s are double-buffered: a stage only
// reads the previous iteration's buffers, which no block writes during the sweep.
template <int D, int NJ, typename T, int TS>
__global__ void __launch_bounds__(256) k_batch_solve(BatchArgs A, BatchVecs<T> V) {
  using TL = BatchTile<D, TS>;
  constexpr int TX = TL::TX, TY = TL::TY, TZ = (D == 3) ? TL::TZ : 1;
  constexpr int HX = TX + 2, HY = TY + 2, HZ = (D == 3) ? TZ + 2 : 1, NH = HX * HY * HZ, NT = TX * TY * TZ;
  constexpr int S = ST<D>::S, NIP = 32 * NJ;
  constexpr bool F64 = std::is_same<T, double>::value;
  extern __shared__ __align__(16) unsigned char fo_batch_smem[];
  T *smU = reinterpret_cast<T *>(fo_batch_smem);             // [NH][NIP] during a sweep
  T *sW = smU + (size_t)NH * NIP;                             // [NT][2 S] own-node weights
  double *part = reinterpret_cast<double *>(fo_batch_smem);  // reduction scratch between sweeps
  __shared__ BatchShared<NIP> sh;
  const Grid &g = A.g;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const long long first = blockIdx.x * (long long)nw + warp, step = (long long)gridDim.x * nw;
  const long long N = g.num_nodes;
  const int nn0 = (int)g.nn[0], nn1 = (int)g.nn[1], nn2 = (int)g.nn[2];
  const int ntx = (nn0 + TX - 1) / TX, nty = (nn1 + TY - 1) / TY, ntz = (D == 3) ? (nn2 + TZ - 1) / TZ : 1;
  const long long ntiles = (long long)ntx * nty * ntz;

  double kk64[NJ], w264[NJ];
  T kk[NJ], w2[NJ];
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    kk64[j] = A.kk[lane + 32 * j];
    w264[j] = A.w2[lane + 32 * j];
    kk[j] = (T)kk64[j];
    w2[j] = (T)w264[j];
  }
  for (int t = threadIdx.x; t < NIP; t += blockDim.x) {
    sh.iters[t] = 0;
    sh.done[t] = 0;
    sh.act[t] = 0;
    sh.upd[t] = 1;
    sh.rn2p[t] = sh.rn2pp[t] = INFINITY;
    sh.res[t] = 0.0;
    sh.bn2[t] = 0.0;
    sh.alpha[t] = sh.beta[t] = sh.gam[t] = sh.gref[t] = 0.0;
    sh.kloc[t] = 0;
  }
  __syncthreads();

  // ---- phases ------------------------------------------------------------------------
  // X += x (FP64) and x = 0 for the instances being updated; on the first call X = 0
  // unless warm-started.
  auto accumulate = [&](bool start) {
    bool mine[NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) mine[j] = sh.upd[lane + 32 * j] != 0;
    for (long long a = first; a < N; a += step)
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        if (!mine[j]) continue;
        const long long q = a * NIP + lane + 32 * j;
        if (start) {
          if (!A.warm) A.X[q] = 0.0;
        } else {
          A.X[q] += (double)V.x[q];
        }
        V.x[q] = T(0);
      }
  };
  // r = b - K X in FP64 for the instances being updated, stored rounded to T in buffer set
  // `buf` (the one the next sweep reads), with the start vectors of a fresh recurrence:
  // w = s = 0 in that set and p = 0.
  auto residual = [&](int buf, double (&red)[2][NJ]) {
    T *rbuf = V.r[buf], *wbuf = V.w[buf], *sbuf = V.s[buf];
    bool mine[NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      red[0][j] = red[1][j] = 0.0;
      mine[j] = sh.upd[lane + 32 * j] != 0;
    }
    for (long long a = first; a < N; a += step) {
      int idx[3];
      node_ijk(g, a, idx);
      double yk[NJ], ym[NJ];
#pragma unroll
      for (int j = 0; j < NJ; ++j) yk[j] = ym[j] = 0.0;
#pragma unroll
      for (int s = 0; s < S; ++s) {
        const long long nb = slot_node<D>(g, idx, a, s);
        if (nb < 0) continue;
        const double wk = A.WK[a * S + s], wm = A.WM[a * S + s];
        if (s > 0 && wk == 0.0 && wm == 0.0) continue;
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
          if (!mine[j]) continue;
          const double xv = A.X[nb * NIP + lane + 32 * j];
          yk[j] = fma(wk, xv, yk[j]);
          ym[j] = fma(wm, xv, ym[j]);
        }
      }
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        if (!mine[j]) continue;
        const long long q = a * NIP + lane + 32 * j;
        const double b = A.bscale * A.B[q];
        const double r = b - fma(kk64[j], yk[j], w264[j] * ym[j]);
        red[0][j] += r * r;
        red[1][j] += b * b;
        rbuf[q] = (T)r;
        wbuf[q] = T(0);
        sbuf[q] = T(0);
        V.p[q] = T(0);
      }
    }
  };
  // One pass over the tiles: step k of the recurrence.  Reads r_{k-1}, w_{k-1}, s_{k-2} from
  // buffer set (k+1)&1, writes r_k, s_{k-1}, w_k to set k&1 and updates p, x; dot products
  // (r_k, u_k), (w_k, u_k) and, in FP64, (r_k, r_k).
  auto sweep = [&](int k, double (&dacc)[3][NJ]) {
    T al[NJ], be[NJ];
    bool on[NJ];   // this lane's instances still iterate; frozen ones are skipped
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      al[j] = (T)sh.alpha[lane + 32 * j];
      be[j] = (T)sh.beta[lane + 32 * j];
      on[j] = sh.act[lane + 32 * j] != 0 && sh.upd[lane + 32 * j] == 0;   // running, not waiting
    }
    const int ob = (k + 1) & 1, nb_ = k & 1;
    const T *ro = V.r[ob], *wo = V.w[ob], *so = V.s[ob];
    T *rn = V.r[nb_], *wn = V.w[nb_], *sn = V.s[nb_];
    T cacc[3][NJ];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        dacc[c][j] = 0.0;
        cacc[c][j] = T(0);
      }
    int chunk = 0;
    auto count = [&]() {   // FP32 partial dot products go to FP64 every DOT_CHUNK nodes
      if (!F64 && ++chunk == DOT_CHUNK) {
        chunk = 0;
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int j = 0; j < NJ; ++j) {
            dacc[c][j] += (double)cacc[c][j];
            cacc[c][j] = T(0);
          }
      }
    };
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
      const int i0 = (int)(tile % ntx) * TX, j0 = (int)((tile / ntx) % nty) * TY;
      const int k0 = (D == 3) ? (int)(tile / ((long long)ntx * nty)) * TZ : 0;
      // stage 1: u_k on the halo box, recurrences on the own nodes.  A warp takes UB halo
      // nodes at a time and issues all their loads before any store, so that several rows
      // per warp are in flight; lanes of frozen or waiting instances neither load nor store.
      constexpr int UB = 4 / NJ;   // rows in flight per warp: UB * NJ = 4
      for (int h0 = warp; h0 < NH; h0 += UB * nw) {
        long long aa[UB];
        int oo[UB];
        bool in[UB], ow[UB];
#pragma unroll
        for (int u = 0; u < UB; ++u) {
          const int h = h0 + u * nw;
          const int hx = h % HX, hy = (h / HX) % HY, hz = h / (HX * HY);
          const int gi = i0 - 1 + hx, gj = j0 - 1 + hy, gk = (D == 3) ? k0 - 1 + hz : 0;
          in[u] = h < NH && gi >= 0 && gi < nn0 && gj >= 0 && gj < nn1 && (D == 2 || (gk >= 0 && gk < nn2));
          ow[u] = in[u] && hx >= 1 && hx <= TX && hy >= 1 && hy <= TY && (D == 2 || (hz >= 1 && hz <= TZ));
          aa[u] = in[u] ? gi + g.stride[1] * gj + (D == 3 ? g.stride[2] * gk : 0) : 0;
          oo[u] = (hx - 1) + TX * ((hy - 1) + TY * (D == 3 ? hz - 1 : 0));
        }
        T rq[UB][NJ], dq[UB][NJ], sq[UB][NJ], wq[UB][NJ], pq[UB][NJ], xq[UB][NJ], wt[UB][2];
#pragma unroll
        for (int u = 0; u < UB; ++u) {
#pragma unroll
          for (int j = 0; j < NJ; ++j) {
            rq[u][j] = dq[u][j] = sq[u][j] = wq[u][j] = pq[u][j] = xq[u][j] = T(0);
            if (in[u] && on[j]) {
              const long long q = aa[u] * NIP + lane + 32 * j;
              rq[u][j] = ro[q];
              dq[u][j] = V.dinv[q];
              sq[u][j] = so[q];
              wq[u][j] = wo[q];
              if (ow[u]) {
                pq[u][j] = V.p[q];
                xq[u][j] = V.x[q];
              }
            }
          }
          wt[u][0] = wt[u][1] = T(0);
          if (ow[u] && lane < S) {
            wt[u][0] = V.WK[aa[u] * S + lane];
            wt[u][1] = V.WM[aa[u] * S + lane];
          }
        }
#pragma unroll
        for (int u = 0; u < UB; ++u) {
          const int h = h0 + u * nw;
          if (h >= NH) continue;
          T *su = smU + (size_t)h * NIP + lane;
          if (!in[u]) {
#pragma unroll
            for (int j = 0; j < NJ; ++j) su[32 * j] = T(0);
            continue;
          }
#pragma unroll
          for (int j = 0; j < NJ; ++j) {
            if (!on[j]) continue;
            // s_{k-1} = w_{k-1} + b s_{k-2},  r_k = r_{k-1} - a s_{k-1},  u_k = D^{-1} r_k
            const T sv = fma(be[j], sq[u][j], wq[u][j]);
            const T rv = fma(-al[j], sv, rq[u][j]);
            const T uv = dq[u][j] * rv;
            su[32 * j] = uv;
            if (ow[u]) {
              const long long q = aa[u] * NIP + lane + 32 * j;
              rn[q] = rv;
              sn[q] = sv;
              const T p_new = fma(be[j], pq[u][j], dq[u][j] * rq[u][j]);   // p_{k-1} = u_{k-1} + b p_{k-2}
              V.x[q] = fma(al[j], p_new, xq[u][j]);                        // x_k = x_{k-1} + a p_{k-1}
              V.p[q] = p_new;
              cacc[0][j] = fma(rv, uv, cacc[0][j]);
              if (F64) cacc[2][j] = fma(rv, rv, cacc[2][j]);
            }
          }
          if (ow[u]) {
            if (lane < S) {
              sW[oo[u] * 2 * S + lane] = wt[u][0];
              sW[oo[u] * 2 * S + S + lane] = wt[u][1];
            }
            count();
          }
        }
      }
      __syncthreads();
      // stage 2: w_k = K u_k on the own nodes, from the shared field and weights
      for (int o = warp; o < NT; o += nw) {
        const int ox = o % TX, oy = (o / TX) % TY, oz = o / (TX * TY);
        const int gi = i0 + ox, gj = j0 + oy, gk = k0 + oz;
        if (gi >= nn0 || gj >= nn1 || (D == 3 && gk >= nn2)) continue;
        const long long a = gi + g.stride[1] * gj + (D == 3 ? g.stride[2] * gk : 0);
        const int h = (ox + 1) + HX * ((oy + 1) + HY * (D == 3 ? oz + 1 : 0));
        const T *sw = sW + o * 2 * S;
        T yk[NJ], ym[NJ];
#pragma unroll
        for (int j = 0; j < NJ; ++j) yk[j] = ym[j] = T(0);
#pragma unroll
        for (int s = 0; s < S; ++s) {
          const T wk = sw[s], wm = sw[S + s];
          if (s > 0 && wk == T(0) && wm == T(0)) continue;   // absent or Dirichlet neighbour
          int dl[3];
          slot_offset<D>(s, dl);
          const T *su = smU + (size_t)(h + dl[0] + HX * (dl[1] + HY * dl[2])) * NIP + lane;
#pragma unroll
          for (int j = 0; j < NJ; ++j) {
            if (!on[j]) continue;
            const T uv = su[32 * j];
            yk[j] = fma(wk, uv, yk[j]);
            ym[j] = fma(wm, uv, ym[j]);
          }
        }
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
          if (!on[j]) continue;
          const long long q = a * NIP + lane + 32 * j;
          const T w_new = fma(kk[j], yk[j], w2[j] * ym[j]);
          wn[q] = w_new;
          cacc[1][j] = fma(w_new, smU[(size_t)h * NIP + lane + 32 * j], cacc[1][j]);
        }
        count();
      }
      __syncthreads();   // the next tile overwrites the shared stencil field
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int j = 0; j < NJ; ++j) dacc[c][j] += (double)cacc[c][j];
  };
  // Per-instance test of the FP64 residual: converged, or at its rounding floor (two
  // consecutive checks that fail to halve it: x is as accurate as FP64 allows).
  auto check_residual = [&](bool first_check, int &nan, int &open) {
    for (int t = threadIdx.x; t < NIP; t += blockDim.x) {
      if (!sh.upd[t]) {
        open |= sh.act[t];
        continue;
      }
      const double rn2 = sh.tot[t];
      if (first_check) sh.bn2[t] = sh.tot[NIP + t];
      const double bn2 = sh.bn2[t];
      if (!isfinite(rn2)) nan = 1;
      const bool conv = rn2 <= A.rtol2 * bn2 || rn2 == 0.0;
      const bool floor = rn2 > 0.25 * sh.rn2p[t] && sh.rn2p[t] > 0.25 * sh.rn2pp[t];
      sh.res[t] = bn2 > 0.0 ? sqrt(rn2 / bn2) : sqrt(rn2);
      sh.rn2pp[t] = sh.rn2p[t];
      sh.rn2p[t] = rn2;
      if (conv || floor) sh.done[t] = 1;
      sh.act[t] = sh.done[t] ? 0 : 1;
      if (sh.done[t]) sh.alpha[t] = sh.beta[t] = 0.0;
      open |= sh.act[t];
    }
  };
  int sweeps = 0, applies = 0, updates = 0, err = DEV_OK;
  bool ok = true;
  double red[2][NJ];
  double dacc[3][NJ];
  accumulate(true);
  if (!(ok = grid_sync(A.bar))) goto finish;
  residual(1, red);
  if (!(ok = batch_allreduce<2, NJ>(A, red, part, sh))) goto finish;
  ++applies;
  {
    int nan = 0, open = 0;
    check_residual(true, nan, open);
    for (int t = threadIdx.x; t < NIP; t += blockDim.x) sh.upd[t] = 0;
    if (__syncthreads_or(nan)) {
      err = DEV_NAN;
      goto finish;
    }
    if (!__syncthreads_or(open)) goto finish;
  }
  // Iterative refinement, per instance.  Each instance runs PCG on K d = r from d = 0 until
  // its inner test holds -- FP64: ||r_k||_2 <= rtol ||b||_2 (the recurrence residual);
  // mixed: (r_k, u_k) <= inner_rtol^2 (r_0, u_0) -- then its d is added to the FP64
  // solution, the FP64 residual b - K x is formed and tested, and, unless it meets rtol (or
  // has reached its rounding floor), the instance restarts PCG from it.  Each instance moves
  // on its own schedule and its trajectory depends on its own data only; the others keep
  // iterating meanwhile.
  for (int k = 0;; ++k) {
    sweep(k, dacc);
    if (!(ok = batch_allreduce<3, NJ>(A, dacc, part, sh))) goto finish;
    ++sweeps;
    ++applies;
    int nan2 = 0, running = 0, waiting = 0;
    const bool at_cap = sweeps >= A.maxit;
    for (int t = threadIdx.x; t < NIP; t += blockDim.x) {
      if (!sh.act[t]) continue;
      if (sh.upd[t]) {   // inner solve ended earlier: idles (frozen) until its refinement step
        waiting += 1;
        continue;
      }
      const double gm = sh.tot[t], dl = sh.tot[NIP + t];
      if (!isfinite(gm) || !isfinite(dl)) nan2 = 1;
      const int kl = sh.kloc[t];   // step of the instance's current inner solve
      if (kl > 0) sh.iters[t] += 1;
      if (kl == 0) sh.gref[t] = gm;
      bool stop = F64 ? sh.tot[2 * NIP + t] <= A.rtol2 * sh.bn2[t] : gm <= A.inner_rtol2 * sh.gref[t];
      stop = stop || !(gm > 0.0) || kl >= A.inner_maxit || at_cap;
      // b = gamma_k / gamma_{k-1},  a = gamma_k / (delta_k - b gamma_k / a_{k-1})
      double beta = 0.0, den = dl;
      if (!stop && kl > 0) {
        beta = gm / sh.gam[t];
        den = dl - beta * gm / sh.alpha[t];
      }
      if (!(den > 0.0)) stop = true;   // breakdown in rounding: refine and restart
      if (stop) {
        sh.alpha[t] = sh.beta[t] = 0.0;
        sh.upd[t] = 1;
        waiting += 1;
      } else {
        sh.alpha[t] = gm / den;
        sh.beta[t] = beta;
        sh.gam[t] = gm;
        sh.kloc[t] = kl + 1;
        running += 1;
      }
    }
    if (__syncthreads_or(nan2)) {
      err = DEV_NAN;
      goto finish;
    }
    // Refinement steps are grouped: one FP64 residual pass serves every waiting instance, and
    // it runs once a quarter of the active instances wait or nothing else iterates.  Waiting
    // changes no instance's state, so the grouping does not change any result.
    const int nrun = __syncthreads_count(running), nwait = __syncthreads_count(waiting);
    if (nwait == 0 || (nrun > 0 && 4 * nwait < nrun + nwait && !at_cap)) continue;
    // refinement step of the instances whose inner solve ended
    accumulate(false);
    if (!(ok = grid_sync(A.bar))) goto finish;
    residual(k & 1, red);
    if (!(ok = batch_allreduce<2, NJ>(A, red, part, sh))) goto finish;
    ++applies;
    ++updates;
    int nan = 0, open = 0;
    check_residual(false, nan, open);
    for (int t = threadIdx.x; t < NIP; t += blockDim.x)
      if (sh.upd[t]) {
        sh.kloc[t] = 0;
        sh.upd[t] = 0;
      }
    if (__syncthreads_or(nan)) {
      err = DEV_NAN;
      goto finish;
    }
    if (!__syncthreads_or(open)) break;
    if (at_cap) {
      err = DEV_NOCONV;
      break;
    }
  }
finish:
  if (blockIdx.x == 0) {
    if (threadIdx.x == 0) {
      A.status[DS_ITERS] = sweeps;
      A.status[DS_APPLIES] = applies;
      A.status[DS_FLAG] = updates;
      if (err != DEV_OK) atomicCAS(A.status + DS_ERR, DEV_OK, err);
    }
    for (int t = threadIdx.x; t < NIP; t += blockDim.x) {
      A.inst_iters[t] = sh.iters[t];
      A.inst_res[t] = sh.res[t];
    }
  }
}

// ------------------------------------------------------------------ costs, volume
template <int NJ>
__global__ void k_batch_costs(long long nn, const double *B, const double *U, double *partials /*[G][NIP]*/) {
  constexpr int NIP = 32 * NJ;
  __shared__ double sp[BATCH_MAX_WARPS * NIP];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double v[NJ];
#pragma unroll
  for (int j = 0; j < NJ; ++j) v[j] = 0.0;
  for (long long a = blockIdx.x * (long long)nw + warp; a < nn; a += (long long)gridDim.x * nw)
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const long long q = a * NIP + lane + 32 * j;
      v[j] = fma(B[q], U[q], v[j]);
    }
#pragma unroll
  for (int j = 0; j < NJ; ++j) sp[warp * NIP + lane + 32 * j] = v[j];
  __syncthreads();
  for (int t = threadIdx.x; t < NIP; t += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += sp[w * NIP + t];
    partials[(size_t)blockIdx.x * NIP + t] = s;
  }
}

__global__ void k_batch_volume(long long ne, double vol_e, const uint8_t *chi, double *partial /*[G]*/) {
  __shared__ double smem[32];
  double v[1] = {0.0};
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ne; e += (long long)gridDim.x * blockDim.x)
    v[0] += chi[e] ? vol_e : 0.0;
  block_sum<1>(v, smem);
  if (threadIdx.x == 0) partial[blockIdx.x] = v[0];
}

// out[i] = sum_b partials[b][i] (i < nip) and out[nip] = sum_b volp[b], fixed order
__global__ void k_batch_costs_finish(int G, int nip, const double *partials, const double *volp, double *out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nip) {
    double s = 0.0;
    for (int b = 0; b < G; ++b) s += partials[(size_t)b * nip + t];
    out[t] = s;
  } else if (t == nip) {
    double s = 0.0;
    for (int b = 0; b < G; ++b) s += volp[b];
    out[nip] = s;
  }
}

// ------------------------------------------------------------- summed shape derivative
// b[D a + k] = sum_i sum_{(p, m) around a} [ |e| A k_i (-|grad u_i|^2 grad lambda_m
//              + 2 grad u_i (grad u_i . grad lambda_m)) + (2 int_e u_i f_i - omega_i^2 int_e u_i^2)
//              grad lambda_m + 2 grad f_i int_e u_i lambda_m ]_k  + lambda / V |e| chi_e grad lambda_m,
// i.e. S0 = 2 u_i grad f_i and S1 = (2 u_i f_i - A k_i |grad u_i|^2 - omega_i^2 u_i^2) I
// + 2 A k_i grad u_i (x) grad u_i summed over the instances (Sec. 6.3 with the zero-order
// term), plus the volume tensor.  The products u f and u^2 are integrated exactly with the
// consistent mass.  Warp per node; each lane sums its instances, then a fixed shuffle tree.
template <int D, int NJ>
__global__ void k_batch_shape(Grid g, const double *coef, const uint8_t *chi, const double *U, const double *F,
                              const double *kk, const double *w2, double lam_over_V, double *b) {
  constexpr int S = ST<D>::S, NIP = 32 * NJ;
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const double mref = g.vol_e / ((D + 1) * (D + 2));
  for (long long a = blockIdx.x * (long long)nw + (threadIdx.x >> 5); a < g.num_nodes; a += (long long)gridDim.x * nw) {
    int idx[3];
    node_ijk(g, a, idx);
    long long nbs[S];
#pragma unroll
    for (int s = 0; s < S; ++s) nbs[s] = slot_node<D>(g, idx, a, s);
    double acc[D];
#pragma unroll
    for (int k = 0; k < D; ++k) acc[k] = 0.0;
    for (int j = 0; j < NJ; ++j) {
      const int i = lane + 32 * j;
      const double ki = kk[i], om2 = w2[i];
      double us[S], fs[S];
#pragma unroll
      for (int s = 0; s < S; ++s) {
        us[s] = nbs[s] >= 0 ? U[nbs[s] * NIP + i] : 0.0;
        fs[s] = nbs[s] >= 0 ? F[nbs[s] * NIP + i] : 0.0;
      }
#pragma unroll
      for (int p = 0; p < KP<D>::P; ++p)
#pragma unroll
        for (int m = 0; m <= D; ++m) {
          long long e;
          if (!elem_of<D>(g, idx, p, m, e)) continue;
          double gu[3] = {0, 0, 0}, gf[3] = {0, 0, 0};
#pragma unroll
          for (int l = 0; l < D; ++l) {
            const int ax = kperm<D>(p, l);
            const int s0 = rel_slot<D>(p, m, l), s1 = rel_slot<D>(p, m, l + 1);
            gu[ax] = (us[s1] - us[s0]) * g.inv_h[ax];
            gf[ax] = (fs[s1] - fs[s0]) * g.inv_h[ax];
          }
          double su = 0, sf = 0, suf = 0, suu = 0;
#pragma unroll
          for (int l = 0; l <= D; ++l) {
            const int sl = rel_slot<D>(p, m, l);
            su += us[sl];
            sf += fs[sl];
            suf += us[sl] * fs[sl];
            suu += us[sl] * us[sl];
          }
          const double Ak = coef[e] * ki;
          double g2 = 0;
#pragma unroll
          for (int k = 0; k < D; ++k) g2 += gu[k] * gu[k];
          const double uf = mref * (suf + su * sf);   // int_e u f
          const double uu = mref * (suu + su * su);   // int_e u^2
          const double Mu = mref * (su + us[0]);      // int_e u lambda_m
          double gl[3] = {0, 0, 0};
          if (m >= 1) gl[kperm<D>(p, m - 1)] += g.inv_h[kperm<D>(p, m - 1)];
          if (m < D) gl[kperm<D>(p, m)] -= g.inv_h[kperm<D>(p, m)];
          double gdot = 0;
#pragma unroll
          for (int k = 0; k < D; ++k) gdot += gu[k] * gl[k];
          const double c0 = 2.0 * uf - om2 * uu;
#pragma unroll
          for (int k = 0; k < D; ++k)
            acc[k] += g.vol_e * Ak * (-g2 * gl[k] + 2.0 * gu[k] * gdot) + c0 * gl[k] + 2.0 * gf[k] * Mu;
        }
    }
#pragma unroll
    for (int k = 0; k < D; ++k)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], o);
    if (lane == 0) {
      if (lam_over_V != 0.0) {
#pragma unroll
        for (int p = 0; p < KP<D>::P; ++p)
#pragma unroll
          for (int m = 0; m <= D; ++m) {
            long long e;
            if (!elem_of<D>(g, idx, p, m, e) || !chi[e]) continue;
            if (m >= 1) acc[kperm<D>(p, m - 1)] += g.vol_e * lam_over_V * g.inv_h[kperm<D>(p, m - 1)];
            if (m < D) acc[kperm<D>(p, m)] -= g.vol_e * lam_over_V * g.inv_h[kperm<D>(p, m)];
          }
      }
#pragma unroll
      for (int k = 0; k < D; ++k) b[a * D + k] = acc[k];
    }
  }
}

// ================================================================================ host
static inline int batch_S(const Grid &g) { return g.dim == 2 ? 7 : 15; }

static size_t batch_bytes(const fo_problem *p, std::vector<std::pair<void **, size_t>> &list) {
  fo_batch *bt = p->batch;
  const Grid &g = p->mesh->g;
  const size_t NN = (size_t)g.num_nodes, nip = (size_t)bt->nip, S = (size_t)batch_S(g);
  list = {
      {(void **)&bt->kk, sizeof(double) * nip},         {(void **)&bt->w2, sizeof(double) * nip},
      {(void **)&bt->f, sizeof(double) * NN * nip},     {(void **)&bt->B, sizeof(double) * NN * nip},
      {(void **)&bt->U, sizeof(double) * NN * nip},     {(void **)&bt->P, sizeof(double) * NN * nip},
      {(void **)&bt->WK, sizeof(double) * NN * S},      {(void **)&bt->WM, sizeof(double) * NN * S},
      {(void **)&bt->WK32, sizeof(float) * NN * S},     {(void **)&bt->WM32, sizeof(float) * NN * S},
      {(void **)&bt->dinv, sizeof(double) * NN * nip},  {(void **)&bt->dinv32, sizeof(float) * NN * nip},
      {(void **)&bt->inst_iters, sizeof(int) * nip},    {(void **)&bt->inst_res, sizeof(double) * nip},
  };
  size_t s = 0;
  for (auto &e : list) s += e.second;
  return s;
}

void fo_batch_destroy(fo_problem *p) {
  if (!p->batch) return;
  fo_bmg_destroy(p);
  std::vector<std::pair<void **, size_t>> list;
  batch_bytes(p, list);
  for (auto &e : list) {
    fo_free(p->ctx, *e.first, e.second);
    *e.first = nullptr;
  }
  delete p->batch;
  p->batch = nullptr;
}

fo_status fo_batch_create(fo_problem *p, const fo_model_desc *desc) {
  fo_ctx *ctx = p->ctx;
  const Grid &g = p->mesh->g;
  const int n = desc->n_inst;
  if (n < 1 || n > FO_MAX_INSTANCES) return fo_fail(ctx, FO_EINVAL, "n_inst must be in [1, %d]", FO_MAX_INSTANCES);
  if (!desc->inst_k || !desc->inst_omega || !desc->inst_f)
    return fo_fail(ctx, FO_EINVAL, "a batch needs inst_k, inst_omega and inst_f");
  for (int i = 0; i < n; ++i)
    if (!(desc->inst_k[i] > 0) || !std::isfinite(desc->inst_omega[i]))
      return fo_fail(ctx, FO_EINVAL, "instance %d: k must be > 0 and omega finite", i);
  fo_batch *bt = new fo_batch();
  p->batch = bt;
  bt->n_inst = n;
  bt->nip = n <= 32 ? 32 : (n <= 64 ? 64 : 128);   // compiled slab counts: 1, 2, 4
  const int nip = bt->nip;
  // Lanes in order of omega_i^2 / k_i, the weight of the well-conditioned mass term: the
  // instances that need the most iterations sit side by side, so that once the others have
  // converged the remaining ones share few memory sectors.  The interface keeps the caller's
  // order (lane_of maps it).
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    return desc->inst_omega[x] * desc->inst_omega[x] / desc->inst_k[x] <
           desc->inst_omega[y] * desc->inst_omega[y] / desc->inst_k[y];
  });
  bt->lane_of.assign(n, 0);
  for (int l = 0; l < n; ++l) bt->lane_of[order[l]] = l;
  bt->h_k.assign(nip, 1.0);
  bt->h_omega.assign(nip, 0.0);
  for (int l = 0; l < n; ++l) {
    bt->h_k[l] = desc->inst_k[order[l]];
    bt->h_omega[l] = desc->inst_omega[order[l]];
  }
  std::vector<std::pair<void **, size_t>> list;
  batch_bytes(p, list);
  for (auto &e : list) FO_TRY(fo_alloc(ctx, e.first, e.second));
  const size_t NN = (size_t)g.num_nodes;
  std::vector<double> w2(nip), fT(NN * nip, 0.0);
  for (int i = 0; i < nip; ++i) w2[i] = bt->h_omega[i] * bt->h_omega[i];
  for (int i = 0; i < n; ++i)
    for (size_t a = 0; a < NN; ++a) fT[a * nip + bt->lane_of[i]] = desc->inst_f[(size_t)i * NN + a];
  cudaStream_t s = ctx->stream;
  FO_CU(ctx, cudaMemcpyAsync(bt->kk, bt->h_k.data(), sizeof(double) * nip, cudaMemcpyHostToDevice, s));
  FO_CU(ctx, cudaMemcpyAsync(bt->w2, w2.data(), sizeof(double) * nip, cudaMemcpyHostToDevice, s));
  FO_CU(ctx, cudaMemcpyAsync(bt->f, fT.data(), sizeof(double) * NN * nip, cudaMemcpyHostToDevice, s));
  FO_CU(ctx, cudaMemsetAsync(bt->U, 0, sizeof(double) * NN * nip, s));
  FO_CU(ctx, cudaMemsetAsync(bt->P, 0, sizeof(double) * NN * nip, s));
  const int blocks = fo_blocks_for((long long)NN * nip, FO_BLOCK, 65536);
  if (g.dim == 2) k_batch_load<2><<<blocks, FO_BLOCK, 0, s>>>(g, p->dir, nip, bt->f, bt->B);
  else k_batch_load<3><<<blocks, FO_BLOCK, 0, s>>>(g, p->dir, nip, bt->f, bt->B);
  fo_note_launch(1);
  FO_CU(ctx, cudaGetLastError());
  FO_CU(ctx, cudaStreamSynchronize(s));   // the host staging buffers die here
  return FO_OK;
}

// WK, WM (FP64, node-major) of grid g from a per-element coefficient and Dirichlet mask; FP32
// copies when WK32 / WM32 are given.
void fo_launch_batch_stencil(cudaStream_t s, const Grid &g, const double *coef, const uint8_t *dir, double *WK,
                             double *WM, float *WK32, float *WM32) {
  const int blocks = fo_blocks_for(g.num_nodes, FO_BLOCK, 65536);
  if (g.dim == 2) k_batch_stencil<2><<<blocks, FO_BLOCK, 0, s>>>(g, coef, dir, WK, WM, WK32, WM32);
  else k_batch_stencil<3><<<blocks, FO_BLOCK, 0, s>>>(g, coef, dir, WK, WM, WK32, WM32);
  fo_note_launch(1);
}

fo_status fo_batch_prepare(fo_problem *p) {
  fo_batch *bt = p->batch;
  const Grid &g = p->mesh->g;
  cudaStream_t s = p->ctx->stream;
  fo_launch_batch_stencil(s, g, p->coef, p->dir, bt->WK, bt->WM, bt->WK32, bt->WM32);
  const int b2 = fo_blocks_for(g.num_nodes * bt->nip, FO_BLOCK, 65536);
  k_batch_dinv<<<b2, FO_BLOCK, 0, s>>>(g.num_nodes, batch_S(g), bt->nip, bt->WK, bt->WM, bt->kk, bt->w2, bt->dinv,
                                        bt->dinv32);
  fo_note_launch(1);
  FO_CU(p->ctx, cudaGetLastError());
  return FO_OK;
}

// ---- solver launch -------------------------------------------------------------------
// One compiled solver: dimension, instance slabs NJ (nip = 32 NJ), inner precision, tile.
struct BatchKernel {
  const void *fn = nullptr;
  size_t smem = 0;     // dynamic shared memory: the halo field, or the reduction scratch
  int tile[3] = {1, 1, 1};
};

template <int D, int NJ, typename T, int TS>
static BatchKernel batch_entry() {
  using TL = BatchTile<D, TS>;
  constexpr int NH = (TL::TX + 2) * (TL::TY + 2) * (D == 3 ? TL::TZ + 2 : 1);
  constexpr int NT = TL::TX * TL::TY * (D == 3 ? TL::TZ : 1);
  BatchKernel k;
  k.fn = (const void *)k_batch_solve<D, NJ, T, TS>;
  k.smem = std::max(((size_t)NH * 32 * NJ + (size_t)NT * 2 * ST<D>::S) * sizeof(T),
                    (size_t)BATCH_MAX_WARPS * 3 * 32 * NJ * sizeof(double));
  k.tile[0] = TL::TX;
  k.tile[1] = TL::TY;
  k.tile[2] = D == 3 ? TL::TZ : 1;
  return k;
}

#define FO_BATCH_TS(DD, NJJ, TT)                                 \
  if (ts == 0) return batch_entry<DD, NJJ, TT, 0>();             \
  return batch_entry<DD, NJJ, TT, 1>();
#define FO_BATCH_T(DD, NJJ)                                      \
  if (f32) { FO_BATCH_TS(DD, NJJ, float) } else { FO_BATCH_TS(DD, NJJ, double) }
static BatchKernel batch_kernel(int d, int nj, bool f32, int ts) {
  if (d == 2) {
    if (nj == 1) { FO_BATCH_T(2, 1) }
    if (nj == 2) { FO_BATCH_T(2, 2) }
    FO_BATCH_T(2, 4)
  }
  if (nj == 1) { FO_BATCH_T(3, 1) }
  if (nj == 2) { FO_BATCH_T(3, 2) }
  FO_BATCH_T(3, 4)
}
#undef FO_BATCH_T
#undef FO_BATCH_TS

// Largest dynamic shared memory a solver block may take (the per-block static part of the
// kernel is below 14 KB; 227 KB is the opt-in limit per block).
#define BATCH_SMEM_LIMIT (200 * 1024)

struct BatchLaunch {
  BatchKernel k;
  int block, grid;
};

template <typename T>
static size_t batch_scratch_bytes(long long nn, int nip, int grid) {
  return sizeof(double) * ((size_t)3 * nip * grid + 3 * nip) + sizeof(T) * 8 * (size_t)nn * nip + 256;
}

template <typename T>
static fo_status batch_launch_t(fo_problem *p, const double *B, double bscale, double *X, const fo_solve_opts *o,
                                const BatchLaunch &L, int warm) {
  fo_batch *bt = p->batch;
  fo_ctx *ctx = p->ctx;
  const Grid &g = p->mesh->g;
  const long long nn = g.num_nodes;
  const int nip = bt->nip;
  char *buf;
  FO_TRY(fo_scratch(p, batch_scratch_bytes<T>(nn, nip, L.grid), (void **)&buf));
  BatchArgs A{};
  A.g = g;
  A.B = B;
  A.bscale = bscale;
  A.X = X;
  A.WK = bt->WK;
  A.WM = bt->WM;
  A.kk = bt->kk;
  A.w2 = bt->w2;
  A.partials = (double *)buf;
  A.totals = A.partials + (size_t)3 * nip * L.grid;
  A.status = p->dev_status;
  A.bar = GridBar{p->bar, p->dev_status + DS_ERR, 2000000000ull};
  A.inst_iters = bt->inst_iters;
  A.inst_res = bt->inst_res;
  A.rtol2 = o->rtol * o->rtol;
  A.inner_rtol2 = o->inner_rtol * o->inner_rtol;
  A.maxit = o->maxit;
  A.inner_maxit = std::is_same<T, double>::value ? o->maxit : o->inner_maxit;
  A.warm = warm;
  T *v = (T *)(A.totals + 3 * nip);
  const size_t n = (size_t)nn * nip;
  BatchVecs<T> V;
  V.x = v;
  V.p = v + n;
  V.r[0] = v + 2 * n;
  V.r[1] = v + 3 * n;
  V.w[0] = v + 4 * n;
  V.w[1] = v + 5 * n;
  V.s[0] = v + 6 * n;
  V.s[1] = v + 7 * n;
  if (std::is_same<T, double>::value) {
    V.dinv = (const T *)bt->dinv;
    V.WK = (const T *)bt->WK;
    V.WM = (const T *)bt->WM;
  } else {
    V.dinv = (const T *)bt->dinv32;
    V.WK = (const T *)bt->WK32;
    V.WM = (const T *)bt->WM32;
  }
  FO_CU(ctx, cudaFuncSetAttribute(L.k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.k.smem));
  FO_CU(ctx, cudaMemsetAsync(p->bar, 0, 64, ctx->stream));
  FO_CU(ctx, cudaMemsetAsync(p->dev_status, 0, sizeof(int) * DS_COUNT, ctx->stream));
  void *argv[] = {(void *)&A, (void *)&V};
  FO_CU(ctx, cudaLaunchCooperativeKernel(L.k.fn, L.grid, L.block, argv, L.k.smem, ctx->stream));
  fo_note_launch(1);
  FO_CU(ctx, cudaGetLastError());
  return FO_OK;
}

static fo_status batch_dispatch(fo_problem *p, int precision, const double *B, double bscale, double *X,
                                const fo_solve_opts *o, const BatchLaunch &L, int warm) {
  if (precision == FO_MIXED) return batch_launch_t<float>(p, B, bscale, X, o, L, warm);
  return batch_launch_t<double>(p, B, bscale, X, o, L, warm);
}

static long long batch_ntiles(const Grid &g, const BatchKernel &k) {
  long long t = 1;
  for (int a = 0; a < g.dim; ++a) t *= (g.nn[a] + k.tile[a] - 1) / k.tile[a];
  return t;
}

// Co-resident blocks of a solver launch shape per SM (0: does not fit).
static int batch_occupancy(fo_problem *p, const BatchKernel &k, int block) {
  if (k.smem > BATCH_SMEM_LIMIT) return 0;
  if (cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem) != cudaSuccess) return 0;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k.fn, block, k.smem) != cudaSuccess) return 0;
  return per_sm;
}

// Launch shape: the autotuned one, or (explicit opts->grid_blocks, or before tuning) the
// first tile that fits with 256 threads and as many blocks as are co-resident.
static fo_status batch_shape(fo_problem *p, int precision, int requested, BatchLaunch *L) {
  fo_batch *bt = p->batch;
  const Grid &g = p->mesh->g;
  const int pi = precision == FO_MIXED ? 1 : 0;
  int ts = bt->tuned_ts[pi], block = bt->tuned_block[pi], bpsm = bt->tuned_bpsm[pi];
  if (requested > 0 || block == 0) {
    block = 256;
    bpsm = 0;
    ts = -1;
    for (int t = 0; t < 2 && ts < 0; ++t)
      if (batch_occupancy(p, batch_kernel(g.dim, bt->nip / 32, precision == FO_MIXED, t), block) > 0) ts = t;
    if (ts < 0) return fo_fail(p->ctx, FO_ECUDA, "no tile of the batched solver fits on an SM");
  }
  L->k = batch_kernel(g.dim, bt->nip / 32, precision == FO_MIXED, ts);
  const int per_sm = batch_occupancy(p, L->k, block);
  if (per_sm < 1) return fo_fail(p->ctx, FO_ECUDA, "batched solver does not fit on an SM");
  if (bpsm <= 0 || bpsm > per_sm) bpsm = per_sm;
  long long grid = requested > 0 ? requested : (long long)bpsm * p->ctx->num_sms;
  grid = std::min(grid, (long long)per_sm * p->ctx->num_sms);
  grid = std::min(grid, batch_ntiles(g, L->k));
  L->block = block;
  L->grid = (int)std::max(grid, 1LL);
  return FO_OK;
}

fo_status fo_batch_read(fo_problem *p, fo_solve_stats *st, const fo_solve_opts *o) {
  fo_ctx *ctx = p->ctx;
  FO_CU(ctx, cudaMemcpyAsync(ctx->h_scalars + 32, p->dev_status, sizeof(int) * DS_COUNT, cudaMemcpyDeviceToHost,
                             ctx->stream));
  std::vector<double> res(p->batch->nip);
  FO_CU(ctx, cudaMemcpyAsync(res.data(), p->batch->inst_res, sizeof(double) * p->batch->nip, cudaMemcpyDeviceToHost,
                             ctx->stream));
  FO_CU(ctx, cudaStreamSynchronize(ctx->stream));
  const int *hs = (const int *)(ctx->h_scalars + 32);
  if (st) {
    st->iterations = hs[DS_ITERS];
    st->operator_applies = hs[DS_APPLIES];
    st->outer_iterations = hs[DS_FLAG];
    double mx = 0;
    for (int i = 0; i < p->batch->n_inst; ++i) mx = std::max(mx, res[i]);
    st->rel_residual = mx;
  }
  if (hs[DS_ERR] == DEV_TIMEOUT) return fo_fail(ctx, FO_ETIMEOUT, "grid barrier timed out in the batched solve");
  if (hs[DS_ERR] == DEV_NAN) return fo_fail(ctx, FO_ENAN, "NaN in the batched solve");
  if (hs[DS_ERR] == DEV_NOCONV)
    return fo_fail(ctx, FO_ENOCONV, "batched solve stopped at maxit=%d (max relative residual %.3e)", o->maxit,
                   st ? st->rel_residual : 0.0);
  return FO_OK;
}

extern "C" fo_status fo_batch_autotune(fo_problem *p, int precision, fo_tune_result *out) {
  if (!p || (precision != FO_FP64 && precision != FO_MIXED)) return FO_EINVAL;
  if (!p->batch) return fo_fail(p->ctx, FO_EINVAL, "not a batch problem");
  fo_ctx *ctx = p->ctx;
  fo_batch *bt = p->batch;
  const Grid &g = p->mesh->g;
  if (!p->coef_valid) FO_TRY(fo_coefficients(p));
  const size_t nx = (size_t)g.num_nodes * bt->nip;
  double *X;
  FO_TRY(fo_alloc(ctx, (void **)&X, sizeof(double) * nx));
  fo_solve_opts o;
  fo_solve_opts_default(&o);
  const int ITERS = 40;
  o.rtol = 0.0;              // never met: every candidate runs the same ITERS iterations
  o.inner_rtol = 0.0;
  o.maxit = ITERS;
  o.inner_maxit = ITERS;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int best_ts = -1, best_block = 0, best_bpsm = 0, cand = 0;
  double best = INFINITY;
  fo_status st = FO_OK;
  const int blocks[2] = {128, 256};
  for (int ts = 0; ts < 2 && st == FO_OK; ++ts)
    for (int bi = 0; bi < 2 && st == FO_OK; ++bi) {
      BatchLaunch L;
      L.k = batch_kernel(g.dim, bt->nip / 32, precision == FO_MIXED, ts);
      L.block = blocks[bi];
      const int per_sm = batch_occupancy(p, L.k, L.block);
      for (int bpsm = 1; bpsm <= std::min(per_sm, 4) && st == FO_OK; ++bpsm) {
        L.grid = (int)std::min((long long)bpsm * ctx->num_sms, batch_ntiles(g, L.k));
        float ms = 0;
        for (int rep = 0; rep < 2 && st == FO_OK; ++rep) {
          cudaEventRecord(e0, ctx->stream);
          st = batch_dispatch(p, precision, bt->B, 1.0, X, &o, L, 0);
          cudaEventRecord(e1, ctx->stream);
          if (st == FO_OK) {
            fo_status r = fo_batch_read(p, nullptr, &o);
            if (r != FO_OK && r != FO_ENOCONV) st = r;
          }
        }
        if (st != FO_OK) break;
        cudaEventElapsedTime(&ms, e0, e1);
        ++cand;
        if (ms < best) {
          best = ms;
          best_ts = ts;
          best_block = L.block;
          best_bpsm = bpsm;
        }
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  fo_free(ctx, X, sizeof(double) * nx);
  if (st != FO_OK) return st;
  if (cand == 0) return fo_fail(ctx, FO_ECUDA, "no launch shape of the batched solver fits");
  const int pi = precision == FO_MIXED ? 1 : 0;
  bt->tuned_ts[pi] = best_ts;
  bt->tuned_block[pi] = best_block;
  bt->tuned_bpsm[pi] = best_bpsm;
  bt->tuned_us[pi] = best * 1000.0 / ITERS;
  if (out) {
    const BatchKernel k = batch_kernel(g.dim, bt->nip / 32, precision == FO_MIXED, best_ts);
    out->block = best_block;
    out->blocks_per_sm = best_bpsm;
    out->us_per_iteration = bt->tuned_us[pi];
    out->candidates = cand;
    out->tile[0] = k.tile[0];
    out->tile[1] = k.tile[1];
    out->tile[2] = k.tile[2];
  }
  return FO_OK;
}

fo_status fo_batch_state(fo_problem *p, bool adjoint, const fo_solve_opts *o, fo_solve_stats *st) {
  fo_batch *bt = p->batch;
  double *X = adjoint ? bt->P : bt->U;
  if (o->precond == FO_PC_MG && fo_mg_applicable(p->mesh->g, 1, false))
    return fo_batch_state_mg(p, bt->B, adjoint ? -1.0 : 1.0, X, o, adjoint ? 0 : o->warm_start, st);
  const int prec = o->precision == FO_MIXED ? FO_MIXED : FO_FP64;
  if (o->grid_blocks <= 0 && bt->tuned_block[prec == FO_MIXED ? 1 : 0] == 0) FO_TRY(fo_batch_autotune(p, prec, nullptr));
  BatchLaunch L;
  FO_TRY(batch_shape(p, prec, o->grid_blocks, &L));
  FO_TRY(batch_dispatch(p, prec, bt->B, adjoint ? -1.0 : 1.0, X, o, L, adjoint ? 0 : o->warm_start));
  fo_solve_stats s;
  memset(&s, 0, sizeof s);
  fo_status r = fo_batch_read(p, &s, o);
  if (st) *st = s;
  return r;
}

fo_status fo_batch_functionals(fo_problem *p, double *J, double *vol, double *J_inst) {
  fo_batch *bt = p->batch;
  fo_ctx *ctx = p->ctx;
  const Grid &g = p->mesh->g;
  const int nip = bt->nip, G = 256;
  // partials [G][nip] + volume [G] + results [nip + 1] in the problem's reduction buffer
  if ((size_t)G * nip + G + nip + 1 > FO_RED_DOUBLES) return fo_fail(ctx, FO_EINVAL, "batch too large");
  double *part = p->red, *volp = part + (size_t)G * nip, *res = volp + G;
  const int nj = nip / 32;
  if (nj == 1) k_batch_costs<1><<<G, 256, 0, ctx->stream>>>(g.num_nodes, bt->B, bt->U, part);
  else if (nj == 2) k_batch_costs<2><<<G, 256, 0, ctx->stream>>>(g.num_nodes, bt->B, bt->U, part);
  else k_batch_costs<4><<<G, 256, 0, ctx->stream>>>(g.num_nodes, bt->B, bt->U, part);
  k_batch_volume<<<G, 256, 0, ctx->stream>>>(g.num_elems, g.vol_e, p->chi, volp);
  k_batch_costs_finish<<<(nip + 1 + 127) / 128, 128, 0, ctx->stream>>>(G, nip, part, volp, res);
  fo_note_launch(3);
  FO_CU(ctx, cudaGetLastError());
  std::vector<double> h(nip + 1);
  FO_CU(ctx, cudaMemcpyAsync(h.data(), res, sizeof(double) * (nip + 1), cudaMemcpyDeviceToHost, ctx->stream));
  FO_CU(ctx, cudaStreamSynchronize(ctx->stream));
  double tot = 0;
  for (int i = 0; i < bt->n_inst; ++i) tot += h[i];
  if (J) *J = tot;
  if (vol) *vol = h[nip];
  if (J_inst)
    for (int i = 0; i < bt->n_inst; ++i) J_inst[i] = h[bt->lane_of[i]];
  return FO_OK;
}

fo_status fo_batch_shape_rhs(fo_problem *p, double lambda) {
  fo_batch *bt = p->batch;
  const Grid &g = p->mesh->g;
  const double V = p->desc.volume_target > 0 ? p->desc.volume_target : 1.0;
  const double lv = lambda / V;
  const int nw = 8, blocks = fo_blocks_for(g.num_nodes, nw, 65536);
  cudaStream_t s = p->ctx->stream;
  const int nj = bt->nip / 32;
#define FO_SHAPE_CASE(DD, NJJ)                                                                                 \
  if (g.dim == DD && nj == NJJ)                                                                               \
    k_batch_shape<DD, NJJ><<<blocks, 32 * nw, 0, s>>>(g, p->coef, p->chi, bt->U, bt->f, bt->kk, bt->w2, lv, p->rhs);
  FO_SHAPE_CASE(2, 1) FO_SHAPE_CASE(2, 2) FO_SHAPE_CASE(2, 4)
  FO_SHAPE_CASE(3, 1) FO_SHAPE_CASE(3, 2) FO_SHAPE_CASE(3, 4)
#undef FO_SHAPE_CASE
  fo_note_launch(1);
  FO_CU(p->ctx, cudaGetLastError());
  return FO_OK;
}

// y = K_i x on instance-minor device arrays [N_n][nip]; fp32: the FP32 stencils.
fo_status fo_batch_apply(fo_problem *p, const double *x, double *y, bool fp32) {
  fo_batch *bt = p->batch;
  const Grid &g = p->mesh->g;
  const int nw = 8, blocks = fo_blocks_for(g.num_nodes, nw, 65536);
  cudaStream_t s = p->ctx->stream;
  const int nj = bt->nip / 32;
#define FO_APPLY_CASE(DD, NJJ)                                                                                    \
  if (g.dim == DD && nj == NJJ) {                                                                                \
    if (fp32) k_batch_apply<DD, NJJ, float><<<blocks, 32 * nw, 0, s>>>(g, bt->WK32, bt->WM32, bt->kk, bt->w2, x, y); \
    else k_batch_apply<DD, NJJ, double><<<blocks, 32 * nw, 0, s>>>(g, bt->WK, bt->WM, bt->kk, bt->w2, x, y);        \
  }
  FO_APPLY_CASE(2, 1) FO_APPLY_CASE(2, 2) FO_APPLY_CASE(2, 4)
  FO_APPLY_CASE(3, 1) FO_APPLY_CASE(3, 2) FO_APPLY_CASE(3, 4)
#undef FO_APPLY_CASE
  fo_note_launch(1);
  FO_CU(p->ctx, cudaGetLastError());
  return FO_OK;
}

extern "C" fo_status fo_batch_costs(fo_problem *p, double *J_inst) {
  if (!p || !J_inst) return FO_EINVAL;
  if (!p->batch) return fo_fail(p->ctx, FO_EINVAL, "not a batch problem");
  if (!p->coef_valid) FO_TRY(fo_coefficients(p));
  return fo_batch_functionals(p, nullptr, nullptr, J_inst);
}

extern "C" fo_status fo_batch_solve_info(fo_problem *p, int *inst_iters, double *inst_res) {
  if (!p) return FO_EINVAL;
  if (!p->batch) return fo_fail(p->ctx, FO_EINVAL, "not a batch problem");
  fo_ctx *ctx = p->ctx;
  fo_batch *bt = p->batch;
  std::vector<int> it(bt->nip);
  std::vector<double> res(bt->nip);
  FO_CU(ctx, cudaMemcpyAsync(it.data(), bt->inst_iters, sizeof(int) * bt->nip, cudaMemcpyDeviceToHost, ctx->stream));
  FO_CU(ctx, cudaMemcpyAsync(res.data(), bt->inst_res, sizeof(double) * bt->nip, cudaMemcpyDeviceToHost, ctx->stream));
  FO_CU(ctx, cudaStreamSynchronize(ctx->stream));
  for (int i = 0; i < bt->n_inst; ++i) {
    if (inst_iters) inst_iters[i] = it[bt->lane_of[i]];
    if (inst_res) inst_res[i] = res[bt->lane_of[i]];
  }
  return FO_OK;
}
