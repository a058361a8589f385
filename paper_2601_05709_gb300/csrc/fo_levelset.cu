// Level-set transport (SUPG / Crank-Nicolson, Sec. 5.6) and reinitialisation (Sec. 5.7).
//
// The transport matrices L, R and the reinitialisation matrix change with theta / phi, so
// they are assembled (node-centrically, deterministic) into stencil form: for every node the
// 7 (2D) / 15 (3D) couplings to its Kuhn neighbours, stored slot-major [S][N_n] so that a
// warp reads consecutive nodes of one slot.  The nonsymmetric systems are solved by a
// persistent, cooperatively launched restarted GMRES; one launch runs every substep.
//
// Quadrature: degree-2 rule (2D: barycentrics (2/3, 1/6, 1/6) and permutations, weights
// |e|/3; 3D: (a, b, b, b), a = (5 + 3 sqrt 5)/20, b = (5 - sqrt 5)/20, weights |e|/4).
#include <cmath>
#include <cstring>

#include "fo_internal.cuh"
#include "fo_ops.cuh"

template <int D>
__device__ __forceinline__ double qbary(int q, int l) {
  if (D == 2) return q == l ? 2.0 / 3.0 : 1.0 / 6.0;
  const double a = 0.58541019662496845446;   // (5 + 3 sqrt 5) / 20
  const double b = 0.13819660112501051518;   // (5 - sqrt 5) / 20
  return q == l ? a : b;
}

// grad lambda_l of simplex p, component k (sparse Kuhn form)
template <int D>
__device__ __forceinline__ double kgrad(const Grid &g, int p, int l, int k) {
  double v = 0;
  if (l >= 1 && kperm<D>(p, l - 1) == k) v += g.inv_h[k];
  if (l < D && kperm<D>(p, l) == k) v -= g.inv_h[k];
  return v;
}

// ------------------------------------------------------------------- transport assembly
// Row m (test function psi^_m) of the element matrices of eq. weak_transport:
//   L = M^ + dt/2 (A + s K^),  R = M^ - dt/2 (A + s K^),
//   M^_ml = int lambda_l psi^_m,  A_ml = int (theta . grad lambda_l) psi^_m,
//   K^_ml = int h^2 grad lambda_l . grad psi^_m,
//   psi^_m = lambda_m + tau theta . grad lambda_m,
//   grad psi^_m = grad lambda_m + (theta . grad lambda_m) grad tau + tau (D theta)^T grad lambda_m.
template <int D>
__global__ void k_transport_assemble(Grid g, const double *theta, double dt, double h, int smooth, double *L,
                                     double *R, double *dinvL) {
  constexpr int S = ST<D>::S;
  const long long N = g.num_nodes;
  for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < N; a += (long long)gridDim.x * blockDim.x) {
    int idx[3];
    node_ijk(g, a, idx);
    double th[S][D];
    load_stencil<D, D, double>(g, idx, a, VecX<double>{theta}, th);
    double Ls[S], Rs[S];
#pragma unroll
    for (int s = 0; s < S; ++s) Ls[s] = Rs[s] = 0.0;
    const double vol = g.vol_e, h2 = h * h, idt2 = 1.0 / (dt * dt), ih2 = 1.0 / h2;
#pragma unroll
    for (int p = 0; p < KP<D>::P; ++p)
#pragma unroll
      for (int m = 0; m <= D; ++m) {
        long long e;
        if (!elem_of<D>(g, idx, p, m, e)) continue;
        int sl[D + 1];
#pragma unroll
        for (int l = 0; l <= D; ++l) sl[l] = rel_slot<D>(p, m, l);
        double Dth[D][D];   // Dth[i][k] = d_k theta_i
#pragma unroll
        for (int l = 0; l < D; ++l) {
          const int ax = kperm<D>(p, l);
#pragma unroll
          for (int i = 0; i < D; ++i) Dth[i][ax] = (th[sl[l + 1]][i] - th[sl[l]][i]) * g.inv_h[ax];
        }
        double Lrow[D + 1], Rrow[D + 1];
#pragma unroll
        for (int l = 0; l <= D; ++l) Lrow[l] = Rrow[l] = 0.0;
#pragma unroll
        for (int q = 0; q <= D; ++q) {
          double thq[D];
#pragma unroll
          for (int i = 0; i < D; ++i) {
            double t = 0;
#pragma unroll
            for (int l = 0; l <= D; ++l) t += qbary<D>(q, l) * th[sl[l]][i];
            thq[i] = t;
          }
          double n2 = 0;
#pragma unroll
          for (int i = 0; i < D; ++i) n2 += thq[i] * thq[i];
          const double s = idt2 + n2 * ih2;
          const double rs = sqrt(s);
          const double tau = 0.5 / rs;
          const double c = -0.5 / (s * rs) * ih2;
          double gtau[D];
#pragma unroll
          for (int k = 0; k < D; ++k) {
            double t = 0;
#pragma unroll
            for (int j = 0; j < D; ++j) t += Dth[j][k] * thq[j];
            gtau[k] = c * t;
          }
          double thg[D + 1];
#pragma unroll
          for (int l = 0; l <= D; ++l) {
            double t = 0;
#pragma unroll
            for (int k = 0; k < D; ++k) t += thq[k] * kgrad<D>(g, p, l, k);
            thg[l] = t;
          }
          const double test = qbary<D>(q, m) + tau * thg[m];
          double gtest[D];
#pragma unroll
          for (int k = 0; k < D; ++k) {
            double t = 0;
#pragma unroll
            for (int j = 0; j < D; ++j) t += Dth[j][k] * kgrad<D>(g, p, m, j);
            gtest[k] = kgrad<D>(g, p, m, k) + thg[m] * gtau[k] + tau * t;
          }
          const double wv = vol / (D + 1);
#pragma unroll
          for (int l = 0; l <= D; ++l) {
            const double mh = wv * test * qbary<D>(q, l);
            const double ad = wv * test * thg[l];
            double df = 0;
            if (smooth) {
              double t = 0;
#pragma unroll
              for (int k = 0; k < D; ++k) t += gtest[k] * kgrad<D>(g, p, l, k);
              df = wv * h2 * t;
            }
            Lrow[l] += mh + 0.5 * dt * (ad + df);
            Rrow[l] += mh - 0.5 * dt * (ad + df);
          }
        }
#pragma unroll
        for (int l = 0; l <= D; ++l) {
          Ls[sl[l]] += Lrow[l];
          Rs[sl[l]] += Rrow[l];
        }
      }
#pragma unroll
    for (int s = 0; s < S; ++s) {
      L[s * N + a] = Ls[s];
      R[s * N + a] = Rs[s];
    }
    dinvL[a] = 1.0 / Ls[0];
  }
}

fo_status fo_launch_transport_assemble(fo_problem *p, double dt, double h, int smooth) {
  const Grid &g = p->mesh->g;
  int blocks = fo_blocks_for(g.num_nodes, FO_BLOCK, 65536);
  if (g.dim == 2)
    k_transport_assemble<2><<<blocks, FO_BLOCK, 0, p->ctx->stream>>>(g, p->theta, dt, h, smooth, p->L, p->R, p->dinvL);
  else
    k_transport_assemble<3><<<blocks, FO_BLOCK, 0, p->ctx->stream>>>(g, p->theta, dt, h, smooth, p->L, p->R, p->dinvL);
  fo_note_launch(1);
  FO_CU(p->ctx, cudaGetLastError());
  return FO_OK;
}

// ----------------------------------------------------------------------- stencil apply
template <int D, class X>
__device__ __forceinline__ double stencil_row(const Grid &g, const double *M, long long a, const int idx[3], const X &x) {
  double acc = 0;
#pragma unroll
  for (int s = 0; s < ST<D>::S; ++s) {
    acc += M[s * g.num_nodes + a] * x(slot_node_or_self<D>(g, idx, a, s));
  }
  return acc;
}

template <int D>
__global__ void k_stencil_apply(Grid g, const double *M, const double *x, double *y) {
  for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < g.num_nodes;
       a += (long long)gridDim.x * blockDim.x) {
    int idx[3];
    node_ijk(g, a, idx);
    y[a] = stencil_row<D>(g, M, a, idx, VecX<double>{x});
  }
}

fo_status fo_launch_stencil_apply(fo_problem *p, const double *S, const double *x, double *y) {
  const Grid &g = p->mesh->g;
  int blocks = fo_blocks_for(g.num_nodes, FO_BLOCK, 65536);
  if (g.dim == 2) k_stencil_apply<2><<<blocks, FO_BLOCK, 0, p->ctx->stream>>>(g, S, x, y);
  else k_stencil_apply<3><<<blocks, FO_BLOCK, 0, p->ctx->stream>>>(g, S, x, y);
  fo_note_launch(1);
  FO_CU(p->ctx, cudaGetLastError());
  return FO_OK;
}

// --------------------------------------------------------------------- persistent GMRES
// Restarted GMRES(GM_M) with right Jacobi preconditioning on a stencil matrix.  The
// Petrov-Galerkin matrices of the transport and, above all, of the reinitialisation are far
// from normal (the streamline term is about half the size of the mass term), where
// BiCGStab breaks down; GMRES minimises the residual and cannot.  Arnoldi uses classical
// Gram-Schmidt with one reorthogonalisation pass (CGS2), each pass one fused grid
// reduction; the Hessenberg matrix, Givens rotations and the small triangular solve live in
// shared memory and are computed identically by every block from the same reduction totals.
#define GM_M 16
#define GM_ONEPASS 1e-3   // one Gram-Schmidt pass while |w - V h|^2 >= GM_ONEPASS |w|^2
#define GM_NR (GM_M + 2)

struct KrylovBufs {
  double *V;             // (GM_M + 1) basis vectors [GM_M + 1][N]
  double *w;             // [N]
  double *rhs;           // [N]
};

template <int NR>
__device__ __forceinline__ bool ls_reduce(double (&v)[NR], double *sred, double *stot, double *partials, int &rk,
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

struct GmresShared {
  double sred[32 * GM_NR];
  double stot[GM_NR];
  double col[GM_M + 1];          // the new Hessenberg column (before the rotations)
  double H[(GM_M + 1) * GM_M];   // column-major: H[j * (GM_M + 1) + i]
  double cs[GM_M], sn[GM_M], g[GM_M + 1], y[GM_M];
  double scal[2];                // a step's |w - V h| and its inverse (formed by warp 0)
  int onepass;                   // the step takes one Gram-Schmidt pass
};

// One thread (thread 32, during the grid barrier after the step's pass): apply the previous
// rotations to column j (col[0..j+1]), form the new one, update the residual estimate g and
// store the rotated column in H.
__device__ __noinline__ void givens_column(GmresShared &sh, int j, double *col) {
  for (int i = 0; i < j; ++i) {
    const double t = sh.cs[i] * col[i] + sh.sn[i] * col[i + 1];
    col[i + 1] = -sh.sn[i] * col[i] + sh.cs[i] * col[i + 1];
    col[i] = t;
  }
  // c, s from one reciprocal norm (no quotients on this serial chain)
  const double a = col[j], b = col[j + 1];
  double c = 1.0, s = 0.0, rnorm = 0.0;
  if (a != 0.0 || b != 0.0) {
    const double rh = rhypot(a, b);
    if (rh >= 1.0e-300 && rh <= 1.0e300) {
      c = a * rh;
      s = b * rh;
      rnorm = a * c + b * s;
    } else {   // |(a, b)| below 1e-300 or above 1e300: the reciprocal would overflow or be subnormal
      rnorm = hypot(a, b);
      c = a / rnorm;
      s = b / rnorm;
    }
  }
  sh.cs[j] = c;
  sh.sn[j] = s;
  col[j] = rnorm;
  col[j + 1] = 0.0;
  sh.g[j + 1] = -s * sh.g[j];
  sh.g[j] = c * sh.g[j];
  for (int i = 0; i <= j; ++i) sh.H[j * (GM_M + 1) + i] = col[i];
}

// One Arnoldi step at compile-time index J: w = M D^{-1} v_J, classical Gram-Schmidt against
// v_0..v_J (one fused grid reduction of the J + 1 dot products and |w|^2), a second pass only
// when the first one left less than GM_ONEPASS of |w|^2 (a Daniel-Gragg-Kaufman-Stewart
// test with a smaller threshold than their 1/2: the mass-dominated transport operators are
// near the identity, so the first projection always removes most of w; above the threshold
// |w - V h|^2 = |w|^2 - |h|^2 loses at most log10(1/GM_ONEPASS) digits to cancellation and the
// basis vector's error is at most eps / sqrt(GM_ONEPASS) of its norm), and v_{J+1} = w' / |w'|.  Every loop runs over
// exactly the J + 1 basis vectors, so no lane issues work for vectors that do not exist yet.
// Leaves the column (h_0..h_J, |w'|) in sh.col.
template <int D, int J>
__device__ bool arnoldi_step(const Grid &g, const double *M, const double *dinv, const KrylovBufs &K,
                             GmresShared &sh, double *partials, int &rk, const GridBar &bar) {
  const long long N = g.num_nodes;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long gs = (long long)gridDim.x * blockDim.x;
  const double *Vj = K.V + (size_t)J * N;
  double h1[J + 2];
#pragma unroll
  for (int i = 0; i < J + 2; ++i) h1[i] = 0.0;
  for (long long a = tid; a < N; a += gs) {
    // the basis entries first: their loads then overlap the stencil's instead of waiting
    // behind the store of w (which the compiler cannot prove distinct from V)
    double va[J + 1];
#pragma unroll
    for (int i = 0; i <= J; ++i) va[i] = K.V[(size_t)i * N + a];
    int idx[3];
    node_ijk(g, a, idx);
    double wa = 0.0;
#pragma unroll
    for (int s = 0; s < ST<D>::S; ++s) {
      const long long nb = slot_node_or_self<D>(g, idx, a, s);
      wa += M[s * N + a] * (dinv[nb] * Vj[nb]);
    }
    K.w[a] = wa;
#pragma unroll
    for (int i = 0; i <= J; ++i) h1[i] += va[i] * wa;
    h1[J + 1] += wa * wa;
  }
  if (!ls_reduce<J + 2>(h1, sh.sred, sh.stot, partials, rk, bar)) return false;
  // the step's scalars once per block, by warp 0 (the FP64 pipe is narrow: 256 threads
  // forming the same square root and quotient cost more than the pass over the vectors, and a
  // single thread's serial chain waits on FP64 latency): |h|^2 by a warp sum, then one
  // reciprocal square root for |w - V h| and its inverse
  if (threadIdx.x < 32) {
    const int l = threadIdx.x;
    double hh = l <= J ? sh.stot[l] * sh.stot[l] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) hh += __shfl_xor_sync(0xffffffffu, hh, o);
    if (l == 0) {
      const double ww = sh.stot[J + 1], wp2 = ww - hh;
      sh.onepass = wp2 >= GM_ONEPASS * ww;
      const double r = (sh.onepass && wp2 > 0.0) ? rsqrt(wp2) : 0.0;
      sh.scal[0] = wp2 * r;
      sh.scal[1] = r;
    }
  }
  __syncthreads();
  double hc[J + 1];
#pragma unroll
  for (int i = 0; i <= J; ++i) hc[i] = sh.stot[i];
  if (sh.onepass) {   // one pass: v_{J+1} = (w - V h) / |w - V h|
    const double hnext = sh.scal[0];
    const double inv = sh.scal[1];
    double *Vn = K.V + (size_t)(J + 1) * N;
    for (long long a = tid; a < N; a += gs) {
      double wa = K.w[a];
#pragma unroll
      for (int i = 0; i <= J; ++i) wa -= hc[i] * K.V[(size_t)i * N + a];
      Vn[a] = wa * inv;
    }
    if (threadIdx.x == 0) {
#pragma unroll
      for (int i = 0; i <= J; ++i) sh.col[i] = hc[i];
      sh.col[J + 1] = hnext;
    }
    return true;
  }
  double h2[J + 2];
#pragma unroll
  for (int i = 0; i < J + 2; ++i) h2[i] = 0.0;
  for (long long a = tid; a < N; a += gs) {
    double wa = K.w[a];
#pragma unroll
    for (int i = 0; i <= J; ++i) wa -= hc[i] * K.V[(size_t)i * N + a];
    K.w[a] = wa;
#pragma unroll
    for (int i = 0; i <= J; ++i) h2[i] += K.V[(size_t)i * N + a] * wa;
    h2[J + 1] += wa * wa;
  }
  if (!ls_reduce<J + 2>(h2, sh.sred, sh.stot, partials, rk, bar)) return false;
  double hn2 = sh.stot[J + 1];
  double h2c[J + 1];
#pragma unroll
  for (int i = 0; i <= J; ++i) {
    h2c[i] = sh.stot[i];
    hc[i] += h2c[i];
    hn2 -= h2c[i] * h2c[i];
  }
  const double hnext = sqrt(fmax(hn2, 0.0));
  double *Vn = K.V + (size_t)(J + 1) * N;
  const double inv = hnext > 0.0 ? 1.0 / hnext : 0.0;
  for (long long a = tid; a < N; a += gs) {
    double wa = K.w[a];
#pragma unroll
    for (int i = 0; i <= J; ++i) wa -= h2c[i] * K.V[(size_t)i * N + a];
    Vn[a] = wa * inv;
  }
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i <= J; ++i) sh.col[i] = hc[i];
    sh.col[J + 1] = hnext;
  }
  return true;
}

template <int D, int J>
__device__ __forceinline__ bool arnoldi_dispatch(int j, const Grid &g, const double *M, const double *dinv,
                                                 const KrylovBufs &K, GmresShared &sh, double *partials, int &rk,
                                                 const GridBar &bar) {
  if constexpr (J + 1 < GM_M) {
    if (j != J) return arnoldi_dispatch<D, J + 1>(j, g, M, dinv, K, sh, partials, rk, bar);
  }
  return arnoldi_step<D, J>(g, M, dinv, K, sh, partials, rk, bar);
}

// Solve M x = rhs (x holds the start value).  When Rm is given, the first residual pass
// also forms rhs = Rm x (the transport's right-hand side R phi^n, gathered from the same
// x before it changes).  With prev given (a sequence of solves, x = phi^n, prev = phi^{n-1},
// prev2 = phi^{n-2}), the solve starts from the polynomial extrapolation of order `order`
// (0: phi^n; 1: 2 phi^n - phi^{n-1}; 2: 3 phi^n - 3 phi^{n-1} + phi^{n-2}) and shifts the
// history for the next one.  Returns the number of Arnoldi steps; err / ok report failures.
template <int D>
__device__ int gmres_solve(const Grid &g, const double *M, const double *dinv, const double *Rm, double *x,
                           KrylovBufs K, double rtol2, int maxit, GmresShared &sh, double *partials, int &rk,
                           const GridBar &bar, int *err, bool *ok, double *prev = nullptr, double *prev2 = nullptr,
                           int order = 0) {
  auto start = [&](long long k) {
    const double xv = x[k];
    return order == 0 ? xv : (order == 1 ? 2.0 * xv - prev[k] : 3.0 * (xv - prev[k]) + prev2[k]);
  };
  const long long N = g.num_nodes;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long gs = (long long)gridDim.x * blockDim.x;
  int total = 0;
  double bb = -1.0;
  *ok = true;
  for (int cycle = 0;; ++cycle) {
    // ---- true residual r = rhs - M x into V_0 (and rhs = Rm x on the first cycle)
    double v2[2] = {0.0, 0.0};
    for (long long a = tid; a < N; a += gs) {
      int idx[3];
      node_ijk(g, a, idx);
      double ra;
      if (cycle == 0 && Rm) {
        ra = 0.0;
        double la = 0.0;
#pragma unroll
        for (int s = 0; s < ST<D>::S; ++s) {
          const long long nb = slot_node_or_self<D>(g, idx, a, s);
          const double xv = x[nb];
          ra += Rm[s * N + a] * xv;
          la += M[s * N + a] * (order == 0 ? xv : start(nb));
        }
        K.rhs[a] = ra;
        ra = ra - la;
        if (prev) K.w[a] = start(a);   // the start value
      } else {
        double la = 0.0;
#pragma unroll
        for (int s = 0; s < ST<D>::S; ++s) {
          la += M[s * N + a] * x[slot_node_or_self<D>(g, idx, a, s)];
        }
        ra = K.rhs[a] - la;
      }
      K.V[a] = ra;
      v2[0] += ra * ra;
      if (cycle == 0) v2[1] += K.rhs[a] * K.rhs[a];
    }
    if (!ls_reduce<2>(v2, sh.sred, sh.stot, partials, rk, bar)) { *ok = false; return total; }
    const double rr = sh.stot[0];
    if (cycle == 0) bb = sh.stot[1];
    if (!(rr == rr)) { *err = DEV_NAN; return total; }
    const bool conv = rr <= rtol2 * bb;
    if (cycle == 0 && Rm && prev) {   // x <- the start value, prev <- phi^n (own nodes)
      for (long long a = tid; a < N; a += gs) {
        prev2[a] = prev[a];
        prev[a] = x[a];
        x[a] = K.w[a];
      }
      if (conv && !grid_sync(bar)) { *ok = false; return total; }
    }
    if (conv) return total;
    if (total >= maxit) { *err = DEV_NOCONV; return total; }
    if (threadIdx.x == 0) {   // beta = |r| and its inverse, once per block
      const double beta = sqrt(rr);
      sh.g[0] = beta;
      sh.scal[1] = 1.0 / beta;
      for (int i = 1; i <= GM_M; ++i) sh.g[i] = 0.0;
    }
    __syncthreads();
    const double ib = sh.scal[1];
    for (long long a = tid; a < N; a += gs) K.V[a] *= ib;
    if (!grid_sync(bar)) { *ok = false; return total; }
    int j = 0;
    bool done = false;
    for (; j < GM_M; ++j) {
      __syncthreads();
      if (!arnoldi_dispatch<D, 0>(j, g, M, dinv, K, sh, partials, rk, bar)) { *ok = false; return total; }
      // v_{j+1} complete before the next apply.  Meanwhile thread 32 rotates the Hessenberg
      // column and updates the residual estimate (the same in every block): a serial FP64
      // chain that would otherwise hold up its warp's share of the pass
      const int jj = j;
      if (!grid_sync_side(bar, [&] {
            double col[GM_M + 1];
            for (int i = 0; i <= jj + 1; ++i) col[i] = sh.col[i];
            givens_column(sh, jj, col);
          })) { *ok = false; return total; }
      const double hnext = sh.col[j + 1];
      ++total;
      const double est = sh.g[j + 1] * sh.g[j + 1];
      done = !(est > rtol2 * bb) || hnext == 0.0 || total >= maxit;
      if (done) { ++j; break; }
    }
    if (j > GM_M) j = GM_M;
    // ---- y = H^{-1} g (upper triangular, j x j), x += D^{-1} V y
    // back substitution by columns in warp 0: lane k holds g_k less the solved terms and
    // the reciprocal of H_kk; y_i = t_i / H_ii goes to every lane, which subtracts its H_ki y_i
    if (threadIdx.x < 32) {
      const int k = threadIdx.x;
      double t = k < j ? sh.g[k] : 0.0;
      const double d = k < j ? sh.H[k * (GM_M + 1) + k] : 0.0;
      const double rinv = d != 0.0 ? 1.0 / d : 0.0;
      double yk = 0.0;
      for (int i = j - 1; i >= 0; --i) {
        const double yi = __shfl_sync(0xffffffffu, t * rinv, i);
        if (k == i) yk = yi;
        if (k < i) t -= sh.H[i * (GM_M + 1) + k] * yi;
      }
      if (k < j) sh.y[k] = yk;
    }
    __syncthreads();
    for (long long a = tid; a < N; a += gs) {
      double s = 0.0;
      for (int i = 0; i < j; ++i) s += sh.y[i] * K.V[(size_t)i * N + a];
      x[a] += dinv[a] * s;
    }
    if (!grid_sync(bar)) { *ok = false; return total; }   // x complete before the residual pass
  }
}

struct TransportArgs {
  KrylovBufs K;
  const double *L, *R, *dinv;
  double *phi;
  double *prev, *prev2;  // the two previous substeps' level sets (start-value extrapolation)
  double rtol2;
  int maxit, nsteps;
  double *partials;
  int *status;
  GridBar bar;
};

template <int D>
__global__ void __launch_bounds__(FO_BLOCK) k_transport_run(Grid g, TransportArgs A) {
  __shared__ GmresShared sh;
  int rk = 0, err = DEV_OK, total = 0;
  bool ok = true;
  for (int step = 0; step < A.nsteps && err == DEV_OK; ++step) {
    // L phi^{n+1} = R phi^n, started from phi^n (first substep), then from the linear and
    // the quadratic extrapolation of the previous level sets; rhs is formed in the first
    // residual pass
    total += gmres_solve<D>(g, A.L, A.dinv, A.R, A.phi, A.K, A.rtol2, A.maxit, sh, A.partials, rk, A.bar, &err, &ok,
                            A.prev, A.prev2, step < 2 ? step : 2);
    if (!ok) return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    A.status[DS_ITERS] = total;
    if (err != DEV_OK) atomicCAS(A.status + DS_ERR, DEV_OK, err);
  }
}

template <class K, class... Args>
static fo_status coop_launch_ls(fo_problem *p, K kernel, int grid, Args... args) {
  void *argv[] = {(void *)&args...};
  FO_CU(p->ctx, cudaMemsetAsync(p->bar, 0, 64, p->ctx->stream));
  FO_CU(p->ctx, cudaMemsetAsync(p->dev_status, 0, sizeof(int) * DS_COUNT, p->ctx->stream));
  FO_CU(p->ctx, cudaLaunchCooperativeKernel((const void *)kernel, grid, FO_BLOCK, argv, 0, p->ctx->stream));
  fo_note_launch(1);
  FO_CU(p->ctx, cudaGetLastError());
  return FO_OK;
}

static fo_status finish_status(fo_problem *p, fo_solve_stats *st, const char *what) {
  fo_ctx *ctx = p->ctx;
  int *hs = (int *)(ctx->h_scalars + 32);
  FO_CU(ctx, cudaMemcpyAsync(hs, p->dev_status, sizeof(int) * DS_COUNT, cudaMemcpyDeviceToHost, ctx->stream));
  FO_CU(ctx, cudaStreamSynchronize(ctx->stream));
  if (st) {
    memset(st, 0, sizeof *st);
    st->iterations = hs[DS_ITERS];
    st->operator_applies = hs[DS_ITERS];
    st->outer_iterations = 1;
  }
  if (hs[DS_ERR] == DEV_TIMEOUT) return fo_fail(ctx, FO_ETIMEOUT, "grid barrier timed out in %s", what);
  if (hs[DS_ERR] == DEV_NAN) return fo_fail(ctx, FO_ENAN, "NaN in %s", what);
  if (hs[DS_ERR] == DEV_NOCONV) return fo_fail(ctx, FO_ENOCONV, "%s GMRES did not converge", what);
  return FO_OK;
}

static fo_status krylov_bufs(fo_problem *p, long long extra, KrylovBufs *K, double **extra_out) {
  const long long N = p->mesh->g.num_nodes;
  double *buf;
  FO_TRY(fo_scratch(p, sizeof(double) * (size_t)((GM_M + 3) * N + extra * N), (void **)&buf));
  K->V = buf;
  K->w = buf + (size_t)(GM_M + 1) * N;
  K->rhs = buf + (size_t)(GM_M + 2) * N;
  if (extra_out) *extra_out = buf + (size_t)(GM_M + 3) * N;
  return FO_OK;
}

fo_status fo_transport_run(fo_problem *p, int nsteps, const fo_solve_opts *o, fo_solve_stats *st) {
  const Grid &g = p->mesh->g;
  const long long N = g.num_nodes;
  TransportArgs A{};
  FO_TRY(krylov_bufs(p, 2, &A.K, &A.prev));
  A.prev2 = A.prev + N;
  A.L = p->L;
  A.R = p->R;
  A.dinv = p->dinvL;
  A.phi = p->phi;
  A.rtol2 = o->rtol * o->rtol;
  A.maxit = o->maxit;
  A.nsteps = nsteps;
  A.partials = p->red;
  A.status = p->dev_status;
  A.bar = GridBar{p->bar, p->dev_status + DS_ERR, 2000000000ull};
  int grid;
  if (g.dim == 2) {
    FO_TRY(fo_cooperative_grid(p, (const void *)k_transport_run<2>, FO_BLOCK, 0, N, o->grid_blocks, &grid));
    FO_TRY(coop_launch_ls(p, k_transport_run<2>, grid, g, A));
  } else {
    FO_TRY(fo_cooperative_grid(p, (const void *)k_transport_run<3>, FO_BLOCK, 0, N, o->grid_blocks, &grid));
    FO_TRY(coop_launch_ls(p, k_transport_run<3>, grid, g, A));
  }
  return finish_status(p, st, "transport");
}

// --------------------------------------------------------------------- reinitialisation
// One step of eq. weak_HJ, row m of the element matrix and element RHS (see the oracle's
// statement of the scheme): P_ml = int lambda_l psi^_m and
//   rhs_m = int (cur + dt S) psi^_m + dt int G(cur, prev, psi^_m)   (AB2), or, on the first
//   step, G -> -H(grad cur) w - h^2 grad cur . grad w (explicit Euler),
// with psi^_m = lambda_m + beta ghat . grad lambda_m, beta = tau S, ghat = grad cur / |grad cur|.
template <int D>
__device__ __forceinline__ void reinit_row(const Grid &g, long long a, const int idx[3], const double *phi0,
                                           const double *cur, const double *prev, double dt, double h, double Ps[],
                                           double &rhs) {
  constexpr int S = ST<D>::S;
  double f0[S][1], fc[S][1], fp[S][1];
  load_stencil<D, 1, double>(g, idx, a, VecX<double>{phi0}, f0);
  load_stencil<D, 1, double>(g, idx, a, VecX<double>{cur}, fc);
  if (prev) load_stencil<D, 1, double>(g, idx, a, VecX<double>{prev}, fp);
#pragma unroll
  for (int s = 0; s < S; ++s) Ps[s] = 0.0;
  rhs = 0.0;
  const double h2 = h * h, idt2 = 1.0 / (dt * dt), ih2 = 1.0 / h2, vol = g.vol_e;
#pragma unroll
  for (int p = 0; p < KP<D>::P; ++p)
#pragma unroll
    for (int m = 0; m <= D; ++m) {
      long long e;
      if (!elem_of<D>(g, idx, p, m, e)) continue;
      int sl[D + 1];
#pragma unroll
      for (int l = 0; l <= D; ++l) sl[l] = rel_slot<D>(p, m, l);
      double gc[D], g0[D], gv[D];
#pragma unroll
      for (int k = 0; k < D; ++k) gc[k] = g0[k] = gv[k] = 0.0;
#pragma unroll
      for (int l = 0; l < D; ++l) {
        const int ax = kperm<D>(p, l);
        gc[ax] = (fc[sl[l + 1]][0] - fc[sl[l]][0]) * g.inv_h[ax];
        g0[ax] = (f0[sl[l + 1]][0] - f0[sl[l]][0]) * g.inv_h[ax];
        if (prev) gv[ax] = (fp[sl[l + 1]][0] - fp[sl[l]][0]) * g.inv_h[ax];
      }
      double nc2 = 0, nv2 = 0;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        nc2 += gc[k] * gc[k];
        nv2 += gv[k] * gv[k];
      }
      const double nc = sqrt(nc2), nv = sqrt(nv2);
      const bool has = nc > 0.0;
      double ghg = 0;   // ghat . grad lambda_m
#pragma unroll
      for (int k = 0; k < D; ++k) ghg += (has ? gc[k] / nc : 0.0) * kgrad<D>(g, p, m, k);
      double gdm[D];   // grad lambda_m
#pragma unroll
      for (int k = 0; k < D; ++k) gdm[k] = kgrad<D>(g, p, m, k);
#pragma unroll
      for (int q = 0; q <= D; ++q) {
        double p0q = 0, cq = 0;
#pragma unroll
        for (int l = 0; l <= D; ++l) {
          p0q += qbary<D>(q, l) * f0[sl[l]][0];
          cq += qbary<D>(q, l) * fc[sl[l]][0];
        }
        const double r2 = p0q * p0q + h2;
        const double sr = sqrt(r2);
        const double Sv = p0q / sr;
        const double dS = h2 / (r2 * sr);
        const double gH = has ? fabs(Sv) : 0.0;
        const double sq = idt2 + gH * gH * ih2;
        const double ssq = sqrt(sq);
        const double tau = 0.5 / ssq;
        const double dtau = -0.5 / (sq * ssq) * Sv * ih2;
        const double beta = has ? tau * Sv : 0.0;
        const double dbeta = has ? (tau + Sv * dtau) * dS : 0.0;
        const double test = qbary<D>(q, m) + beta * ghg;
        double gtest[D];
#pragma unroll
        for (int k = 0; k < D; ++k) gtest[k] = gdm[k] + ghg * dbeta * g0[k];
        const double wv = vol / (D + 1);
#pragma unroll
        for (int l = 0; l <= D; ++l) Ps[sl[l]] += wv * test * qbary<D>(q, l);
        const double Hc = Sv * nc;
        double src, fl = 0;
        if (!prev) {
          src = cq + dt * Sv - dt * Hc;
#pragma unroll
          for (int k = 0; k < D; ++k) fl += -h2 * gc[k] * gtest[k];
        } else {
          const double Hv = Sv * nv;
          src = cq + dt * Sv + dt * 0.5 * (Hv - 3.0 * Hc);
#pragma unroll
          for (int k = 0; k < D; ++k) fl += h2 * 0.5 * (gv[k] - 3.0 * gc[k]) * gtest[k];
        }
        rhs += wv * (src * test + dt * fl);
      }
    }
}

struct ReinitArgs {
  KrylovBufs K;
  double *Pm, *dinvP;    // P stencil (rewritten every step) and its inverse diagonal
  const double *phi0;    // level set at the start (copy)
  double *bufA, *bufB;   // rotating storage for prev / next
  double *phi;           // in/out
  double dt, h;
  double rtol2;
  int maxit, nsteps;
  double *partials;
  int *status;
  GridBar bar;
};

template <int D>
__global__ void __launch_bounds__(FO_BLOCK) k_reinit_run(Grid g, ReinitArgs A) {
  constexpr int S = ST<D>::S;
  __shared__ GmresShared sh;
  const long long N = g.num_nodes;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long gs = (long long)gridDim.x * blockDim.x;
  int rk = 0, err = DEV_OK, total = 0;
  bool ok = true;
  // storage: cur, prev, next rotate through {phi, bufA, bufB}; the result ends in phi
  double *cur = A.phi, *prev = nullptr, *next = A.bufA, *spare = A.bufB;
  for (int step = 0; step < A.nsteps && err == DEV_OK; ++step) {
    for (long long a = tid; a < N; a += gs) {
      int idx[3];
      node_ijk(g, a, idx);
      double Ps[S], rhs;
      reinit_row<D>(g, a, idx, A.phi0, cur, prev, A.dt, A.h, Ps, rhs);
#pragma unroll
      for (int s = 0; s < S; ++s) A.Pm[s * N + a] = Ps[s];
      A.dinvP[a] = 1.0 / Ps[0];
      A.K.rhs[a] = rhs;
      next[a] = cur[a];
    }
    if (!grid_sync(A.bar)) return;   // P rows, D^{-1} and the start value complete
    total += gmres_solve<D>(g, A.Pm, A.dinvP, nullptr, next, A.K, A.rtol2, A.maxit, sh, A.partials, rk, A.bar, &err,
                            &ok);
    if (!ok) return;
    double *old_prev = prev;
    prev = cur;
    cur = next;
    next = old_prev ? old_prev : spare;
  }
  if (cur != A.phi) {
    for (long long a = tid; a < N; a += gs) A.phi[a] = cur[a];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    A.status[DS_ITERS] = total;
    if (err != DEV_OK) atomicCAS(A.status + DS_ERR, DEV_OK, err);
  }
}

fo_status fo_reinit_run(fo_problem *p, int nsteps, double dt, double h, const fo_solve_opts *o, fo_solve_stats *st) {
  const Grid &g = p->mesh->g;
  const long long N = g.num_nodes;
  ReinitArgs A{};
  double *extra;
  FO_TRY(krylov_bufs(p, 3, &A.K, &extra));
  double *phi0 = extra;
  A.bufA = extra + N;
  A.bufB = extra + 2 * N;
  A.Pm = p->L;           // the transport matrices are rebuilt before the next transport
  A.dinvP = p->dinvL;
  A.phi0 = phi0;
  A.phi = p->phi;
  A.dt = dt;
  A.h = h;
  A.rtol2 = o->rtol * o->rtol;
  A.maxit = o->maxit;
  A.nsteps = nsteps;
  A.partials = p->red;
  A.status = p->dev_status;
  A.bar = GridBar{p->bar, p->dev_status + DS_ERR, 2000000000ull};
  p->transport_valid = false;
  FO_CU(p->ctx, cudaMemcpyAsync(phi0, p->phi, sizeof(double) * N, cudaMemcpyDeviceToDevice, p->ctx->stream));
  int grid;
  if (g.dim == 2) {
    FO_TRY(fo_cooperative_grid(p, (const void *)k_reinit_run<2>, FO_BLOCK, 0, N, o->grid_blocks, &grid));
    FO_TRY(coop_launch_ls(p, k_reinit_run<2>, grid, g, A));
  } else {
    FO_TRY(fo_cooperative_grid(p, (const void *)k_reinit_run<3>, FO_BLOCK, 0, N, o->grid_blocks, &grid));
    FO_TRY(coop_launch_ls(p, k_reinit_run<3>, grid, g, A));
  }
  return finish_status(p, st, "reinitialisation");
}
