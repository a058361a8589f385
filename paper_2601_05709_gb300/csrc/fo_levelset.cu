// Level-set transport (SUPG / Crank-Nicolson, Sec. 5.6) and reinitialisation (Sec. 5.7).
//
// The transport matrices L, R and the reinitialisation matrix change with theta / phi, so
// they are assembled (node-centrically, deterministic) into stencil form: for every node the
// 7 (2D) / 15 (3D) couplings to its Kuhn neighbours, stored slot-major [S][N_n] so that a
// warp reads consecutive nodes of one slot.  The nonsymmetric systems are solved by a
// persistent, cooperatively launched Jacobi-BiCGStab; one launch runs every substep.
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
    const long long nb = slot_node<D>(g, idx, a, s);
    if (nb >= 0) acc += M[s * g.num_nodes + a] * x(nb);
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

// ------------------------------------------------------------------- persistent BiCGStab
struct BcgBufs {
  double *x, *rhs, *r, *rhat, *p0, *p1, *v0, *v1, *s, *t;
  const double *M;       // stencil matrix [S][N]
  const double *dinv;    // [N]
};

template <int NR>
__device__ __forceinline__ bool bcg_reduce(double (&v)[NR], double *sred, double *stot, double *partials, int &rk,
                                           const GridBar &bar) {
  block_sum<NR>(v, sred);
  double *part = partials + (size_t)(rk & 1) * gridDim.x * 4;
  if (threadIdx.x == 0)
#pragma unroll
    for (int j = 0; j < NR; ++j) part[(size_t)blockIdx.x * 4 + j] = v[j];
  if (!grid_sync(bar)) return false;
  // fixed-order total of the first NR of the 4 slots
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (warp == 0) {
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      double t = 0.0;
      for (int b = lane; b < (int)gridDim.x; b += 32) t += __ldcg(part + (size_t)b * 4 + j);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
      if (lane == 0) stot[j] = t;
    }
  }
  __syncthreads();
  ++rk;
  return true;
}

// BiCGStab (right Jacobi preconditioning) on M x = rhs, x holding the start value and r,
// rhat holding rhs - M x (set by the caller's phase, followed by a reduction giving
// rr = r.r, bb = rhs.rhs, rho = rhat.r).  Three grid reductions per iteration; the search
// direction and s = r - alpha v are formed inside the gathers of the two applies.
template <int D>
__device__ int bicgstab_loop(const Grid &g, BcgBufs B, double rr, double bb, double rho_new, double rtol2, int maxit,
                             double *sred, double *stot, double *partials, int &rk, const GridBar &bar, int *err,
                             bool *ok) {
  const long long N = g.num_nodes;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long gs = (long long)gridDim.x * blockDim.x;
  double rho = 1.0, alpha = 1.0, omega = 1.0;
  double *pold = B.p0, *pnew = B.p1, *vold = B.v0, *vnew = B.v1;
  // v_old = p_old = 0 is ensured by the caller
  int it = 0;
  *ok = true;
  while (rr > rtol2 * bb) {
    if (it >= maxit) { *err = DEV_NOCONV; break; }
    if (!(rr == rr)) { *err = DEV_NAN; break; }
    const double beta = (rho_new / rho) * (alpha / omega);
    // phase 1: p = r + beta (p_old - omega v_old); v = M D^{-1} p
    double w1[1] = {0.0};
    for (long long a = tid; a < N; a += gs) {
      int idx[3];
      node_ijk(g, a, idx);
      double acc = 0;
#pragma unroll
      for (int s = 0; s < ST<D>::S; ++s) {
        const long long nb = slot_node<D>(g, idx, a, s);
        if (nb >= 0) {
          const double pn = B.r[nb] + beta * (pold[nb] - omega * vold[nb]);
          acc += B.M[s * N + a] * (B.dinv[nb] * pn);
        }
      }
      pnew[a] = B.r[a] + beta * (pold[a] - omega * vold[a]);
      vnew[a] = acc;
      w1[0] += B.rhat[a] * acc;
    }
    __syncthreads();
    if (!bcg_reduce<1>(w1, sred, stot, partials, rk, bar)) { *ok = false; return it; }
    const double rv = stot[0];
    alpha = (rv != 0.0) ? rho_new / rv : 0.0;
    // phase 2: s = r - alpha v; t = M D^{-1} s
    double w2[2] = {0.0, 0.0};
    for (long long a = tid; a < N; a += gs) {
      int idx[3];
      node_ijk(g, a, idx);
      double acc = 0;
#pragma unroll
      for (int s = 0; s < ST<D>::S; ++s) {
        const long long nb = slot_node<D>(g, idx, a, s);
        if (nb >= 0) acc += B.M[s * N + a] * (B.dinv[nb] * (B.r[nb] - alpha * vnew[nb]));
      }
      const double sa = B.r[a] - alpha * vnew[a];
      B.s[a] = sa;
      B.t[a] = acc;
      w2[0] += acc * sa;
      w2[1] += acc * acc;
    }
    if (!bcg_reduce<2>(w2, sred, stot, partials, rk, bar)) { *ok = false; return it; }
    omega = (stot[1] > 0.0) ? stot[0] / stot[1] : 0.0;
    // phase 3: x += alpha D^{-1} p + omega D^{-1} s; r = s - omega t
    double w3[2] = {0.0, 0.0};
    for (long long a = tid; a < N; a += gs) {
      const double di = B.dinv[a];
      B.x[a] += alpha * di * pnew[a] + omega * di * B.s[a];
      const double ra = B.s[a] - omega * B.t[a];
      B.r[a] = ra;
      w3[0] += ra * ra;
      w3[1] += B.rhat[a] * ra;
    }
    if (!bcg_reduce<2>(w3, sred, stot, partials, rk, bar)) { *ok = false; return it; }
    rr = stot[0];
    rho = rho_new;
    rho_new = stot[1];
    double *t = pold; pold = pnew; pnew = t;
    t = vold; vold = vnew; vnew = t;
    ++it;
    if (omega == 0.0 || rho_new == 0.0) {   // breakdown: stop here, caller sees the residual
      if (rr > rtol2 * bb) *err = DEV_NOCONV;
      break;
    }
  }
  return it;
}

struct TransportArgs {
  BcgBufs B;
  const double *Rm;      // R stencil
  double rtol2;
  int maxit, nsteps;
  double *partials;
  int *status;
  GridBar bar;
};

template <int D>
__global__ void __launch_bounds__(FO_BLOCK) k_transport_run(Grid g, TransportArgs A) {
  __shared__ double sred[32 * 3];
  __shared__ double stot[4];
  const long long N = g.num_nodes;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long gs = (long long)gridDim.x * blockDim.x;
  int rk = 0, err = DEV_OK, total = 0;
  bool ok = true;
  for (int step = 0; step < A.nsteps && err == DEV_OK; ++step) {
    // rhs = R phi^n, r = rhs - L phi^n (x starts at phi^n), zero the directions
    double v[3] = {0, 0, 0};
    for (long long a = tid; a < N; a += gs) {
      int idx[3];
      node_ijk(g, a, idx);
      const double ra = stencil_row<D>(g, A.Rm, a, idx, VecX<double>{A.B.x});
      const double la = stencil_row<D>(g, A.B.M, a, idx, VecX<double>{A.B.x});
      A.B.rhs[a] = ra;
      const double r = ra - la;
      A.B.r[a] = r;
      A.B.rhat[a] = r;
      A.B.p0[a] = A.B.p1[a] = A.B.v0[a] = A.B.v1[a] = 0.0;
      v[0] += r * r;
      v[1] += ra * ra;
      v[2] += r * r;
    }
    if (!bcg_reduce<3>(v, sred, stot, A.partials, rk, A.bar)) return;
    const double rr = stot[0], bb = stot[1], rho = stot[2];
    // the first-step x update writes phi in place; every block has finished gathering phi^n
    total += bicgstab_loop<D>(g, A.B, rr, bb, rho, A.rtol2, A.maxit, sred, stot, A.partials, rk, A.bar, &err, &ok);
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
    st->operator_applies = 2 * hs[DS_ITERS];
    st->outer_iterations = 1;
  }
  if (hs[DS_ERR] == DEV_TIMEOUT) return fo_fail(ctx, FO_ETIMEOUT, "grid barrier timed out in %s", what);
  if (hs[DS_ERR] == DEV_NAN) return fo_fail(ctx, FO_ENAN, "NaN in %s", what);
  if (hs[DS_ERR] == DEV_NOCONV) return fo_fail(ctx, FO_ENOCONV, "%s BiCGStab did not converge", what);
  return FO_OK;
}

fo_status fo_transport_run(fo_problem *p, int nsteps, const fo_solve_opts *o, fo_solve_stats *st) {
  const Grid &g = p->mesh->g;
  const long long N = g.num_nodes;
  double *buf;
  FO_TRY(fo_scratch(p, sizeof(double) * 9 * N, (void **)&buf));
  TransportArgs A{};
  A.B.x = p->phi;
  A.B.rhs = buf;
  A.B.r = buf + N;
  A.B.rhat = buf + 2 * N;
  A.B.p0 = buf + 3 * N;
  A.B.p1 = buf + 4 * N;
  A.B.v0 = buf + 5 * N;
  A.B.v1 = buf + 6 * N;
  A.B.s = buf + 7 * N;
  A.B.t = buf + 8 * N;
  A.B.M = p->L;
  A.B.dinv = p->dinvL;
  A.Rm = p->R;
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
  BcgBufs B;             // B.M = P stencil (rewritten each step), B.dinv = its inverse diagonal
  double *Pm, *dinvP;
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
  __shared__ double sred[32 * 3];
  __shared__ double stot[4];
  const long long N = g.num_nodes;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long gs = (long long)gridDim.x * blockDim.x;
  int rk = 0, err = DEV_OK, total = 0;
  bool ok = true;
  // storage: cur, prev, next rotate through {phi, bufA, bufB}; the result ends in phi
  double *cur = A.phi, *prev = nullptr, *next = A.bufA, *spare = A.bufB;
  for (int step = 0; step < A.nsteps && err == DEV_OK; ++step) {
    double v[3] = {0, 0, 0};
    for (long long a = tid; a < N; a += gs) {
      int idx[3];
      node_ijk(g, a, idx);
      double Ps[S], rhs;
      reinit_row<D>(g, a, idx, A.phi0, cur, prev, A.dt, A.h, Ps, rhs);
      double px = 0;
#pragma unroll
      for (int s = 0; s < S; ++s) {
        A.Pm[s * N + a] = Ps[s];
        const long long nb = slot_node<D>(g, idx, a, s);
        if (nb >= 0) px += Ps[s] * cur[nb];
      }
      A.dinvP[a] = 1.0 / Ps[0];
      next[a] = cur[a];
      A.B.rhs[a] = rhs;
      const double r = rhs - px;
      A.B.r[a] = r;
      A.B.rhat[a] = r;
      A.B.p0[a] = A.B.p1[a] = A.B.v0[a] = A.B.v1[a] = 0.0;
      v[0] += r * r;
      v[1] += rhs * rhs;
      v[2] += r * r;
    }
    if (!bcg_reduce<3>(v, sred, stot, A.partials, rk, A.bar)) return;
    BcgBufs B = A.B;
    B.x = next;
    total += bicgstab_loop<D>(g, B, stot[0], stot[1], stot[2], A.rtol2, A.maxit, sred, stot, A.partials, rk, A.bar,
                              &err, &ok);
    if (!ok) return;
    // rotate: prev <- cur, cur <- next
    double *old_prev = prev;
    prev = cur;
    cur = next;
    next = old_prev ? old_prev : spare;
  }
  // copy the result into phi when it ended elsewhere
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
  double *buf;
  FO_TRY(fo_scratch(p, sizeof(double) * 12 * N, (void **)&buf));
  ReinitArgs A{};
  A.B.rhs = buf;
  A.B.r = buf + N;
  A.B.rhat = buf + 2 * N;
  A.B.p0 = buf + 3 * N;
  A.B.p1 = buf + 4 * N;
  A.B.v0 = buf + 5 * N;
  A.B.v1 = buf + 6 * N;
  A.B.s = buf + 7 * N;
  A.B.t = buf + 8 * N;
  double *phi0 = buf + 9 * N;
  A.bufA = buf + 10 * N;
  A.bufB = buf + 11 * N;
  A.Pm = p->L;           // the transport matrices are rebuilt before the next transport
  A.dinvP = p->dinvL;
  A.B.M = p->L;
  A.B.dinv = p->dinvL;
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
