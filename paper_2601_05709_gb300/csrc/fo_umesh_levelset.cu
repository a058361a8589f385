// Level-set transport and reinitialisation on general simplicial meshes: node-centric
// assembly of the Petrov-Galerkin matrices into the node graph (CSR, one row per thread, sums
// over the node's elements in element order) and one persistent BiCGStab launch per solve
// (right Jacobi preconditioning; for the transport all substeps in one launch).
#include <cmath>
#include <cstring>
#include <algorithm>

#include "fo_internal.cuh"
#include "fo_umesh.cuh"

// Degree-2 rule: 2D (2/3, 1/6, 1/6) and permutations, weights 1/3; 3D (a, b, b, b) and
// permutations, a = (5 + 3 sqrt 5)/20, b = (5 - sqrt 5)/20, weights 1/4 (fractions of |e|).
template <int D>
__device__ __forceinline__ double u_qbary(int q, int b) {
  if (D == 2) return q == b ? 2.0 / 3.0 : 1.0 / 6.0;
  const double s5 = 2.2360679774997896964;   // sqrt(5) to double precision
  return q == b ? (5.0 + 3.0 * s5) / 20.0 : (5.0 - s5) / 20.0;
}

// ------------------------------------------------------------------------ transport
// Rows of L = M^ + dt/2 (C + s h^2 K^) and R = M^ - dt/2 (C + s h^2 K^) (Sec. 5.6, eq.
// weak_transport): test function psi^ = psi + tau theta . grad psi with tau of eq. tau_lv at
// the quadrature points, and the diffusion tested with the full
// grad psi^ = grad psi + (theta . grad psi) grad tau + tau (D theta)^T grad psi.
template <int D>
__global__ void k_u_transport_assemble(UMeshView m, const double *theta, double dt, double h, int smooth, double *Lv,
                                       double *Rv, double *dinvL) {
  for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < m.nn; a += (long long)gridDim.x * blockDim.x) {
    for (int k = m.row_ptr[a]; k < m.row_ptr[a + 1]; ++k) Lv[k] = Rv[k] = 0.0;
    for (int q0 = m.adj_ptr[a]; q0 < m.adj_ptr[a + 1]; ++q0) {
      const long long e = m.adj[q0] / (D + 1);
      const int la = m.adj[q0] % (D + 1);
      double th[D + 1][D], g[D + 1][D];
#pragma unroll
      for (int b = 0; b <= D; ++b) {
        const long long nb = m.cells[e * (D + 1) + b];
#pragma unroll
        for (int k = 0; k < D; ++k) {
          th[b][k] = theta[nb * D + k];
          g[b][k] = m.g(e, b, k);
        }
      }
      double Dth[D][D];   // (D theta)_ij = d_j theta_i
#pragma unroll
      for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) {
          double s = 0;
#pragma unroll
          for (int b = 0; b <= D; ++b) s += th[b][i] * g[b][j];
          Dth[i][j] = s;
        }
      double Mrow[D + 1], Frow[D + 1];
#pragma unroll
      for (int b = 0; b <= D; ++b) Mrow[b] = Frow[b] = 0.0;
      const double wv = m.vol[e] / (D + 1);
#pragma unroll
      for (int q = 0; q <= D; ++q) {
        double lam[D + 1], thq[D];
#pragma unroll
        for (int b = 0; b <= D; ++b) lam[b] = u_qbary<D>(q, b);
#pragma unroll
        for (int i = 0; i < D; ++i) {
          double s = 0;
#pragma unroll
          for (int b = 0; b <= D; ++b) s += lam[b] * th[b][i];
          thq[i] = s;
        }
        double t2 = 0;
#pragma unroll
        for (int i = 0; i < D; ++i) t2 += thq[i] * thq[i];
        const double s = 1.0 / (dt * dt) + t2 / (h * h);
        const double tau = 0.5 / sqrt(s);
        const double gfac = -0.5 / (s * sqrt(s)) / (h * h);
        double gtau[D];
#pragma unroll
        for (int i = 0; i < D; ++i) {
          double v = 0;
#pragma unroll
          for (int j = 0; j < D; ++j) v += Dth[j][i] * thq[j];
          gtau[i] = gfac * v;
        }
        double thg[D + 1];
#pragma unroll
        for (int b = 0; b <= D; ++b) {
          double v = 0;
#pragma unroll
          for (int k = 0; k < D; ++k) v += thq[k] * g[b][k];
          thg[b] = v;
        }
        const double test = lam[la] + tau * thg[la];
        double gtest[D];
#pragma unroll
        for (int i = 0; i < D; ++i) {
          double v = 0;
#pragma unroll
          for (int j = 0; j < D; ++j) v += Dth[j][i] * g[la][j];
          gtest[i] = g[la][i] + thg[la] * gtau[i] + tau * v;
        }
#pragma unroll
        for (int b = 0; b <= D; ++b) {
          double gd = 0;
#pragma unroll
          for (int k = 0; k < D; ++k) gd += gtest[k] * g[b][k];
          Mrow[b] += wv * test * lam[b];
          Frow[b] += wv * test * thg[b] + (smooth ? wv * h * h * gd : 0.0);
        }
      }
#pragma unroll
      for (int b = 0; b <= D; ++b) {
        const long long pos = m.adj_pos[(long long)q0 * (D + 1) + b];
        Lv[pos] += Mrow[b] + 0.5 * dt * Frow[b];
        Rv[pos] += Mrow[b] - 0.5 * dt * Frow[b];
      }
    }
    dinvL[a] = 1.0 / Lv[m.diag[a]];
  }
}

// ------------------------------------------------------------------- reinitialisation
// Row of one step of eq. weak_HJ: P[a, b] = int psi^_a lambda_b and the right-hand side
//   int (cur + dt S) psi^_a + dt int G(cur, prev, psi^_a)
// with S = phi0 / sqrt(phi0^2 + h^2) at the quadrature points, grad H = S grad cur / |grad cur|
// (0 on elements where grad cur = 0), psi^ = psi + beta ghat . grad psi, beta = tau S,
// tau = (1/2)(1/dt^2 + S^2/h^2)^(-1/2), grad psi^ including grad beta along grad phi0;
// prev == null: the explicit Euler first step (G = -H(grad u) w - h^2 grad u . grad w).
template <int D>
__global__ void k_u_reinit_assemble(UMeshView m, const double *phi0, const double *cur, const double *prev, double dt,
                                    double h, double *Pv, double *rhs, double *dinv) {
  for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < m.nn; a += (long long)gridDim.x * blockDim.x) {
    for (int k = m.row_ptr[a]; k < m.row_ptr[a + 1]; ++k) Pv[k] = 0.0;
    double ra = 0.0;
    for (int q0 = m.adj_ptr[a]; q0 < m.adj_ptr[a + 1]; ++q0) {
      const long long e = m.adj[q0] / (D + 1);
      const int la = m.adj[q0] % (D + 1);
      double p0[D + 1], ce[D + 1], pv[D + 1], g[D + 1][D];
#pragma unroll
      for (int b = 0; b <= D; ++b) {
        const long long nb = m.cells[e * (D + 1) + b];
        p0[b] = phi0[nb];
        ce[b] = cur[nb];
        pv[b] = prev ? prev[nb] : 0.0;
#pragma unroll
        for (int k = 0; k < D; ++k) g[b][k] = m.g(e, b, k);
      }
      double gc[D], gp0[D], gv[D];
#pragma unroll
      for (int k = 0; k < D; ++k) {
        double s1 = 0, s2 = 0, s3 = 0;
#pragma unroll
        for (int b = 0; b <= D; ++b) {
          s1 += ce[b] * g[b][k];
          s2 += p0[b] * g[b][k];
          s3 += pv[b] * g[b][k];
        }
        gc[k] = s1;
        gp0[k] = s2;
        gv[k] = s3;
      }
      double nc2 = 0, nv2 = 0;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        nc2 += gc[k] * gc[k];
        nv2 += gv[k] * gv[k];
      }
      const double nc = sqrt(nc2), nvv = sqrt(nv2);
      const bool has = nc > 0.0;
      double ghg[D + 1];
#pragma unroll
      for (int b = 0; b <= D; ++b) {
        double v = 0;
#pragma unroll
        for (int k = 0; k < D; ++k) v += (has ? gc[k] / nc : 0.0) * g[b][k];
        ghg[b] = v;
      }
      double Prow[D + 1];
#pragma unroll
      for (int b = 0; b <= D; ++b) Prow[b] = 0.0;
      const double wv = m.vol[e] / (D + 1);
#pragma unroll
      for (int q = 0; q <= D; ++q) {
        double lam[D + 1], p0q = 0, cq = 0;
#pragma unroll
        for (int b = 0; b <= D; ++b) {
          lam[b] = u_qbary<D>(q, b);
          p0q += p0[b] * lam[b];
          cq += ce[b] * lam[b];
        }
        const double r2 = p0q * p0q + h * h;
        const double S = p0q / sqrt(r2);
        const double dS = h * h / (r2 * sqrt(r2));
        const double gH = has ? fabs(S) : 0.0;
        const double sq = 1.0 / (dt * dt) + gH * gH / (h * h);
        const double tau = 0.5 / sqrt(sq);
        const double dtau = -0.5 / (sq * sqrt(sq)) * S / (h * h);
        const double beta = has ? tau * S : 0.0;
        const double dbeta = has ? (tau + S * dtau) * dS : 0.0;
        const double test = lam[la] + beta * ghg[la];
        double gtest[D];
#pragma unroll
        for (int k = 0; k < D; ++k) gtest[k] = g[la][k] + ghg[la] * dbeta * gp0[k];
#pragma unroll
        for (int b = 0; b <= D; ++b) Prow[b] += wv * test * lam[b];
        const double Hc = S * nc;
        double src, fl = 0;
        if (!prev) {
          src = cq + dt * S - dt * Hc;
#pragma unroll
          for (int k = 0; k < D; ++k) fl += -(h * h) * gc[k] * gtest[k];
        } else {
          const double Hv = S * nvv;
          src = cq + dt * S + dt * 0.5 * (Hv - 3.0 * Hc);
#pragma unroll
          for (int k = 0; k < D; ++k) fl += (h * h) * 0.5 * (gv[k] - 3.0 * gc[k]) * gtest[k];
        }
        ra += wv * (src * test + dt * fl);
      }
#pragma unroll
      for (int b = 0; b <= D; ++b) Pv[m.adj_pos[(long long)q0 * (D + 1) + b]] += Prow[b];
    }
    rhs[a] = ra;
    dinv[a] = 1.0 / Pv[m.diag[a]];
  }
}

// ----------------------------------------------------------------------- BiCGStab
// One persistent launch: nsys solves of A x = b with A in the node graph (scalar CSR), right
// Jacobi preconditioning M = diag(A)^{-1}, start value x (in place).  With R (transport) each
// solve's right-hand side is b = R x of the previous solve's result (all Crank-Nicolson
// substeps in one launch); otherwise b is given.  Per iteration five grid phases (two
// operator passes, four deterministic reductions); stop when ||r|| <= rtol ||b||.
struct BicgArgs {
  const int *row_ptr, *col;
  const double *A, *R, *dinv;
  double *x, *b;
  double *r, *rh, *p, *v, *y, *s, *z, *t;
  long long n;
  int nsys, maxit;
  double rtol2;
  double *partials, *out;   // out: [0] iterations, [1] last ||r||^2, [2] last ||b||^2
  int *status;
  GridBar bar;
};

__device__ __forceinline__ double u_row(const int *rp, const int *col, const double *A, const double *x, long long a) {
  double s = 0;
  for (int k = rp[a]; k < rp[a + 1]; ++k) s = fma(A[k], x[col[k]], s);
  return s;
}

__global__ void __launch_bounds__(FO_BLOCK) k_u_bicgstab(BicgArgs B) {
  __shared__ double sred[32 * 3];
  __shared__ double stot[3];
  const long long first = blockIdx.x * (long long)blockDim.x + threadIdx.x, step = (long long)gridDim.x * blockDim.x;
  int rk = 0, total = 0, err = DEV_OK;
  double rr = 0, bb = 0;
  for (int sys = 0; sys < B.nsys; ++sys) {
    // b (transport: R x), r = b - A x, rhat = r, p = v = 0
    double w3[3] = {0, 0, 0};
    for (long long a = first; a < B.n; a += step) {
      const double ba = B.R ? u_row(B.row_ptr, B.col, B.R, B.x, a) : B.b[a];
      if (B.R) B.b[a] = ba;
      const double ra = ba - u_row(B.row_ptr, B.col, B.A, B.x, a);
      B.r[a] = ra;
      B.rh[a] = ra;
      B.p[a] = 0.0;
      B.v[a] = 0.0;
      w3[0] += ba * ba;
      w3[1] += ra * ra;
    }
    if (!reduce_grid<3>(w3, sred, stot, B.partials, rk, B.bar)) return;
    bb = stot[0];
    rr = stot[1];
    double rho = 1.0, alpha = 1.0, omega = 1.0, rho_new = rr;   // (rhat, r) = ||r||^2 at the start
    int it = 0;
    while (rr > B.rtol2 * bb && bb > 0.0) {
      if (it >= B.maxit) {
        err = DEV_NOCONV;
        break;
      }
      if (!(rr == rr)) {
        err = DEV_NAN;
        break;
      }
      const double beta = (rho_new / rho) * (alpha / omega);
      rho = rho_new;
      // p = r + beta (p - omega v); y = M p
      for (long long a = first; a < B.n; a += step) {
        const double pa = B.r[a] + beta * (B.p[a] - omega * B.v[a]);
        B.p[a] = pa;
        B.y[a] = B.dinv[a] * pa;
      }
      if (!grid_sync(B.bar)) return;
      // v = A y; (rhat, v)
      double w1[1] = {0};
      for (long long a = first; a < B.n; a += step) {
        const double va = u_row(B.row_ptr, B.col, B.A, B.y, a);
        B.v[a] = va;
        w1[0] += B.rh[a] * va;
      }
      if (!reduce_grid<1>(w1, sred, stot, B.partials, rk, B.bar)) return;
      const double rv = stot[0];
      if (rv == 0.0) break;   // breakdown: keep x
      alpha = rho / rv;
      // s = r - alpha v; z = M s; ||s||^2
      double w2[1] = {0};
      for (long long a = first; a < B.n; a += step) {
        const double sa = B.r[a] - alpha * B.v[a];
        B.s[a] = sa;
        B.z[a] = B.dinv[a] * sa;
        w2[0] += sa * sa;
      }
      if (!reduce_grid<1>(w2, sred, stot, B.partials, rk, B.bar)) return;
      ++it;
      if (stot[0] <= B.rtol2 * bb) {   // x += alpha y and stop
        for (long long a = first; a < B.n; a += step) B.x[a] += alpha * B.y[a];
        rr = stot[0];
        if (!grid_sync(B.bar)) return;
        break;
      }
      // t = A z; (t, s), (t, t)
      double w4[3] = {0, 0, 0};
      for (long long a = first; a < B.n; a += step) {
        const double ta = u_row(B.row_ptr, B.col, B.A, B.z, a);
        B.t[a] = ta;
        w4[0] += ta * B.s[a];
        w4[1] += ta * ta;
      }
      if (!reduce_grid<3>(w4, sred, stot, B.partials, rk, B.bar)) return;
      if (stot[1] == 0.0) break;
      omega = stot[0] / stot[1];
      // x += alpha y + omega z; r = s - omega t; (rhat, r), ||r||^2
      double w5[3] = {0, 0, 0};
      for (long long a = first; a < B.n; a += step) {
        B.x[a] += alpha * B.y[a] + omega * B.z[a];
        const double ra = B.s[a] - omega * B.t[a];
        B.r[a] = ra;
        w5[0] += B.rh[a] * ra;
        w5[1] += ra * ra;
      }
      if (!reduce_grid<3>(w5, sred, stot, B.partials, rk, B.bar)) return;
      rho_new = stot[0];
      rr = stot[1];
      if (omega == 0.0) break;
    }
    total += it;
    if (err != DEV_OK) break;
    if (!grid_sync(B.bar)) return;   // x complete before the next right-hand side
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    B.out[0] = (double)total;
    B.out[1] = rr;
    B.out[2] = bb;
    B.status[DS_ITERS] = total;
    if (err != DEV_OK) atomicCAS(B.status + DS_ERR, DEV_OK, err);
  }
}

static fo_status u_bicgstab(fo_problem *p, const double *A, const double *R, const double *dinv, double *x, double *b,
                            int nsys, const fo_solve_opts *o, fo_solve_stats *st) {
  fo_ctx *ctx = p->ctx;
  const long long n = p->mesh->um->nn;
  double *buf;
  FO_TRY(fo_scratch(p, sizeof(double) * 9 * n, (void **)&buf));
  BicgArgs B{};
  B.row_ptr = p->mesh->um->row_ptr;
  B.col = p->mesh->um->col;
  B.A = A;
  B.R = R;
  B.dinv = dinv;
  B.x = x;
  B.b = R ? buf + 8 * n : b;
  B.r = buf;
  B.rh = buf + n;
  B.p = buf + 2 * n;
  B.v = buf + 3 * n;
  B.y = buf + 4 * n;
  B.s = buf + 5 * n;
  B.z = buf + 6 * n;
  B.t = buf + 7 * n;
  B.n = n;
  B.nsys = nsys;
  B.maxit = o->maxit;
  B.rtol2 = o->rtol * o->rtol;
  B.partials = p->red;
  B.out = p->red + (FO_RED_DOUBLES - 64);
  B.status = p->dev_status;
  B.bar = GridBar{p->bar, p->dev_status + DS_ERR, 2000000000ull};
  int grid;
  FO_TRY(fo_cooperative_grid(p, (const void *)k_u_bicgstab, FO_BLOCK, 0, n, o->grid_blocks, &grid));
  void *argv[] = {(void *)&B};
  FO_CU(ctx, cudaMemsetAsync(p->bar, 0, 64, ctx->stream));
  FO_CU(ctx, cudaMemsetAsync(p->dev_status, 0, sizeof(int) * DS_COUNT, ctx->stream));
  FO_CU(ctx, cudaLaunchCooperativeKernel((const void *)k_u_bicgstab, grid, FO_BLOCK, argv, 0, ctx->stream));
  fo_note_launch(1);
  FO_CU(ctx, cudaGetLastError());
  FO_CU(ctx, cudaMemcpyAsync(ctx->h_scalars, B.out, 3 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  FO_CU(ctx, cudaMemcpyAsync(ctx->h_scalars + 32, p->dev_status, sizeof(int) * DS_COUNT, cudaMemcpyDeviceToHost,
                             ctx->stream));
  FO_CU(ctx, cudaStreamSynchronize(ctx->stream));
  const int *hs = (const int *)(ctx->h_scalars + 32);
  if (st) {
    st->iterations += hs[DS_ITERS];
    st->operator_applies += 2 * hs[DS_ITERS] + nsys * (R ? 2 : 1);
    st->outer_iterations = 1;
    st->rel_residual = ctx->h_scalars[2] > 0 ? std::sqrt(ctx->h_scalars[1] / ctx->h_scalars[2]) : 0.0;
  }
  if (hs[DS_ERR] == DEV_TIMEOUT) return fo_fail(ctx, FO_ETIMEOUT, "grid barrier timed out in BiCGStab");
  if (hs[DS_ERR] == DEV_NAN) return fo_fail(ctx, FO_ENAN, "NaN in BiCGStab");
  if (hs[DS_ERR] == DEV_NOCONV) return fo_fail(ctx, FO_ENOCONV, "BiCGStab reached maxit=%d", o->maxit);
  return FO_OK;
}

// ------------------------------------------------------------------------- host drivers
fo_status fo_umesh_transport_assemble(fo_problem *p, double dt, double h, int smooth) {
  const UMeshView m = umesh_view(p->mesh);
  const int blocks = fo_blocks_for(m.nn, FO_BLOCK, 65536);
  if (m.dim == 2)
    k_u_transport_assemble<2><<<blocks, FO_BLOCK, 0, p->ctx->stream>>>(m, p->theta, dt, h, smooth, p->L, p->R, p->dinvL);
  else
    k_u_transport_assemble<3><<<blocks, FO_BLOCK, 0, p->ctx->stream>>>(m, p->theta, dt, h, smooth, p->L, p->R, p->dinvL);
  fo_note_launch(1);
  FO_CU(p->ctx, cudaGetLastError());
  return FO_OK;
}

__global__ void k_u_csr_apply(long long n, const int *rp, const int *col, const double *A, const double *x, double *y) {
  for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < n; a += (long long)gridDim.x * blockDim.x)
    y[a] = u_row(rp, col, A, x, a);
}

fo_status fo_umesh_transport_apply(fo_problem *p, int which, const double *x, double *y) {
  const fo_umesh *u = p->mesh->um;
  const int blocks = fo_blocks_for(u->nn, FO_BLOCK, 65536);
  k_u_csr_apply<<<blocks, FO_BLOCK, 0, p->ctx->stream>>>(u->nn, u->row_ptr, u->col, which == 0 ? p->L : p->R, x, y);
  fo_note_launch(1);
  FO_CU(p->ctx, cudaGetLastError());
  return FO_OK;
}

fo_status fo_umesh_levelset_step(fo_problem *p, double t_end, int nsteps, double h, int smooth,
                                 const fo_solve_opts *o, fo_solve_stats *st) {
  const double dt = t_end / nsteps;
  FO_TRY(fo_umesh_transport_assemble(p, dt, h, smooth));
  if (st) memset(st, 0, sizeof *st);
  return u_bicgstab(p, p->L, p->R, p->dinvL, p->phi, nullptr, nsteps, o, st);
}

fo_status fo_umesh_reinit(fo_problem *p, int nsteps, double t_final, double h, const fo_solve_opts *o,
                          fo_solve_stats *st) {
  fo_ctx *ctx = p->ctx;
  const UMeshView m = umesh_view(p->mesh);
  const long long n = m.nn;
  // phi0 (the input), prev, cur and the step's right-hand side live beside the solver scratch
  double *keep;
  FO_TRY(fo_scratch(p, sizeof(double) * 13 * n, (void **)&keep));
  double *phi0 = keep + 9 * n, *prev = keep + 10 * n, *rhs = keep + 11 * n;
  FO_CU(ctx, cudaMemcpyAsync(phi0, p->phi, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
  if (st) memset(st, 0, sizeof *st);
  const double dt = t_final / nsteps;
  const int blocks = fo_blocks_for(n, FO_BLOCK, 65536);
  for (int k = 0; k < nsteps; ++k) {
    // cur = p->phi; the new iterate overwrites it after prev takes a copy
    const double *pv = k == 0 ? nullptr : prev;
    if (m.dim == 2)
      k_u_reinit_assemble<2><<<blocks, FO_BLOCK, 0, ctx->stream>>>(m, phi0, p->phi, pv, dt, h, p->L, rhs, p->dinvL);
    else
      k_u_reinit_assemble<3><<<blocks, FO_BLOCK, 0, ctx->stream>>>(m, phi0, p->phi, pv, dt, h, p->L, rhs, p->dinvL);
    fo_note_launch(1);
    FO_CU(ctx, cudaGetLastError());
    FO_CU(ctx, cudaMemcpyAsync(prev, p->phi, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
    FO_TRY(u_bicgstab(p, p->L, nullptr, p->dinvL, p->phi, rhs, 1, o, st));
  }
  p->transport_valid = false;   // L held the reinitialisation matrix
  return FO_OK;
}
