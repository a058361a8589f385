// Inverse elasticity by a Kohn-Vogelius-type cost (Sec. 3, Sec. 6.1) on the box grid.
//
// For every force-displacement pair k (a load case): the state u_k with Gamma0 clamped and the
// force f_k on Gamma1 (eq. w-f), the state v_k vanishing on the whole boundary with
// int A sigma(v_k + g_k):eps(w) = 0 (eq. w-g; g_k the measurement extended into D), the cost
//   J = sum_k alpha/2 int |u_k - v_k - g_k|^2 + beta/2 int_Gamma1 |u_k - g_k|^2     (eq. cost),
// the adjoints p_k (Gamma0 clamped) and q_k (boundary clamped) with right-hand sides
//   -alpha M w_k - beta M_Gamma1 (u_k - g_k)  and  alpha M w_k   (w_k = u_k - v_k - g_k),
// and the shape derivative (eq. SDelast_inv) with S0 = -alpha Dg^T w (the grad(eps(g)) term
// vanishes for a P1 g) and
//   S1 = (alpha/2 |w|^2 + A sigma(u):eps(p) + A sigma(v+g):eps(q)) I
//        - A (Du^T sigma(p) + Dp^T sigma(u) + Dv^T sigma(q) + Dq^T sigma(v+g)).
// M is the consistent P1 mass (|e| (1 + delta) / ((d+1)(d+2)) per simplex), M_Gamma1 the facet
// mass on the Gamma1 faces (|f| (1 + delta) / (d (d+1)) per facet); every integral is exact for
// P1 data.  u_k and p_k use the problem's own operator (Gamma0 = its Dirichlet faces); v_k and
// q_k an operator with every boundary DOF clamped, built by the same stencil builder from the
// same coefficients (Jacobi-PCG).  The lifting -K g_k of v_k's right-hand side needs the
// operator without any clamped DOF, built into the same rows just before.
#include <cmath>
#include <cstring>
#include <vector>

#include "fo_internal.cuh"
#include "fo_ops.cuh"

// Per node: the bits (2 axis + side) of the Gamma1 faces it lies on; per DOF: on the boundary.
template <int D>
__global__ void k_inv_masks(Grid g, uint32_t gamma1, uint8_t *gam, uint8_t *dirb) {
  for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < g.num_nodes;
       a += (long long)gridDim.x * blockDim.x) {
    int idx[3];
    node_ijk(g, a, idx);
    unsigned bits = 0;
    bool onb = false;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      if (idx[c] == 0) {
        onb = true;
        if (gamma1 & (1u << (2 * c))) bits |= 1u << (2 * c);
      }
      if (idx[c] == g.n[c]) {
        onb = true;
        if (gamma1 & (1u << (2 * c + 1))) bits |= 1u << (2 * c + 1);
      }
    }
    gam[a] = (uint8_t)bits;
#pragma unroll
    for (int c = 0; c < D; ++c) dirb[a * D + c] = onb ? 1 : 0;
  }
}

// y = scale * K x at the DOFs that mask_out leaves free (0 elsewhere); K from rows W, unmasked x.
template <int D>
__global__ void k_inv_apply(StencilOp<D, D, true, double> op, const double *x, const uint8_t *mask_out, double scale,
                            double *y) {
  op.sweep(VecX<double>{x}, [&](long long a, const double (&ax)[D]) {
#pragma unroll
    for (int c = 0; c < D; ++c) y[a * D + c] = mask_out[a * D + c] ? 0.0 : scale * ax[c];
  });
}

// (M w)_a and (M_Gamma1 e)_a of node a, w = u - v - g and e = u - g (D components each).
template <int D>
__device__ __forceinline__ void inv_mass_rows(const Grid &g, const int idx[3], long long a, const double *u,
                                              const double *v, const double *gm, unsigned gbits, double Mw[D],
                                              double Me[D]) {
  const double mref = g.vol_e / ((D + 1) * (D + 2));
#pragma unroll
  for (int c = 0; c < D; ++c) Mw[c] = Me[c] = 0.0;
  auto wv = [&](long long n, int c) { return u[n * D + c] - v[n * D + c] - gm[n * D + c]; };
  auto ev = [&](long long n, int c) { return u[n * D + c] - gm[n * D + c]; };
#pragma unroll
  for (int p = 0; p < KP<D>::P; ++p)
#pragma unroll
    for (int m = 0; m <= D; ++m) {
      long long e;
      if (!elem_of<D>(g, idx, p, m, e)) continue;
#pragma unroll
      for (int l = 0; l <= D; ++l) {
        const long long nb = slot_node<D>(g, idx, a, rel_slot<D>(p, m, l));
        const double f = l == m ? 2.0 : 1.0;
#pragma unroll
        for (int c = 0; c < D; ++c) Mw[c] += f * mref * wv(nb, c);
      }
    }
  if (!gbits) return;
#pragma unroll
  for (int c = 0; c < D; ++c)        // the face normal to axis c, at side 0 or 1
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      if (!(gbits & (1u << (2 * c + side)))) continue;
      const double fm = g.facet_area[c] / (D * (D + 1));
      if (D == 2) {
        const int o = 1 - c;
#pragma unroll
        for (int sg = -1; sg <= 1; sg += 2) {
          if (idx[o] + sg < 0 || idx[o] + sg > g.n[o]) continue;
          int dl[3] = {0, 0, 0};
          dl[o] = sg;
          const long long nb = slot_node<D>(g, idx, a, stencil_slot<D>(dl));
#pragma unroll
          for (int k = 0; k < D; ++k) Me[k] += fm * (2.0 * ev(a, k) + ev(nb, k));
        }
      } else {
        const int o1 = c == 0 ? 1 : 0, o2 = c == 2 ? 1 : 2;
#pragma unroll
        for (int q = 0; q < 2; ++q)   // face-local Kuhn triangles, paths (o1, o2) and (o2, o1)
#pragma unroll
          for (int m = 0; m <= 2; ++m) {
            const int ax[2] = {q == 0 ? o1 : o2, q == 0 ? o2 : o1};
            int cc[3] = {idx[0], idx[1], idx[2]};
            for (int l = 0; l < m; ++l) cc[ax[l]] -= 1;
            if (cc[o1] < 0 || cc[o1] >= g.n[o1] || cc[o2] < 0 || cc[o2] >= g.n[o2]) continue;
#pragma unroll
            for (int k = 0; k < D; ++k) Me[k] += 2.0 * fm * ev(a, k);
#pragma unroll
            for (int l = 0; l <= 2; ++l) {
              if (l == m) continue;
              int dl[3] = {0, 0, 0};
              for (int j = 0; j < 2; ++j) {
                if (l > m && j >= m && j < l) dl[ax[j]] += 1;
                if (l < m && j >= l && j < m) dl[ax[j]] -= 1;
              }
              const long long nb = slot_node<D>(g, idx, a, stencil_slot<D>(dl));
#pragma unroll
              for (int k = 0; k < D; ++k) Me[k] += fm * ev(nb, k);
            }
          }
      }
    }
}

// Per-block partials of int |w|^2 and int_Gamma1 |e|^2; with rp / rq the adjoint right-hand
// sides -alpha M w - beta M_G1 e (zero on Gamma0 DOFs) and alpha M w (zero on boundary DOFs).
template <int D>
__global__ void k_inv_cost_rhs(Grid g, const double *u, const double *v, const double *gm, const uint8_t *gam,
                               const uint8_t *dir0, const uint8_t *dirb, double alpha, double beta, double *rp,
                               double *rq, double *partials) {
  __shared__ double smem[64];
  double s[2] = {0.0, 0.0};
  for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < g.num_nodes;
       a += (long long)gridDim.x * blockDim.x) {
    int idx[3];
    node_ijk(g, a, idx);
    double Mw[D], Me[D];
    inv_mass_rows<D>(g, idx, a, u, v, gm, gam[a], Mw, Me);
#pragma unroll
    for (int c = 0; c < D; ++c) {
      const long long k = a * D + c;
      s[0] += (u[k] - v[k] - gm[k]) * Mw[c];
      s[1] += (u[k] - gm[k]) * Me[c];
      if (rp) rp[k] = dir0[k] ? 0.0 : -alpha * Mw[c] - beta * Me[c];
      if (rq) rq[k] = dirb[k] ? 0.0 : alpha * Mw[c];
    }
  }
  block_sum<2>(s, smem);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = s[0];
    partials[2 * blockIdx.x + 1] = s[1];
  }
}

__global__ void k_inv_total(const double *partials, int nblocks, double *out) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (w >= 2) return;
  double t = 0.0;
  for (int b = lane; b < nblocks; b += 32) t += partials[2 * b + w];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  if (lane == 0) out[w] = t;
}

// b[D a + k] (+)= sum over the simplices (p, m) of node a of int_e S0_k lambda_m + (S1 grad lambda_m)_k
template <int D>
__global__ void k_inv_shape(Grid g, const double *coef, double lam, double mu, double alpha, const double *u,
                            const double *v, const double *pa, const double *q, const double *gm, double *b,
                            int add) {
  const double ve = g.vol_e, mref = g.vol_e / ((D + 1) * (D + 2));
  for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < g.num_nodes;
       a += (long long)gridDim.x * blockDim.x) {
    int idx[3];
    node_ijk(g, a, idx);
    double acc[D];
#pragma unroll
    for (int k = 0; k < D; ++k) acc[k] = 0.0;
#pragma unroll 1
    for (int p = 0; p < KP<D>::P; ++p)
#pragma unroll 1
      for (int m = 0; m <= D; ++m) {
        long long e;
        if (!elem_of<D>(g, idx, p, m, e)) continue;
        long long vx[D + 1];
#pragma unroll
        for (int l = 0; l <= D; ++l) vx[l] = slot_node<D>(g, idx, a, rel_slot<D>(p, m, l));
        // Jacobians along the Kuhn path: (D x)_{i, ax} = (x_{l+1} - x_l)_i / h_ax, ax = pi_l
        double Du[D][D], Dv[D][D], Dp[D][D], Dq[D][D], Dg[D][D];
#pragma unroll
        for (int l = 0; l < D; ++l) {
          const int ax = kperm<D>(p, l);
          const long long n0 = vx[l] * D, n1 = vx[l + 1] * D;
#pragma unroll
          for (int i = 0; i < D; ++i) {
            Du[i][ax] = (u[n1 + i] - u[n0 + i]) * g.inv_h[ax];
            Dv[i][ax] = (v[n1 + i] - v[n0 + i]) * g.inv_h[ax];
            Dp[i][ax] = (pa[n1 + i] - pa[n0 + i]) * g.inv_h[ax];
            Dq[i][ax] = (q[n1 + i] - q[n0 + i]) * g.inv_h[ax];
            Dg[i][ax] = (gm[n1 + i] - gm[n0 + i]) * g.inv_h[ax];
          }
        }
        // w = u - v - g at the vertices: int_e |w|^2 and the node's own mass row of w
        double ww = 0.0, Mw[D];
#pragma unroll
        for (int i = 0; i < D; ++i) {
          double sw = 0.0, sq = 0.0, wm = 0.0;
#pragma unroll
          for (int l = 0; l <= D; ++l) {
            const long long k = vx[l] * D + i;
            const double wl = u[k] - v[k] - gm[k];
            sw += wl;
            sq += wl * wl;
            if (l == m) wm = wl;
          }
          ww += mref * (sw * sw + sq);
          Mw[i] = mref * (sw + wm);
        }
        // stresses: sigma(x) = lam tr(eps) I + mu (Dx + Dx^T)
        auto sigma = [&](const double (&Dx)[D][D], double (&s)[D][D]) {
          double tr = 0.0;
#pragma unroll
          for (int i = 0; i < D; ++i) tr += Dx[i][i];
#pragma unroll
          for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j) s[i][j] = (i == j ? lam * tr : 0.0) + mu * (Dx[i][j] + Dx[j][i]);
        };
        double su[D][D], sp[D][D], sq[D][D], svg[D][D], Dvg[D][D];
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
          for (int j = 0; j < D; ++j) Dvg[i][j] = Dv[i][j] + Dg[i][j];
        sigma(Du, su);
        sigma(Dp, sp);
        sigma(Dq, sq);
        sigma(Dvg, svg);
        double up = 0.0, vq = 0.0;   // sigma(u):eps(p), sigma(v+g):eps(q)
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
          for (int j = 0; j < D; ++j) {
            up += su[i][j] * 0.5 * (Dp[i][j] + Dp[j][i]);
            vq += svg[i][j] * 0.5 * (Dq[i][j] + Dq[j][i]);
          }
        const double A = coef[e];
        const double scal = 0.5 * alpha * ww + ve * A * (up + vq);
        double gmv[3];
        kuhn_grad<D>(g, p, m, gmv);
#pragma unroll
        for (int k = 0; k < D; ++k) {
          double t = 0.0;   // (T grad lambda_m)_k, T = Du^T sp + Dp^T su + Dv^T sq + Dq^T svg
#pragma unroll
          for (int j = 0; j < D; ++j) {
            double tkj = 0.0;
#pragma unroll
            for (int r = 0; r < D; ++r)
              tkj += Du[r][k] * sp[r][j] + Dp[r][k] * su[r][j] + Dv[r][k] * sq[r][j] + Dq[r][k] * svg[r][j];
            t += tkj * gmv[j];
          }
          double s0 = 0.0;   // int_e S0_k lambda_m = -alpha sum_j (Dg)_{jk} (M_e w_j)_m
#pragma unroll
          for (int j = 0; j < D; ++j) s0 += Dg[j][k] * Mw[j];
          acc[k] += scal * gmv[k] - ve * A * t - alpha * s0;
        }
      }
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const long long i = (long long)D * a + k;
      b[i] = add ? b[i] + acc[k] : acc[k];
    }
  }
}

// ------------------------------------------------------------------------------ host
fo_status fo_inverse_create(fo_problem *p, const fo_model_desc *desc) {
  fo_ctx *ctx = p->ctx;
  const Grid &g = p->mesh->g;
  fo_inv *iv = new fo_inv();
  p->inv = iv;
  const size_t nd = (size_t)p->ndof, nc = (size_t)p->ncases, S = g.dim == 2 ? 7 : 15, blk = (size_t)g.dim * g.dim;
  auto add = [&](void **ptr, size_t bytes) { iv->allocs.push_back({ptr, bytes}); };
  add((void **)&iv->v, sizeof(double) * nd * nc);
  add((void **)&iv->q, sizeof(double) * nd * nc);
  add((void **)&iv->g, sizeof(double) * nd * nc);
  add((void **)&iv->r, sizeof(double) * nd);
  add((void **)&iv->W, sizeof(double) * S * blk * (size_t)g.num_nodes);
  add((void **)&iv->W32, sizeof(float) * S * blk * (size_t)g.num_nodes);
  add((void **)&iv->dinv, sizeof(double) * nd);
  add((void **)&iv->dinv32, sizeof(float) * nd);
  add((void **)&iv->dirb, nd);
  add((void **)&iv->none, nd);
  add((void **)&iv->gamma1, (size_t)g.num_nodes);
  for (auto &e : iv->allocs) FO_TRY(fo_alloc(ctx, e.first, e.second));
  cudaStream_t s = ctx->stream;
  FO_CU(ctx, cudaMemcpyAsync(iv->g, desc->meas, sizeof(double) * nd * nc, cudaMemcpyHostToDevice, s));
  FO_CU(ctx, cudaMemsetAsync(iv->v, 0, sizeof(double) * nd * nc, s));
  FO_CU(ctx, cudaMemsetAsync(iv->q, 0, sizeof(double) * nd * nc, s));
  FO_CU(ctx, cudaMemsetAsync(iv->none, 0, nd, s));
  const int blocks = fo_blocks_for(g.num_nodes, FO_BLOCK, 65536);
  if (g.dim == 2) k_inv_masks<2><<<blocks, FO_BLOCK, 0, s>>>(g, desc->gamma1_faces, iv->gamma1, iv->dirb);
  else k_inv_masks<3><<<blocks, FO_BLOCK, 0, s>>>(g, desc->gamma1_faces, iv->gamma1, iv->dirb);
  fo_note_launch(1);
  FO_CU(ctx, cudaGetLastError());
  FO_CU(ctx, cudaStreamSynchronize(s));   // the host array may be reused
  return FO_OK;
}

void fo_inverse_destroy(fo_problem *p) {
  if (!p->inv) return;
  for (auto &e : p->inv->allocs) fo_free(p->ctx, *e.first, e.second);
  delete p->inv;
  p->inv = nullptr;
}

// Runs f with the problem's operator replaced by the boundary-clamped one (the solvers read the
// problem's rows, inverse diagonals and Dirichlet mask).
template <class F>
static fo_status with_boundary_rows(fo_problem *p, F &&f) {
  fo_inv *iv = p->inv;
  std::swap(p->Wst, iv->W);
  std::swap(p->Wst32, iv->W32);
  std::swap(p->dinv_state, iv->dinv);
  std::swap(p->dinv_state32, iv->dinv32);
  std::swap(p->dir, iv->dirb);
  const fo_status s = f();
  std::swap(p->Wst, iv->W);
  std::swap(p->Wst32, iv->W32);
  std::swap(p->dinv_state, iv->dinv);
  std::swap(p->dinv_state32, iv->dinv32);
  std::swap(p->dir, iv->dirb);
  return s;
}

static fo_status inv_rows(fo_problem *p, const uint8_t *mask) {
  fo_inv *iv = p->inv;
  return fo_launch_stencil_on(p, p->mesh->g, p->coef, mask, iv->W, iv->W32, iv->dinv, iv->dinv32);
}

static void add_stats(fo_solve_stats &t, const fo_solve_stats &s) {
  t.iterations += s.iterations;
  t.outer_iterations += s.outer_iterations;
  t.operator_applies += s.operator_applies;
  t.rel_residual = std::max(t.rel_residual, s.rel_residual);
}

fo_status fo_inverse_states(fo_problem *p, const fo_solve_opts *o, fo_solve_stats *st) {
  fo_ctx *ctx = p->ctx;
  fo_inv *iv = p->inv;
  const Grid &g = p->mesh->g;
  const long long nd = p->ndof;
  const int blocks = fo_blocks_for(g.num_nodes, FO_BLOCK, 65536);
  // v_k's right-hand sides -K g_k at the interior DOFs (held in q_k until the solves), with the
  // operator that clamps nothing; then the boundary-clamped rows for the solves
  FO_TRY(inv_rows(p, iv->none));
  for (int k = 0; k < p->ncases; ++k) {
    const double *gk = iv->g + (size_t)k * nd;
    double *rk = iv->q + (size_t)k * nd;
    if (g.dim == 2) {
      StencilOp<2, 2, true, double> op;
      op.g = g;
      op.W = iv->W;
      k_inv_apply<2><<<blocks, FO_BLOCK, 0, ctx->stream>>>(op, gk, iv->dirb, -1.0, rk);
    } else {
      StencilOp<3, 3, true, double> op;
      op.g = g;
      op.W = iv->W;
      k_inv_apply<3><<<blocks, FO_BLOCK, 0, ctx->stream>>>(op, gk, iv->dirb, -1.0, rk);
    }
    fo_note_launch(1);
    FO_CU(ctx, cudaGetLastError());
  }
  FO_TRY(inv_rows(p, iv->dirb));
  iv->rows_epoch = p->coef_epoch;
  fo_solve_stats tot;
  memset(&tot, 0, sizeof tot);
  fo_status res = FO_OK;
  for (int k = 0; k < p->ncases; ++k) {
    fo_solve_stats s;
    memset(&s, 0, sizeof s);
    fo_status r = fo_state_pcg(p, p->load + (size_t)k * nd, p->u + (size_t)k * nd, o, &s);
    if (r != FO_OK && r != FO_ENOCONV) return r;
    if (r != FO_OK) res = r;
    add_stats(tot, s);
  }
  fo_solve_opts oj = *o;
  oj.precond = FO_PC_JACOBI;
  for (int k = 0; k < p->ncases; ++k) {
    fo_solve_stats s;
    memset(&s, 0, sizeof s);
    const fo_status r = with_boundary_rows(
        p, [&] { return fo_state_pcg(p, iv->q + (size_t)k * nd, iv->v + (size_t)k * nd, &oj, &s); });
    if (r != FO_OK && r != FO_ENOCONV) return r;
    if (r != FO_OK) res = r;
    add_stats(tot, s);
  }
  FO_CU(ctx, cudaMemsetAsync(iv->q, 0, sizeof(double) * nd * p->ncases, ctx->stream));   // until the adjoints
  if (st) *st = tot;
  return res;
}

fo_status fo_inverse_adjoints(fo_problem *p, const fo_solve_opts *o, fo_solve_stats *st) {
  fo_ctx *ctx = p->ctx;
  fo_inv *iv = p->inv;
  const Grid &g = p->mesh->g;
  const long long nd = p->ndof;
  if (iv->rows_epoch != p->coef_epoch) {
    FO_TRY(inv_rows(p, iv->dirb));
    iv->rows_epoch = p->coef_epoch;
  }
  const int blocks = fo_blocks_for(g.num_nodes, FO_BLOCK, 1024);
  const double al = p->desc.kv_alpha, be = p->desc.kv_beta;
  fo_solve_opts oa = *o;
  oa.warm_start = 0;
  fo_solve_opts oj = oa;
  oj.precond = FO_PC_JACOBI;
  fo_solve_stats tot;
  memset(&tot, 0, sizeof tot);
  fo_status res = FO_OK;
  for (int k = 0; k < p->ncases; ++k) {
    const double *uk = p->u + (size_t)k * nd, *vk = iv->v + (size_t)k * nd, *gk = iv->g + (size_t)k * nd;
    if (g.dim == 2)
      k_inv_cost_rhs<2><<<blocks, FO_BLOCK, 0, ctx->stream>>>(g, uk, vk, gk, iv->gamma1, p->dir, iv->dirb, al, be, p->rhs,
                                                             iv->r, p->red);
    else
      k_inv_cost_rhs<3><<<blocks, FO_BLOCK, 0, ctx->stream>>>(g, uk, vk, gk, iv->gamma1, p->dir, iv->dirb, al, be, p->rhs,
                                                             iv->r, p->red);
    fo_note_launch(1);
    FO_CU(ctx, cudaGetLastError());
    fo_solve_stats s;
    memset(&s, 0, sizeof s);
    fo_status r = fo_state_pcg(p, p->rhs, p->p + (size_t)k * nd, &oa, &s);
    if (r != FO_OK && r != FO_ENOCONV) return r;
    if (r != FO_OK) res = r;
    add_stats(tot, s);
    memset(&s, 0, sizeof s);
    r = with_boundary_rows(p, [&] { return fo_state_pcg(p, iv->r, iv->q + (size_t)k * nd, &oj, &s); });
    if (r != FO_OK && r != FO_ENOCONV) return r;
    if (r != FO_OK) res = r;
    add_stats(tot, s);
  }
  p->rhs_valid = false;
  if (st) *st = tot;
  return res;
}

fo_status fo_inverse_cost(fo_problem *p, double *J) {
  fo_ctx *ctx = p->ctx;
  fo_inv *iv = p->inv;
  const Grid &g = p->mesh->g;
  const long long nd = p->ndof;
  const int blocks = fo_blocks_for(g.num_nodes, FO_BLOCK, 1024);
  double tot = 0.0;
  for (int k = 0; k < p->ncases; ++k) {
    const double *uk = p->u + (size_t)k * nd, *vk = iv->v + (size_t)k * nd, *gk = iv->g + (size_t)k * nd;
    if (g.dim == 2)
      k_inv_cost_rhs<2><<<blocks, FO_BLOCK, 0, ctx->stream>>>(g, uk, vk, gk, iv->gamma1, p->dir, iv->dirb, 0.0, 0.0,
                                                             nullptr, nullptr, p->red);
    else
      k_inv_cost_rhs<3><<<blocks, FO_BLOCK, 0, ctx->stream>>>(g, uk, vk, gk, iv->gamma1, p->dir, iv->dirb, 0.0, 0.0,
                                                             nullptr, nullptr, p->red);
    k_inv_total<<<1, 64, 0, ctx->stream>>>(p->red, blocks, p->red + 4096);
    fo_note_launch(2);
    FO_CU(ctx, cudaGetLastError());
    FO_CU(ctx, cudaMemcpyAsync(ctx->h_scalars, p->red + 4096, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    FO_CU(ctx, cudaStreamSynchronize(ctx->stream));
    tot += 0.5 * p->desc.kv_alpha * ctx->h_scalars[0] + 0.5 * p->desc.kv_beta * ctx->h_scalars[1];
  }
  *J = tot;
  return FO_OK;
}

fo_status fo_inverse_shape(fo_problem *p) {
  fo_ctx *ctx = p->ctx;
  fo_inv *iv = p->inv;
  const Grid &g = p->mesh->g;
  const long long nd = p->ndof;
  const int blocks = fo_blocks_for(g.num_nodes, FO_BLOCK, 65536);
  for (int k = 0; k < p->ncases; ++k) {
    const size_t o = (size_t)k * nd;
    if (g.dim == 2)
      k_inv_shape<2><<<blocks, FO_BLOCK, 0, ctx->stream>>>(g, p->coef, p->lame_lambda, p->lame_mu, p->desc.kv_alpha,
                                                          p->u + o, iv->v + o, p->p + o, iv->q + o, iv->g + o, p->rhs,
                                                          k > 0);
    else
      k_inv_shape<3><<<blocks, FO_BLOCK, 0, ctx->stream>>>(g, p->coef, p->lame_lambda, p->lame_mu, p->desc.kv_alpha,
                                                          p->u + o, iv->v + o, p->p + o, iv->q + o, iv->g + o, p->rhs,
                                                          k > 0);
    fo_note_launch(1);
    FO_CU(ctx, cudaGetLastError());
  }
  return FO_OK;
}
