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
// same coefficients, with a multigrid hierarchy of its own.  The lifting -K g_k of v_k's right-hand side needs the
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
  const size_t nd = (size_t)p->ndof, nc = (size_t)p->ncases, S = (size_t)fo_row_slots(g.dim), blk = (size_t)g.dim * g.dim;
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
  fo_mg_release(p->ctx, p->inv->mgb);
  for (auto &e : p->inv->allocs) fo_free(p->ctx, *e.first, e.second);
  delete p->inv;
  p->inv = nullptr;
}

// Runs f with the problem's operator replaced by the boundary-clamped one (the solvers read the
// problem's rows, inverse diagonals, Dirichlet mask and multigrid hierarchy; the clamped
// operator keeps a hierarchy of its own, built from the same coefficients on first use).
template <class F>
static fo_status with_boundary_rows(fo_problem *p, F &&f) {
  fo_inv *iv = p->inv;
  auto swap_all = [&] {
    std::swap(p->Wst, iv->W);
    std::swap(p->Wst32, iv->W32);
    std::swap(p->dinv_state, iv->dinv);
    std::swap(p->dinv_state32, iv->dinv32);
    std::swap(p->dir, iv->dirb);
    std::swap(p->mg, iv->mgb);
  };
  swap_all();
  const fo_status s = f();
  swap_all();
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
  for (int k = 0; k < p->ncases; ++k) {
    fo_solve_stats s;
    memset(&s, 0, sizeof s);
    const fo_status r = with_boundary_rows(
        p, [&] { return fo_state_pcg(p, iv->q + (size_t)k * nd, iv->v + (size_t)k * nd, o, &s); });
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
    r = with_boundary_rows(p, [&] { return fo_state_pcg(p, iv->r, iv->q + (size_t)k * nd, &oa, &s); });
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

// ------------------------------------------------------------- Dirichlet extension (Sec. 5.7)
// Per component: eta = the given values on the nodes of the listed faces, and the P1 Laplacian of
// eta vanishes at every other node (int D eta : D zeta = 0 for zeta zero on those faces).  Written
// eta = fix + x with fix the values on the faces (zero elsewhere) and x zero there:
// L_b x = -(L fix) at the free nodes, L the Laplacian rows without clamped nodes and L_b with the
// face nodes clamped; Jacobi-preconditioned CG per component, host-driven.
template <int D>
__global__ void k_ext_setup(Grid g, uint32_t faces, const double *vals, uint8_t *mask, double *fix, double *ones_e) {
  const long long N = g.num_nodes;
  for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < N; a += (long long)gridDim.x * blockDim.x) {
    int idx[3];
    node_ijk(g, a, idx);
    bool on = false;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      if (idx[c] == 0 && (faces & (1u << (2 * c)))) on = true;
      if (idx[c] == g.n[c] && (faces & (1u << (2 * c + 1)))) on = true;
    }
    mask[a] = on ? 1 : 0;
#pragma unroll
    for (int c = 0; c < D; ++c) fix[c * N + a] = on ? vals[a * D + c] : 0.0;   // component-major
  }
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < g.num_elems;
       e += (long long)gridDim.x * blockDim.x)
    ones_e[e] = 1.0;
}

// y = scale * L x at the nodes mask leaves free (0 at masked nodes); x read unmasked
template <int D>
__global__ void k_ext_apply(StencilOp<D, 1, true, double> op, const double *x, const uint8_t *mask, double scale,
                            double *y) {
  op.sweep(VecX<double>{x}, [&](long long a, const double (&ax)[1]) { y[a] = mask[a] ? 0.0 : scale * ax[0]; });
}

// per-block partials of (a . b) and (c . d)
__global__ void k_ext_dots(const double *a, const double *b, const double *c, const double *d, long long n,
                           double *partials) {
  __shared__ double smem[64];
  double s[2] = {0.0, 0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    s[0] += a[i] * b[i];
    s[1] += c[i] * d[i];
  }
  block_sum<2>(s, smem);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = s[0];
    partials[2 * blockIdx.x + 1] = s[1];
  }
}

// x += alpha p; r -= alpha q; z = dinv r
__global__ void k_ext_update(double *x, double *r, double *z, const double *p, const double *q, const double *dinv,
                             double alpha, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    x[i] += alpha * p[i];
    const double ri = r[i] - alpha * q[i];
    r[i] = ri;
    z[i] = dinv[i] * ri;
  }
}

// p = z + beta p
__global__ void k_ext_dir(double *p, const double *z, double beta, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] = z[i] + beta * p[i];
}

// eta (interleaved) = fix + x (component-major)
__global__ void k_ext_out(const double *fix, const double *x, long long N, int D, double *eta) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N * D; i += (long long)gridDim.x * blockDim.x) {
    const long long a = i / D, c = i % D;
    eta[i] = fix[c * N + a] + x[c * N + a];
  }
}

extern "C" fo_status fo_dirichlet_extension(fo_mesh *m, uint32_t faces, const double *values, double *out,
                                            const fo_solve_opts *opts) {
  if (!m || !values || !out) return FO_EINVAL;
  fo_ctx *ctx = m->ctx;
  if (m->um) return fo_fail(ctx, FO_EINVAL, "the Dirichlet extension runs on box meshes");
  if (faces == 0) return fo_fail(ctx, FO_EINVAL, "no face to extend from");
  fo_solve_opts def;
  fo_solve_opts_default(&def);
  const fo_solve_opts *o = opts ? opts : &def;
  const Grid &g = m->g;
  const int D = g.dim;
  const long long N = g.num_nodes, S = fo_row_slots(D);
  std::vector<std::pair<void **, size_t>> al;
  double *vals, *fix, *x, *r, *z, *p, *q, *W, *dinv, *ones, *part;
  float *W32, *dinv32;
  uint8_t *mask;
  al.push_back({(void **)&vals, sizeof(double) * N * D});
  al.push_back({(void **)&fix, sizeof(double) * N * D});
  al.push_back({(void **)&x, sizeof(double) * N * D});
  al.push_back({(void **)&r, sizeof(double) * N});
  al.push_back({(void **)&z, sizeof(double) * N});
  al.push_back({(void **)&p, sizeof(double) * N});
  al.push_back({(void **)&q, sizeof(double) * N});
  al.push_back({(void **)&W, sizeof(double) * S * N});
  al.push_back({(void **)&W32, sizeof(float) * S * N});
  al.push_back({(void **)&dinv, sizeof(double) * N});
  al.push_back({(void **)&dinv32, sizeof(float) * N});
  al.push_back({(void **)&ones, sizeof(double) * g.num_elems});
  al.push_back({(void **)&mask, (size_t)N});
  al.push_back({(void **)&part, sizeof(double) * 2048});
  fo_status st = FO_OK;
  size_t done = 0;
  for (; done < al.size() && st == FO_OK; ++done) st = fo_alloc(ctx, al[done].first, al[done].second);
  auto release = [&] {
    cudaStreamSynchronize(ctx->stream);
    for (size_t i = 0; i < done; ++i) fo_free(ctx, *al[i].first, al[i].second);
  };
  if (st != FO_OK) {
    release();
    return st;
  }
  cudaStream_t s = ctx->stream;
  const int blocks = fo_blocks_for(N, FO_BLOCK, 1024);
  std::vector<double> hp(2048);
  int iters = 0;
  auto run = [&]() -> fo_status {
    FO_CU(ctx, cudaMemcpyAsync(vals, values, sizeof(double) * N * D, cudaMemcpyHostToDevice, s));
    if (D == 2) k_ext_setup<2><<<fo_blocks_for(std::max(N, g.num_elems), FO_BLOCK, 65536), FO_BLOCK, 0, s>>>(
        g, faces, vals, mask, fix, ones);
    else k_ext_setup<3><<<fo_blocks_for(std::max(N, g.num_elems), FO_BLOCK, 65536), FO_BLOCK, 0, s>>>(
        g, faces, vals, mask, fix, ones);
    fo_note_launch(1);
    FO_CU(ctx, cudaMemsetAsync(x, 0, sizeof(double) * N * D, s));
    // right-hand sides -(L fix) with the rows that clamp nothing (mask of zeros: r as scratch)
    FO_CU(ctx, cudaMemsetAsync(r, 0, (size_t)N, s));   // r's first N bytes, zero, serve as the empty mask
    FO_TRY(fo_launch_scalar_stencil(ctx, g, ones, (const uint8_t *)r, W, W32, dinv, dinv32));
    for (int c = 0; c < D; ++c) {
      if (D == 2) {
        StencilOp<2, 1, true, double> op;
        op.g = g;
        op.W = W;
        k_ext_apply<2><<<blocks, FO_BLOCK, 0, s>>>(op, fix + c * N, mask, -1.0, x + c * N);   // rhs in x for now
      } else {
        StencilOp<3, 1, true, double> op;
        op.g = g;
        op.W = W;
        k_ext_apply<3><<<blocks, FO_BLOCK, 0, s>>>(op, fix + c * N, mask, -1.0, x + c * N);
      }
      fo_note_launch(1);
    }
    FO_TRY(fo_launch_scalar_stencil(ctx, g, ones, mask, W, W32, dinv, dinv32));
    for (int c = 0; c < D; ++c) {
      double *xc = x + c * N;
      // r = b (x = 0), z = D^{-1} r, p = z; the right-hand side moves from xc into r
      FO_CU(ctx, cudaMemcpyAsync(r, xc, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
      FO_CU(ctx, cudaMemsetAsync(xc, 0, sizeof(double) * N, s));
      FO_CU(ctx, cudaMemsetAsync(p, 0, sizeof(double) * N, s));   // (read, times zero, by the update)
      FO_CU(ctx, cudaMemsetAsync(q, 0, sizeof(double) * N, s));
      k_ext_update<<<blocks, FO_BLOCK, 0, s>>>(xc, r, z, p, q, dinv, 0.0, N);   // z = D^{-1} r
      FO_CU(ctx, cudaMemcpyAsync(p, z, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
      k_ext_dots<<<blocks, FO_BLOCK, 0, s>>>(r, z, r, r, N, part);
      fo_note_launch(2);
      auto sums = [&](double *a, double *b2) -> fo_status {
        FO_CU(ctx, cudaMemcpyAsync(hp.data(), part, sizeof(double) * 2 * blocks, cudaMemcpyDeviceToHost, s));
        FO_CU(ctx, cudaStreamSynchronize(s));
        double t0 = 0, t1 = 0;
        for (int b = 0; b < blocks; ++b) {
          t0 += hp[2 * b];
          t1 += hp[2 * b + 1];
        }
        *a = t0;
        *b2 = t1;
        return FO_OK;
      };
      double rz = 0, rr = 0;
      FO_TRY(sums(&rz, &rr));
      const double bb = rr;
      int it = 0;
      while (rr > o->rtol * o->rtol * bb && it < o->maxit && bb > 0) {
        if (D == 2) {
          StencilOp<2, 1, true, double> op;
          op.g = g;
          op.W = W;
          k_ext_apply<2><<<blocks, FO_BLOCK, 0, s>>>(op, p, mask, 1.0, q);
        } else {
          StencilOp<3, 1, true, double> op;
          op.g = g;
          op.W = W;
          k_ext_apply<3><<<blocks, FO_BLOCK, 0, s>>>(op, p, mask, 1.0, q);
        }
        k_ext_dots<<<blocks, FO_BLOCK, 0, s>>>(p, q, p, q, N, part);
        fo_note_launch(2);
        double pq = 0, unused = 0;
        FO_TRY(sums(&pq, &unused));
        if (!(pq > 0)) break;
        const double alpha = rz / pq;
        k_ext_update<<<blocks, FO_BLOCK, 0, s>>>(xc, r, z, p, q, dinv, alpha, N);
        k_ext_dots<<<blocks, FO_BLOCK, 0, s>>>(r, z, r, r, N, part);
        fo_note_launch(2);
        double rz1 = 0;
        FO_TRY(sums(&rz1, &rr));
        k_ext_dir<<<blocks, FO_BLOCK, 0, s>>>(p, z, rz1 / rz, N);
        fo_note_launch(1);
        rz = rz1;
        ++it;
      }
      iters += it;
      if (!std::isfinite(rr)) return fo_fail(ctx, FO_ENAN, "NaN in the Dirichlet extension");
      if (it >= o->maxit) return fo_fail(ctx, FO_ENOCONV, "Dirichlet extension reached maxit=%d", o->maxit);
    }
    // eta = fix + x, interleaved, into vals (device) and out to the host
    k_ext_out<<<fo_blocks_for(N * D, FO_BLOCK, 65536), FO_BLOCK, 0, s>>>(fix, x, N, D, vals);
    fo_note_launch(1);
    FO_CU(ctx, cudaGetLastError());
    FO_CU(ctx, cudaMemcpyAsync(out, vals, sizeof(double) * N * D, cudaMemcpyDeviceToHost, s));
    FO_CU(ctx, cudaStreamSynchronize(s));
    return FO_OK;
  };
  st = run();
  release();
  return st;
}
