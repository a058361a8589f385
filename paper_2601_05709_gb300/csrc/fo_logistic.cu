// The logistic population model on the box grid (Sec. 6.4): Newton's method for the nonlinear
// state, the linear adjoint and the shape-derivative right-hand side.
//
// State: F(u)(v) = int grad u . grad v - r int u (1 - u / K) v = 0 for all P1 v (eq. log_weak),
// K = K_e the element coefficient (carrying capacity: a_in inside, a_out outside, eq.
// log_KOmega).  Jacobian DF(u)(du, v) = int grad du . grad v + int w du v with the P1 weight
// w = r (2u / K_e - 1) on each element.  The cubic integrals are exact: on a simplex e with
// vertex values x, y, z of three P1 functions,
//   int_e x y z = c3 |e| (Sx Sy Sz + Sx (y.z) + Sy (x.z) + Sz (x.y) + 2 sum_c x_c y_c z_c),
// c3 = d! / (d + 3)!, S. the vertex sums (the monomial integrals over a simplex, d! a1! a2!
// ... / (d + sum a)!, summed over the products).  Per node a (vertex m of each of its
// simplices) this gives
//   int_e w psi_m psi_l = c3 |e| (Sw + w_m + w_l)  (l != m),   c3 |e| (2 Sw + 4 w_m)  (l = m),
//   int_e u^2 psi_m     = c3 |e| (Su^2 + Qu + 2 Su u_m + 2 u_m^2)   (Qu = sum u_c^2),
//   int_e u psi_m       = |e| (Su + u_m) / ((d + 1)(d + 2)).
// One kernel per Newton step writes the Jacobian's stencil rows (difference form, the exact
// row sum c3 |e| (d + 3)(Sw + w_m) in slot 0, the stiffness rows summing to zero) and -F(u),
// and the host solves DF du = -F with the Jacobi-preconditioned CG of the state options.
//
// Adjoint (linear): DF(u) p = (int psi_a)_a (DF is symmetric).  Cost J = -int u.
// Shape derivative: S0^J = 0, S1^J = (grad u . grad p - u - r u (1 - u / K) p) I
// - (grad u (x) grad p + grad p (x) grad u), plus lambda chi / V I; b[a, k] = sum over the
// simplices of node a of int_e (S1 grad psi_a)_k.
#include <cmath>
#include <cstring>

#include "fo_internal.cuh"
#include "fo_ops.cuh"

namespace {

template <int D>
struct LogC {
  static constexpr double c3 = D == 2 ? 1.0 / 60.0 : 1.0 / 120.0;   // d! / (d + 3)!
};

// Block maximum of two non-negative values (thread 0 holds the result); order-independent.
__device__ __forceinline__ void block_max2(double (&v)[2], double *smem /* [64] */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v[0] = fmax(v[0], __shfl_xor_sync(0xffffffffu, v[0], o));
    v[1] = fmax(v[1], __shfl_xor_sync(0xffffffffu, v[1], o));
  }
  __syncthreads();
  if (lane == 0) {
    smem[warp] = v[0];
    smem[32 + warp] = v[1];
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int w = 1; w < nw; ++w) {
      v[0] = fmax(v[0], smem[w]);
      v[1] = fmax(v[1], smem[32 + w]);
    }
}

}  // namespace

// Jacobian rows W (slot-major, difference form), their FP32 copy, the inverse diagonals, -F
// (zero on Dirichlet DOFs) and per-block partial sums of ||F||^2 over the free DOFs.
template <int D>
__global__ void k_logistic_newton(Grid g, const double *Kc, const uint8_t *dir, double r, const double *u, double *W,
                                  float *W32, double *dinv, float *dinv32, double *mF, double *partials) {
  constexpr int S = ST<D>::S;
  __shared__ double smem[32];
  const long long N = g.num_nodes;
  const double ve = g.vol_e, c3 = g.vol_e * LogC<D>::c3, mref = g.vol_e / ((D + 1) * (D + 2));
  double nrm[1] = {0.0};
  for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < N; a += (long long)gridDim.x * blockDim.x) {
    int idx[3];
    node_ijk(g, a, idx);
    double us[S][1];
    load_stencil<D, 1, double>(g, idx, a, VecX<double>{u}, us);
    double w[S];
#pragma unroll
    for (int s = 0; s < S; ++s) w[s] = 0.0;
    double R = 0.0, F = 0.0;
#pragma unroll
    for (int p = 0; p < KP<D>::P; ++p)
#pragma unroll
      for (int m = 0; m <= D; ++m) {
        long long e;
        if (!elem_of<D>(g, idx, p, m, e)) continue;
        const double iK = 1.0 / Kc[e];
        double uv[D + 1], wv[D + 1], Su = 0.0, Qu = 0.0, Sw = 0.0;
#pragma unroll
        for (int l = 0; l <= D; ++l) {
          uv[l] = us[rel_slot<D>(p, m, l)][0];
          wv[l] = r * (2.0 * uv[l] * iK - 1.0);
          Su += uv[l];
          Qu += uv[l] * uv[l];
          Sw += wv[l];
        }
        double gm[3];
        kuhn_grad<D>(g, p, m, gm);
        double gum = 0.0;   // grad u . grad lambda_m
#pragma unroll
        for (int l = 0; l <= D; ++l) {
          double gl[3];
          kuhn_grad<D>(g, p, l, gl);
          double dot = 0.0;
#pragma unroll
          for (int k = 0; k < D; ++k) dot += gm[k] * gl[k];
          gum += uv[l] * dot;
          w[rel_slot<D>(p, m, l)] += ve * dot + c3 * (l == m ? 2.0 * Sw + 4.0 * wv[m] : Sw + wv[m] + wv[l]);
        }
        R += c3 * (D + 3) * (Sw + wv[m]);
        F += ve * gum - r * mref * (Su + uv[m]) + r * iK * c3 * (Su * Su + Qu + 2.0 * Su * uv[m] + 2.0 * uv[m] * uv[m]);
      }
    // eliminated Dirichlet columns leave the row; Dirichlet rows become identity rows
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const long long nb = slot_node<D>(g, idx, a, s);
      if (nb >= 0 && dir[nb]) {
        R -= w[s];
        w[s] = 0.0;
      }
    }
    const bool da = dir[a] != 0;
    const double diag = da ? 1.0 : w[0];
    dinv[a] = 1.0 / diag;
    dinv32[a] = (float)(1.0 / diag);
    if (da) {
#pragma unroll
      for (int s = 0; s < S; ++s) w[s] = 0.0;
      R = 1.0;
      F = 0.0;
    }
    w[0] = R;
#pragma unroll
    for (int s = 0; s < ST<D>::SH; ++s) {   // the stored slots (the Jacobian is symmetric)
      W[s * N + a] = w[s];
      W32[s * N + a] = (float)w[s];
    }
    mF[a] = -F;
    nrm[0] += F * F;
  }
  block_sum<1>(nrm, smem);
  if (threadIdx.x == 0) partials[blockIdx.x] = nrm[0];
}

// the block partials summed by one warp in a fixed order
__global__ void k_logistic_total(const double *partials, int nblocks, double *out) {
  double t = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += 32) t += partials[b];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  if (threadIdx.x == 0) out[0] = t;
}

// u += du; per-block maxima of |du| and |u| (after the update)
__global__ void k_logistic_update(double *u, const double *du, long long n, double *partials) {
  __shared__ double smem[64];
  double v[2] = {0.0, 0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double ui = u[i] + du[i];
    u[i] = ui;
    v[0] = fmax(v[0], fabs(du[i]));
    v[1] = fmax(v[1], fabs(ui));
  }
  block_max2(v, smem);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = v[0];
    partials[2 * blockIdx.x + 1] = v[1];
  }
}

__global__ void k_logistic_max_total(const double *partials, int nblocks, double *out) {
  double a = 0.0, b = 0.0;
  for (int k = threadIdx.x; k < nblocks; k += 32) {
    a = fmax(a, partials[2 * k]);
    b = fmax(b, partials[2 * k + 1]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a = fmax(a, __shfl_down_sync(0xffffffffu, a, o));
    b = fmax(b, __shfl_down_sync(0xffffffffu, b, o));
  }
  if (threadIdx.x == 0) {
    out[0] = a;
    out[1] = b;
  }
}

// adjoint load (int psi_a)_a = |e| / (d + 1) per simplex around node a; zero on Dirichlet DOFs
template <int D>
__global__ void k_logistic_adjoint_load(Grid g, const uint8_t *dir, double *b) {
  for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < g.num_nodes;
       a += (long long)gridDim.x * blockDim.x) {
    int idx[3];
    node_ijk(g, a, idx);
    int count = 0;
#pragma unroll
    for (int p = 0; p < KP<D>::P; ++p)
#pragma unroll
      for (int m = 0; m <= D; ++m) {
        long long e;
        if (elem_of<D>(g, idx, p, m, e)) ++count;
      }
    b[a] = dir[a] ? 0.0 : count * (g.vol_e / (D + 1));
  }
}

// b[D a + k] (+)= sum over the simplices (p, m) of node a of int_e (S1 grad lambda_m)_k
template <int D>
__global__ void k_logistic_shape(Grid g, const double *Kc, const uint8_t *chi, const double *chif, double r,
                                 double cvol, const double *u, const double *pa, double *b, int add) {
  constexpr int S = ST<D>::S;
  const double ve = g.vol_e, c3 = g.vol_e * LogC<D>::c3, mref = g.vol_e / ((D + 1) * (D + 2));
  for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < g.num_nodes;
       a += (long long)gridDim.x * blockDim.x) {
    int idx[3];
    node_ijk(g, a, idx);
    double us[S][1], ps[S][1];
    load_stencil<D, 1, double>(g, idx, a, VecX<double>{u}, us);
    load_stencil<D, 1, double>(g, idx, a, VecX<double>{pa}, ps);
    double acc[D];
#pragma unroll
    for (int k = 0; k < D; ++k) acc[k] = 0.0;
#pragma unroll
    for (int p = 0; p < KP<D>::P; ++p)
#pragma unroll
      for (int m = 0; m <= D; ++m) {
        long long e;
        if (!elem_of<D>(g, idx, p, m, e)) continue;
        double gu[3] = {0, 0, 0}, gp[3] = {0, 0, 0};
#pragma unroll
        for (int l = 0; l < D; ++l) {
          const int ax = kperm<D>(p, l);
          const int s0 = rel_slot<D>(p, m, l), s1 = rel_slot<D>(p, m, l + 1);
          gu[ax] = (us[s1][0] - us[s0][0]) * g.inv_h[ax];
          gp[ax] = (ps[s1][0] - ps[s0][0]) * g.inv_h[ax];
        }
        double Su = 0.0, Sp = 0.0, Qu = 0.0, Uup = 0.0, UUP = 0.0;
#pragma unroll
        for (int l = 0; l <= D; ++l) {
          const int sl = rel_slot<D>(p, m, l);
          const double ul = us[sl][0], pl = ps[sl][0];
          Su += ul;
          Sp += pl;
          Qu += ul * ul;
          Uup += ul * pl;
          UUP += ul * ul * pl;
        }
        const double int_u = ve * Su / (D + 1);
        const double int_up = mref * (Su * Sp + Uup);
        const double int_uup = c3 * (Su * Su * Sp + 2.0 * Su * Uup + Sp * Qu + 2.0 * UUP);
        double gug = 0.0;
#pragma unroll
        for (int k = 0; k < D; ++k) gug += gu[k] * gp[k];
        const double cv = chif ? chif[e] * cvol : (chi[e] ? cvol : 0.0);
        const double scal = ve * (gug + cv) - int_u - r * int_up + (r / Kc[e]) * int_uup;
        double gm[3];
        kuhn_grad<D>(g, p, m, gm);
        double gpm = 0.0, gum = 0.0;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          gpm += gp[k] * gm[k];
          gum += gu[k] * gm[k];
        }
#pragma unroll
        for (int k = 0; k < D; ++k) acc[k] += scal * gm[k] - ve * (gu[k] * gpm + gp[k] * gum);
      }
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const long long i = (long long)D * a + k;
      b[i] = add ? b[i] + acc[k] : acc[k];
    }
  }
}

// ------------------------------------------------------------------------------ host
static fo_status logistic_rows(fo_problem *p, const double *u, double *mF, double *normF) {
  fo_ctx *ctx = p->ctx;
  const Grid &g = p->mesh->g;
  const int blocks = fo_blocks_for(g.num_nodes, FO_BLOCK, 1024);
  double *part = p->red, *res = p->red + 2048;
  const double r = p->desc.growth_rate;
  if (g.dim == 2)
    k_logistic_newton<2><<<blocks, FO_BLOCK, 0, ctx->stream>>>(g, p->coef, p->dir, r, u, p->Wst, p->Wst32,
                                                                p->dinv_state, p->dinv_state32, mF, part);
  else
    k_logistic_newton<3><<<blocks, FO_BLOCK, 0, ctx->stream>>>(g, p->coef, p->dir, r, u, p->Wst, p->Wst32,
                                                                p->dinv_state, p->dinv_state32, mF, part);
  k_logistic_total<<<1, 32, 0, ctx->stream>>>(part, blocks, res);
  fo_note_launch(2);
  FO_CU(ctx, cudaGetLastError());
  if (normF) {
    FO_CU(ctx, cudaMemcpyAsync(ctx->h_scalars, res, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    FO_CU(ctx, cudaStreamSynchronize(ctx->stream));
    *normF = std::sqrt(ctx->h_scalars[0]);
  }
  return FO_OK;
}

// Newton's method: each step builds DF(u) and -F(u) in one pass, stops on the residual
// criterion, else solves DF du = -F (Jacobi-PCG, FP64 or mixed per the options) and updates u.
// Work vectors: -F in the load field, du in the right-hand-side field (both free for this model
// while the state is solved).
fo_status fo_logistic_state(fo_problem *p, const fo_solve_opts *o, fo_solve_stats *st, int *steps_out) {
  fo_ctx *ctx = p->ctx;
  const long long n = p->ndof;
  const fo_model_desc &d = p->desc;
  const double rtol = d.newton_rtol > 0 ? d.newton_rtol : 1e-13;
  const double atol = d.newton_atol > 0 ? d.newton_atol : 0.0;
  const int maxit = d.newton_maxit > 0 ? d.newton_maxit : 50;
  if (!o->warm_start || !p->u_valid)
    FO_CU(ctx, cudaMemcpyAsync(p->u, p->f, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
  fo_solve_opts lo = *o;
  lo.warm_start = 0;
  lo.precond = FO_PC_JACOBI;
  fo_solve_stats tot;
  memset(&tot, 0, sizeof tot);
  double *mF = p->load, *du = p->rhs;
  p->rhs_valid = false;
  double F0 = 0.0, Fk = 0.0;
  int k = 0;
  bool done = false;
  for (;; ++k) {
    FO_TRY(logistic_rows(p, p->u, mF, &Fk));
    if (!std::isfinite(Fk)) return fo_fail(ctx, FO_ENAN, "non-finite Newton residual at step %d", k);
    if (k == 0) F0 = Fk;
    if (Fk <= rtol * F0 + atol) {
      done = true;
      break;
    }
    if (k >= maxit) break;
    fo_solve_stats ls;
    memset(&ls, 0, sizeof ls);
    const fo_status s = fo_state_pcg(p, mF, du, &lo, &ls);
    if (s != FO_OK && s != FO_ENOCONV) return s;
    tot.iterations += ls.iterations;
    tot.operator_applies += ls.operator_applies;
    const int blocks = fo_blocks_for(n, FO_BLOCK, 1024);
    k_logistic_update<<<blocks, FO_BLOCK, 0, ctx->stream>>>(p->u, du, n, p->red);
    k_logistic_max_total<<<1, 32, 0, ctx->stream>>>(p->red, blocks, p->red + 2048);
    fo_note_launch(2);
    FO_CU(ctx, cudaGetLastError());
    FO_CU(ctx, cudaMemcpyAsync(ctx->h_scalars, p->red + 2048, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                               ctx->stream));
    FO_CU(ctx, cudaStreamSynchronize(ctx->stream));
    if (ctx->h_scalars[0] <= 1e-14 * ctx->h_scalars[1]) {   // stagnation: the update is at rounding level
      FO_TRY(logistic_rows(p, p->u, mF, &Fk));
      done = true;
      ++k;
      break;
    }
  }
  p->u_valid = true;
  tot.outer_iterations = k;
  tot.rel_residual = F0 > 0 ? Fk / F0 : 0.0;
  if (st) *st = tot;
  if (steps_out) *steps_out = k;
  if (!done) return fo_fail(ctx, FO_ENOCONV, "Newton reached %d steps (||F|| / ||F0|| = %.3e)", maxit, tot.rel_residual);
  return FO_OK;
}

// DF(u) p = (int psi_a)_a with the rows rebuilt at the current state.
fo_status fo_logistic_adjoint(fo_problem *p, const fo_solve_opts *o, fo_solve_stats *st) {
  fo_ctx *ctx = p->ctx;
  const Grid &g = p->mesh->g;
  FO_TRY(logistic_rows(p, p->u, p->load, nullptr));
  const int blocks = fo_blocks_for(g.num_nodes, FO_BLOCK, 65536);
  if (g.dim == 2) k_logistic_adjoint_load<2><<<blocks, FO_BLOCK, 0, ctx->stream>>>(g, p->dir, p->rhs);
  else k_logistic_adjoint_load<3><<<blocks, FO_BLOCK, 0, ctx->stream>>>(g, p->dir, p->rhs);
  fo_note_launch(1);
  FO_CU(ctx, cudaGetLastError());
  fo_solve_opts lo = *o;
  lo.warm_start = 0;
  lo.precond = FO_PC_JACOBI;
  const fo_status s = fo_state_pcg(p, p->rhs, p->p, &lo, st);
  p->rhs_valid = false;
  return s;
}

// b = sum_e int_e S1 grad psi (Sec. 6.4) + lambda chi / V I, into p->rhs (add: accumulate)
fo_status fo_launch_logistic_shape(fo_problem *p, double lambda, const double *chif, double inv_V, int add) {
  fo_ctx *ctx = p->ctx;
  const Grid &g = p->mesh->g;
  const int blocks = fo_blocks_for(g.num_nodes, FO_BLOCK, 65536);
  const double r = p->desc.growth_rate, cv = lambda * inv_V;
  if (g.dim == 2)
    k_logistic_shape<2><<<blocks, FO_BLOCK, 0, ctx->stream>>>(g, p->coef, p->chi, chif, r, cv, p->u, p->p, p->rhs, add);
  else
    k_logistic_shape<3><<<blocks, FO_BLOCK, 0, ctx->stream>>>(g, p->coef, p->chi, chif, r, cv, p->u, p->p, p->rhs, add);
  fo_note_launch(1);
  FO_CU(ctx, cudaGetLastError());
  return FO_OK;
}
