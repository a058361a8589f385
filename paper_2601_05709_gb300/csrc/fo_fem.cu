// Element-level kernels: mesh build, masks, loads, ersatz coefficient, operator applies and
// diagonals, functionals, the shape-derivative right-hand side and the initial level set.
#include <cmath>
#include <vector>

#include "fo_internal.cuh"
#include "fo_ops.cuh"
#include "fo_umesh.cuh"

// -------------------------------------------------------------------------- mesh build
// Coordinates lo + (hi - lo) * i / n in that operation order; connectivity of simplex
// P*c + p along the Kuhn path of permutation p.
template <int D>
__global__ void k_mesh_build(Grid g, int32_t *cells, double *coords) {
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long a = tid; a < g.num_nodes; a += stride) {
    int idx[3];
    node_ijk(g, a, idx);
#pragma unroll
    for (int k = 0; k < D; ++k) {
      double t = (g.hi[k] - g.lo[k]) * (double)idx[k];
      t = t / (double)g.n[k];
      coords[a * D + k] = g.lo[k] + t;
    }
  }
  for (long long e = tid; e < g.num_elems; e += stride) {
    const long long c = e / KP<D>::P;
    const int p = (int)(e % KP<D>::P);
    int ci[3];
    ci[0] = (int)(c % g.n[0]);
    long long t = c / g.n[0];
    ci[1] = (int)(t % g.n[1]);
    ci[2] = (int)(t / g.n[1]);
    long long v = ci[0] + g.stride[1] * ci[1] + (D == 3 ? g.stride[2] * ci[2] : 0);
    cells[e * (D + 1)] = (int32_t)v;
#pragma unroll
    for (int l = 0; l < D; ++l) {
      v += g.stride[kperm<D>(p, l)];
      cells[e * (D + 1) + l + 1] = (int32_t)v;
    }
  }
}

fo_status fo_launch_mesh_build(fo_mesh *m) {
  const Grid &g = m->g;
  long long n = g.num_nodes > g.num_elems ? g.num_nodes : g.num_elems;
  int blocks = fo_blocks_for(n, FO_BLOCK, 65536);
  if (g.dim == 2) k_mesh_build<2><<<blocks, FO_BLOCK, 0, m->ctx->stream>>>(g, m->d_cells, m->d_coords);
  else k_mesh_build<3><<<blocks, FO_BLOCK, 0, m->ctx->stream>>>(g, m->d_cells, m->d_coords);
  fo_note_launch(1);
  FO_CU(m->ctx, cudaGetLastError());
  return FO_OK;
}

// -------------------------------------------------------------------------------- masks
struct MaskArgs {
  Grid g;
  uint32_t faces;     // Dirichlet faces of the state
  int ncomp;
  int vel_dirichlet;
  int n_omega0;
  double o_lo[4][3], o_hi[4][3];
  int n_vol;                       // constraint regions (bit j of regmask)
  double v_lo[4][3], v_hi[4][3];
};

template <int D>
__global__ void k_masks(MaskArgs m, const double *coords, uint8_t *dir, uint8_t *vdir, uint8_t *omega0,
                        uint8_t *regmask) {
  const Grid &g = m.g;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long a = tid; a < g.num_nodes; a += stride) {
    int idx[3];
    node_ijk(g, a, idx);
    bool on = false, bd = false;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      if (idx[k] == 0) { bd = true; on |= (m.faces >> (2 * k)) & 1u; }
      if (idx[k] == g.n[k]) { bd = true; on |= (m.faces >> (2 * k + 1)) & 1u; }
    }
    for (int c = 0; c < m.ncomp; ++c) dir[a * m.ncomp + c] = on ? 1 : 0;
    vdir[a] = (m.vel_dirichlet && bd) ? 1 : 0;
  }
  // Omega_0: centroid ((x_0 + x_1) + x_2 (+ x_3)) / (D+1) strictly inside one of the boxes
  for (long long e = tid; e < g.num_elems; e += stride) {
    const long long c = e / KP<D>::P;
    const int p = (int)(e % KP<D>::P);
    int ci[3];
    ci[0] = (int)(c % g.n[0]);
    long long t = c / g.n[0];
    ci[1] = (int)(t % g.n[1]);
    ci[2] = (int)(t / g.n[1]);
    long long v = ci[0] + g.stride[1] * ci[1] + (D == 3 ? g.stride[2] * ci[2] : 0);
    double s[3];
#pragma unroll
    for (int k = 0; k < D; ++k) s[k] = coords[v * D + k];
#pragma unroll
    for (int l = 0; l < D; ++l) {
      v += g.stride[kperm<D>(p, l)];
#pragma unroll
      for (int k = 0; k < D; ++k) s[k] = s[k] + coords[v * D + k];
    }
    bool in = false;
    for (int b = 0; b < m.n_omega0; ++b) {
      bool ok = true;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const double x = s[k] / (double)(D + 1);
        ok = ok && (x > m.o_lo[b][k]) && (x < m.o_hi[b][k]);
      }
      in = in || ok;
    }
    omega0[e] = in ? 1 : 0;
    unsigned rm = 0;
    for (int b = 0; b < m.n_vol; ++b) {
      bool ok = true;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const double x = s[k] / (double)(D + 1);
        ok = ok && (x > m.v_lo[b][k]) && (x < m.v_hi[b][k]);
      }
      if (ok) rm |= 1u << b;
    }
    regmask[e] = (uint8_t)rm;
  }
}

fo_status fo_launch_masks(fo_problem *p) {
  const Grid &g = p->mesh->g;
  MaskArgs m{};
  m.g = g;
  m.faces = p->desc.dirichlet_faces;
  m.ncomp = p->ncomp;
  m.vel_dirichlet = p->desc.velocity_dirichlet;
  m.n_omega0 = p->desc.omega0_weight != 0.0 ? p->desc.n_omega0 : 0;
  for (int b = 0; b < 4; ++b)
    for (int k = 0; k < 3; ++k) {
      m.o_lo[b][k] = p->desc.omega0_lo[b][k];
      m.o_hi[b][k] = p->desc.omega0_hi[b][k];
      m.v_lo[b][k] = p->desc.volume_lo[b][k];
      m.v_hi[b][k] = p->desc.volume_hi[b][k];
    }
  m.n_vol = p->nvol;
  long long n = g.num_nodes > g.num_elems ? g.num_nodes : g.num_elems;
  int blocks = fo_blocks_for(n, FO_BLOCK, 65536);
  if (g.dim == 2)
    k_masks<2><<<blocks, FO_BLOCK, 0, p->ctx->stream>>>(m, p->mesh->d_coords, p->dir, p->vdir, p->omega0, p->regmask);
  else
    k_masks<3><<<blocks, FO_BLOCK, 0, p->ctx->stream>>>(m, p->mesh->d_coords, p->dir, p->vdir, p->omega0, p->regmask);
  fo_note_launch(1);
  FO_CU(p->ctx, cudaGetLastError());
  return FO_OK;
}

// -------------------------------------------------------------------------------- loads
struct LoadArgs {
  Grid g;
  int ncomp;
  int n_tr;
  int tr_face[4];
  double tr_vec[4][3];
  double mref;   // |e| / ((D+1)(D+2))
};

// F = M f (P1 body source) + constant tractions (|f| / D per facet vertex); point loads are
// added on the host side of the launch; Dirichlet DOFs are zeroed.
template <int D>
__global__ void k_loads(LoadArgs L, const double *f, const uint8_t *dir, double *F) {
  const Grid &g = L.g;
  for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < g.num_nodes;
       a += (long long)gridDim.x * blockDim.x) {
    int idx[3];
    node_ijk(g, a, idx);
    double acc[3] = {0, 0, 0};
    if (f) {
      double fs[ST<D>::S][1];
      load_stencil<D, 1, double>(g, idx, a, VecX<double>{f}, fs);
      double s = 0;
#pragma unroll
      for (int p = 0; p < KP<D>::P; ++p)
#pragma unroll
        for (int m = 0; m <= D; ++m) {
          long long e;
          if (!elem_of<D>(g, idx, p, m, e)) continue;
          double sum = fs[0][0];
#pragma unroll
          for (int l = 0; l <= D; ++l) sum += fs[rel_slot<D>(p, m, l)][0];
          s += L.mref * sum;
        }
      acc[0] = s;
    }
    for (int t = 0; t < L.n_tr; ++t) {
      const int axis = L.tr_face[t] >> 1, side = L.tr_face[t] & 1;
      if (idx[axis] != (side ? g.n[axis] : 0)) continue;
      int cnt = 0;
      if (D == 2) {
        const int o = 1 - axis;
        cnt = (idx[o] + 1 <= g.n[o]) + (idx[o] - 1 >= 0);
      } else {
        const int o1 = axis == 0 ? 1 : 0, o2 = axis == 2 ? 1 : 2;
        for (int q = 0; q < 2; ++q)
          for (int m = 0; m <= 2; ++m) {
            const int ax[2] = {q == 0 ? o1 : o2, q == 0 ? o2 : o1};
            int c[3] = {idx[0], idx[1], idx[2]};
            for (int l = 0; l < m; ++l) c[ax[l]] -= 1;
            if (c[o1] < 0 || c[o1] >= g.n[o1] || c[o2] < 0 || c[o2] >= g.n[o2]) continue;
            ++cnt;
          }
      }
      const double w = g.facet_area[axis] / D * cnt;
      for (int c = 0; c < L.ncomp; ++c) acc[c] += w * L.tr_vec[t][c];
    }
    for (int c = 0; c < L.ncomp; ++c) F[a * L.ncomp + c] = dir[a * L.ncomp + c] ? 0.0 : acc[c];
  }
}

__global__ void k_point_loads(int n, const long long *node, const double *vec, int ncomp, const uint8_t *dir,
                              double *F) {
  // single thread: point loads applied in order (deterministic)
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  for (int i = 0; i < n; ++i)
    for (int c = 0; c < ncomp; ++c) {
      long long k = node[i] * ncomp + c;
      if (!dir[k]) F[k] += vec[i * 3 + c];
    }
}

// One load vector per load case k (case-major at p->load + k N_dof): f in case 0 only, each
// case's own tractions and point loads.
fo_status fo_launch_loads(fo_problem *p) {
  const Grid &g = p->mesh->g;
  fo_ctx *ctx = p->ctx;
  for (int k = 0; k < p->ncases; ++k) {
    double *F = p->load + (size_t)k * p->ndof;
    LoadArgs L{};
    L.g = g;
    L.ncomp = p->ncomp;
    for (int t = 0; t < p->desc.n_tractions; ++t) {
      if (p->desc.traction_case[t] != k && p->ncases > 1) continue;
      L.tr_face[L.n_tr] = p->desc.traction_face[t];
      for (int c = 0; c < 3; ++c) L.tr_vec[L.n_tr][c] = p->desc.traction_vec[t][c];
      ++L.n_tr;
    }
    L.mref = g.vol_e / ((g.dim + 1) * (g.dim + 2));
    const double *f = (p->desc.kind != FO_ELASTIC && k == 0) ? p->f : nullptr;
    int blocks = fo_blocks_for(g.num_nodes, FO_BLOCK, 65536);
    if (g.dim == 2) k_loads<2><<<blocks, FO_BLOCK, 0, ctx->stream>>>(L, f, p->dir, F);
    else k_loads<3><<<blocks, FO_BLOCK, 0, ctx->stream>>>(L, f, p->dir, F);
    fo_note_launch(1);
    FO_CU(ctx, cudaGetLastError());
    long long nodes[4];
    double vec[12];
    int np = 0;
    for (int i = 0; i < p->desc.n_point_loads; ++i) {
      if (p->desc.point_case[i] != k && p->ncases > 1) continue;
      nodes[np] = p->desc.point_node[i];
      for (int c = 0; c < 3; ++c) vec[np * 3 + c] = p->desc.point_vec[i][c];
      ++np;
    }
    if (np > 0) {
      // stage the point loads through the reduction buffer (fits: <= 4 * (1 + 3) doubles)
      char *stage = (char *)p->red;
      FO_CU(ctx, cudaMemcpyAsync(stage, nodes, sizeof(long long) * np, cudaMemcpyHostToDevice, ctx->stream));
      FO_CU(ctx, cudaMemcpyAsync(stage + 64, vec, sizeof(double) * 3 * np, cudaMemcpyHostToDevice, ctx->stream));
      k_point_loads<<<1, 1, 0, ctx->stream>>>(np, (const long long *)stage, (const double *)(stage + 64), p->ncomp,
                                              p->dir, F);
      fo_note_launch(1);
      FO_CU(ctx, cudaGetLastError());
      FO_CU(ctx, cudaStreamSynchronize(ctx->stream));   // host staging arrays go out of scope
    }
  }
  return FO_OK;
}

// -------------------------------------------------------------------------- coefficient
// chi_e = [(phi_0 + phi_1) + phi_2 (+ phi_3) < 0], A_e = chi ? a_in : a_out (times k).
template <int D>
__global__ void k_coefficients(Grid g, const double *phi, double a_in, double a_out, double *coef, float *coef32,
                               uint8_t *chi, int cut, double *chif) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < g.num_elems;
       e += (long long)gridDim.x * blockDim.x) {
    const long long c = e / KP<D>::P;
    const int p = (int)(e % KP<D>::P);
    int ci[3];
    ci[0] = (int)(c % g.n[0]);
    long long t = c / g.n[0];
    ci[1] = (int)(t % g.n[1]);
    ci[2] = (int)(t / g.n[1]);
    long long v = ci[0] + g.stride[1] * ci[1] + (D == 3 ? g.stride[2] * ci[2] : 0);
    double pv[D + 1];
    pv[0] = phi[v];
    double s = pv[0];
#pragma unroll
    for (int l = 0; l < D; ++l) {
      v += g.stride[kperm<D>(p, l)];
      pv[l + 1] = phi[v];
      s = s + pv[l + 1];
    }
    if (cut) {   // exact cut-cell fraction (FO_COEF_CUT)
      const double f = cut_fraction<D>(pv);
      const double A = a_out + (a_in - a_out) * f;
      coef[e] = A;
      coef32[e] = (float)A;
      chi[e] = f > 0.0 ? 1 : 0;
      chif[e] = f;
      continue;
    }
    const bool in = s < 0.0;
    const double A = in ? a_in : a_out;
    coef[e] = A;
    coef32[e] = (float)A;
    chi[e] = in ? 1 : 0;
    chif[e] = in ? 1.0 : 0.0;
  }
}

fo_status fo_launch_coefficients(fo_problem *p) {
  const Grid &g = p->mesh->g;
  const double k = p->desc.kind == FO_HELMHOLTZ ? p->desc.k : 1.0;
  const int cut = p->desc.coef_rule == FO_COEF_CUT;
  int blocks = fo_blocks_for(g.num_elems, FO_BLOCK, 65536);
  if (g.dim == 2)
    k_coefficients<2><<<blocks, FO_BLOCK, 0, p->ctx->stream>>>(g, p->phi, p->desc.a_in * k, p->desc.a_out * k,
                                                                p->coef, p->coef32, p->chi, cut, p->chif);
  else
    k_coefficients<3><<<blocks, FO_BLOCK, 0, p->ctx->stream>>>(g, p->phi, p->desc.a_in * k, p->desc.a_out * k,
                                                                p->coef, p->coef32, p->chi, cut, p->chif);
  fo_note_launch(1);
  FO_CU(p->ctx, cudaGetLastError());
  return FO_OK;
}

// generic node-parallel apply / diag
template <int D, class Op, class X, typename T>
__global__ void k_apply(Op op, X x, T *y) {
  for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < op.g.num_nodes;
       a += (long long)gridDim.x * blockDim.x) {
    int idx[3];
    node_ijk(op.g, a, idx);
    T out[Op::NPN];
    op.row(a, idx, x, out);
#pragma unroll
    for (int c = 0; c < Op::NPN; ++c) y[a * Op::NPN + c] = out[c];
  }
}

template <int D, class Op, typename T>
__global__ void k_diag_inv(Op op, T *dinv, float *dinv32) {
  for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < op.g.num_nodes;
       a += (long long)gridDim.x * blockDim.x) {
    int idx[3];
    node_ijk(op.g, a, idx);
    T out[Op::NPN];
    op.diag(a, idx, out);
#pragma unroll
    for (int c = 0; c < Op::NPN; ++c) {
      dinv[a * Op::NPN + c] = T(1) / out[c];
      if (dinv32) dinv32[a * Op::NPN + c] = (float)(T(1) / out[c]);
    }
  }
}

__global__ void k_d2f(const double *x, float *y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}
__global__ void k_f2d(const float *x, double *y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = (double)x[i];
}

// ------------------------------------------------------------------ stored stencils
// Stored rows are kept in difference form: slot 0 holds the row sum R (an NPN x NPN block, or
// its diagonal), slots s >= 1 the neighbour blocks W_s, and the row is applied as
//   (A x)_a = R x_a + sum_{s >= 1} W_s (x_{nb(s)} - x_a),
// which is the same operator.  R is formed from the exact row sums of the element matrices: the
// stiffness rows sum to zero exactly (sum_l grad lambda_l = 0), so R holds only the mass-type and
// penalty terms, minus the weights of eliminated Dirichlet columns.  Rounding in the stored
// weights then perturbs the operator like rounding in the differences of a matrix-free apply:
// it keeps the constant (rigid translation) kernel, which matters in FP32 for these
// ill-conditioned systems.  Dirichlet DOFs: identity row, eliminated column.  The Jacobi
// inverse diagonal of the (eliminated) operator is written alongside.
//
// State rows of node a, summed over the simplices (p, m) around it (the node is vertex m):
// scalar (NPN = 1): A_e|e| grad lambda_m . grad lambda_l + omega^2 |e| (1 + delta_ml) / ((D+1)(D+2))
// with A_e = coef (A times k); elastic (NPN = D): the block
// A_e|e| [lam (g_m)_i (g_l)_j + mu (g_m)_j (g_l)_i + mu delta_ij g_m . g_l] coupling component i of
// the node with component j of vertex l (plane strain / 3D Lame constants).
template <int D, int NPN>
__device__ __forceinline__ void state_stencil_node(const Grid &g, long long a, const double *coef, const uint8_t *dir,
                                                   double lam, double mu, double w2, double *W, float *W32,
                                                   double *dinv, float *dinv32) {
  constexpr int S = ST<D>::S, BLK = NPN * NPN;
  const long long N = g.num_nodes;
  const double mref = g.vol_e / ((D + 1) * (D + 2));
  int idx[3];
  node_ijk(g, a, idx);
  double w[S][BLK];
  double R[BLK];
#pragma unroll
  for (int k = 0; k < BLK; ++k) R[k] = 0.0;
#pragma unroll
  for (int s = 0; s < S; ++s)
#pragma unroll
    for (int k = 0; k < BLK; ++k) w[s][k] = 0.0;
#pragma unroll
  for (int p = 0; p < KP<D>::P; ++p)
#pragma unroll
    for (int m = 0; m <= D; ++m) {
      long long e;
      if (!elem_of<D>(g, idx, p, m, e)) continue;
      const double Av = coef[e] * g.vol_e;
      double gm[3];
      kuhn_grad<D>(g, p, m, gm);
      if (NPN == 1 && w2 != 0.0) R[0] += w2 * mref * (D + 2);   // mass row sum
#pragma unroll
      for (int l = 0; l <= D; ++l) {
        const int sl = rel_slot<D>(p, m, l);
        double gl[3];
        kuhn_grad<D>(g, p, l, gl);
        double dot = 0.0;
#pragma unroll
        for (int k = 0; k < D; ++k) dot += gm[k] * gl[k];
        if (NPN == 1) {
          w[sl][0] += Av * dot + (w2 != 0.0 ? w2 * mref * (l == m ? 2.0 : 1.0) : 0.0);
        } else {
#pragma unroll
          for (int i = 0; i < NPN; ++i)
#pragma unroll
            for (int j = 0; j < NPN; ++j)
              w[sl][i * NPN + j] += Av * (lam * gm[i] * gl[j] + mu * gm[j] * gl[i] + (i == j ? mu * dot : 0.0));
        }
      }
    }
  // eliminated Dirichlet columns leave the row: their weight comes off the row sum
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const long long nb = slot_node<D>(g, idx, a, s);
#pragma unroll
    for (int j = 0; j < NPN; ++j)
      if (nb >= 0 && dir[nb * NPN + j])
#pragma unroll
        for (int i = 0; i < NPN; ++i) {
          R[i * NPN + j] -= w[s][i * NPN + j];
          w[s][i * NPN + j] = 0.0;
        }
  }
#pragma unroll
  for (int i = 0; i < NPN; ++i) {
    const double diag = dir[a * NPN + i] ? 1.0 : w[0][i * NPN + i];
    dinv[a * NPN + i] = 1.0 / diag;
    dinv32[a * NPN + i] = (float)(1.0 / diag);
    if (dir[a * NPN + i]) {   // identity row
#pragma unroll
      for (int s = 0; s < S; ++s)
#pragma unroll
        for (int j = 0; j < NPN; ++j) w[s][i * NPN + j] = 0.0;
#pragma unroll
      for (int j = 0; j < NPN; ++j) R[i * NPN + j] = (i == j) ? 1.0 : 0.0;
    }
  }
#pragma unroll
  for (int k = 0; k < BLK; ++k) w[0][k] = R[k];
#pragma unroll
  for (int s = 0; s < ST<D>::SH; ++s)   // the stored slots (symmetric operator)
#pragma unroll
    for (int k = 0; k < BLK; ++k) {
      W[(s * BLK + k) * N + a] = w[s][k];
      W32[(s * BLK + k) * N + a] = (float)w[s][k];
    }
}

template <int D, int NPN>
__global__ void k_state_stencil(Grid g, const double *coef, const uint8_t *dir, double lam, double mu, double w2,
                                double *W, float *W32, double *dinv, float *dinv32) {
  for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < g.num_nodes;
       a += (long long)gridDim.x * blockDim.x)
    state_stencil_node<D, NPN>(g, a, coef, dir, lam, mu, w2, W, W32, dinv, dinv32);
}

// The rows of several grids in one launch (the coarse levels of a multigrid hierarchy: each
// launch of a small level is latency bound, ~30 us whatever its size, so one launch for all
// of them costs about what one did).  Blocks first_block[k] .. first_block[k + 1] - 1 take
// level k, one node per thread.
template <int D, int NPN>
__global__ void k_state_stencil_levels(StencilLevels L, double lam, double mu, double w2) {
  int k = 0;
  while (k + 1 < L.n && (int)blockIdx.x >= L.first_block[k + 1]) ++k;
  const long long a = (long long)((int)blockIdx.x - L.first_block[k]) * blockDim.x + threadIdx.x;
  if (a < L.g[k].num_nodes)
    state_stencil_node<D, NPN>(L.g[k], a, L.coef[k], L.dir[k], lam, mu, w2, L.W[k], L.W32[k], L.di[k], L.di32[k]);
}

// Rows of the velocity form B of node a (component-diagonal), in difference form as above: for
// every component the P1 Laplacian plus (alpha + gamma_0 chi_Omega0) times the consistent mass;
// for component c on a face normal to axis c also gamma_b times the facet mass of that face (the
// normal penalty couples only the normal component on an axis-aligned box).  H^1_0: identity
// rows on boundary nodes, eliminated columns.  The mass-type coefficient of element e is
// mcoef[e] when given (coarse multigrid levels: children means), else alpha + gamma_0 chi_Omega0;
// the H^1_0 mask of node a is vmask[a * vstride].  FP32 copies are written when W32 / dinv32
// are given.
template <int D>
__global__ void k_velocity_stencil(Grid g, const uint8_t *omega0, const double *mcoef, const uint8_t *vmask,
                                   int vstride, double alpha, double gamma0, double gammab, double *W, float *W32,
                                   double *dinv, float *dinv32) {
  constexpr int S = ST<D>::S;
  const long long N = g.num_nodes;
  const double mref = g.vol_e / ((D + 1) * (D + 2));
  for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < N; a += (long long)gridDim.x * blockDim.x) {
    int idx[3];
    node_ijk(g, a, idx);
    double w[S][D], R[D];
#pragma unroll
    for (int c = 0; c < D; ++c) R[c] = 0.0;
#pragma unroll
    for (int s = 0; s < S; ++s)
#pragma unroll
      for (int c = 0; c < D; ++c) w[s][c] = 0.0;
    if (vmask[a * vstride]) {
#pragma unroll
      for (int c = 0; c < D; ++c) {
        R[c] = 1.0;
        dinv[a * D + c] = 1.0;
        if (dinv32) dinv32[a * D + c] = 1.0f;
      }
    } else {
#pragma unroll
      for (int p = 0; p < KP<D>::P; ++p)
#pragma unroll
        for (int m = 0; m <= D; ++m) {
          long long e;
          if (!elem_of<D>(g, idx, p, m, e)) continue;
          const double wm = (mcoef ? mcoef[e] : alpha + (omega0[e] ? gamma0 : 0.0)) * mref;
#pragma unroll
          for (int c = 0; c < D; ++c) R[c] += wm * (D + 2);
          double gm[3];
          kuhn_grad<D>(g, p, m, gm);
#pragma unroll
          for (int l = 0; l <= D; ++l) {
            const int sl = rel_slot<D>(p, m, l);
            double gl[3];
            kuhn_grad<D>(g, p, l, gl);
            double dot = 0.0;
#pragma unroll
            for (int k = 0; k < D; ++k) dot += gm[k] * gl[k];
            const double v = g.vol_e * dot + wm * (l == m ? 2.0 : 1.0);
#pragma unroll
            for (int c = 0; c < D; ++c) w[sl][c] += v;
          }
        }
      if (gammab != 0.0) {
#pragma unroll
        for (int c = 0; c < D; ++c) {
          if (!(idx[c] == 0 || idx[c] == g.n[c])) continue;
          const double fm = gammab * g.facet_area[c] / (D * (D + 1));   // facet mass unit
          if (D == 2) {
            const int o = 1 - c;
#pragma unroll
            for (int sg = -1; sg <= 1; sg += 2) {
              if (idx[o] + sg < 0 || idx[o] + sg > g.n[o]) continue;
              int dl[3] = {0, 0, 0};
              dl[o] = sg;
              w[0][c] += 2.0 * fm;
              w[stencil_slot<D>(dl)][c] += fm;
              R[c] += 3.0 * fm;
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
                w[0][c] += 2.0 * fm;
                R[c] += 4.0 * fm;
#pragma unroll
                for (int l = 0; l <= 2; ++l) {
                  if (l == m) continue;
                  int dl[3] = {0, 0, 0};
                  for (int j = 0; j < 2; ++j) {
                    if (l > m && j >= m && j < l) dl[ax[j]] += 1;
                    if (l < m && j >= l && j < m) dl[ax[j]] -= 1;
                  }
                  w[stencil_slot<D>(dl)][c] += fm;
                }
              }
          }
        }
      }
#pragma unroll
      for (int s = 1; s < S; ++s) {
        const long long nb = slot_node<D>(g, idx, a, s);
        if (nb >= 0 && vmask[nb * vstride])
#pragma unroll
          for (int c = 0; c < D; ++c) {
            R[c] -= w[s][c];
            w[s][c] = 0.0;
          }
      }
#pragma unroll
      for (int c = 0; c < D; ++c) {
        dinv[a * D + c] = 1.0 / w[0][c];
        if (dinv32) dinv32[a * D + c] = (float)(1.0 / w[0][c]);
      }
    }
#pragma unroll
    for (int c = 0; c < D; ++c) w[0][c] = R[c];
#pragma unroll
    for (int s = 0; s < ST<D>::SH; ++s)   // the stored slots (symmetric operator)
#pragma unroll
      for (int c = 0; c < D; ++c) {
        W[(s * D + c) * N + a] = w[s][c];
        if (W32) W32[(s * D + c) * N + a] = (float)w[s][c];
      }
  }
}

// The state operator's stencil rows on grid g (the problem's grid or a coarser one) from
// element coefficients `coef` and the Dirichlet mask `dir` of that grid.
fo_status fo_launch_stencil_on(fo_problem *p, const Grid &g, const double *coef, const uint8_t *dir, double *W,
                               float *W32, double *di, float *di32) {
  int blocks = fo_blocks_for(g.num_nodes, FO_BLOCK, 65536);
  cudaStream_t s = p->ctx->stream;
  const double w2 = p->desc.kind == FO_HELMHOLTZ ? p->desc.omega * p->desc.omega : 0.0;
  if (p->desc.kind == FO_ELASTIC) {
    if (g.dim == 2)
      k_state_stencil<2, 2><<<blocks, FO_BLOCK, 0, s>>>(g, coef, dir, p->lame_lambda, p->lame_mu, 0.0, W, W32, di, di32);
    else
      k_state_stencil<3, 3><<<blocks, FO_BLOCK, 0, s>>>(g, coef, dir, p->lame_lambda, p->lame_mu, 0.0, W, W32, di, di32);
  } else {
    if (g.dim == 2) k_state_stencil<2, 1><<<blocks, FO_BLOCK, 0, s>>>(g, coef, dir, 0.0, 0.0, w2, W, W32, di, di32);
    else k_state_stencil<3, 1><<<blocks, FO_BLOCK, 0, s>>>(g, coef, dir, 0.0, 0.0, w2, W, W32, di, di32);
  }
  fo_note_launch(1);
  FO_CU(p->ctx, cudaGetLastError());
  return FO_OK;
}

fo_status fo_launch_stencil_levels(fo_problem *p, const StencilLevels &L) {
  if (L.n == 0) return FO_OK;
  const int blocks = L.first_block[L.n];
  cudaStream_t s = p->ctx->stream;
  const double w2 = p->desc.kind == FO_HELMHOLTZ ? p->desc.omega * p->desc.omega : 0.0;
  const int dim = L.g[0].dim;
  if (p->desc.kind == FO_ELASTIC) {
    if (dim == 2) k_state_stencil_levels<2, 2><<<blocks, FO_BLOCK, 0, s>>>(L, p->lame_lambda, p->lame_mu, 0.0);
    else k_state_stencil_levels<3, 3><<<blocks, FO_BLOCK, 0, s>>>(L, p->lame_lambda, p->lame_mu, 0.0);
  } else {
    if (dim == 2) k_state_stencil_levels<2, 1><<<blocks, FO_BLOCK, 0, s>>>(L, 0.0, 0.0, w2);
    else k_state_stencil_levels<3, 1><<<blocks, FO_BLOCK, 0, s>>>(L, 0.0, 0.0, w2);
  }
  fo_note_launch(1);
  FO_CU(p->ctx, cudaGetLastError());
  return FO_OK;
}

// Scalar P1 rows (coef-weighted Laplacian, no mass) on grid g with the Dirichlet mask dir.
fo_status fo_launch_scalar_stencil(fo_ctx *ctx, const Grid &g, const double *coef, const uint8_t *dir, double *W,
                                   float *W32, double *di, float *di32) {
  const int blocks = fo_blocks_for(g.num_nodes, FO_BLOCK, 65536);
  if (g.dim == 2) k_state_stencil<2, 1><<<blocks, FO_BLOCK, 0, ctx->stream>>>(g, coef, dir, 0.0, 0.0, 0.0, W, W32, di, di32);
  else k_state_stencil<3, 1><<<blocks, FO_BLOCK, 0, ctx->stream>>>(g, coef, dir, 0.0, 0.0, 0.0, W, W32, di, di32);
  fo_note_launch(1);
  FO_CU(ctx, cudaGetLastError());
  return FO_OK;
}

fo_status fo_launch_state_diag(fo_problem *p) {
  // the state operator's stencil rows (from the current coefficients) and its Jacobi diagonal
  return fo_launch_stencil_on(p, p->mesh->g, p->coef, p->dir, p->Wst, p->Wst32, p->dinv_state, p->dinv_state32);
}

// Velocity rows on grid g (the problem's or a coarser one) from a per-element mass-type
// coefficient and a per-DOF H^1_0 mask of that grid (component 0 of each node is read).
fo_status fo_launch_velocity_stencil_on(fo_problem *p, const Grid &g, const double *mcoef, const uint8_t *dofmask,
                                        double *W, float *W32, double *dinv, float *dinv32) {
  const int blocks = fo_blocks_for(g.num_nodes, FO_BLOCK, 65536);
  cudaStream_t s = p->ctx->stream;
  const double gb = p->desc.normal_penalty;
  if (g.dim == 2)
    k_velocity_stencil<2><<<blocks, FO_BLOCK, 0, s>>>(g, nullptr, mcoef, dofmask, 2, 0.0, 0.0, gb, W, W32, dinv, dinv32);
  else
    k_velocity_stencil<3><<<blocks, FO_BLOCK, 0, s>>>(g, nullptr, mcoef, dofmask, 3, 0.0, 0.0, gb, W, W32, dinv, dinv32);
  fo_note_launch(1);
  FO_CU(p->ctx, cudaGetLastError());
  return FO_OK;
}

fo_status fo_launch_velocity_diag(fo_problem *p) {
  // the velocity form does not depend on phi: its stencil is built once per problem
  const Grid &g = p->mesh->g;
  int blocks = fo_blocks_for(g.num_nodes, FO_BLOCK, 65536);
  cudaStream_t s = p->ctx->stream;
  const double gb = p->desc.normal_penalty, g0 = p->desc.omega0_weight, al = p->desc.alpha_mass;
  if (g.dim == 2)
    k_velocity_stencil<2><<<blocks, FO_BLOCK, 0, s>>>(g, p->omega0, nullptr, p->vdir, 1, al, g0, gb, p->Wvel, nullptr,
                                                      p->dinv_vel, nullptr);
  else
    k_velocity_stencil<3><<<blocks, FO_BLOCK, 0, s>>>(g, p->omega0, nullptr, p->vdir, 1, al, g0, gb, p->Wvel, nullptr,
                                                      p->dinv_vel, nullptr);
  fo_note_launch(1);
  FO_CU(p->ctx, cudaGetLastError());
  return FO_OK;
}

fo_status fo_launch_state_apply(fo_problem *p, const double *x, double *y, bool mask) {
  if (p->mesh->um) return fo_umesh_state_apply(p, x, y, false);   // general mesh (input masked)
  const Grid &g = p->mesh->g;
  int blocks = fo_blocks_for(g.num_nodes, FO_BLOCK, 65536);
  cudaStream_t s = p->ctx->stream;
  if (p->desc.kind == FO_ELASTIC) {
    if (g.dim == 2) {
      auto op = make_elastic_stencil<2, double>(p);
      if (mask) k_apply<2><<<blocks, FO_BLOCK, 0, s>>>(op, MaskedX<double>{x, p->dir}, y);
      else k_apply<2><<<blocks, FO_BLOCK, 0, s>>>(op, VecX<double>{x}, y);
    } else {
      auto op = make_elastic_stencil<3, double>(p);
      if (mask) k_apply<3><<<blocks, FO_BLOCK, 0, s>>>(op, MaskedX<double>{x, p->dir}, y);
      else k_apply<3><<<blocks, FO_BLOCK, 0, s>>>(op, VecX<double>{x}, y);
    }
  } else {
    if (g.dim == 2) {
      auto op = make_scalar_stencil<2, double>(p);
      if (mask) k_apply<2><<<blocks, FO_BLOCK, 0, s>>>(op, MaskedX<double>{x, p->dir}, y);
      else k_apply<2><<<blocks, FO_BLOCK, 0, s>>>(op, VecX<double>{x}, y);
    } else {
      auto op = make_scalar_stencil<3, double>(p);
      if (mask) k_apply<3><<<blocks, FO_BLOCK, 0, s>>>(op, MaskedX<double>{x, p->dir}, y);
      else k_apply<3><<<blocks, FO_BLOCK, 0, s>>>(op, VecX<double>{x}, y);
    }
  }
  fo_note_launch(1);
  FO_CU(p->ctx, cudaGetLastError());
  return FO_OK;
}

// FP32 operator of the mixed path, applied to double vectors (x masked, converted in the gather)
template <typename T>
struct MaskedCastX {
  const double *v;
  const uint8_t *dir;
  __device__ __forceinline__ T operator()(long long i) const { return dir[i] ? T(0) : (T)v[i]; }
};

template <int D, class Op>
__global__ void k_apply32(Op op, MaskedCastX<float> x, double *y) {
  for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < op.g.num_nodes;
       a += (long long)gridDim.x * blockDim.x) {
    int idx[3];
    node_ijk(op.g, a, idx);
    float out[Op::NPN];
    op.row(a, idx, x, out);
#pragma unroll
    for (int c = 0; c < Op::NPN; ++c) y[a * Op::NPN + c] = (double)out[c];
  }
}

fo_status fo_launch_state_apply32(fo_problem *p, const double *x, double *y) {
  const Grid &g = p->mesh->g;
  int blocks = fo_blocks_for(g.num_nodes, FO_BLOCK, 65536);
  cudaStream_t s = p->ctx->stream;
  MaskedCastX<float> mx{x, p->dir};
  if (p->desc.kind == FO_ELASTIC) {
    if (g.dim == 2) k_apply32<2><<<blocks, FO_BLOCK, 0, s>>>(make_elastic_stencil<2, float>(p), mx, y);
    else k_apply32<3><<<blocks, FO_BLOCK, 0, s>>>(make_elastic_stencil<3, float>(p), mx, y);
  } else {
    if (g.dim == 2) k_apply32<2><<<blocks, FO_BLOCK, 0, s>>>(make_scalar_stencil<2, float>(p), mx, y);
    else k_apply32<3><<<blocks, FO_BLOCK, 0, s>>>(make_scalar_stencil<3, float>(p), mx, y);
  }
  fo_note_launch(1);
  FO_CU(p->ctx, cudaGetLastError());
  return FO_OK;
}

fo_status fo_launch_velocity_apply(fo_problem *p, const double *x, double *y) {
  const Grid &g = p->mesh->g;
  int blocks = fo_blocks_for(g.num_nodes, FO_BLOCK, 65536);
  // H^1_0: boundary columns are dropped (rows are identity), as in the reduced system
  if (g.dim == 2)
    k_apply<2><<<blocks, FO_BLOCK, 0, p->ctx->stream>>>(make_velocity_stencil<2>(p), NodeMaskedX<double, 2>{x, p->vdir}, y);
  else
    k_apply<3><<<blocks, FO_BLOCK, 0, p->ctx->stream>>>(make_velocity_stencil<3>(p), NodeMaskedX<double, 3>{x, p->vdir}, y);
  fo_note_launch(1);
  FO_CU(p->ctx, cudaGetLastError());
  return FO_OK;
}

// --------------------------------------------------------------------------- functionals
// J and |Omega| as element sums: block partials, then one block adds them in a fixed order.
struct FuncArgs {
  Grid g;
  int kind;
  double lam, mu;
};

template <int D>
__global__ void k_functionals(FuncArgs f, const double *coef, const uint8_t *chi, const double *chif, const double *u,
                              const double *load, double *partials) {
  __shared__ double smem[32 * 2];
  const Grid &g = f.g;
  double v[2] = {0.0, 0.0};
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = tid; e < g.num_elems; e += stride) {
    const long long c = e / KP<D>::P;
    const int p = (int)(e % KP<D>::P);
    int ci[3];
    ci[0] = (int)(c % g.n[0]);
    long long t = c / g.n[0];
    ci[1] = (int)(t % g.n[1]);
    ci[2] = (int)(t / g.n[1]);
    long long vtx[D + 1];
    vtx[0] = ci[0] + g.stride[1] * ci[1] + (D == 3 ? g.stride[2] * ci[2] : 0);
#pragma unroll
    for (int l = 0; l < D; ++l) vtx[l + 1] = vtx[l] + g.stride[kperm<D>(p, l)];
    const double A = coef[e];
    if (f.kind == FO_ELASTIC) {
      double du[D][D];
#pragma unroll
      for (int l = 0; l < D; ++l) {
        const int ax = kperm<D>(p, l);
#pragma unroll
        for (int i = 0; i < D; ++i) du[i][ax] = (u[vtx[l + 1] * D + i] - u[vtx[l] * D + i]) * g.inv_h[ax];
      }
      double tr = 0;
#pragma unroll
      for (int i = 0; i < D; ++i) tr += du[i][i];
      double se = 0;   // sigma : eps = lam tr^2 + 2 mu eps : eps
#pragma unroll
      for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) {
          const double eij = 0.5 * (du[i][j] + du[j][i]);
          se += 2.0 * f.mu * eij * eij;
        }
      se += f.lam * tr * tr;
      v[0] += A * g.vol_e * se;
    } else if (f.kind == FO_HEAT) {
      double g2 = 0;
#pragma unroll
      for (int l = 0; l < D; ++l) {
        const int ax = kperm<D>(p, l);
        const double d = (u[vtx[l + 1]] - u[vtx[l]]) * g.inv_h[ax];
        g2 += d * d;
      }
      v[0] += A * g.vol_e * g2;
    } else if (f.kind == FO_LOGISTIC) {   // J = -int u
      double su = 0;
#pragma unroll
      for (int l = 0; l <= D; ++l) su += u[vtx[l]];
      v[0] -= g.vol_e * su / (D + 1);
    }
    v[1] += chif ? chif[e] * g.vol_e : (chi[e] ? g.vol_e : 0.0);
  }
  if (f.kind == FO_HELMHOLTZ) {   // J = F . u
    for (long long a = tid; a < g.num_nodes; a += stride) v[0] += load[a] * u[a];
  }
  block_sum<2>(v, smem);
  if (threadIdx.x == 0) {
    partials[blockIdx.x * 2 + 0] = v[0];
    partials[blockIdx.x * 2 + 1] = v[1];
  }
}

__global__ void k_finish_sum(const double *partials, int nblocks, int nr, double *out) {
  // one warp per value, fixed order
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (w >= nr) return;
  double t = 0;
  for (int b = lane; b < nblocks; b += 32) t += partials[(size_t)b * nr + w];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  if (lane == 0) out[w] = t;
}

fo_status fo_launch_functionals_on(fo_problem *p, const double *u, const double *load, double *J, double *vol) {
  const Grid &g = p->mesh->g;
  fo_ctx *ctx = p->ctx;
  FuncArgs f{g, p->desc.kind, p->lame_lambda, p->lame_mu};
  const int blocks = fo_blocks_for(g.num_elems, FO_BLOCK, 1024);
  double *part = p->red, *res = p->red + 2 * 1024;
  const double *chif = p->desc.coef_rule == FO_COEF_CUT ? p->chif : nullptr;
  if (g.dim == 2) k_functionals<2><<<blocks, FO_BLOCK, 0, ctx->stream>>>(f, p->coef, p->chi, chif, u, load, part);
  else k_functionals<3><<<blocks, FO_BLOCK, 0, ctx->stream>>>(f, p->coef, p->chi, chif, u, load, part);
  k_finish_sum<<<1, 64, 0, ctx->stream>>>(part, blocks, 2, res);
  fo_note_launch(2);
  FO_CU(ctx, cudaGetLastError());
  FO_CU(ctx, cudaMemcpyAsync(ctx->h_scalars, res, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  FO_CU(ctx, cudaStreamSynchronize(ctx->stream));
  *J = ctx->h_scalars[0];
  *vol = ctx->h_scalars[1];
  return FO_OK;
}

fo_status fo_launch_functionals(fo_problem *p, double *J, double *vol) {
  return fo_launch_functionals_on(p, p->u, p->load, J, vol);
}

// Volume of Omega in each constraint region: sum_e w_e |e| [e in R_j], w_e = chif_e (the
// material fraction, 0 / 1 for the one-point rule); |e| constant on the box grid (vol null).
__global__ void k_region_volumes(long long ne, const double *vol, double vol_e, const double *chif,
                                 const uint8_t *regmask, int nreg, double *partials) {
  __shared__ double smem[32 * 4];
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ne; e += (long long)gridDim.x * blockDim.x) {
    const double w = chif[e] * (vol ? vol[e] : vol_e);
    const unsigned rm = regmask[e];
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (j < nreg && ((rm >> j) & 1u)) v[j] += w;
  }
  block_sum<4>(v, smem);
  if (threadIdx.x == 0)
#pragma unroll
    for (int j = 0; j < 4; ++j) partials[blockIdx.x * 4 + j] = v[j];
}

// w_e = chif_e [e in R_j]: the weights of constraint j's volume term in the shape derivative
__global__ void k_region_weight(long long ne, const double *chif, const uint8_t *regmask, int j, double *w) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ne; e += (long long)gridDim.x * blockDim.x)
    w[e] = ((regmask[e] >> j) & 1u) ? chif[e] : 0.0;
}

fo_status fo_region_volumes(fo_problem *p, const double *vol, double *out) {
  fo_ctx *ctx = p->ctx;
  const long long ne = p->mesh->g.num_elems;
  const int blocks = fo_blocks_for(ne, FO_BLOCK, 1024);
  double *part = p->red, *res = p->red + 4 * 1024;
  k_region_volumes<<<blocks, FO_BLOCK, 0, ctx->stream>>>(ne, vol, p->mesh->g.vol_e, p->chif, p->regmask, p->nvol, part);
  k_finish_sum<<<1, 128, 0, ctx->stream>>>(part, blocks, 4, res);
  fo_note_launch(2);
  FO_CU(ctx, cudaGetLastError());
  FO_CU(ctx, cudaMemcpyAsync(ctx->h_scalars, res, 4 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  FO_CU(ctx, cudaStreamSynchronize(ctx->stream));
  for (int j = 0; j < 4; ++j) out[j] = ctx->h_scalars[j];
  return FO_OK;
}

fo_status fo_region_weight(fo_problem *p, int j, double *w) {
  const long long ne = p->mesh->g.num_elems;
  k_region_weight<<<fo_blocks_for(ne, FO_BLOCK, 65536), FO_BLOCK, 0, p->ctx->stream>>>(ne, p->chif, p->regmask, j, w);
  fo_note_launch(1);
  FO_CU(p->ctx, cudaGetLastError());
  return FO_OK;
}

// ------------------------------------------------------------------ shape derivative RHS
// b[D a + k] = sum over the simplices (p, m) of node a of
//   |e| (S1 grad lambda_m)_k + int_e S0_k lambda_m,   S1 = S1^J + lambda chi / V I.
struct ShapeArgs {
  Grid g;
  int kind;
  double lam_e, mu_e;       // Lame
  double lam_ppl, inv_V;    // PPL multiplier and 1 / V
  double mref;              // |e| / ((D+1)(D+2))
};

template <int D>
__global__ void k_shape_rhs(ShapeArgs s, const double *coef, const uint8_t *chi, const double *chif, const double *u,
                            const double *f, double *b, int add) {
  const Grid &g = s.g;
  for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < g.num_nodes;
       a += (long long)gridDim.x * blockDim.x) {
    int idx[3];
    node_ijk(g, a, idx);
    double acc[D];
#pragma unroll
    for (int k = 0; k < D; ++k) acc[k] = 0;
    if (s.kind == FO_ELASTIC) {
      double us[ST<D>::S][D];
      load_stencil<D, D, double>(g, idx, a, VecX<double>{u}, us);
#pragma unroll
      for (int p = 0; p < KP<D>::P; ++p)
#pragma unroll
        for (int m = 0; m <= D; ++m) {
          long long e;
          if (!elem_of<D>(g, idx, p, m, e)) continue;
          double du[D][D];
#pragma unroll
          for (int l = 0; l < D; ++l) {
            const int ax = kperm<D>(p, l);
            const int s0 = rel_slot<D>(p, m, l), s1 = rel_slot<D>(p, m, l + 1);
#pragma unroll
            for (int i = 0; i < D; ++i) du[i][ax] = (us[s1][i] - us[s0][i]) * g.inv_h[ax];
          }
          double tr = 0;
#pragma unroll
          for (int i = 0; i < D; ++i) tr += du[i][i];
          double sig[D][D], se = 0;
#pragma unroll
          for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j) {
              sig[i][j] = (i == j ? s.lam_e * tr : 0.0) + s.mu_e * (du[i][j] + du[j][i]);
              se += sig[i][j] * 0.5 * (du[i][j] + du[j][i]);
            }
          const double A = coef[e];
          const double cv = chif ? chif[e] * (s.lam_ppl * s.inv_V) : (chi[e] ? s.lam_ppl * s.inv_V : 0.0);
          // S1[i][j] = A (2 sum_k du[k][i] sig[k][j] - se delta_ij) + cv delta_ij
#pragma unroll
          for (int side = 0; side < 2; ++side) {
            if (side == 0 && m < 1) continue;
            if (side == 1 && m >= D) continue;
            const int j = side == 0 ? kperm<D>(p, m - 1) : kperm<D>(p, m);
            const double sgn = side == 0 ? g.inv_h[j] : -g.inv_h[j];
#pragma unroll
            for (int i = 0; i < D; ++i) {
              double t = 0;
#pragma unroll
              for (int k = 0; k < D; ++k) t += du[k][i] * sig[k][j];
              const double S1ij = A * (2.0 * t - (i == j ? se : 0.0)) + (i == j ? cv : 0.0);
              acc[i] += g.vol_e * sgn * S1ij;
            }
          }
        }
    } else {   // heat: S0 = 2u grad f, S1 = (2uf - A|grad u|^2) I + 2A grad u (x) grad u
      double us[ST<D>::S][1], fs[ST<D>::S][1];
      load_stencil<D, 1, double>(g, idx, a, VecX<double>{u}, us);
      load_stencil<D, 1, double>(g, idx, a, VecX<double>{f}, fs);
#pragma unroll
      for (int p = 0; p < KP<D>::P; ++p)
#pragma unroll
        for (int m = 0; m <= D; ++m) {
          long long e;
          if (!elem_of<D>(g, idx, p, m, e)) continue;
          double gu[3] = {0, 0, 0}, gf[3] = {0, 0, 0};
          double su = 0, sf = 0, suf = 0;
#pragma unroll
          for (int l = 0; l < D; ++l) {
            const int ax = kperm<D>(p, l);
            const int s0 = rel_slot<D>(p, m, l), s1 = rel_slot<D>(p, m, l + 1);
            gu[ax] = (us[s1][0] - us[s0][0]) * g.inv_h[ax];
            gf[ax] = (fs[s1][0] - fs[s0][0]) * g.inv_h[ax];
          }
#pragma unroll
          for (int l = 0; l <= D; ++l) {
            const int sl = rel_slot<D>(p, m, l);
            su += us[sl][0];
            sf += fs[sl][0];
            suf += us[sl][0] * fs[sl][0];
          }
          const double A = coef[e];
          double g2 = 0;
#pragma unroll
          for (int k = 0; k < D; ++k) g2 += gu[k] * gu[k];
          const double uf = s.mref * (suf + su * sf);          // int_e u f
          const double Mu = s.mref * (su + us[0][0]);          // int_e u lambda_m
          const double cv = chif ? chif[e] * (s.lam_ppl * s.inv_V) : (chi[e] ? s.lam_ppl * s.inv_V : 0.0);
          // grad lambda_m components
          double gl[3] = {0, 0, 0};
          if (m >= 1) gl[kperm<D>(p, m - 1)] += g.inv_h[kperm<D>(p, m - 1)];
          if (m < D) gl[kperm<D>(p, m)] -= g.inv_h[kperm<D>(p, m)];
          double gdot = 0;
#pragma unroll
          for (int k = 0; k < D; ++k) gdot += gu[k] * gl[k];
#pragma unroll
          for (int i = 0; i < D; ++i) {
            const double S1gl = A * (-g2 * gl[i] + 2.0 * gu[i] * gdot) + cv * gl[i];
            acc[i] += g.vol_e * S1gl + 2.0 * uf * gl[i] + 2.0 * gf[i] * Mu;
          }
        }
    }
#pragma unroll
    for (int k = 0; k < D; ++k) b[a * D + k] = add ? b[a * D + k] + acc[k] : acc[k];
  }
}

// b (+)= the RHS of state u (source f) with multiplier lambda on the volume weights w
// (chi_e, or any element weights, over V = 1 / inv_V); add = 0 overwrites b.
fo_status fo_launch_shape_rhs_ex(fo_problem *p, const double *u, const double *f, double lambda, const double *w,
                                 double inv_V, int add) {
  const Grid &g = p->mesh->g;
  if (p->desc.kind == FO_HELMHOLTZ)
    return fo_fail(p->ctx, FO_EINVAL, "the single-instance shape derivative covers FO_HEAT and FO_ELASTIC");
  ShapeArgs s{g, p->desc.kind, p->lame_lambda, p->lame_mu, lambda, inv_V, g.vol_e / ((g.dim + 1) * (g.dim + 2))};
  int blocks = fo_blocks_for(g.num_nodes, FO_BLOCK, 65536);
  if (g.dim == 2) k_shape_rhs<2><<<blocks, FO_BLOCK, 0, p->ctx->stream>>>(s, p->coef, p->chi, w, u, f, p->rhs, add);
  else k_shape_rhs<3><<<blocks, FO_BLOCK, 0, p->ctx->stream>>>(s, p->coef, p->chi, w, u, f, p->rhs, add);
  fo_note_launch(1);
  FO_CU(p->ctx, cudaGetLastError());
  return FO_OK;
}

fo_status fo_launch_shape_rhs(fo_problem *p, double lambda) {
  const Grid &g = p->mesh->g;
  if (p->desc.kind == FO_HELMHOLTZ)
    return fo_fail(p->ctx, FO_EINVAL, "the single-instance shape derivative covers FO_HEAT and FO_ELASTIC");
  ShapeArgs s{g, p->desc.kind, p->lame_lambda, p->lame_mu, lambda,
              p->desc.volume_target > 0 ? 1.0 / p->desc.volume_target : 1.0, g.vol_e / ((g.dim + 1) * (g.dim + 2))};
  int blocks = fo_blocks_for(g.num_nodes, FO_BLOCK, 65536);
  const double *chif = p->desc.coef_rule == FO_COEF_CUT ? p->chif : nullptr;
  if (g.dim == 2) k_shape_rhs<2><<<blocks, FO_BLOCK, 0, p->ctx->stream>>>(s, p->coef, p->chi, chif, p->u, p->f, p->rhs, 0);
  else k_shape_rhs<3><<<blocks, FO_BLOCK, 0, p->ctx->stream>>>(s, p->coef, p->chi, chif, p->u, p->f, p->rhs, 0);
  fo_note_launch(1);
  FO_CU(p->ctx, cudaGetLastError());
  return FO_OK;
}

// --------------------------------------------------------------------------- initial level
// phi0(x) = factor * max_k (r_k - |x - c_k|_ord)   (ord 2 or infinity)
__global__ void k_initial_level(int dim, long long nn, const double *coords, int count, const double *cr,
                                double factor, int ord, double *phi) {
  for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < nn; a += (long long)gridDim.x * blockDim.x) {
    double best = -INFINITY;
    for (int k = 0; k < count; ++k) {
      double dist = 0;
      for (int j = 0; j < dim; ++j) {
        const double d = coords[a * dim + j] - cr[k * 4 + j];
        if (ord == 2) dist += d * d;
        else dist = fmax(dist, fabs(d));
      }
      if (ord == 2) dist = sqrt(dist);
      best = fmax(best, cr[k * 4 + 3] - dist);
    }
    phi[a] = factor * best;
  }
}

fo_status fo_launch_initial_level(fo_problem *p, int count, const double *centers, const double *radii, double factor,
                                  int ord) {
  const Grid &g = p->mesh->g;
  fo_ctx *ctx = p->ctx;
  std::vector<double> cr(4 * (size_t)count);
  for (int k = 0; k < count; ++k) {
    for (int j = 0; j < g.dim; ++j) cr[k * 4 + j] = centers[k * g.dim + j];
    cr[k * 4 + 3] = radii[k];
  }
  double *d_cr;
  FO_TRY(fo_alloc(ctx, (void **)&d_cr, sizeof(double) * cr.size()));
  fo_status st = fo_cuda_check(ctx, cudaMemcpyAsync(d_cr, cr.data(), sizeof(double) * cr.size(),
                                                    cudaMemcpyHostToDevice, ctx->stream), "copy centres");
  if (st == FO_OK) {
    k_initial_level<<<fo_blocks_for(g.num_nodes, FO_BLOCK, 65536), FO_BLOCK, 0, ctx->stream>>>(
        g.dim, g.num_nodes, p->mesh->d_coords, count, d_cr, factor, ord, p->phi);
    fo_note_launch(1);
    st = fo_cuda_check(ctx, cudaGetLastError(), "initial level");
  }
  if (st == FO_OK) st = fo_cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "initial level sync");
  fo_free(ctx, d_cr, sizeof(double) * cr.size());
  return st;
}

// ------------------------------------------------------------------ Gaussian-bump level set
// phi(x) = sum_k exp(-|x - c_k|^2 / (2 width^2)) - offset, the terms added in k order
// (the random-bump initial shapes of the 3D and serving workloads).
__global__ void k_phi_bumps(int dim, long long nn, const double *coords, int count, const double *c, double inv2w2,
                            double offset, double *phi) {
  for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < nn; a += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < count; ++k) {
      double d2 = 0.0;
      for (int j = 0; j < dim; ++j) {
        const double d = coords[a * dim + j] - c[k * dim + j];
        d2 += d * d;
      }
      s += exp(-d2 * inv2w2);
    }
    phi[a] = s - offset;
  }
}

fo_status fo_launch_phi_bumps(fo_problem *p, int count, const double *centers, double width, double offset) {
  const Grid &g = p->mesh->g;
  fo_ctx *ctx = p->ctx;
  const size_t nc = (size_t)count * g.dim;
  double *d_c;
  FO_TRY(fo_alloc(ctx, (void **)&d_c, sizeof(double) * nc));
  fo_status st = fo_cuda_check(ctx, cudaMemcpyAsync(d_c, centers, sizeof(double) * nc, cudaMemcpyHostToDevice,
                                                    ctx->stream), "copy bump centres");
  if (st == FO_OK) {
    k_phi_bumps<<<fo_blocks_for(g.num_nodes, FO_BLOCK, 65536), FO_BLOCK, 0, ctx->stream>>>(
        g.dim, g.num_nodes, p->mesh->d_coords, count, d_c, 1.0 / (2.0 * width * width), offset, p->phi);
    fo_note_launch(1);
    st = fo_cuda_check(ctx, cudaGetLastError(), "bump level set");
  }
  if (st == FO_OK) st = fo_cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "bump level set sync");
  fo_free(ctx, d_c, sizeof(double) * nc);
  return st;
}
