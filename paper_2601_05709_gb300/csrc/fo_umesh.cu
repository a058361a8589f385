// General simplicial meshes given as arrays: host construction of the adjacency, node graph
// and boundary facets; element geometry, coefficients, masks, loads, assembled state and
// velocity operators, functionals and the shape-derivative right-hand side on the GPU.
// (Transport, reinitialisation and their Krylov solver: fo_umesh_levelset.cu.)
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "fo_internal.cuh"
#include "fo_ops.cuh"
#include "fo_umesh.cuh"

// ------------------------------------------------------------------------- host build
template <class T>
static fo_status up(fo_mesh *m, T **dst, const std::vector<T> &src) {
  fo_umesh *u = m->um;
  const size_t bytes = sizeof(T) * std::max<size_t>(src.size(), 1);
  FO_TRY(fo_alloc(m->ctx, (void **)dst, bytes));
  u->allocs.push_back({(void **)dst, bytes});
  if (!src.empty())
    FO_CU(m->ctx, cudaMemcpyAsync(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice, m->ctx->stream));
  return FO_OK;
}
template <class T>
static fo_status dev_alloc(fo_mesh *m, T **dst, size_t count) {
  const size_t bytes = sizeof(T) * std::max<size_t>(count, 1);
  FO_TRY(fo_alloc(m->ctx, (void **)dst, bytes));
  m->um->allocs.push_back({(void **)dst, bytes});
  return FO_OK;
}

void fo_umesh_release(fo_mesh *m) {
  if (!m->um) return;
  for (auto &a : m->um->allocs) fo_free(m->ctx, *a.first, a.second);
  delete m->um;
  m->um = nullptr;
}

template <int D>
__global__ void k_u_geometry(long long nt, const int32_t *cells, const double *X, double *vol, double *grad) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nt; e += (long long)gridDim.x * blockDim.x) {
    int v[D + 1];
#pragma unroll
    for (int a = 0; a <= D; ++a) v[a] = cells[e * (D + 1) + a];
    double E[D][D];   // columns x_m - x_0
#pragma unroll
    for (int m = 0; m < D; ++m)
#pragma unroll
      for (int k = 0; k < D; ++k) E[k][m] = X[(long long)v[m + 1] * D + k] - X[(long long)v[0] * D + k];
    double inv[D][D], det;
    if (D == 2) {
      det = E[0][0] * E[1][1] - E[0][1] * E[1][0];
      inv[0][0] = E[1][1] / det;
      inv[0][1] = -E[0][1] / det;
      inv[1][0] = -E[1][0] / det;
      inv[1][1] = E[0][0] / det;
    } else {
      const double c00 = E[1][1] * E[2][2] - E[1][2] * E[2][1];
      const double c01 = E[1][2] * E[2][0] - E[1][0] * E[2][2];
      const double c02 = E[1][0] * E[2][1] - E[1][1] * E[2][0];
      det = E[0][0] * c00 + E[0][1] * c01 + E[0][2] * c02;
      inv[0][0] = c00 / det;
      inv[1][0] = c01 / det;
      inv[2][0] = c02 / det;
      inv[0][1] = (E[0][2] * E[2][1] - E[0][1] * E[2][2]) / det;
      inv[1][1] = (E[0][0] * E[2][2] - E[0][2] * E[2][0]) / det;
      inv[2][1] = (E[0][1] * E[2][0] - E[0][0] * E[2][1]) / det;
      inv[0][2] = (E[0][1] * E[1][2] - E[0][2] * E[1][1]) / det;
      inv[1][2] = (E[0][2] * E[1][0] - E[0][0] * E[1][2]) / det;
      inv[2][2] = (E[0][0] * E[1][1] - E[0][1] * E[1][0]) / det;
    }
    vol[e] = fabs(det) / (D == 2 ? 2.0 : 6.0);
    // grad lambda_m (m >= 1) = row m-1 of E^{-1}; grad lambda_0 = -(sum of the others)
#pragma unroll
    for (int k = 0; k < D; ++k) {
      double s = 0;
#pragma unroll
      for (int m = 1; m <= D; ++m) {
        grad[((long long)m * D + k) * nt + e] = inv[m - 1][k];
        s += inv[m - 1][k];
      }
      grad[(long long)k * nt + e] = -s;
    }
  }
}

fo_status fo_umesh_build(fo_mesh *m, const double *coords, const int32_t *cells) {
  fo_ctx *ctx = m->ctx;
  fo_umesh *u = m->um;
  const int d = u->dim, nv = d + 1;
  const long long nn = u->nn, nt = u->nt;
  // bounding box and box-face membership
  for (int a = 0; a < d; ++a) {
    u->lo[a] = INFINITY;
    u->hi[a] = -INFINITY;
  }
  for (long long i = 0; i < nn; ++i)
    for (int a = 0; a < d; ++a) {
      u->lo[a] = std::min(u->lo[a], coords[i * d + a]);
      u->hi[a] = std::max(u->hi[a], coords[i * d + a]);
    }
  std::vector<uint8_t> fmask(nn, 0);
  for (long long i = 0; i < nn; ++i)
    for (int a = 0; a < d; ++a) {
      if (coords[i * d + a] == u->lo[a]) fmask[i] |= (uint8_t)(1u << (2 * a));
      if (coords[i * d + a] == u->hi[a]) fmask[i] |= (uint8_t)(1u << (2 * a + 1));
    }
  // node -> element adjacency in element order
  std::vector<int> aptr(nn + 1, 0), adj((size_t)nt * nv);
  for (long long e = 0; e < nt; ++e)
    for (int a = 0; a < nv; ++a) aptr[cells[e * nv + a] + 1]++;
  for (long long i = 0; i < nn; ++i) aptr[i + 1] += aptr[i];
  {
    std::vector<int> fill(aptr.begin(), aptr.end() - 1);
    for (long long e = 0; e < nt; ++e)
      for (int a = 0; a < nv; ++a) adj[fill[cells[e * nv + a]]++] = (int)(e * nv + a);
  }
  // node graph: sorted neighbour lists (the node itself included)
  std::vector<int> rptr(nn + 1, 0), col, diag(nn);
  std::vector<int> nb;
  for (long long i = 0; i < nn; ++i) {
    nb.clear();
    for (int k = aptr[i]; k < aptr[i + 1]; ++k) {
      const long long e = adj[k] / nv;
      for (int b = 0; b < nv; ++b) nb.push_back(cells[e * nv + b]);
    }
    if (nb.empty()) nb.push_back((int)i);   // an isolated node keeps its diagonal
    std::sort(nb.begin(), nb.end());
    nb.erase(std::unique(nb.begin(), nb.end()), nb.end());
    for (int c : nb) {
      if (c == i) diag[i] = (int)col.size();
      col.push_back(c);
    }
    rptr[i + 1] = (int)col.size();
  }
  auto pos_of = [&](long long row, int c) {
    const int *b = col.data() + rptr[row], *e = col.data() + rptr[row + 1];
    return (int)(std::lower_bound(b, e, c) - col.data());
  };
  std::vector<int> apos((size_t)nt * nv * nv);
  for (long long i = 0; i < nn; ++i)
    for (int k = aptr[i]; k < aptr[i + 1]; ++k) {
      const long long e = adj[k] / nv;
      for (int b = 0; b < nv; ++b) apos[(size_t)k * nv + b] = pos_of(i, cells[e * nv + b]);
    }
  // boundary facets: the facets of exactly one element (sort the (d)-tuples of all facets)
  struct Fc {
    int v[3];
    long long e;
    int m;
  };
  std::vector<Fc> all((size_t)nt * nv);
  for (long long e = 0; e < nt; ++e)
    for (int mm = 0; mm < nv; ++mm) {
      Fc f{{0, 0, 0}, e, mm};
      int q = 0;
      for (int a = 0; a < nv; ++a)
        if (a != mm) f.v[q++] = cells[e * nv + a];
      std::sort(f.v, f.v + d);
      all[(size_t)e * nv + mm] = f;
    }
  auto less = [d](const Fc &x, const Fc &y) {
    for (int i = 0; i < d; ++i)
      if (x.v[i] != y.v[i]) return x.v[i] < y.v[i];
    return x.e < y.e;
  };
  std::sort(all.begin(), all.end(), less);
  auto same = [d](const Fc &x, const Fc &y) {
    for (int i = 0; i < d; ++i)
      if (x.v[i] != y.v[i]) return false;
    return true;
  };
  std::vector<Fc> bnd;
  for (size_t i = 0; i < all.size();) {
    size_t j = i + 1;
    while (j < all.size() && same(all[i], all[j])) ++j;
    if (j - i == 1) bnd.push_back(all[i]);
    else if (j - i > 2) return fo_fail(ctx, FO_EINVAL, "a facet is shared by more than two elements");
    i = j;
  }
  // facets in element order (facet vertices in the element's vertex order)
  std::sort(bnd.begin(), bnd.end(), [](const Fc &x, const Fc &y) { return x.e != y.e ? x.e < y.e : x.m < y.m; });
  const long long nf = (long long)bnd.size();
  u->nf = nf;
  std::vector<int> fn((size_t)nf * d), ff(nf, -1);
  std::vector<double> fa(nf), fnorm((size_t)nf * d);
  for (long long f = 0; f < nf; ++f) {
    const Fc &c = bnd[f];
    int q = 0;
    for (int a = 0; a < nv; ++a)
      if (a != c.m) fn[f * d + q++] = cells[c.e * nv + a];
    const double *x0 = coords + (long long)fn[f * d] * d, *x1 = coords + (long long)fn[f * d + 1] * d;
    double nrm[3] = {0, 0, 0};
    if (d == 2) {
      const double tx = x1[0] - x0[0], ty = x1[1] - x0[1];
      fa[f] = std::sqrt(tx * tx + ty * ty);
      nrm[0] = ty;
      nrm[1] = -tx;
    } else {
      const double *x2 = coords + (long long)fn[f * d + 2] * d;
      const double a1[3] = {x1[0] - x0[0], x1[1] - x0[1], x1[2] - x0[2]};
      const double a2[3] = {x2[0] - x0[0], x2[1] - x0[1], x2[2] - x0[2]};
      nrm[0] = a1[1] * a2[2] - a1[2] * a2[1];
      nrm[1] = a1[2] * a2[0] - a1[0] * a2[2];
      nrm[2] = a1[0] * a2[1] - a1[1] * a2[0];
      fa[f] = 0.5 * std::sqrt(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
    }
    // box face: all vertices on it
    uint8_t common = 0xff;
    for (int q2 = 0; q2 < d; ++q2) common &= fmask[fn[f * d + q2]];
    int face = -1;
    for (int b = 0; b < 2 * d; ++b)
      if (common & (1u << b)) {
        face = b;
        break;
      }
    ff[f] = face;
    if (face >= 0) {   // axis-aligned: the exact outward normal
      for (int k = 0; k < d; ++k) fnorm[f * d + k] = 0.0;
      fnorm[f * d + face / 2] = (face & 1) ? 1.0 : -1.0;
    } else {   // orient away from the opposite vertex
      const double *xo = coords + (long long)cells[c.e * nv + c.m] * d;
      double dotp = 0, len = 0;
      for (int k = 0; k < d; ++k) {
        dotp += nrm[k] * (x0[k] - xo[k]);
        len += nrm[k] * nrm[k];
      }
      len = std::sqrt(len);
      for (int k = 0; k < d; ++k) fnorm[f * d + k] = (dotp < 0 ? -nrm[k] : nrm[k]) / len;
    }
  }
  // node -> facet adjacency with graph positions
  std::vector<int> fptr(nn + 1, 0), fadj((size_t)nf * d), fpos((size_t)nf * d * d);
  for (long long f = 0; f < nf; ++f)
    for (int a = 0; a < d; ++a) fptr[fn[f * d + a] + 1]++;
  for (long long i = 0; i < nn; ++i) fptr[i + 1] += fptr[i];
  {
    std::vector<int> fill(fptr.begin(), fptr.end() - 1);
    for (long long f = 0; f < nf; ++f)
      for (int a = 0; a < d; ++a) fadj[fill[fn[f * d + a]]++] = (int)(f * d + a);
  }
  for (long long i = 0; i < nn; ++i)
    for (int k = fptr[i]; k < fptr[i + 1]; ++k) {
      const long long f = fadj[k] / d;
      for (int b = 0; b < d; ++b) fpos[(size_t)k * d + b] = pos_of(i, fn[f * d + b]);
    }
  u->nnz = (long long)col.size();
  FO_TRY(up(m, &u->adj_ptr, aptr));
  FO_TRY(up(m, &u->adj, adj));
  FO_TRY(up(m, &u->adj_pos, apos));
  FO_TRY(up(m, &u->row_ptr, rptr));
  FO_TRY(up(m, &u->col, col));
  FO_TRY(up(m, &u->diag, diag));
  FO_TRY(up(m, &u->fnodes, fn));
  FO_TRY(up(m, &u->farea, fa));
  FO_TRY(up(m, &u->fnormal, fnorm));
  FO_TRY(up(m, &u->fface, ff));
  FO_TRY(up(m, &u->nf_ptr, fptr));
  FO_TRY(up(m, &u->nf_adj, fadj));
  FO_TRY(up(m, &u->nf_pos, fpos));
  FO_TRY(up(m, &u->face_mask, fmask));
  FO_TRY(dev_alloc(m, &u->vol, nt));
  FO_TRY(dev_alloc(m, &u->grad, (size_t)nt * nv * d));
  const int blocks = fo_blocks_for(nt, FO_BLOCK, 65536);
  if (d == 2) k_u_geometry<2><<<blocks, FO_BLOCK, 0, ctx->stream>>>(nt, m->d_cells, m->d_coords, u->vol, u->grad);
  else k_u_geometry<3><<<blocks, FO_BLOCK, 0, ctx->stream>>>(nt, m->d_cells, m->d_coords, u->vol, u->grad);
  fo_note_launch(1);
  FO_CU(ctx, cudaGetLastError());
  // |D| = sum of the element measures (host, for the mesh diameter)
  std::vector<double> hv(nt);
  FO_CU(ctx, cudaMemcpyAsync(hv.data(), u->vol, sizeof(double) * nt, cudaMemcpyDeviceToHost, ctx->stream));
  FO_CU(ctx, cudaStreamSynchronize(ctx->stream));
  double s = 0;
  for (double v : hv) {
    if (!(v > 0)) return fo_fail(ctx, FO_EINVAL, "degenerate element (zero measure)");
    s += v;
  }
  u->volume = s;
  return FO_OK;
}

// ------------------------------------------------------------------ coefficients, masks
// A_e, chi_e from phi (eqs heat_AOmega / compli_AOmega): the vertex values summed in the
// element's vertex order, < 0 inside (strict: a zero sum is outside); A_e times k (Helmholtz).
template <int D>
__global__ void k_u_coefficients(UMeshView m, const double *phi, double a_in, double a_out, double *coef,
                                 float *coef32, uint8_t *chi, int cut, double *chif) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < m.nt; e += (long long)gridDim.x * blockDim.x) {
    double pv[D + 1];
#pragma unroll
    for (int a = 0; a <= D; ++a) pv[a] = phi[m.cells[e * (D + 1) + a]];
    if (cut) {   // exact cut-cell fraction (FO_COEF_CUT)
      const double f = cut_fraction<D>(pv);
      const double A = a_out + (a_in - a_out) * f;
      coef[e] = A;
      coef32[e] = (float)A;
      chi[e] = f > 0.0 ? 1 : 0;
      chif[e] = f;
      continue;
    }
    double s = pv[0];
#pragma unroll
    for (int a = 1; a <= D; ++a) s = s + pv[a];
    const bool in = s < 0.0;
    const double A = in ? a_in : a_out;
    coef[e] = A;
    coef32[e] = (float)A;
    chi[e] = in ? 1 : 0;
    chif[e] = in ? 1.0 : 0.0;
  }
}

struct UMaskArgs {
  uint32_t faces;
  int ncomp, vel_dirichlet, n_omega0;
  double o_lo[4][3], o_hi[4][3];
  int n_vol;
  double v_lo[4][3], v_hi[4][3];
};

// State Dirichlet mask per DOF (nodes on a selected box face), the H^1_0 velocity mask (nodes
// on any box face), and Omega_0 per element: its centroid (vertex coordinates summed in vertex
// order, then / (d+1)) strictly inside one of the boxes (Sec. 5.7, eq. sub_dom).
template <int D>
__global__ void k_u_masks(UMeshView m, UMaskArgs a, uint8_t *dir, uint8_t *vdir, uint8_t *omega0, uint8_t *regmask) {
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x, st = (long long)gridDim.x * blockDim.x;
  for (long long i = tid; i < m.nn; i += st) {
    const uint32_t fm = m.face_mask[i];
    const bool on = (fm & a.faces) != 0;
    for (int c = 0; c < a.ncomp; ++c) dir[i * a.ncomp + c] = on ? 1 : 0;
    vdir[i] = (a.vel_dirichlet && fm != 0) ? 1 : 0;
  }
  for (long long e = tid; e < m.nt; e += st) {
    double s[3];
#pragma unroll
    for (int k = 0; k < D; ++k) s[k] = m.coords[(long long)m.cells[e * (D + 1)] * D + k];
#pragma unroll
    for (int v = 1; v <= D; ++v)
#pragma unroll
      for (int k = 0; k < D; ++k) s[k] = s[k] + m.coords[(long long)m.cells[e * (D + 1) + v] * D + k];
    bool in = false;
    for (int b = 0; b < a.n_omega0; ++b) {
      bool ok = true;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const double x = s[k] / (double)(D + 1);
        ok = ok && (x > a.o_lo[b][k]) && (x < a.o_hi[b][k]);
      }
      in = in || ok;
    }
    omega0[e] = in ? 1 : 0;
    unsigned rm = 0;
    for (int b = 0; b < a.n_vol; ++b) {
      bool ok = true;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const double x = s[k] / (double)(D + 1);
        ok = ok && (x > a.v_lo[b][k]) && (x < a.v_hi[b][k]);
      }
      if (ok) rm |= 1u << b;
    }
    regmask[e] = (uint8_t)rm;
  }
}

fo_status fo_umesh_masks(fo_problem *p) {
  const UMeshView m = umesh_view(p->mesh);
  UMaskArgs a{};
  a.faces = p->desc.dirichlet_faces;
  a.ncomp = p->ncomp;
  a.vel_dirichlet = p->desc.velocity_dirichlet;
  a.n_omega0 = p->desc.omega0_weight != 0.0 ? p->desc.n_omega0 : 0;
  for (int b = 0; b < 4; ++b)
    for (int k = 0; k < 3; ++k) {
      a.o_lo[b][k] = p->desc.omega0_lo[b][k];
      a.o_hi[b][k] = p->desc.omega0_hi[b][k];
      a.v_lo[b][k] = p->desc.volume_lo[b][k];
      a.v_hi[b][k] = p->desc.volume_hi[b][k];
    }
  a.n_vol = p->nvol;
  const int blocks = fo_blocks_for(std::max(m.nn, m.nt), FO_BLOCK, 65536);
  if (m.dim == 2) k_u_masks<2><<<blocks, FO_BLOCK, 0, p->ctx->stream>>>(m, a, p->dir, p->vdir, p->omega0, p->regmask);
  else k_u_masks<3><<<blocks, FO_BLOCK, 0, p->ctx->stream>>>(m, a, p->dir, p->vdir, p->omega0, p->regmask);
  fo_note_launch(1);
  FO_CU(p->ctx, cudaGetLastError());
  return FO_OK;
}

// ------------------------------------------------------------------------------ loads
struct ULoadArgs {
  int ncomp;
  int n_tr;
  int tr_face[4];
  double tr_vec[4][3];
  int n_pt;
  long long pt_node[4];
  double pt_vec[4][3];
};

// F_a = int f psi_a (f the P1 interpolant: the consistent mass row, |e| (f_a + sum_b f_b) /
// ((d+1)(d+2)) per element) + sum over the node's boundary facets on a traction face of
// t |f| / d (eq. compli_weak) + point loads; zero on Dirichlet DOFs.  Sums in element / facet
// order.
template <int D>
__global__ void k_u_loads(UMeshView m, ULoadArgs L, const double *f, const uint8_t *dir, double *F) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m.nn; i += (long long)gridDim.x * blockDim.x) {
    double acc[3] = {0, 0, 0};
    if (f) {
      for (int k = m.adj_ptr[i]; k < m.adj_ptr[i + 1]; ++k) {
        const long long e = m.adj[k] / (D + 1);
        double s = f[m.cells[e * (D + 1)]];
#pragma unroll
        for (int b = 1; b <= D; ++b) s = s + f[m.cells[e * (D + 1) + b]];
        acc[0] += m.vol[e] / ((D + 1) * (D + 2)) * (s + f[i]);
      }
    }
    for (int k = m.nf_ptr[i]; k < m.nf_ptr[i + 1]; ++k) {
      const long long fc = m.nf_adj[k] / D;
      const int face = m.fface[fc];
      for (int t = 0; t < L.n_tr; ++t)
        if (face == L.tr_face[t]) {
          const double w = m.farea[fc] / D;
          for (int c = 0; c < L.ncomp; ++c) acc[c] += w * L.tr_vec[t][c];
        }
    }
    for (int t = 0; t < L.n_pt; ++t)
      if (L.pt_node[t] == i)
        for (int c = 0; c < L.ncomp; ++c) acc[c] += L.pt_vec[t][c];
    for (int c = 0; c < L.ncomp; ++c) F[i * L.ncomp + c] = dir[i * L.ncomp + c] ? 0.0 : acc[c];
  }
}

fo_status fo_umesh_loads(fo_problem *p) {
  const UMeshView m = umesh_view(p->mesh);
  for (int kc = 0; kc < p->ncases; ++kc) {
    ULoadArgs L{};
    L.ncomp = p->ncomp;
    for (int t = 0; t < p->desc.n_tractions; ++t) {
      if (p->desc.traction_case[t] != kc && p->ncases > 1) continue;
      L.tr_face[L.n_tr] = p->desc.traction_face[t];
      for (int c = 0; c < 3; ++c) L.tr_vec[L.n_tr][c] = p->desc.traction_vec[t][c];
      ++L.n_tr;
    }
    for (int t = 0; t < p->desc.n_point_loads; ++t) {
      if (p->desc.point_case[t] != kc && p->ncases > 1) continue;
      L.pt_node[L.n_pt] = p->desc.point_node[t];
      for (int c = 0; c < 3; ++c) L.pt_vec[L.n_pt][c] = p->desc.point_vec[t][c];
      ++L.n_pt;
    }
    const double *f = (p->desc.kind != FO_ELASTIC && kc == 0) ? p->f : nullptr;
    double *F = p->load + (size_t)kc * p->ndof;
    const int blocks = fo_blocks_for(m.nn, FO_BLOCK, 65536);
    if (m.dim == 2) k_u_loads<2><<<blocks, FO_BLOCK, 0, p->ctx->stream>>>(m, L, f, p->dir, F);
    else k_u_loads<3><<<blocks, FO_BLOCK, 0, p->ctx->stream>>>(m, L, f, p->dir, F);
    fo_note_launch(1);
    FO_CU(p->ctx, cudaGetLastError());
  }
  return FO_OK;
}

// ------------------------------------------------------------- assembled operators
// Turn the raw block row of node a (rows of element blocks summed at W[r0..r1)) into
// difference form with Dirichlet rows as identity and Dirichlet columns eliminated (see
// CsrOp); the raw diagonal gives the Jacobi inverse.  dirn(c, j): DOF j of node c is fixed.
template <int NPN, class Dir>
__device__ void u_finish_row(const UMeshView &m, long long a, const Dir &dirn, double *W, float *W32, double *dinv,
                             float *dinv32) {
  constexpr int BLK = NPN * NPN;
  const int r0 = m.row_ptr[a], r1 = m.row_ptr[a + 1], dg = m.diag[a];
  double R[BLK];
#pragma unroll
  for (int q = 0; q < BLK; ++q) R[q] = 0.0;
#pragma unroll
  for (int i = 0; i < NPN; ++i) {
    const double di = W[(long long)dg * BLK + i * NPN + i];
    const bool fixed = dirn(a, i);
    dinv[a * NPN + i] = fixed ? 1.0 : 1.0 / di;
    if (dinv32) dinv32[a * NPN + i] = (float)(fixed ? 1.0 : 1.0 / di);
  }
  for (int k = r0; k < r1; ++k) {
    const long long c = m.col[k];
#pragma unroll
    for (int i = 0; i < NPN; ++i)
#pragma unroll
      for (int j = 0; j < NPN; ++j) {
        double w = W[(long long)k * BLK + i * NPN + j];
        if (dirn(a, i) || dirn(c, j)) w = 0.0;
        R[i * NPN + j] += w;
        if (k != dg) {
          W[(long long)k * BLK + i * NPN + j] = w;
          if (W32) W32[(long long)k * BLK + i * NPN + j] = (float)w;
        }
      }
  }
#pragma unroll
  for (int i = 0; i < NPN; ++i)
#pragma unroll
    for (int j = 0; j < NPN; ++j) {
      const double v = dirn(a, i) ? (i == j ? 1.0 : 0.0) : R[i * NPN + j];
      W[(long long)dg * BLK + i * NPN + j] = v;
      if (W32) W32[(long long)dg * BLK + i * NPN + j] = (float)v;
    }
}

struct DofDir {
  const uint8_t *dir;
  int npn;
  __device__ __forceinline__ bool operator()(long long c, int j) const { return dir[c * npn + j] != 0; }
};
struct NodeDir {
  const uint8_t *mask;   // per node, or null
  __device__ __forceinline__ bool operator()(long long c, int) const { return mask && mask[c] != 0; }
};

// State operator: K_e = A_e |e| G G^T (+ omega^2 M_e) for scalar models (eqs heat_weak and the
// screened family), A_e |e| [lam g_ai g_bj + mu g_aj g_bi + mu delta_ij g_a . g_b] for
// elasticity (eq. compli_weak), summed row by row over the node's elements.
template <int D, int NPN>
__global__ void k_u_state_assemble(UMeshView m, double lam, double mu, double w2, const double *coef,
                                   const uint8_t *dir, double *W, float *W32, double *dinv, float *dinv32) {
  constexpr int BLK = NPN * NPN;
  for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < m.nn; a += (long long)gridDim.x * blockDim.x) {
    for (int k = m.row_ptr[a] * BLK; k < m.row_ptr[a + 1] * BLK; ++k) W[k] = 0.0;
    for (int q = m.adj_ptr[a]; q < m.adj_ptr[a + 1]; ++q) {
      const long long e = m.adj[q] / (D + 1);
      const int la = m.adj[q] % (D + 1);
      const double Av = coef[e] * m.vol[e];
      double ga[D];
#pragma unroll
      for (int k = 0; k < D; ++k) ga[k] = m.g(e, la, k);
#pragma unroll
      for (int lb = 0; lb <= D; ++lb) {
        const long long pos = m.adj_pos[(long long)q * (D + 1) + lb];
        double gb[D], dot = 0;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          gb[k] = m.g(e, lb, k);
          dot += ga[k] * gb[k];
        }
        if (NPN == 1) {
          double v = Av * dot;
          if (w2 != 0.0) v += w2 * m.vol[e] * (la == lb ? 2.0 : 1.0) / ((D + 1) * (D + 2));
          W[pos] += v;
        } else {
#pragma unroll
          for (int i = 0; i < NPN; ++i)
#pragma unroll
            for (int j = 0; j < NPN; ++j)
              W[pos * BLK + i * NPN + j] += Av * (lam * ga[i] * gb[j] + mu * ga[j] * gb[i] + (i == j ? mu * dot : 0.0));
        }
      }
    }
    u_finish_row<NPN>(m, a, DofDir{dir, NPN}, W, W32, dinv, dinv32);
  }
}

fo_status fo_umesh_coefficients(fo_problem *p) {
  const UMeshView m = umesh_view(p->mesh);
  cudaStream_t s = p->ctx->stream;
  const double k = p->desc.kind == FO_HELMHOLTZ ? p->desc.k : 1.0;
  const int cut = p->desc.coef_rule == FO_COEF_CUT;
  int blocks = fo_blocks_for(m.nt, FO_BLOCK, 65536);
  if (m.dim == 2)
    k_u_coefficients<2><<<blocks, FO_BLOCK, 0, s>>>(m, p->phi, p->desc.a_in * k, p->desc.a_out * k, p->coef, p->coef32, p->chi,
                                                    cut, p->chif);
  else
    k_u_coefficients<3><<<blocks, FO_BLOCK, 0, s>>>(m, p->phi, p->desc.a_in * k, p->desc.a_out * k, p->coef, p->coef32, p->chi,
                                                    cut, p->chif);
  blocks = fo_blocks_for(m.nn, FO_BLOCK, 65536);
  const double w2 = p->desc.kind == FO_HELMHOLTZ ? p->desc.omega * p->desc.omega : 0.0;
  if (p->desc.kind == FO_ELASTIC) {
    if (m.dim == 2)
      k_u_state_assemble<2, 2><<<blocks, FO_BLOCK, 0, s>>>(m, p->lame_lambda, p->lame_mu, 0.0, p->coef, p->dir, p->Wst,
                                                           p->Wst32, p->dinv_state, p->dinv_state32);
    else
      k_u_state_assemble<3, 3><<<blocks, FO_BLOCK, 0, s>>>(m, p->lame_lambda, p->lame_mu, 0.0, p->coef, p->dir, p->Wst,
                                                           p->Wst32, p->dinv_state, p->dinv_state32);
  } else {
    if (m.dim == 2)
      k_u_state_assemble<2, 1><<<blocks, FO_BLOCK, 0, s>>>(m, 0.0, 0.0, w2, p->coef, p->dir, p->Wst, p->Wst32,
                                                           p->dinv_state, p->dinv_state32);
    else
      k_u_state_assemble<3, 1><<<blocks, FO_BLOCK, 0, s>>>(m, 0.0, 0.0, w2, p->coef, p->dir, p->Wst, p->Wst32,
                                                           p->dinv_state, p->dinv_state32);
  }
  fo_note_launch(2);
  FO_CU(p->ctx, cudaGetLastError());
  return FO_OK;
}

// Velocity form (Sec. 5.5, eqs velocity, bd_plt, sub_dom): per element (|e| g_a . g_b +
// (alpha_m + gamma_0 chi_Omega0) M_e[a, b]) I, per boundary facet gamma_b |f| (1 + delta_ab) /
// (d (d+1)) n n^T; H^1_0 rows and columns of box-face nodes eliminated when asked.
template <int D>
__global__ void k_u_velocity_assemble(UMeshView m, double alpha, double gamma0, double gammab, const uint8_t *omega0,
                                      const uint8_t *vdir, double *W, double *dinv) {
  constexpr int BLK = D * D;
  for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < m.nn; a += (long long)gridDim.x * blockDim.x) {
    for (int k = m.row_ptr[a] * BLK; k < m.row_ptr[a + 1] * BLK; ++k) W[k] = 0.0;
    for (int q = m.adj_ptr[a]; q < m.adj_ptr[a + 1]; ++q) {
      const long long e = m.adj[q] / (D + 1);
      const int la = m.adj[q] % (D + 1);
      const double v = m.vol[e], mc = alpha + (omega0[e] ? gamma0 : 0.0);
#pragma unroll
      for (int lb = 0; lb <= D; ++lb) {
        const long long pos = m.adj_pos[(long long)q * (D + 1) + lb];
        double dot = 0;
#pragma unroll
        for (int k = 0; k < D; ++k) dot += m.g(e, la, k) * m.g(e, lb, k);
        const double val = v * dot + mc * v * (la == lb ? 2.0 : 1.0) / ((D + 1) * (D + 2));
#pragma unroll
        for (int i = 0; i < D; ++i) W[pos * BLK + i * D + i] += val;
      }
    }
    if (gammab != 0.0)
      for (int q = m.nf_ptr[a]; q < m.nf_ptr[a + 1]; ++q) {
        const long long f = m.nf_adj[q] / D;
        const int la = m.nf_adj[q] % D;
        double n[D];
#pragma unroll
        for (int k = 0; k < D; ++k) n[k] = m.fnormal[f * D + k];
#pragma unroll
        for (int lb = 0; lb < D; ++lb) {
          const long long pos = m.nf_pos[(long long)q * D + lb];
          const double w = gammab * m.farea[f] * (la == lb ? 2.0 : 1.0) / (D * (D + 1));
#pragma unroll
          for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j) W[pos * BLK + i * D + j] += w * n[i] * n[j];
        }
      }
    u_finish_row<D>(m, a, NodeDir{vdir}, W, nullptr, dinv, nullptr);
  }
}

fo_status fo_umesh_velocity_setup(fo_problem *p) {
  const UMeshView m = umesh_view(p->mesh);
  const int blocks = fo_blocks_for(m.nn, FO_BLOCK, 65536);
  const uint8_t *vd = p->desc.velocity_dirichlet ? p->vdir : nullptr;
  const double g0 = p->desc.n_omega0 > 0 ? p->desc.omega0_weight : 0.0;
  if (m.dim == 2)
    k_u_velocity_assemble<2><<<blocks, FO_BLOCK, 0, p->ctx->stream>>>(m, p->desc.alpha_mass, g0, p->desc.normal_penalty,
                                                                      p->omega0, vd, p->Wvel, p->dinv_vel);
  else
    k_u_velocity_assemble<3><<<blocks, FO_BLOCK, 0, p->ctx->stream>>>(m, p->desc.alpha_mass, g0, p->desc.normal_penalty,
                                                                      p->omega0, vd, p->Wvel, p->dinv_vel);
  fo_note_launch(1);
  FO_CU(p->ctx, cudaGetLastError());
  return FO_OK;
}

template <class Op, class X, typename T>
__global__ void k_u_apply(Op op, X x, double *y) {
  op.sweep(x, [&](long long a, const T *out) {
#pragma unroll
    for (int c = 0; c < Op::NPN; ++c) y[a * Op::NPN + c] = (double)out[c];
  });
}

struct UCastX {   // FP32 gather of a double vector, Dirichlet DOFs read as zero
  const double *v;
  const uint8_t *dir;
  __device__ __forceinline__ float operator()(long long i) const { return dir[i] ? 0.f : (float)v[i]; }
};

fo_status fo_umesh_state_apply(fo_problem *p, const double *x, double *y, bool fp32) {
  const fo_mesh *me = p->mesh;
  const int blocks = fo_blocks_for(me->um->nn, FO_BLOCK, 65536);
  cudaStream_t s = p->ctx->stream;
  const int d = me->um->dim;
  const MaskedX<double> mx{x, p->dir};
  const UCastX cx{x, p->dir};
#define FO_U_APPLY(NPN)                                                                                      \
  if (fp32) k_u_apply<CsrOp<NPN, float>, UCastX, float><<<blocks, FO_BLOCK, 0, s>>>(make_csr_op<NPN>(me, p->Wst32), cx, y); \
  else k_u_apply<CsrOp<NPN, double>, MaskedX<double>, double><<<blocks, FO_BLOCK, 0, s>>>(make_csr_op<NPN>(me, (const double *)p->Wst), mx, y);
  if (p->ncomp == 1) {
    FO_U_APPLY(1)
  } else if (d == 2) {
    FO_U_APPLY(2)
  } else {
    FO_U_APPLY(3)
  }
#undef FO_U_APPLY
  fo_note_launch(1);
  FO_CU(p->ctx, cudaGetLastError());
  return FO_OK;
}

fo_status fo_umesh_velocity_apply(fo_problem *p, const double *x, double *y) {
  const fo_mesh *me = p->mesh;
  const int blocks = fo_blocks_for(me->um->nn, FO_BLOCK, 65536);
  cudaStream_t s = p->ctx->stream;
  const uint8_t *vd = p->desc.velocity_dirichlet ? p->vdir : nullptr;
  if (me->um->dim == 2) {
    if (vd) k_u_apply<CsrOp<2, double>, NodeMaskedX<double, 2>, double><<<blocks, FO_BLOCK, 0, s>>>(make_csr_op<2>(me, (const double *)p->Wvel), NodeMaskedX<double, 2>{x, vd}, y);
    else k_u_apply<CsrOp<2, double>, VecX<double>, double><<<blocks, FO_BLOCK, 0, s>>>(make_csr_op<2>(me, (const double *)p->Wvel), VecX<double>{x}, y);
  } else {
    if (vd) k_u_apply<CsrOp<3, double>, NodeMaskedX<double, 3>, double><<<blocks, FO_BLOCK, 0, s>>>(make_csr_op<3>(me, (const double *)p->Wvel), NodeMaskedX<double, 3>{x, vd}, y);
    else k_u_apply<CsrOp<3, double>, VecX<double>, double><<<blocks, FO_BLOCK, 0, s>>>(make_csr_op<3>(me, (const double *)p->Wvel), VecX<double>{x}, y);
  }
  fo_note_launch(1);
  FO_CU(p->ctx, cudaGetLastError());
  return FO_OK;
}

// --------------------------------------------------------------------------- functionals
// J (heat: sum A_e |e| |grad u|^2, eq. heat_cost; elasticity: sum A_e |e| sigma : eps,
// eq. compli_cost; screened family: F . u) and |Omega| = sum chi_e |e| (eq. compli_constr):
// block partials, then one warp per value adds them in a fixed order.
template <int D>
__global__ void k_u_functionals(UMeshView m, int kind, double lam, double mu, const double *coef, const uint8_t *chi,
                                const double *chif, const double *u, const double *load, double *partials) {
  __shared__ double smem[32 * 2];
  double v[2] = {0.0, 0.0};
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x, st = (long long)gridDim.x * blockDim.x;
  for (long long e = tid; e < m.nt; e += st) {
    const double A = coef[e], vol = m.vol[e];
    if (kind == FO_ELASTIC) {
      double du[D][D];
#pragma unroll
      for (int i = 0; i < D; ++i)
#pragma unroll
        for (int k = 0; k < D; ++k) du[i][k] = 0.0;
#pragma unroll
      for (int b = 0; b <= D; ++b) {
        const long long nb = m.cells[e * (D + 1) + b];
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
          for (int k = 0; k < D; ++k) du[i][k] += u[nb * D + i] * m.g(e, b, k);
      }
      double tr = 0, se = 0;
#pragma unroll
      for (int i = 0; i < D; ++i) tr += du[i][i];
#pragma unroll
      for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) {
          const double eij = 0.5 * (du[i][j] + du[j][i]);
          se += 2.0 * mu * eij * eij;
        }
      se += lam * tr * tr;
      v[0] += A * vol * se;
    } else if (kind == FO_HEAT) {
      double gu[D];
#pragma unroll
      for (int k = 0; k < D; ++k) gu[k] = 0.0;
#pragma unroll
      for (int b = 0; b <= D; ++b) {
        const double ub = u[m.cells[e * (D + 1) + b]];
#pragma unroll
        for (int k = 0; k < D; ++k) gu[k] += ub * m.g(e, b, k);
      }
      double g2 = 0;
#pragma unroll
      for (int k = 0; k < D; ++k) g2 += gu[k] * gu[k];
      v[0] += A * vol * g2;
    }
    v[1] += chif ? chif[e] * vol : (chi[e] ? vol : 0.0);
  }
  if (kind == FO_HELMHOLTZ)
    for (long long a = tid; a < m.nn; a += st) v[0] += load[a] * u[a];
  block_sum<2>(v, smem);
  if (threadIdx.x == 0) {
    partials[blockIdx.x * 2 + 0] = v[0];
    partials[blockIdx.x * 2 + 1] = v[1];
  }
}

__global__ void k_u_finish2(const double *partials, int nblocks, double *out) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (w >= 2) return;
  double t = 0;
  for (int b = lane; b < nblocks; b += 32) t += partials[(size_t)b * 2 + w];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  if (lane == 0) out[w] = t;
}

fo_status fo_umesh_functionals_on(fo_problem *p, const double *u, const double *load, double *J, double *vol) {
  const UMeshView m = umesh_view(p->mesh);
  fo_ctx *ctx = p->ctx;
  const int blocks = fo_blocks_for(std::max(m.nt, m.nn), FO_BLOCK, 1024);
  double *part = p->red, *res = p->red + 2 * 1024;
  const double *chif = p->desc.coef_rule == FO_COEF_CUT ? p->chif : nullptr;
  if (m.dim == 2)
    k_u_functionals<2><<<blocks, FO_BLOCK, 0, ctx->stream>>>(m, p->desc.kind, p->lame_lambda, p->lame_mu, p->coef,
                                                             p->chi, chif, u, load, part);
  else
    k_u_functionals<3><<<blocks, FO_BLOCK, 0, ctx->stream>>>(m, p->desc.kind, p->lame_lambda, p->lame_mu, p->coef,
                                                             p->chi, chif, u, load, part);
  k_u_finish2<<<1, 64, 0, ctx->stream>>>(part, blocks, res);
  fo_note_launch(2);
  FO_CU(ctx, cudaGetLastError());
  FO_CU(ctx, cudaMemcpyAsync(ctx->h_scalars, res, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  FO_CU(ctx, cudaStreamSynchronize(ctx->stream));
  *J = ctx->h_scalars[0];
  *vol = ctx->h_scalars[1];
  return FO_OK;
}

fo_status fo_umesh_functionals(fo_problem *p, double *J, double *vol) {
  return fo_umesh_functionals_on(p, p->u, p->load, J, vol);
}

// ------------------------------------------------------------------ shape derivative RHS
// b[d a + i] = sum over the node's elements of |e| (S1 grad lambda_a)_i + int_e S0_i lambda_a,
// S1 = S1^J + lambda chi_e / V I (eq. S0andS1; S^J of Sec. 6.2 for elasticity with p = -2u:
// A (2 Du^T sigma(u) - sigma : eps I); of Sec. 6.3 for heat with p = -u: S0 = 2u grad f,
// S1 = (2uf - A |grad u|^2) I + 2A grad u (x) grad u, f the P1 interpolant).
template <int D>
__global__ void k_u_shape_rhs(UMeshView m, int kind, double lam_e, double mu_e, double lam_ppl, double inv_V,
                              const double *coef, const uint8_t *chi, const double *chif, const double *u,
                              const double *f, double *b, int add) {
  for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < m.nn; a += (long long)gridDim.x * blockDim.x) {
    double acc[D];
#pragma unroll
    for (int k = 0; k < D; ++k) acc[k] = 0.0;
    for (int q = m.adj_ptr[a]; q < m.adj_ptr[a + 1]; ++q) {
      const long long e = m.adj[q] / (D + 1);
      const int la = m.adj[q] % (D + 1);
      const double A = coef[e], vol = m.vol[e];
      const double cv = chif ? chif[e] * (lam_ppl * inv_V) : (chi[e] ? lam_ppl * inv_V : 0.0);
      double gl[D];
#pragma unroll
      for (int k = 0; k < D; ++k) gl[k] = m.g(e, la, k);
      if (kind == FO_ELASTIC) {
        double du[D][D];
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
          for (int k = 0; k < D; ++k) du[i][k] = 0.0;
#pragma unroll
        for (int bb = 0; bb <= D; ++bb) {
          const long long nb = m.cells[e * (D + 1) + bb];
#pragma unroll
          for (int i = 0; i < D; ++i)
#pragma unroll
            for (int k = 0; k < D; ++k) du[i][k] += u[nb * D + i] * m.g(e, bb, k);
        }
        double tr = 0;
#pragma unroll
        for (int i = 0; i < D; ++i) tr += du[i][i];
        double sig[D][D], se = 0;
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
          for (int j = 0; j < D; ++j) {
            sig[i][j] = (i == j ? lam_e * tr : 0.0) + mu_e * (du[i][j] + du[j][i]);
            se += sig[i][j] * 0.5 * (du[i][j] + du[j][i]);
          }
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
          for (int j = 0; j < D; ++j) {
            double t = 0;
#pragma unroll
            for (int k = 0; k < D; ++k) t += du[k][i] * sig[k][j];
            const double S1ij = A * (2.0 * t - (i == j ? se : 0.0)) + (i == j ? cv : 0.0);
            acc[i] += vol * S1ij * gl[j];
          }
      } else {
        double gu[D], gf[D];
#pragma unroll
        for (int k = 0; k < D; ++k) gu[k] = gf[k] = 0.0;
        double su = 0, sf = 0, suf = 0;
#pragma unroll
        for (int bb = 0; bb <= D; ++bb) {
          const long long nb = m.cells[e * (D + 1) + bb];
          const double ub = u[nb], fb = f[nb];
          su += ub;
          sf += fb;
          suf += ub * fb;
#pragma unroll
          for (int k = 0; k < D; ++k) {
            gu[k] += ub * m.g(e, bb, k);
            gf[k] += fb * m.g(e, bb, k);
          }
        }
        const double mref = vol / ((D + 1) * (D + 2));
        const double uf = mref * (suf + su * sf);       // int_e u f
        const double Mu = mref * (su + u[a]);           // int_e u lambda_a
        double g2 = 0, gdot = 0;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          g2 += gu[k] * gu[k];
          gdot += gu[k] * gl[k];
        }
#pragma unroll
        for (int i = 0; i < D; ++i) {
          const double S1gl = A * (-g2 * gl[i] + 2.0 * gu[i] * gdot) + cv * gl[i];
          acc[i] += vol * S1gl + 2.0 * uf * gl[i] + 2.0 * gf[i] * Mu;
        }
      }
    }
#pragma unroll
    for (int k = 0; k < D; ++k) b[a * D + k] = add ? b[a * D + k] + acc[k] : acc[k];
  }
}

fo_status fo_umesh_shape_rhs_ex(fo_problem *p, const double *u, const double *f, double lambda, const double *w,
                                double inv_V, int add) {
  if (p->desc.kind == FO_HELMHOLTZ)
    return fo_fail(p->ctx, FO_EINVAL, "the single-instance shape derivative covers FO_HEAT and FO_ELASTIC");
  const UMeshView m = umesh_view(p->mesh);
  const int blocks = fo_blocks_for(m.nn, FO_BLOCK, 65536);
  if (m.dim == 2)
    k_u_shape_rhs<2><<<blocks, FO_BLOCK, 0, p->ctx->stream>>>(m, p->desc.kind, p->lame_lambda, p->lame_mu, lambda, inv_V,
                                                              p->coef, p->chi, w, u, f, p->rhs, add);
  else
    k_u_shape_rhs<3><<<blocks, FO_BLOCK, 0, p->ctx->stream>>>(m, p->desc.kind, p->lame_lambda, p->lame_mu, lambda, inv_V,
                                                              p->coef, p->chi, w, u, f, p->rhs, add);
  fo_note_launch(1);
  FO_CU(p->ctx, cudaGetLastError());
  return FO_OK;
}

fo_status fo_umesh_shape_rhs(fo_problem *p, double lambda) {
  if (p->desc.kind == FO_HELMHOLTZ)
    return fo_fail(p->ctx, FO_EINVAL, "the single-instance shape derivative covers FO_HEAT and FO_ELASTIC");
  const UMeshView m = umesh_view(p->mesh);
  const double inv_V = p->desc.volume_target > 0 ? 1.0 / p->desc.volume_target : 1.0;
  const int blocks = fo_blocks_for(m.nn, FO_BLOCK, 65536);
  const double *chif = p->desc.coef_rule == FO_COEF_CUT ? p->chif : nullptr;
  if (m.dim == 2)
    k_u_shape_rhs<2><<<blocks, FO_BLOCK, 0, p->ctx->stream>>>(m, p->desc.kind, p->lame_lambda, p->lame_mu, lambda, inv_V,
                                                              p->coef, p->chi, chif, p->u, p->f, p->rhs, 0);
  else
    k_u_shape_rhs<3><<<blocks, FO_BLOCK, 0, p->ctx->stream>>>(m, p->desc.kind, p->lame_lambda, p->lame_mu, lambda, inv_V,
                                                              p->coef, p->chi, chif, p->u, p->f, p->rhs, 0);
  fo_note_launch(1);
  FO_CU(p->ctx, cudaGetLastError());
  return FO_OK;
}
