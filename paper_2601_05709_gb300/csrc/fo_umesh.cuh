// General simplicial meshes given as arrays (fo_mesh_from_arrays): connectivity, element data
// and the assembled node-block operators that the solvers apply on them.
//
// The paper runs on Gmsh / DOLFINx meshes (Sec. 5.1 helpers, Sec. 6 examples); this is the
// path for such meshes, beside the structured Kuhn grid that derives everything from grid
// indices.  Layout (all device arrays, built once per mesh):
//   cells [N_T][d+1] int32, coords [N_n][d] FP64 (as given);
//   element data: |e| [N_T] and barycentric gradients grad[(a d + k) N_T + e] (slot-major, so
//   a warp reading one gradient entry of 32 consecutive elements is coalesced);
//   node -> element adjacency in CSR over nodes, entries e (d+1) + local vertex, in element
//   order (every per-node sum runs over the node's elements in a fixed order: deterministic,
//   no atomics);
//   the node graph (CSR over nodes, sorted columns, diagonal included) and, per adjacency
//   entry, the graph position of each of the element's vertices in the node's row, so that a
//   thread owning a row adds element blocks straight into it;
//   boundary facets (those of one element only) with their measure, outward unit normal and
//   box face (2 axis + side, or -1), and the node -> facet adjacency with graph positions.
// Box faces are those of the nodes' bounding box: a node lies on face (axis, side) when its
// coordinate equals the box's bound exactly.
#pragma once
#include "fo_internal.cuh"

struct fo_umesh {
  int dim = 0;
  long long nn = 0, nt = 0, nnz = 0, nf = 0;
  double volume = 0;                // sum of the element measures
  double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  int *adj_ptr = nullptr;           // [nn + 1]
  int *adj = nullptr;               // [nt (d+1)]
  int *adj_pos = nullptr;           // [nt (d+1)][d+1]
  int *row_ptr = nullptr;           // [nn + 1]
  int *col = nullptr;               // [nnz]
  int *diag = nullptr;              // [nn]
  double *vol = nullptr;            // [nt]
  double *grad = nullptr;           // [(d+1) d][nt]
  int *fnodes = nullptr;            // [nf][d]
  double *farea = nullptr;          // [nf]
  double *fnormal = nullptr;        // [nf][d]
  int *fface = nullptr;             // [nf]
  int *nf_ptr = nullptr;            // [nn + 1]
  int *nf_adj = nullptr;            // [nf d]: f d + local vertex
  int *nf_pos = nullptr;            // [nf d][d]
  uint8_t *face_mask = nullptr;     // [nn]: bit (2 axis + side)
  std::vector<std::pair<void **, size_t>> allocs;   // for release
};

// Device view of a general mesh for kernels.
struct UMeshView {
  int dim;
  long long nn, nt;
  const int32_t *cells;
  const double *coords;
  const int *adj_ptr, *adj, *adj_pos, *row_ptr, *col, *diag;
  const double *vol, *grad;
  const int *fnodes, *fface, *nf_ptr, *nf_adj, *nf_pos;
  const double *farea, *fnormal;
  const uint8_t *face_mask;
  __device__ __forceinline__ double g(long long e, int a, int k) const { return grad[(a * dim + k) * nt + e]; }
};

inline UMeshView umesh_view(const fo_mesh *m) {
  const fo_umesh *u = m->um;
  UMeshView v;
  v.dim = u->dim;
  v.nn = u->nn;
  v.nt = u->nt;
  v.cells = m->d_cells;
  v.coords = m->d_coords;
  v.adj_ptr = u->adj_ptr;
  v.adj = u->adj;
  v.adj_pos = u->adj_pos;
  v.row_ptr = u->row_ptr;
  v.col = u->col;
  v.diag = u->diag;
  v.vol = u->vol;
  v.grad = u->grad;
  v.fnodes = u->fnodes;
  v.fface = u->fface;
  v.nf_ptr = u->nf_ptr;
  v.nf_adj = u->nf_adj;
  v.nf_pos = u->nf_pos;
  v.farea = u->farea;
  v.fnormal = u->fnormal;
  v.face_mask = u->face_mask;
  return v;
}

// Assembled operator in node-block CSR, in difference form: the entry at the diagonal
// position of row a holds the block row sum R_a, the others the off-diagonal blocks W, and
//   (A x)_a = R_a x_a + sum_{c != a} W_ac (x_c - x_a),
// which keeps the constant kernel of a stiffness matrix exact under rounding of the stored
// weights (FP32 copies included), as the structured path's stencil rows do.  Dirichlet rows are
// identity rows and Dirichlet columns are eliminated (baked in by the assembly).  Blocks are
// stored entry-major, W[k BLK + i NPN + j], so a thread reads its row as one contiguous run.
// Node ownership: one node per thread, grid-stride (the persistent solvers' sweep / each).
template <int NPN_, typename T>
struct CsrOp {
  static constexpr int NPN = NPN_;
  static constexpr int BLK = NPN * NPN;
  static constexpr size_t smem_bytes = 0;
  Grid g;   // only g.num_nodes is read
  const int *row_ptr, *col, *diag;
  const T *W;

  template <class X>
  __device__ __forceinline__ void row(long long a, const X &x, T out[NPN]) const {
    T xa[NPN], acc[NPN];
#pragma unroll
    for (int j = 0; j < NPN; ++j) xa[j] = (T)x(a * NPN + j);
    const int dg = diag[a];
#pragma unroll
    for (int i = 0; i < NPN; ++i) {
      T s = T(0);
#pragma unroll
      for (int j = 0; j < NPN; ++j) s = fma(W[(long long)dg * BLK + i * NPN + j], xa[j], s);
      acc[i] = s;
    }
    const int k1 = row_ptr[a + 1];
    for (int k = row_ptr[a]; k < k1; ++k) {
      if (k == dg) continue;
      const long long c = col[k];
      T dx[NPN];
#pragma unroll
      for (int j = 0; j < NPN; ++j) dx[j] = (T)x(c * NPN + j) - xa[j];
#pragma unroll
      for (int i = 0; i < NPN; ++i)
#pragma unroll
        for (int j = 0; j < NPN; ++j) acc[i] = fma(W[(long long)k * BLK + i * NPN + j], dx[j], acc[i]);
    }
#pragma unroll
    for (int i = 0; i < NPN; ++i) out[i] = acc[i];
  }
  template <class X, class F>
  __device__ __forceinline__ void sweep(const X &x, F &&f) const {
    const long long gs = (long long)gridDim.x * blockDim.x;
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < g.num_nodes; a += gs) {
      T out[NPN];
      row(a, x, out);
      f(a, out);
    }
  }
  template <class F>
  __device__ __forceinline__ void each(F &&f) const {
    const long long gs = (long long)gridDim.x * blockDim.x;
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < g.num_nodes; a += gs) f(a);
  }
};

template <int NPN, typename T>
inline CsrOp<NPN, T> make_csr_op(const fo_mesh *m, const T *W) {
  CsrOp<NPN, T> op;
  op.g = Grid{};
  op.g.dim = m->um->dim;
  op.g.num_nodes = m->um->nn;
  op.row_ptr = m->um->row_ptr;
  op.col = m->um->col;
  op.diag = m->um->diag;
  op.W = W;
  return op;
}

// Entry points of the general-mesh path (fo_umesh.cu unless noted).
fo_status fo_umesh_build(fo_mesh *m, const double *coords, const int32_t *cells);
void fo_umesh_release(fo_mesh *m);
fo_status fo_umesh_masks(fo_problem *p);
fo_status fo_umesh_loads(fo_problem *p);
fo_status fo_umesh_coefficients(fo_problem *p);       // also assembles the state operator
fo_status fo_umesh_velocity_setup(fo_problem *p);
fo_status fo_umesh_state_apply(fo_problem *p, const double *x, double *y, bool fp32);
fo_status fo_umesh_velocity_apply(fo_problem *p, const double *x, double *y);
fo_status fo_umesh_functionals(fo_problem *p, double *J, double *vol);
fo_status fo_umesh_shape_rhs(fo_problem *p, double lambda);
fo_status fo_umesh_shape_rhs_ex(fo_problem *p, const double *u, const double *f, double lambda, const double *w,
                                double inv_V, int add);
fo_status fo_umesh_functionals_on(fo_problem *p, const double *u, const double *load, double *J, double *vol);
fo_status fo_umesh_transport_assemble(fo_problem *p, double dt, double h, int smooth);
fo_status fo_umesh_transport_apply(fo_problem *p, int which, const double *x, double *y);
fo_status fo_umesh_levelset_step(fo_problem *p, double t_end, int nsteps, double h, int smooth,
                                 const fo_solve_opts *o, fo_solve_stats *st);
fo_status fo_umesh_reinit(fo_problem *p, int nsteps, double t_final, double h, const fo_solve_opts *o,
                          fo_solve_stats *st);
// fo_krylov.cu: Jacobi-PCG on the assembled operators (state: FP64, or FP32 inner solves in
// FP64 refinement; velocity: the coupled d-component system)
fo_status fo_umesh_state_pcg(fo_problem *p, const double *b, double *x, const fo_solve_opts *o, fo_solve_stats *st);
fo_status fo_umesh_velocity_pcg(fo_problem *p, const fo_solve_opts *o, double *Btt, fo_solve_stats *st);
