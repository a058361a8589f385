// Node-centric helpers of the structured Kuhn grid and the stored-stencil operator.
//
// Every simplex of the Kuhn triangulation is a path v_0 -> v_1 -> ... -> v_D with
// v_{l+1} = v_l + e_{pi_l}; its barycentric gradients are sparse,
//   grad lambda_l = e_{pi_{l-1}} / h_{pi_{l-1}}  (l >= 1)  -  e_{pi_l} / h_{pi_l}  (l <= D-1),
// and the Jacobian of a P1 field w is the path difference D w [:, pi_l] = (w_{l+1} - w_l) / h_{pi_l}.
// A node's 7 (2D) / 15 (3D) stencil neighbours are its slots (self, the positive Kuhn
// neighbours by bitmask, the negative ones); its 6 / 24 simplices (p, m) are those in which it
// is vertex m of simplex p.  The element-level kernels (stencil builders, loads, shape
// derivative) visit them from a thread per node with the field at the slots in registers;
// the solvers apply the operators as stored rows (StencilOp).  Sums run in a fixed order, so
// results are deterministic and no atomics are needed.
#pragma once
#include <type_traits>
#include "fo_internal.cuh"

// ---- field views ------------------------------------------------------------------------
template <typename T>
struct VecX {
  const T *v;
  __device__ __forceinline__ T operator()(long long i) const { return v[i]; }
};
template <typename T>
struct MaskedX {   // Dirichlet DOFs read as zero
  const T *v;
  const uint8_t *dir;
  __device__ __forceinline__ T operator()(long long i) const { return dir[i] ? T(0) : v[i]; }
};
template <typename T, int NPN>
struct NodeMaskedX {   // all components of masked nodes read as zero
  const T *v;
  const uint8_t *mask;   // per node
  __device__ __forceinline__ T operator()(long long i) const { return mask[i / NPN] ? T(0) : v[i]; }
};
// z + beta_c p with one beta per system; system c = dof % NC (NC = 1: a single system)
template <typename T, int NC>
struct CombX {
  const T *z;
  const T *p;
  T beta[NC];
  __device__ __forceinline__ T operator()(long long i) const {
    const int c = (NC == 1) ? 0 : (int)(i % NC);
    return z[i] + beta[c] * p[i];
  }
};

// ---- node ownership ---------------------------------------------------------------------
// A persistent kernel walks "its" nodes through the operator: `sweep(x, f)` applies the
// operator to the field view x and calls f(a, row[NPN]) for every node a the calling
// thread owns; `each(f)` calls f(a) for the same nodes without applying anything.  The
// node-centric operators own nodes grid-stride, one per thread.
template <int NPN, typename OUT, class Op, class X, class F>
__device__ __forceinline__ void node_sweep(const Op &op, const Grid &g, const X &x, F &&f) {
  const long long gs = (long long)gridDim.x * blockDim.x;
  for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < g.num_nodes; a += gs) {
    int idx[3];
    node_ijk(g, a, idx);
    OUT out[NPN];
    op.row(a, idx, x, out);
    f(a, out);
  }
}
template <class F>
__device__ __forceinline__ void node_each(const Grid &g, F &&f) {
  const long long gs = (long long)gridDim.x * blockDim.x;
  for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < g.num_nodes; a += gs) f(a);
}
#define FO_NODE_OWNERSHIP(OUT)                                                                           \
  static constexpr size_t smem_bytes = 0;                                                                \
  template <class X, class F>                                                                            \
  __device__ __forceinline__ void sweep(const X &x, F &&f) const { node_sweep<NPN, OUT>(*this, g, x, f); } \
  template <class F>                                                                                     \
  __device__ __forceinline__ void each(F &&f) const { node_each(g, f); }

// Slot (stencil index) of vertex l of simplex p as seen from its vertex m.
template <int D>
__device__ __forceinline__ int rel_slot(int p, int m, int l) {
  int delta[3] = {0, 0, 0};
#pragma unroll
  for (int j = 0; j < D; ++j) {
    if (l > m && j >= m && j < l) delta[kperm<D>(p, j)] += 1;
    if (l < m && j >= l && j < m) delta[kperm<D>(p, j)] -= 1;
  }
  return stencil_slot<D>(delta);
}

// Node id of stencil slot s around node a (returns -1 outside the grid).
template <int D>
__device__ __forceinline__ long long slot_node(const Grid &g, const int idx[3], long long a, int s) {
  int dl[3];
  slot_offset<D>(s, dl);
  long long id = a;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    int q = idx[k] + dl[k];
    if (q < 0 || q >= (int)g.nn[k]) return -1;
    id += dl[k] * g.stride[k];
  }
  return id;
}

// slot_node with a slot outside the grid mapped to the node itself.  Every stored row has zero
// weight in such a slot (no element reaches it), and a difference-form row sees a zero
// difference there, so an apply may read x_a instead of branching: without the branch the
// loads of all slots can be issued together (cantilever 256x128 state CG: 4.16 -> 3.53 ms
// per optimisation step).
template <int D>
__device__ __forceinline__ long long slot_node_or_self(const Grid &g, const int idx[3], long long a, int s) {
  const long long nb = slot_node<D>(g, idx, a, s);
  return nb < 0 ? a : nb;
}

// Is the cell of simplex (p, m) around idx inside the grid?  Writes its element id.
template <int D>
__device__ __forceinline__ bool elem_of(const Grid &g, const int idx[3], int p, int m, long long &elem) {
  int c[3] = {idx[0], idx[1], idx[2]};
#pragma unroll
  for (int l = 0; l < D; ++l)
    if (l < m) c[kperm<D>(p, l)] -= 1;
#pragma unroll
  for (int k = 0; k < D; ++k)
    if (c[k] < 0 || c[k] >= g.n[k]) return false;
  long long cell = c[0] + g.cstride[1] * c[1] + (D == 3 ? g.cstride[2] * c[2] : 0);
  elem = (long long)KP<D>::P * cell + p;
  return true;
}

// grad lambda_l of the Kuhn simplex p: e_{pi_{l-1}} / h - e_{pi_l} / h (sparse)
template <int D>
__device__ __forceinline__ void kuhn_grad(const Grid &g, int p, int l, double gr[3]) {
  gr[0] = gr[1] = gr[2] = 0.0;
  if (l >= 1) gr[kperm<D>(p, l - 1)] += g.inv_h[kperm<D>(p, l - 1)];
  if (l < D) gr[kperm<D>(p, l)] -= g.inv_h[kperm<D>(p, l)];
}

// Load NPN components of the field at every stencil neighbour (0 outside the grid).
template <int D, int NPN, typename T, class X>
__device__ __forceinline__ void load_stencil(const Grid &g, const int idx[3], long long a, const X &x,
                                             T xs[ST<D>::S][NPN]) {
#pragma unroll
  for (int s = 0; s < ST<D>::S; ++s) {
    long long nb = slot_node<D>(g, idx, a, s);
#pragma unroll
    for (int c = 0; c < NPN; ++c) xs[s][c] = (nb >= 0) ? x(nb * NPN + c) : T(0);
  }
}

// ---- stored per-node stencils --------------------------------------------------------------
// A problem's operator kept as its matrix rows in stencil form: for every stencil slot s (the
// node itself, then its Kuhn neighbours) an NPN x NPN block (FULL) or only its diagonal (the
// velocity form, whose component systems are decoupled).  Slot-major layout
// W[(s * BLK + k) * N_n + a], so that a warp's loads of one entry are coalesced.  Rows are in
// difference form: slot 0 holds the row sum R and the row is
//   (A x)_a = R x_a + sum_{s >= 1} W_s (x_{nb(s)} - x_a)
// (R is exact, the stiffness rows summing to zero), so that rounding in the stored weights,
// FP32 ones included, keeps the operator's constant kernel as a matrix-free apply that
// differences the field does.  Dirichlet rows are identity rows and Dirichlet columns are
// eliminated (the builders bake both in).  An apply costs a subtraction and an FMA per stored
// entry; on GB300, whose FP64 rate is 1/58 of its FP32 rate, that is several times less FP64
// work than recomputing element matrices, and a single problem's stencils stay resident in the
// 129 MB L2.  Built once per coefficient update (state) or once per problem (velocity).
//
// WT is the storage type of the weights (T, or BF16 rows of a multigrid level applied in FP32:
// the difference form keeps the rounded operator's constant kernel and its symmetry).
// Where the weight of entry e of slot s in node a's row is stored (nb: the slot's neighbour,
// or a itself outside the grid).  Slots below SH are the node's own; slot s >= SH (offset -m,
// m = s - SH + 1) is the transpose of the neighbour's slot-m block: entry (i, j) is read as
// (j, i) of row nb.  Outside the grid nb = a reads an arbitrary stored weight, which the
// difference form multiplies by x_a - x_a = 0.
template <int D, int NPN, bool FULL, class WT>
__device__ __forceinline__ const WT *slot_weight(const WT *W, long long N, long long a, long long nb, int s, int e) {
  constexpr int BLK = FULL ? NPN * NPN : NPN;
  if (s < ST<D>::SH) return W + ((long long)s * BLK + e) * N + a;
  const int m = s - ST<D>::SH + 1;
  const int et = FULL ? (e % NPN) * NPN + e / NPN : e;
  return W + ((long long)m * BLK + et) * N + nb;
}

template <typename T, typename WT>
__device__ __forceinline__ T stencil_weight(const WT *w) {
  return (T)*w;
}
template <>
__device__ __forceinline__ float stencil_weight<float, __nv_bfloat16>(const __nv_bfloat16 *w) {
  return __bfloat162float(*w);
}

template <int D, int NPN_, bool FULL, typename T, typename WT = T>
struct StencilOp {
  static constexpr int NPN = NPN_;
  static constexpr int BLK = FULL ? NPN * NPN : NPN;
  Grid g;
  FO_NODE_OWNERSHIP(T)
  const WT *W;

  template <class X>
  __device__ __forceinline__ void row(long long a, const int idx[3], const X &x, T out[NPN]) const {
    const long long N = g.num_nodes;
    T acc[NPN], xa[NPN];
#pragma unroll
    for (int j = 0; j < NPN; ++j) xa[j] = (T)x(a * NPN + j);
#pragma unroll
    for (int c = 0; c < NPN; ++c) acc[c] = T(0);
#pragma unroll
    for (int s = 0; s < ST<D>::S; ++s) {
      const long long nb = slot_node_or_self<D>(g, idx, a, s);
      T xv[NPN];   // x_a on slot 0, x_nb - x_a on the others (zero outside the grid)
#pragma unroll
      for (int j = 0; j < NPN; ++j) xv[j] = s == 0 ? xa[j] : (T)x(nb * NPN + j) - xa[j];
      if (FULL) {
#pragma unroll
        for (int i = 0; i < NPN; ++i)
#pragma unroll
          for (int j = 0; j < NPN; ++j)
            acc[i] = fma(stencil_weight<T>(slot_weight<D, NPN, FULL>(W, N, a, nb, s, i * NPN + j)), xv[j], acc[i]);
      } else {
#pragma unroll
        for (int c = 0; c < NPN; ++c)
          acc[c] = fma(stencil_weight<T>(slot_weight<D, NPN, FULL>(W, N, a, nb, s, c)), xv[c], acc[c]);
      }
    }
#pragma unroll
    for (int c = 0; c < NPN; ++c) out[c] = acc[c];
  }

};


// --------------------------------------------------------------- operator construction
// Stored-stencil operators of a problem (state: scalar or elastic; velocity).
template <int D, typename T>
inline StencilOp<D, 1, true, T> make_scalar_stencil(const fo_problem *p) {
  StencilOp<D, 1, true, T> op;
  op.g = p->mesh->g;
  op.W = std::is_same<T, float>::value ? (const T *)p->Wst32 : (const T *)p->Wst;
  return op;
}
template <int D, typename T>
inline StencilOp<D, D, true, T> make_elastic_stencil(const fo_problem *p) {
  StencilOp<D, D, true, T> op;
  op.g = p->mesh->g;
  op.W = std::is_same<T, float>::value ? (const T *)p->Wst32 : (const T *)p->Wst;
  return op;
}
template <int D>
inline StencilOp<D, D, false, double> make_velocity_stencil(const fo_problem *p) {
  StencilOp<D, D, false, double> op;
  op.g = p->mesh->g;
  op.W = p->Wvel;
  return op;
}
