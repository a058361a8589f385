// Matrix-free P1 operators on the structured Kuhn grid, written node-centrically.
//
// Every simplex of the Kuhn triangulation is a path v_0 -> v_1 -> ... -> v_D with
// v_{l+1} = v_l + e_{pi_l}; its barycentric gradients are sparse,
//   grad lambda_l = e_{pi_{l-1}} / h_{pi_{l-1}}  (l >= 1)  -  e_{pi_l} / h_{pi_l}  (l <= D-1),
// and the Jacobian of a P1 field w is the path difference D w [:, pi_l] = (w_{l+1} - w_l) / h_{pi_l}.
// A thread owns one node: it loads the field at the node's 7 (2D) / 15 (3D) stencil
// neighbours into registers once, then visits the node's 6 / 24 simplices (p, m) -- the
// node is vertex m of simplex p -- reading each vertex from the register stencil.  Sums
// run in a fixed order, so results are deterministic and no atomics are needed.
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

// A field view read in single precision (the gathered FP64 value rounded once to FP32).
template <class X>
struct CastX {
  X x;
  __device__ __forceinline__ float operator()(long long i) const { return (float)x(i); }
};

// Operator adapter of the mixed path: the element arithmetic of the wrapped FP32 operator
// (FP32 element data, FP32 accumulation) on FP64 vectors, so that the Krylov recurrence
// around it stays in FP64.  On GB300 the FP64 pipe is about 1/58 of the FP32 one, and the
// element arithmetic is most of the FP64 work of an iteration.
template <class Op32>
struct Fp32ApplyOp {
  static constexpr int NPN = Op32::NPN;
  Op32 op;
  Grid g;
  FO_NODE_OWNERSHIP(double)
  template <class X>
  __device__ __forceinline__ void row(long long a, const int idx[3], const X &x, double out[NPN]) const {
    float o[NPN];
    op.row(a, idx, CastX<X>{x}, o);
#pragma unroll
    for (int c = 0; c < NPN; ++c) out[c] = (double)o[c];
  }
};

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

// ---- scalar state operator: int A k grad u . grad v (+ omega^2 int u v) ------------------
template <int D, typename T>
struct ScalarStateOp {
  static constexpr int NPN = 1;
  Grid g;
  FO_NODE_OWNERSHIP(T)
  const T *coef;       // A_e * k per element
  const uint8_t *dir;  // per node
  T sk[3];             // |e| / h_a^2
  T w2m;               // omega^2 |e| / ((D+1)(D+2)); 0 = no mass term

  template <class X>
  __device__ __forceinline__ void row(long long a, const int idx[3], const X &x, T out[1]) const {
    if (dir[a]) { out[0] = x(a); return; }
    T xs[ST<D>::S][1];
    load_stencil<D, 1, T>(g, idx, a, x, xs);
    T acc = 0;
#pragma unroll
    for (int p = 0; p < KP<D>::P; ++p)
#pragma unroll
      for (int m = 0; m <= D; ++m) {
        long long e;
        if (!elem_of<D>(g, idx, p, m, e)) continue;
        const T Ae = coef[e];
        T s = 0;
        if (m >= 1) s += (xs[0][0] - xs[rel_slot<D>(p, m, m - 1)][0]) * sk[kperm<D>(p, m - 1)];
        if (m < D) s -= (xs[rel_slot<D>(p, m, m + 1)][0] - xs[0][0]) * sk[kperm<D>(p, m)];
        acc += Ae * s;
        if (w2m != T(0)) {
          T sum = xs[0][0];
#pragma unroll
          for (int l = 0; l <= D; ++l) sum += xs[rel_slot<D>(p, m, l)][0];
          acc += w2m * sum;
        }
      }
    out[0] = acc;
  }

  __device__ __forceinline__ void diag(long long a, const int idx[3], T out[1]) const {
    if (dir[a]) { out[0] = 1; return; }
    T acc = 0;
#pragma unroll
    for (int p = 0; p < KP<D>::P; ++p)
#pragma unroll
      for (int m = 0; m <= D; ++m) {
        long long e;
        if (!elem_of<D>(g, idx, p, m, e)) continue;
        T s = 0;
        if (m >= 1) s += sk[kperm<D>(p, m - 1)];
        if (m < D) s += sk[kperm<D>(p, m)];
        acc += coef[e] * s + 2 * w2m;
      }
    out[0] = acc;
  }
};

// ---- linear elasticity: int A sigma(u) : eps(v) -------------------------------------------
template <int D, typename T>
struct ElasticStateOp {
  static constexpr int NPN = D;
  Grid g;
  FO_NODE_OWNERSHIP(T)
  const T *coef;
  const uint8_t *dir;   // per DOF
  T lam, mu, vol;
  T ih[3];

  // Contribution of simplex (p, m) with gathered vertex values to the residual of vertex m.
  __device__ __forceinline__ void elem_row(int p, int m, const T (&xs)[ST<D>::S][D], T Ae, T acc[D]) const {
    T du[D][D];   // du[i][j] = d_j u_i
#pragma unroll
    for (int l = 0; l < D; ++l) {
      const int ax = kperm<D>(p, l);
      const int s0 = rel_slot<D>(p, m, l), s1 = rel_slot<D>(p, m, l + 1);
#pragma unroll
      for (int i = 0; i < D; ++i) du[i][ax] = (xs[s1][i] - xs[s0][i]) * ih[ax];
    }
    T tr = 0;
#pragma unroll
    for (int i = 0; i < D; ++i) tr += du[i][i];
    const T w = Ae * vol;
    if (m >= 1) {
      const int j = kperm<D>(p, m - 1);
#pragma unroll
      for (int i = 0; i < D; ++i) acc[i] += w * ih[j] * ((i == j ? lam * tr : T(0)) + mu * (du[i][j] + du[j][i]));
    }
    if (m < D) {
      const int j = kperm<D>(p, m);
#pragma unroll
      for (int i = 0; i < D; ++i) acc[i] -= w * ih[j] * ((i == j ? lam * tr : T(0)) + mu * (du[i][j] + du[j][i]));
    }
  }

  template <class X>
  __device__ __forceinline__ void row(long long a, const int idx[3], const X &x, T out[D]) const {
    T xs[ST<D>::S][D];
    load_stencil<D, D, T>(g, idx, a, x, xs);
    T acc[D];
#pragma unroll
    for (int i = 0; i < D; ++i) acc[i] = 0;
#pragma unroll
    for (int p = 0; p < KP<D>::P; ++p)
#pragma unroll
      for (int m = 0; m <= D; ++m) {
        long long e;
        if (!elem_of<D>(g, idx, p, m, e)) continue;
        elem_row(p, m, xs, coef[e], acc);
      }
#pragma unroll
    for (int i = 0; i < D; ++i) out[i] = dir[a * D + i] ? xs[0][i] : acc[i];
  }

  // diag of component i: A|e| [(lam + mu) (d_i psi)^2 + mu |grad psi|^2]
  __device__ __forceinline__ void diag(long long a, const int idx[3], T out[D]) const {
    T acc[D];
#pragma unroll
    for (int i = 0; i < D; ++i) acc[i] = 0;
#pragma unroll
    for (int p = 0; p < KP<D>::P; ++p)
#pragma unroll
      for (int m = 0; m <= D; ++m) {
        long long e;
        if (!elem_of<D>(g, idx, p, m, e)) continue;
        T gr[3] = {0, 0, 0};
        if (m >= 1) gr[kperm<D>(p, m - 1)] += ih[kperm<D>(p, m - 1)];
        if (m < D) gr[kperm<D>(p, m)] -= ih[kperm<D>(p, m)];
        T g2 = 0;
#pragma unroll
        for (int k = 0; k < D; ++k) g2 += gr[k] * gr[k];
        const T w = coef[e] * vol;
#pragma unroll
        for (int i = 0; i < D; ++i) acc[i] += w * ((lam + mu) * gr[i] * gr[i] + mu * g2);
      }
#pragma unroll
    for (int i = 0; i < D; ++i) out[i] = dir[a * D + i] ? T(1) : acc[i];
  }
};

// ---- velocity form B (component-blocked, D independent scalar systems) --------------------
// B_c = alpha_m M + K + gamma_0 M_{Omega_0} + gamma_b M_{faces normal to e_c}; H^1_0 rows
// are identity on boundary nodes.
template <int D, typename T>
struct VelocityOp {
  static constexpr int NPN = D;
  Grid g;
  FO_NODE_OWNERSHIP(T)
  const uint8_t *omega0;   // per element
  const uint8_t *vdir;     // per node (H^1_0)
  T sk[3];                 // |e| / h_a^2
  T mref;                  // |e| / ((D+1)(D+2))
  T alpha, gamma0, gammab;
  T fref[3];               // |f| / (D (D+1)) for facets on faces normal to axis a

  // facet-mass row of the face normal to `axis` through this node, for component values v[s]
  __device__ __forceinline__ T facet_row(const int idx[3], int axis, const T (&xs)[ST<D>::S][D], int comp) const {
    T acc = 0;
    if (D == 2) {
      const int o = 1 - axis;
      int dl[3] = {0, 0, 0};
      if (idx[o] + 1 <= g.n[o]) { dl[o] = 1; acc += fref[axis] * (2 * xs[0][comp] + xs[stencil_slot<D>(dl)][comp]); }
      if (idx[o] - 1 >= 0) { dl[o] = -1; acc += fref[axis] * (2 * xs[0][comp] + xs[stencil_slot<D>(dl)][comp]); }
    } else {
      const int o1 = axis == 0 ? 1 : 0, o2 = axis == 2 ? 1 : 2;
#pragma unroll
      for (int q = 0; q < 2; ++q)          // face-local Kuhn paths (o1, o2) and (o2, o1)
#pragma unroll
        for (int m = 0; m <= 2; ++m) {
          const int ax[2] = {q == 0 ? o1 : o2, q == 0 ? o2 : o1};
          int c[3] = {idx[0], idx[1], idx[2]};
          for (int l = 0; l < m; ++l) c[ax[l]] -= 1;
          if (c[o1] < 0 || c[o1] >= g.n[o1] || c[o2] < 0 || c[o2] >= g.n[o2]) continue;
          T sum = 2 * xs[0][comp];
#pragma unroll
          for (int l = 0; l <= 2; ++l) {
            if (l == m) continue;
            int dl[3] = {0, 0, 0};
            for (int j = 0; j < 2; ++j) {
              if (l > m && j >= m && j < l) dl[ax[j]] += 1;
              if (l < m && j >= l && j < m) dl[ax[j]] -= 1;
            }
            sum += xs[stencil_slot<D>(dl)][comp];
          }
          acc += fref[axis] * sum;
        }
    }
    return acc;
  }

  template <class X>
  __device__ __forceinline__ void row(long long a, const int idx[3], const X &x, T out[D]) const {
    T xs[ST<D>::S][D];
    load_stencil<D, D, T>(g, idx, a, x, xs);
    if (vdir[a]) {
#pragma unroll
      for (int c = 0; c < D; ++c) out[c] = xs[0][c];
      return;
    }
    T acc[D];
#pragma unroll
    for (int c = 0; c < D; ++c) acc[c] = 0;
#pragma unroll
    for (int p = 0; p < KP<D>::P; ++p)
#pragma unroll
      for (int m = 0; m <= D; ++m) {
        long long e;
        if (!elem_of<D>(g, idx, p, m, e)) continue;
        const T wm = (alpha + (omega0[e] ? gamma0 : T(0))) * mref;
#pragma unroll
        for (int c = 0; c < D; ++c) {
          T s = 0;
          if (m >= 1) s += (xs[0][c] - xs[rel_slot<D>(p, m, m - 1)][c]) * sk[kperm<D>(p, m - 1)];
          if (m < D) s -= (xs[rel_slot<D>(p, m, m + 1)][c] - xs[0][c]) * sk[kperm<D>(p, m)];
          T sum = xs[0][c];
#pragma unroll
          for (int l = 0; l <= D; ++l) sum += xs[rel_slot<D>(p, m, l)][c];
          acc[c] += s + wm * sum;
        }
      }
    if (gammab != T(0)) {
#pragma unroll
      for (int c = 0; c < D; ++c)
        if (idx[c] == 0 || idx[c] == g.n[c]) acc[c] += gammab * facet_row(idx, c, xs, c);
    }
#pragma unroll
    for (int c = 0; c < D; ++c) out[c] = acc[c];
  }

  __device__ __forceinline__ void diag(long long a, const int idx[3], T out[D]) const {
    if (vdir[a]) {
#pragma unroll
      for (int c = 0; c < D; ++c) out[c] = 1;
      return;
    }
    T acc = 0;
#pragma unroll
    for (int p = 0; p < KP<D>::P; ++p)
#pragma unroll
      for (int m = 0; m <= D; ++m) {
        long long e;
        if (!elem_of<D>(g, idx, p, m, e)) continue;
        T s = 0;
        if (m >= 1) s += sk[kperm<D>(p, m - 1)];
        if (m < D) s += sk[kperm<D>(p, m)];
        acc += s + (alpha + (omega0[e] ? gamma0 : T(0))) * mref * 2;
      }
#pragma unroll
    for (int c = 0; c < D; ++c) {
      T v = acc;
      if (gammab != T(0) && (idx[c] == 0 || idx[c] == g.n[c])) {
        // number of face facets through the node times 2 |f| / (D (D+1))
        int cnt = 0;
        if (D == 2) {
          const int o = 1 - c;
          cnt = (idx[o] + 1 <= g.n[o]) + (idx[o] - 1 >= 0);
        } else {
          const int o1 = c == 0 ? 1 : 0, o2 = c == 2 ? 1 : 2;
          for (int q = 0; q < 2; ++q)
            for (int m = 0; m <= 2; ++m) {
              const int ax[2] = {q == 0 ? o1 : o2, q == 0 ? o2 : o1};
              int cc[3] = {idx[0], idx[1], idx[2]};
              for (int l = 0; l < m; ++l) cc[ax[l]] -= 1;
              if (cc[o1] < 0 || cc[o1] >= g.n[o1] || cc[o2] < 0 || cc[o2] >= g.n[o2]) continue;
              ++cnt;
            }
        }
        v += gammab * fref[c] * 2 * cnt;
      }
      out[c] = v;
    }
  }
};

// ---- tiled linear elasticity: element data computed once per simplex -----------------------
// A block owns a tile of TX x TY (x TZ) nodes.  Stage 1 stages the field on the tile and a
// one-node halo in shared memory (the view x is evaluated once per node); stage 2 computes,
// for every simplex of the cells touching the tile, the scaled stress A_e |e| sigma(u_e)
// once (the node-centric operator recomputes it for each of the simplex's vertices);
// stage 3 forms each tile node's row from the stresses of its simplices:
//   row_m = sum_{(p,m)} S_e[:, pi_{m-1}] / h_{pi_{m-1}} - S_e[:, pi_m] / h_{pi_m}.
// T is the element arithmetic (double, or float for the mixed path); rows are returned in
// double.  Needs smem_bytes of dynamic shared memory and blocks of TX*TY*TZ threads.
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
template <int D, int NPN_, bool FULL, typename T>
struct StencilOp {
  static constexpr int NPN = NPN_;
  static constexpr int BLK = FULL ? NPN * NPN : NPN;
  Grid g;
  FO_NODE_OWNERSHIP(T)
  const T *W;

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
      const long long nb = slot_node<D>(g, idx, a, s);
      if (nb < 0) continue;
      T xv[NPN];   // x_a on slot 0, x_nb - x_a on the others
#pragma unroll
      for (int j = 0; j < NPN; ++j) xv[j] = s == 0 ? xa[j] : (T)x(nb * NPN + j) - xa[j];
      if (FULL) {
#pragma unroll
        for (int i = 0; i < NPN; ++i)
#pragma unroll
          for (int j = 0; j < NPN; ++j) acc[i] = fma(W[(s * BLK + i * NPN + j) * N + a], xv[j], acc[i]);
      } else {
#pragma unroll
        for (int c = 0; c < NPN; ++c) acc[c] = fma(W[(s * BLK + c) * N + a], xv[c], acc[c]);
      }
    }
#pragma unroll
    for (int c = 0; c < NPN; ++c) out[c] = acc[c];
  }

};

template <int D, typename T>
struct TiledElasticOp {
  static constexpr int NPN = D;
  static constexpr int TX = (D == 2) ? 16 : 8, TY = (D == 2) ? 8 : 4, TZ = (D == 2) ? 1 : 4;
  static constexpr int THREADS = TX * TY * TZ;
  static constexpr int HX = TX + 2, HY = TY + 2, HZ = (D == 2) ? 1 : TZ + 2;   // halo node box
  static constexpr int CX = TX + 1, CY = TY + 1, CZ = (D == 2) ? 1 : TZ + 1;   // cells touching the tile
  static constexpr int P = KP<D>::P;
  static constexpr int NS = (D == 2) ? 3 : 6;                                  // symmetric stress entries
  static constexpr size_t smem_bytes = sizeof(T) * ((size_t)HX * HY * HZ * D + (size_t)CX * CY * CZ * P * NS);
  Grid g;
  const T *coef;
  const uint8_t *dir;   // per DOF
  T lam, mu, vol;
  T ih[3];
  int ntile[3];
  long long ntiles;

  __device__ __forceinline__ static int sidx(int i, int j) {   // symmetric index
    if (i == j) return i;
    const int a = i < j ? i : j, b = i < j ? j : i;
    return (D == 2) ? 2 : (a == 0 ? (b == 1 ? 3 : 4) : 5);
  }

  template <class X, class F>
  __device__ void sweep(const X &x, F &&f) const {
    extern __shared__ __align__(16) unsigned char fo_dyn_smem[];
    T *U = reinterpret_cast<T *>(fo_dyn_smem);                 // [HZ][HY][HX][D]
    T *S = U + HX * HY * HZ * D;                                // [CZ][CY][CX][P][NS]
    const int tx = threadIdx.x % TX, ty = (threadIdx.x / TX) % TY, tz = threadIdx.x / (TX * TY);
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
      const int i0 = (int)(t % ntile[0]) * TX;
      const int j0 = (int)((t / ntile[0]) % ntile[1]) * TY;
      const int k0 = (D == 3) ? (int)(t / ((long long)ntile[0] * ntile[1])) * TZ : 0;
      __syncthreads();   // the previous tile's shared data is no longer read
      // stage 1: field on the halo box [i0-1, i0+TX] x [j0-1, j0+TY] (x [k0-1, k0+TZ])
      for (int s = threadIdx.x; s < HX * HY * HZ; s += blockDim.x) {
        const int hx = s % HX, hy = (s / HX) % HY, hz = s / (HX * HY);
        const int gi = i0 - 1 + hx, gj = j0 - 1 + hy, gk = (D == 3) ? k0 - 1 + hz : 0;
        const bool in = gi >= 0 && gi < (int)g.nn[0] && gj >= 0 && gj < (int)g.nn[1] &&
                        (D == 2 || (gk >= 0 && gk < (int)g.nn[2]));
        const long long a = gi + g.stride[1] * gj + (D == 3 ? g.stride[2] * gk : 0);
#pragma unroll
        for (int c = 0; c < D; ++c) U[s * D + c] = in ? (T)x(a * D + c) : T(0);
      }
      __syncthreads();
      // stage 2: scaled stress of the P simplices of every cell [i0-1, i0+TX-1] x ...
      for (int cs = threadIdx.x; cs < CX * CY * CZ; cs += blockDim.x) {
        const int cx = cs % CX, cy = (cs / CX) % CY, cz = cs / (CX * CY);
        const int gi = i0 - 1 + cx, gj = j0 - 1 + cy, gk = (D == 3) ? k0 - 1 + cz : 0;
        if (gi < 0 || gi >= g.n[0] || gj < 0 || gj >= g.n[1] || (D == 3 && (gk < 0 || gk >= g.n[2]))) continue;
        const long long e0 = (long long)P * (gi + g.cstride[1] * gj + (D == 3 ? g.cstride[2] * gk : 0));
        // field at the 2^D cell corners; corner bit k set = +1 along axis k
        T uc[1 << D][D];
#pragma unroll
        for (int b = 0; b < (1 << D); ++b) {
          const int h = (cx + (b & 1)) + HX * ((cy + ((b >> 1) & 1)) + HY * (D == 3 ? cz + ((b >> 2) & 1) : 0));
#pragma unroll
          for (int i = 0; i < D; ++i) uc[b][i] = U[h * D + i];
        }
#pragma unroll
        for (int p = 0; p < P; ++p) {
          // walk the Kuhn path of permutation p from the cell corner
          T du[D][D];
          int at = 0;
#pragma unroll
          for (int l = 0; l < D; ++l) {
            const int ax = kperm<D>(p, l);
            const int next = at | (1 << ax);
#pragma unroll
            for (int i = 0; i < D; ++i) du[i][ax] = (uc[next][i] - uc[at][i]) * ih[ax];
            at = next;
          }
          T tr = 0;
#pragma unroll
          for (int i = 0; i < D; ++i) tr += du[i][i];
          const T w = coef[e0 + p] * vol;
          T *Se = S + ((size_t)cs * P + p) * NS;
#pragma unroll
          for (int i = 0; i < D; ++i) Se[i] = w * (lam * tr + 2 * mu * du[i][i]);
#pragma unroll
          for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = i + 1; j < D; ++j) Se[sidx(i, j)] = w * mu * (du[i][j] + du[j][i]);
        }
      }
      __syncthreads();
      // stage 3: rows of the tile's nodes
      const int gi = i0 + tx, gj = j0 + ty, gk = k0 + tz;
      if (gi < (int)g.nn[0] && gj < (int)g.nn[1] && (D == 2 || gk < (int)g.nn[2])) {
        const long long a = gi + g.stride[1] * gj + (D == 3 ? g.stride[2] * gk : 0);
        double out[D];
        const int hself = (tx + 1) + HX * ((ty + 1) + HY * (D == 3 ? tz + 1 : 0));
        T acc[D];
#pragma unroll
        for (int i = 0; i < D; ++i) acc[i] = 0;
#pragma unroll
        for (int p = 0; p < P; ++p)
#pragma unroll
          for (int m = 0; m <= D; ++m) {
            int c[3] = {gi, gj, gk};
#pragma unroll
            for (int l = 0; l < D; ++l)
              if (l < m) c[kperm<D>(p, l)] -= 1;
            bool ok = true;
#pragma unroll
            for (int k = 0; k < D; ++k) ok = ok && c[k] >= 0 && c[k] < g.n[k];
            if (!ok) continue;
            const int cx = c[0] - (i0 - 1), cy = c[1] - (j0 - 1), cz = (D == 3) ? c[2] - (k0 - 1) : 0;
            const T *Se = S + ((size_t)((cx + CX * (cy + CY * cz)) * P + p)) * NS;
            if (m >= 1) {
              const int j = kperm<D>(p, m - 1);
#pragma unroll
              for (int i = 0; i < D; ++i) acc[i] += ih[j] * Se[sidx(i, j)];
            }
            if (m < D) {
              const int j = kperm<D>(p, m);
#pragma unroll
              for (int i = 0; i < D; ++i) acc[i] -= ih[j] * Se[sidx(i, j)];
            }
          }
#pragma unroll
        for (int i = 0; i < D; ++i) out[i] = dir[a * D + i] ? (double)U[hself * D + i] : (double)acc[i];
        f(a, out);
      }
    }
  }

  template <class F>
  __device__ void each(F &&f) const {
    const int tx = threadIdx.x % TX, ty = (threadIdx.x / TX) % TY, tz = threadIdx.x / (TX * TY);
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
      const int gi = (int)(t % ntile[0]) * TX + tx;
      const int gj = (int)((t / ntile[0]) % ntile[1]) * TY + ty;
      const int gk = (D == 3) ? (int)(t / ((long long)ntile[0] * ntile[1])) * TZ + tz : 0;
      if (gi < (int)g.nn[0] && gj < (int)g.nn[1] && (D == 2 || gk < (int)g.nn[2]))
        f(gi + g.stride[1] * gj + (D == 3 ? g.stride[2] * gk : 0));
    }
  }
};

// --------------------------------------------------------------- operator construction
template <int D, typename T>
inline ScalarStateOp<D, T> make_scalar_op(const fo_problem *p) {
  const Grid &g = p->mesh->g;
  ScalarStateOp<D, T> op;
  op.g = g;
  op.coef = std::is_same<T, float>::value ? (const T *)p->coef32 : (const T *)p->coef;
  op.dir = p->dir;
  for (int a = 0; a < 3; ++a) op.sk[a] = (T)(g.vol_e * g.inv_h[a] * g.inv_h[a]);
  const double w = p->desc.kind == FO_HELMHOLTZ ? p->desc.omega * p->desc.omega : 0.0;
  op.w2m = (T)(w * g.vol_e / ((D + 1) * (D + 2)));
  return op;
}

template <int D, typename T>
inline ElasticStateOp<D, T> make_elastic_op(const fo_problem *p) {
  const Grid &g = p->mesh->g;
  ElasticStateOp<D, T> op;
  op.g = g;
  op.coef = std::is_same<T, float>::value ? (const T *)p->coef32 : (const T *)p->coef;
  op.dir = p->dir;
  op.lam = (T)p->lame_lambda;
  op.mu = (T)p->lame_mu;
  op.vol = (T)g.vol_e;
  for (int a = 0; a < 3; ++a) op.ih[a] = (T)g.inv_h[a];
  return op;
}

template <int D, typename T>
inline VelocityOp<D, T> make_velocity_op(const fo_problem *p) {
  const Grid &g = p->mesh->g;
  VelocityOp<D, T> op;
  op.g = g;
  op.omega0 = p->omega0;
  op.vdir = p->vdir;
  for (int a = 0; a < 3; ++a) {
    op.sk[a] = (T)(g.vol_e * g.inv_h[a] * g.inv_h[a]);
    op.fref[a] = (T)(g.facet_area[a] / (D * (D + 1)));
  }
  op.mref = (T)(g.vol_e / ((D + 1) * (D + 2)));
  op.alpha = (T)p->desc.alpha_mass;
  op.gamma0 = (T)p->desc.omega0_weight;
  op.gammab = (T)p->desc.normal_penalty;
  return op;
}


template <int D, typename T>
inline TiledElasticOp<D, T> make_tiled_elastic_op(const fo_problem *p) {
  const Grid &g = p->mesh->g;
  using Op = TiledElasticOp<D, T>;
  Op op;
  op.g = g;
  op.coef = std::is_same<T, float>::value ? (const T *)p->coef32 : (const T *)p->coef;
  op.dir = p->dir;
  op.lam = (T)p->lame_lambda;
  op.mu = (T)p->lame_mu;
  op.vol = (T)g.vol_e;
  for (int a = 0; a < 3; ++a) op.ih[a] = (T)g.inv_h[a];
  op.ntile[0] = (int)((g.nn[0] + Op::TX - 1) / Op::TX);
  op.ntile[1] = (int)((g.nn[1] + Op::TY - 1) / Op::TY);
  op.ntile[2] = (D == 3) ? (int)((g.nn[2] + Op::TZ - 1) / Op::TZ) : 1;
  op.ntiles = (long long)op.ntile[0] * op.ntile[1] * op.ntile[2];
  return op;
}

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
