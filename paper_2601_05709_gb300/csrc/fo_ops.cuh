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

