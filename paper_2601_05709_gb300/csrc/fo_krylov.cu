// Persistent, cooperatively launched Jacobi-preconditioned conjugate gradients for the
// state and velocity systems, and the FP32-inner / FP64-refinement driver of the mixed path.
//
// The recurrence is the single-reduction form of PCG due to Chronopoulos and Gear:
//   p_i = u_i + b_i p_{i-1},  s_i = w_i + b_i s_{i-1}          (s_i = A p_i)
//   x_{i+1} = x_i + a_i p_i,  r_{i+1} = r_i - a_i s_i,  u_{i+1} = D^{-1} r_{i+1},  w_{i+1} = A u_{i+1}
//   g_{i+1} = (r_{i+1}, u_{i+1}),  d_{i+1} = (w_{i+1}, u_{i+1}),
//   b_{i+1} = g_{i+1} / g_i,  a_{i+1} = g_{i+1} / (d_{i+1} - b_{i+1} g_{i+1} / a_i).
// Its three dot products are reduced together, so an iteration needs one grid barrier:
// the apply w_{i+1} = A u_{i+1} gathers u_{i+1} at the stencil neighbours and forms it
// there from the previous iteration's r_i, w_i and s_{i-1},
//   u_{i+1}[nb] = D^{-1}[nb] (r_i[nb] - a_i (w_i[nb] + b_i s_{i-1}[nb])),
// which are final once the previous barrier has passed.  r, w and s are double-buffered
// so that a phase never overwrites a value another block may still gather.
// All dot products are accumulated in FP64 with a fixed reduction order (block partials,
// then every block sums all partials in the same order): every block takes the same
// branch, and the result does not depend on timing.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <map>
#include <mutex>

#include "fo_internal.cuh"
#include "fo_ops.cuh"
#include "fo_umesh.cuh"

// ----------------------------------------------------------------------------- scratch
fo_status fo_scratch(fo_problem *p, size_t bytes, void **out) {
  if (bytes > p->scratch.bytes) {
    fo_free(p->ctx, p->scratch.buf, p->scratch.bytes);
    p->scratch.buf = nullptr;
    p->scratch.bytes = 0;
    FO_TRY(fo_alloc(p->ctx, &p->scratch.buf, bytes));
    p->scratch.bytes = bytes;
  }
  if (out) *out = p->scratch.buf;
  return FO_OK;
}

// Grid of a persistent kernel: enough blocks to cover `work` items (one per thread), at
// most what fits co-resident on the device (divided by the context's grid share).
fo_status fo_cooperative_grid(fo_problem *p, const void *kernel, int block, size_t smem, long long work,
                              int requested, int *grid) {
  int per_sm = 0;
  FO_CU(p->ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem));
  if (per_sm < 1) return fo_fail(p->ctx, FO_ECUDA, "persistent kernel does not fit on an SM");
  long long cap = (long long)per_sm * p->ctx->num_sms;
  if (p->ctx->grid_share > 1) cap = std::max(1LL, cap / p->ctx->grid_share);
  long long want = requested > 0 ? requested : (work + block - 1) / block;
  if (want > cap) want = cap;
  if (want > 4096) want = 4096;
  if (want < 1) want = 1;
  *grid = (int)want;
  return FO_OK;
}

std::mutex &fo_launch_mutex() {
  static std::mutex m;
  return m;
}

fo_status fo_smem_limit(fo_ctx *ctx, const void *kernel, size_t bytes) {
  static std::map<std::pair<int, const void *>, size_t> limit;
  size_t &cur = limit[{ctx->device, kernel}];
  if (bytes > cur) {
    FO_CU(ctx, cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    cur = bytes;
  }
  return FO_OK;
}

// Threads per block for a persistent kernel over n nodes: 256, or fewer (>= 64) so that a
// small problem still spreads over every SM (the FP64 work is ALU-bound per SM).
int fo_persistent_block(const fo_problem *p, long long n) {
  const long long sms = p->ctx->num_sms > 0 ? p->ctx->num_sms : 1;
  long long per = (n + sms - 1) / sms;
  int b = 64;
  while (b < 256 && b < per) b *= 2;
  return b;
}

// ------------------------------------------------------------------------------ kernel
template <int NC, typename T>
struct PcgArgs {
  T *x, *u, *p;          // single buffers (own nodes only)
  T *r[2], *s[2], *w[2]; // double buffers (gathered at neighbours)
  const double *b;       // right-hand side (FP64), scaled by bscale
  const T *bT;           // right-hand side in T when non-null (inner solves)
  const uint8_t *bmask;  // per node: nonzero rows get a zero right-hand side (H^1_0 rows)
  double bscale;
  const T *dinv;
  double *partials;      // [2][G][3 NC]: two buffers used alternately
  double *out;           // [4 NC]: rr, bb, b.x
  int *status;           // DS_* words
  GridBar bar;
  double rtol2;
  int maxit;
  int warm;
};

// u_{i+1} at any DOF, formed from the previous iteration's r, w, s (see the file comment)
template <typename T, int NC>
struct NextU {
  const T *r, *w, *s, *dinv;
  T a[NC], b[NC];
  __device__ __forceinline__ T operator()(long long k) const {
    const int c = (NC == 1) ? 0 : (int)(k % NC);
    return dinv[k] * (r[k] - a[c] * (w[k] + b[c] * s[k]));
  }
};

template <int D, class Op, typename T, int NC>
__global__ void __launch_bounds__(FO_BLOCK) k_pcg(Op op, PcgArgs<NC, T> S) {
  constexpr int NPN = Op::NPN;
  constexpr int NR = 3 * NC;
  __shared__ double sred[32 * NR];
  __shared__ double stot[NR];
  const Grid &g = op.g;
  const long long N = g.num_nodes;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long gstride = (long long)gridDim.x * blockDim.x;
  int rk = 0;

  // ---- start 1: r_0 = b - A x_0, u_0 = D^{-1} r_0, s_{-1} = 0; ||b||^2
  double v[NR];
#pragma unroll
  for (int j = 0; j < NR; ++j) v[j] = 0.0;
  auto start1 = [&](long long a, const auto *ax) {
#pragma unroll
    for (int c = 0; c < NPN; ++c) {
      const long long k = a * NPN + c;
      const int sy = (NC == 1) ? 0 : c;
      const double bk = (S.bmask && S.bmask[a]) ? 0.0 : (S.bT ? (double)S.bT[k] : S.bscale * S.b[k]);
      double axc = 0.0;
      if (ax) axc = (double)ax[c];
      else S.x[k] = T(0);
      const T rk0 = (T)(bk - axc);
      S.r[0][k] = rk0;
      S.u[k] = S.dinv[k] * rk0;
      S.s[1][k] = T(0);
      S.p[k] = T(0);
      v[sy * 3 + 0] += (double)rk0 * (double)rk0;
      v[sy * 3 + 1] += bk * bk;
    }
  };
  if (S.warm) op.sweep(VecX<T>{S.x}, start1);
  else op.each([&](long long a) { start1(a, (const double *)nullptr); });
  if (!reduce_grid<NR>(v, sred, stot, S.partials, rk, S.bar)) return;
  double rr[NC], bb[NC], gam[NC], alpha[NC], beta[NC];
#pragma unroll
  for (int s = 0; s < NC; ++s) {
    rr[s] = stot[s * 3 + 0];
    bb[s] = stot[s * 3 + 1];
  }
  // ---- start 2: w_0 = A u_0, g_0 = (r_0, u_0), d_0 = (w_0, u_0)
  __syncthreads();
#pragma unroll
  for (int j = 0; j < NR; ++j) v[j] = 0.0;
  op.sweep(VecX<T>{S.u}, [&](long long a, const auto *wa) {
#pragma unroll
    for (int c = 0; c < NPN; ++c) {
      const long long k = a * NPN + c;
      const int sy = (NC == 1) ? 0 : c;
      const T wk = (T)wa[c];
      S.w[0][k] = wk;
      const double uk = (double)S.u[k];
      v[sy * 3 + 0] += (double)S.r[0][k] * uk;
      v[sy * 3 + 1] += (double)wk * uk;
    }
  });
  if (!reduce_grid<NR>(v, sred, stot, S.partials, rk, S.bar)) return;
#pragma unroll
  for (int s = 0; s < NC; ++s) {
    gam[s] = stot[s * 3 + 0];
    const double del = stot[s * 3 + 1];
    alpha[s] = (del != 0.0) ? gam[s] / del : 0.0;
    beta[s] = 0.0;
  }

  int it = 0, err = DEV_OK;
  for (;;) {
    bool any = false;
#pragma unroll
    for (int s = 0; s < NC; ++s) {
      if (!(rr[s] == rr[s]) || !(alpha[s] == alpha[s])) err = DEV_NAN;
      if (rr[s] > S.rtol2 * bb[s]) any = true;
    }
    if (err != DEV_OK || !any) break;
    if (it >= S.maxit) { err = DEV_NOCONV; break; }
    // converged systems keep x: their step length is zero from here on
#pragma unroll
    for (int s = 0; s < NC; ++s)
      if (!(rr[s] > S.rtol2 * bb[s])) alpha[s] = 0.0, beta[s] = 0.0;
    const int cur = it & 1, nxt = cur ^ 1;
    T *rc = S.r[cur], *rn = S.r[nxt], *wc = S.w[cur], *wn = S.w[nxt], *sp = S.s[nxt], *sc = S.s[cur];
    NextU<T, NC> nu;
    nu.r = rc;
    nu.w = wc;
    nu.s = sp;
    nu.dinv = S.dinv;
#pragma unroll
    for (int s = 0; s < NC; ++s) {
      nu.a[s] = (T)alpha[s];
      nu.b[s] = (T)beta[s];
    }
    __syncthreads();   // stot is rewritten by the reduction below
#pragma unroll
    for (int j = 0; j < NR; ++j) v[j] = 0.0;
    op.sweep(nu, [&](long long a, const auto *wa) {   // wa = w_{i+1} = A u_{i+1}
#pragma unroll
      for (int c = 0; c < NPN; ++c) {
        const long long k = a * NPN + c;
        const int sy = (NC == 1) ? 0 : c;
        const T al = nu.a[sy], be = nu.b[sy];
        const T pk = S.u[k] + be * S.p[k];
        const T sk = wc[k] + be * sp[k];
        S.p[k] = pk;
        sc[k] = sk;
        S.x[k] += al * pk;
        const T rk1 = rc[k] - al * sk;
        const T uk1 = S.dinv[k] * rk1;
        const T wk1 = (T)wa[c];
        rn[k] = rk1;
        S.u[k] = uk1;
        wn[k] = wk1;
        v[sy * 3 + 0] += (double)rk1 * (double)uk1;
        v[sy * 3 + 1] += (double)wk1 * (double)uk1;
        v[sy * 3 + 2] += (double)rk1 * (double)rk1;
      }
    });
    if (!reduce_grid<NR>(v, sred, stot, S.partials, rk, S.bar)) return;
#pragma unroll
    for (int s = 0; s < NC; ++s) {
      const double gn = stot[s * 3 + 0], del = stot[s * 3 + 1];
      rr[s] = stot[s * 3 + 2];
      if (alpha[s] != 0.0) {
        const double bn = (gam[s] != 0.0) ? gn / gam[s] : 0.0;
        const double den = del - bn * gn / alpha[s];
        beta[s] = bn;
        alpha[s] = (den != 0.0) ? gn / den : 0.0;
        gam[s] = gn;
      }
    }
    ++it;
  }
  // ---- b . x per system (B(theta, theta) = -b . theta for the velocity)
  __syncthreads();
  double bx[NR];
#pragma unroll
  for (int j = 0; j < NR; ++j) bx[j] = 0.0;
  op.each([&](long long a) {
#pragma unroll
    for (int c = 0; c < NPN; ++c) {
      const long long k = a * NPN + c;
      const int sy = (NC == 1) ? 0 : c;
      const double bk = (S.bmask && S.bmask[a]) ? 0.0 : (S.bT ? (double)S.bT[k] : S.bscale * S.b[k]);
      bx[sy * 3] += bk * (double)S.x[k];
    }
  });
  if (!reduce_grid<NR>(bx, sred, stot, S.partials, rk, S.bar)) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    for (int s = 0; s < NC; ++s) {
      S.out[s * 4 + 0] = rr[s];
      S.out[s * 4 + 1] = bb[s];
      S.out[s * 4 + 2] = stot[s * 3];
    }
    S.status[DS_ITERS] = it;
    if (err != DEV_OK) atomicCAS(S.status + DS_ERR, DEV_OK, err);
  }
}

// ------------------------------------------------------------------------- host driver
template <class K, class... Args>
static fo_status coop_launch(fo_problem *p, K kernel, int grid, int block, size_t smem, Args... args) {
  void *argv[] = {(void *)&args...};
  FO_CU(p->ctx, cudaMemsetAsync(p->bar, 0, 64, p->ctx->stream));
  FO_CU(p->ctx, cudaMemsetAsync(p->dev_status, 0, sizeof(int) * DS_COUNT, p->ctx->stream));
  FO_CU(p->ctx, cudaLaunchCooperativeKernel((const void *)kernel, grid, block, argv, smem, p->ctx->stream));
  fo_note_launch(1);
  return FO_OK;
}

// Block size, work items and dynamic shared memory of a persistent sweep with operator Op:
// node-centric operators take one node per thread; tiled operators one tile per block.
template <class Op>
static void sweep_shape(const fo_problem *p, const Op &op, long long nodes, int *block, long long *work, size_t *smem) {
  if constexpr (Op::smem_bytes > 0) {
    *block = Op::THREADS;
    *work = op.ntiles * Op::THREADS;
    *smem = Op::smem_bytes;
  } else {
    *block = fo_persistent_block(p, nodes);
    *work = nodes;
    *smem = 0;
  }
}

struct SolveOut {
  int status[DS_COUNT];
  double out[16];
};

static double *out_area(fo_problem *p) { return p->red + FO_RED_DOUBLES - 64; }

static fo_status read_out(fo_problem *p, double *out_dev, SolveOut *o, int nout) {
  fo_ctx *ctx = p->ctx;
  FO_CU(ctx, cudaMemcpyAsync(ctx->h_scalars, out_dev, sizeof(double) * nout, cudaMemcpyDeviceToHost, ctx->stream));
  FO_CU(ctx, cudaMemcpyAsync(ctx->h_scalars + 32, p->dev_status, sizeof(int) * DS_COUNT, cudaMemcpyDeviceToHost,
                             ctx->stream));
  FO_CU(ctx, cudaStreamSynchronize(ctx->stream));
  memcpy(o->out, ctx->h_scalars, sizeof(double) * nout);
  memcpy(o->status, ctx->h_scalars + 32, sizeof(int) * DS_COUNT);
  return FO_OK;
}

// 9 vectors of n entries of T: x is external; u, p, r[2], s[2], w[2] come from `buf`
template <int NC, typename T>
static void bind_vectors(PcgArgs<NC, T> &a, T *x, T *buf, long long n) {
  a.x = x;
  a.u = buf;
  a.p = buf + n;
  a.r[0] = buf + 2 * n;
  a.r[1] = buf + 3 * n;
  a.s[0] = buf + 4 * n;
  a.s[1] = buf + 5 * n;
  a.w[0] = buf + 6 * n;
  a.w[1] = buf + 7 * n;
}

template <int D, class Op, typename T, int NC>
static fo_status run_pcg(fo_problem *p, const Op &op, PcgArgs<NC, T> a, long long nodes, int requested, SolveOut *o) {
  auto kern = k_pcg<D, Op, T, NC>;
  int block, grid;
  long long work;
  size_t smem;
  sweep_shape(p, op, nodes, &block, &work, &smem);
  std::unique_lock<std::mutex> lk(fo_launch_mutex());
  if (smem > 48 * 1024) FO_TRY(fo_smem_limit(p->ctx, (const void *)kern, smem));
  FO_TRY(fo_cooperative_grid(p, (const void *)kern, block, smem, work, requested, &grid));
  a.partials = p->red;
  a.out = out_area(p);
  a.status = p->dev_status;
  a.bar = GridBar{p->bar, p->dev_status + DS_ERR, 2000000000ull};
  fo_ctx *ctx = p->ctx;
  const bool tm = ctx->timing != 0 && ctx->ev_solve[0] != nullptr;
  if (tm) FO_CU(ctx, cudaEventRecord(ctx->ev_solve[0], ctx->stream));
  FO_TRY(coop_launch(p, kern, grid, block, smem, op, a));
  FO_CU(p->ctx, cudaGetLastError());
  lk.unlock();
  if (tm) FO_CU(ctx, cudaEventRecord(ctx->ev_solve[1], ctx->stream));
  FO_TRY(read_out(p, out_area(p), o, 4 * NC));
  if (tm) {   // device time of the persistent PCG launch alone, summed over restarts
    float ms = 0.f;
    FO_CU(ctx, cudaEventElapsedTime(&ms, ctx->ev_solve[0], ctx->ev_solve[1]));
    ctx->last_solve_ms += ms;
  }
  if (o->status[DS_ERR] == DEV_TIMEOUT) return fo_fail(p->ctx, FO_ETIMEOUT, "grid barrier timed out in PCG");
  if (o->status[DS_ERR] == DEV_NAN) return fo_fail(p->ctx, FO_ENAN, "NaN in the PCG recurrence");
  return FO_OK;
}

__global__ void k_residual_norms(const double *b, const double *ax, double *r, long long n, double *partials) {
  __shared__ double sm[64];
  double v[2] = {0, 0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double ri = b[i] - ax[i];
    r[i] = ri;
    v[0] += ri * ri;
    v[1] += b[i] * b[i];
  }
  block_sum<2>(v, sm);
  if (threadIdx.x == 0) {
    partials[blockIdx.x * 2] = v[0];
    partials[blockIdx.x * 2 + 1] = v[1];
  }
}
__global__ void k_finish_sum2(const double *partials, int nblocks, double *out) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (w >= 2) return;
  double t = 0;
  for (int b = lane; b < nblocks; b += 32) t += partials[(size_t)b * 2 + w];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  if (lane == 0) out[w] = t;
}
__global__ void k_axpy(double *x, const double *d, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] += d[i];
}

// op64: the FP64 operator; op_mixed: the operator of the inner solve of the mixed path
// (FP32 element arithmetic, FP64 vectors)
template <int D, class Op64, class OpMixed>
static fo_status state_solve_impl(fo_problem *p, const Op64 &op64, const OpMixed &op_mixed, const double *b,
                                  double *x, const fo_solve_opts *o, fo_solve_stats *st) {
  const Grid &g = p->mesh->g;
  const long long n = p->ndof;
  fo_solve_stats s;
  memset(&s, 0, sizeof s);
  if (o->precision == FO_FP64) {
    double *buf;
    FO_TRY(fo_scratch(p, sizeof(double) * 8 * n, (void **)&buf));
    PcgArgs<1, double> a{};
    bind_vectors(a, x, buf, n);
    a.b = b;
    a.bscale = 1.0;
    a.dinv = p->dinv_state;
    a.rtol2 = o->rtol * o->rtol;
    a.maxit = o->maxit;
    a.warm = o->warm_start;
    SolveOut out;
    FO_TRY(run_pcg<D>(p, op64, a, g.num_nodes, o->grid_blocks, &out));
    s.iterations = out.status[DS_ITERS];
    s.operator_applies = s.iterations + 1 + (o->warm_start ? 1 : 0);
    s.outer_iterations = 1;
    s.rel_residual = out.out[1] > 0 ? std::sqrt(out.out[0] / out.out[1]) : 0.0;
    // The single-reduction recurrence updates its residual recursively; over thousands of
    // iterations that residual drifts from b - A x.  Check the true residual and, while it is
    // above rtol, restart from x (the warm start forms b - A x afresh): at most two restarts.
    if (out.status[DS_ERR] != DEV_NOCONV) {
      fo_ctx *ctx = p->ctx;
      double *ax64 = buf, *r64 = buf + n;   // the solver's scratch, free after the launch
      const int blocks = fo_blocks_for(n, FO_BLOCK, 1024);
      for (int restart = 0; restart < 3; ++restart) {
        FO_TRY(fo_launch_state_apply(p, x, ax64, true));
        k_residual_norms<<<blocks, FO_BLOCK, 0, ctx->stream>>>(b, ax64, r64, n, p->red);
        k_finish_sum2<<<1, 64, 0, ctx->stream>>>(p->red, blocks, out_area(p) + 8);
        fo_note_launch(2);
        FO_CU(ctx, cudaGetLastError());
        FO_CU(ctx, cudaMemcpyAsync(ctx->h_scalars, out_area(p) + 8, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                                   ctx->stream));
        FO_CU(ctx, cudaStreamSynchronize(ctx->stream));
        const double rn2 = ctx->h_scalars[0], bn2 = ctx->h_scalars[1];
        s.operator_applies += 1;
        s.rel_residual = bn2 > 0 ? std::sqrt(rn2 / bn2) : 0.0;
        if (!(rn2 > o->rtol * o->rtol * bn2) || restart == 2 || s.iterations >= o->maxit) break;
        a.warm = 1;
        a.maxit = o->maxit - s.iterations;
        bind_vectors(a, x, buf, n);
        FO_TRY(run_pcg<D>(p, op64, a, g.num_nodes, o->grid_blocks, &out));
        s.iterations += out.status[DS_ITERS];
        s.operator_applies += out.status[DS_ITERS] + 2;
        s.outer_iterations += 1;
        if (out.status[DS_ERR] == DEV_NOCONV) break;
      }
    }
    if (st) *st = s;
    if (out.status[DS_ERR] == DEV_NOCONV) return fo_fail(p->ctx, FO_ENOCONV, "PCG reached maxit=%d", o->maxit);
    return FO_OK;
  }
  // ---- mixed: FP64 iterative refinement around an inner PCG whose operator applies run in
  // FP32 (FP32 element data and accumulation); the inner recurrence, its dot products and
  // the refinement residual stay in FP64.
  double *buf;
  FO_TRY(fo_scratch(p, sizeof(double) * 11 * n, (void **)&buf));
  double *r64 = buf, *ax64 = buf + n, *d64 = buf + 2 * n, *vec64 = buf + 3 * n;
  fo_ctx *ctx = p->ctx;
  const int blocks = fo_blocks_for(n, FO_BLOCK, 1024);
  if (!o->warm_start) FO_CU(ctx, cudaMemsetAsync(x, 0, sizeof(double) * n, ctx->stream));
  double bnorm2 = -1, prev_rn2 = INFINITY, prev2_rn2 = INFINITY;
  const int max_outer = 60;
  const char *tr = getenv("FORMOPT_TRACE");   // trace the refinement on stderr when set
  const bool trace = tr && tr[0] && tr[0] != '0';
  for (int outer = 0;; ++outer) {
    // FP64 residual r = b - A x (the operator masks Dirichlet columns; rows are identity)
    FO_TRY(fo_launch_state_apply(p, x, ax64, true));
    k_residual_norms<<<blocks, FO_BLOCK, 0, ctx->stream>>>(b, ax64, r64, n, p->red);
    k_finish_sum2<<<1, 64, 0, ctx->stream>>>(p->red, blocks, out_area(p) + 8);
    fo_note_launch(2);
    FO_CU(ctx, cudaGetLastError());
    FO_CU(ctx, cudaMemcpyAsync(ctx->h_scalars, out_area(p) + 8, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    FO_CU(ctx, cudaStreamSynchronize(ctx->stream));
    const double rn2 = ctx->h_scalars[0];
    if (bnorm2 < 0) bnorm2 = ctx->h_scalars[1];
    s.operator_applies += 1;
    s.rel_residual = bnorm2 > 0 ? std::sqrt(rn2 / bnorm2) : 0.0;
    if (trace)
      fprintf(stderr, "[formopt] refinement step %d: ||b - Ax||/||b|| = %.3e after %d inner iterations\n", outer,
              s.rel_residual, s.iterations);
    if (!std::isfinite(rn2)) return fo_fail(ctx, FO_ENAN, "NaN in the refinement residual");
    if (rn2 <= o->rtol * o->rtol * bnorm2 || bnorm2 == 0) break;
    // The FP64 residual cannot fall below its own rounding floor (about eps * ||A|| ||x||,
    // i.e. kappa * eps relative to ||b|| on ill-conditioned systems).  Two consecutive steps
    // that fail to halve it mean the floor is reached: x is as accurate as FP64 allows.
    if (outer >= 2 && rn2 > 0.25 * prev_rn2 && prev_rn2 > 0.25 * prev2_rn2) break;
    prev2_rn2 = prev_rn2;
    prev_rn2 = rn2;
    if (outer >= max_outer || s.iterations >= o->maxit) {
      if (st) *st = s;
      return fo_fail(ctx, FO_ENOCONV, "iterative refinement stalled at %.3e", s.rel_residual);
    }
    PcgArgs<1, double> a{};
    bind_vectors(a, d64, vec64, n);
    a.b = r64;
    a.bscale = 1.0;
    a.dinv = p->dinv_state;
    a.rtol2 = o->inner_rtol * o->inner_rtol;
    a.maxit = o->inner_maxit;
    a.warm = 0;
    SolveOut out;
    FO_TRY(run_pcg<D>(p, op_mixed, a, g.num_nodes, o->grid_blocks, &out));
    s.iterations += out.status[DS_ITERS];
    s.operator_applies += out.status[DS_ITERS] + 1;
    s.outer_iterations = outer + 1;
    k_axpy<<<blocks, FO_BLOCK, 0, ctx->stream>>>(x, d64, n);
    fo_note_launch(1);
    FO_CU(ctx, cudaGetLastError());
  }
  if (st) *st = s;
  return FO_OK;
}

fo_status fo_state_pcg(fo_problem *p, const double *b, double *x, const fo_solve_opts *o, fo_solve_stats *st) {
  const Grid &g = p->mesh->g;
  if (p->mesh->um) return fo_umesh_state_pcg(p, b, x, o, st);   // general mesh: Jacobi-PCG
  if (o->precond == FO_PC_MG && !p->batch && fo_mg_applicable(g, p->ncomp)) return fo_state_pcg_mg(p, b, x, o, st);
  // stored-stencil operators: FP64 rows for the FP64 solve and the refinement residual, FP32
  // rows for the inner solve of the mixed path
  if (p->desc.kind == FO_ELASTIC) {
    if (g.dim == 2)
      return state_solve_impl<2>(p, make_elastic_stencil<2, double>(p), make_elastic_stencil<2, float>(p), b, x, o, st);
    return state_solve_impl<3>(p, make_elastic_stencil<3, double>(p), make_elastic_stencil<3, float>(p), b, x, o, st);
  }
  if (g.dim == 2)
    return state_solve_impl<2>(p, make_scalar_stencil<2, double>(p), make_scalar_stencil<2, float>(p), b, x, o, st);
  return state_solve_impl<3>(p, make_scalar_stencil<3, double>(p), make_scalar_stencil<3, float>(p), b, x, o, st);
}

// General meshes: the assembled node-block operators (FP64 rows; FP32 rows for the inner
// solves of the mixed path) under the same Jacobi-PCG and refinement driver.
fo_status fo_umesh_state_pcg(fo_problem *p, const double *b, double *x, const fo_solve_opts *o, fo_solve_stats *st) {
  const fo_mesh *m = p->mesh;
  if (p->ncomp == 1)
    return state_solve_impl<2>(p, make_csr_op<1>(m, (const double *)p->Wst), make_csr_op<1>(m, (const float *)p->Wst32),
                               b, x, o, st);
  if (m->um->dim == 2)
    return state_solve_impl<2>(p, make_csr_op<2>(m, (const double *)p->Wst), make_csr_op<2>(m, (const float *)p->Wst32),
                               b, x, o, st);
  return state_solve_impl<3>(p, make_csr_op<3>(m, (const double *)p->Wst), make_csr_op<3>(m, (const float *)p->Wst32),
                             b, x, o, st);
}

// General meshes: B theta = -b as one coupled system (the normal penalty n n^T of a facet
// that is not axis-aligned couples the components); B(theta, theta) = -b . theta.
template <int D>
static fo_status umesh_velocity_impl(fo_problem *p, const fo_solve_opts *o, double *Btt, fo_solve_stats *st) {
  const long long nn = p->mesh->um->nn, n = (long long)D * nn;
  double *buf;
  FO_TRY(fo_scratch(p, sizeof(double) * 8 * n, (void **)&buf));
  PcgArgs<1, double> a{};
  bind_vectors(a, p->theta, buf, n);
  a.b = p->rhs;
  a.bscale = -1.0;
  a.bmask = p->desc.velocity_dirichlet ? p->vdir : nullptr;
  a.dinv = p->dinv_vel;
  a.rtol2 = o->rtol * o->rtol;
  a.maxit = o->maxit;
  a.warm = o->warm_start;
  SolveOut out;
  FO_TRY(run_pcg<D>(p, make_csr_op<D>(p->mesh, (const double *)p->Wvel), a, nn, o->grid_blocks, &out));
  if (Btt) *Btt = out.out[2];
  if (st) {
    st->iterations = out.status[DS_ITERS];
    st->operator_applies = out.status[DS_ITERS] + 1 + (o->warm_start ? 1 : 0);
    st->outer_iterations = 1;
    st->rel_residual = out.out[1] > 0 ? std::sqrt(out.out[0] / out.out[1]) : 0.0;
  }
  if (out.status[DS_ERR] == DEV_NOCONV) return fo_fail(p->ctx, FO_ENOCONV, "velocity PCG reached maxit");
  return FO_OK;
}

fo_status fo_umesh_velocity_pcg(fo_problem *p, const fo_solve_opts *o, double *Btt, fo_solve_stats *st) {
  return p->mesh->um->dim == 2 ? umesh_velocity_impl<2>(p, o, Btt, st) : umesh_velocity_impl<3>(p, o, Btt, st);
}

template <int D>
static fo_status velocity_impl(fo_problem *p, const fo_solve_opts *o, double *Btt, fo_solve_stats *st) {
  const Grid &g = p->mesh->g;
  const long long n = (long long)D * g.num_nodes;
  double *buf;
  FO_TRY(fo_scratch(p, sizeof(double) * 8 * n, (void **)&buf));
  PcgArgs<D, double> a{};
  bind_vectors(a, p->theta, buf, n);
  a.b = p->rhs;
  a.bscale = -1.0;                // B theta = -b
  a.bmask = p->desc.velocity_dirichlet ? p->vdir : nullptr;
  a.dinv = p->dinv_vel;
  a.rtol2 = o->rtol * o->rtol;
  a.maxit = o->maxit;
  a.warm = o->warm_start;
  SolveOut out;
  FO_TRY(run_pcg<D>(p, make_velocity_stencil<D>(p), a, g.num_nodes, o->grid_blocks, &out));
  double rr = 0, bb = 0, bx = 0;
  for (int s = 0; s < D; ++s) {
    rr += out.out[s * 4];
    bb += out.out[s * 4 + 1];
    bx += out.out[s * 4 + 2];   // (-b) . theta summed over components
  }
  if (Btt) *Btt = bx;           // B(theta, theta) = -b . theta
  if (st) {
    st->iterations = out.status[DS_ITERS];
    st->operator_applies = out.status[DS_ITERS] + 1 + (o->warm_start ? 1 : 0);
    st->outer_iterations = 1;
    st->rel_residual = bb > 0 ? std::sqrt(rr / bb) : 0.0;
  }
  if (out.status[DS_ERR] == DEV_NOCONV) return fo_fail(p->ctx, FO_ENOCONV, "velocity PCG reached maxit");
  return FO_OK;
}

fo_status fo_velocity_pcg(fo_problem *p, const fo_solve_opts *o, double *Btt, fo_solve_stats *st) {
  if (p->mesh->um) return fo_umesh_velocity_pcg(p, o, Btt, st);
  if (o->precond == FO_PC_MG && fo_mg_applicable(p->mesh->g, p->mesh->g.dim)) return fo_velocity_pcg_mg(p, o, Btt, st);
  if (p->mesh->g.dim == 2) return velocity_impl<2>(p, o, Btt, st);
  return velocity_impl<3>(p, o, Btt, st);
}

// ============================================================ state solve without allocation
// Some callers cannot let a library allocate device memory while they run: cudaMalloc and
// cudaFree may synchronise the whole device (a stall in a latency-bound loop), and another
// framework's caching allocator or a fixed memory budget may already own the device memory.  fo_state_solve_noalloc gives them a state solve whose
// working memory -- the Krylov vectors, the reduction partials, the grid-barrier counter and
// the status words of the persistent PCG -- is this fixed array, which every GPU that loads
// the library holds until the process exits.  The caller passes the right-hand side and the
// solution; nothing is allocated or freed by the call.
//
// Layout (doubles): [0, 8) barrier counter, [8, 16) status words, [16, 48) solver outputs,
// [64, 64 + 2*4096*3) reduction partials, from FO_NOALLOC_HEADER on: 8 vectors of N_dof.
#define FO_NOALLOC_HEADER 32768
#define FO_NOALLOC_DOUBLES (FO_NOALLOC_SCRATCH_BYTES / 8)
static __device__ __align__(256) double g_noalloc_scratch[FO_NOALLOC_DOUBLES];

static fo_status noalloc_scratch_address(fo_ctx *ctx, double **out) {
  // The array's device address is looked up once per device, with that device current.
  // Host code cannot use the symbol itself: on the host it names a stand-in, not GPU memory.
  // std::call_once publishes the address to every thread that calls later (two threads making
  // their first call at once do not race), and the caller's current device is restored.
  static std::once_flag once[64];
  static double *addr[64] = {};
  static cudaError_t err[64] = {};
  const int dev = ctx->device;
  if (dev < 0 || dev >= 64) return fo_fail(ctx, FO_EINVAL, "device index out of range");
  std::call_once(once[dev], [dev]() {
    int prev = -1;
    cudaError_t e = cudaGetDevice(&prev);
    if (e == cudaSuccess && prev != dev) e = cudaSetDevice(dev);
    void *p = nullptr;
    if (e == cudaSuccess) e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (prev >= 0 && prev != dev) {
      const cudaError_t r = cudaSetDevice(prev);
      if (e == cudaSuccess) e = r;
    }
    err[dev] = e;
    addr[dev] = e == cudaSuccess ? (double *)p : nullptr;
  });
  if (err[dev] != cudaSuccess) return fo_cuda_check(ctx, err[dev], "cudaGetSymbolAddress(no-alloc scratch)");
  *out = addr[dev];
  return FO_OK;
}

template <int D, class Op>
static fo_status noalloc_pcg(fo_problem *p, const Op &op, const double *b, double *x, const fo_solve_opts *o,
                             fo_solve_stats *st) {
  fo_ctx *ctx = p->ctx;
  const long long n = p->ndof;
  double *base;
  FO_TRY(noalloc_scratch_address(ctx, &base));
  unsigned *bar = (unsigned *)base;
  int *status = (int *)(base + 8);
  double *out = base + 16;
  auto kern = k_pcg<D, Op, double, 1>;
  const int block = fo_persistent_block(p, p->mesh->g.num_nodes);
  int grid;
  FO_TRY(fo_cooperative_grid(p, (const void *)kern, block, 0, p->mesh->g.num_nodes, o->grid_blocks, &grid));
  const int *hs = (const int *)(ctx->h_scalars + 32);
  // one persistent launch (warm: from x, forming b - A x afresh); its iterations and status
  auto launch = [&](int warm, int maxit) -> fo_status {
    // the counter must start at zero and the status words are read back: clear them (the
    // array keeps whatever the previous launch or call left there)
    FO_CU(ctx, cudaMemsetAsync(base, 0, 64 * sizeof(double), ctx->stream));
    PcgArgs<1, double> a{};
    bind_vectors(a, x, base + FO_NOALLOC_HEADER, n);
    a.b = b;
    a.bscale = 1.0;
    a.dinv = p->dinv_state;
    a.rtol2 = o->rtol * o->rtol;
    a.maxit = maxit;
    a.warm = warm;
    a.partials = base + 64;
    a.out = out;
    a.status = status;
    a.bar = GridBar{bar, status + DS_ERR, 2000000000ull};
    void *argv[] = {(void *)&op, (void *)&a};
    FO_CU(ctx, cudaLaunchCooperativeKernel((const void *)kern, grid, block, argv, 0, ctx->stream));
    fo_note_launch(1);
    FO_CU(ctx, cudaMemcpyAsync(ctx->h_scalars, out, 4 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    FO_CU(ctx, cudaMemcpyAsync(ctx->h_scalars + 32, status, sizeof(int) * DS_COUNT, cudaMemcpyDeviceToHost,
                               ctx->stream));
    FO_CU(ctx, cudaStreamSynchronize(ctx->stream));
    return FO_OK;
  };
  FO_TRY(launch(o->warm_start, o->maxit));
  int iters = hs[DS_ITERS], launches = 1;
  // The single-reduction recurrence updates its residual recursively and may drift from
  // b - A x over many iterations.  As in fo_state_solve, restart from x at most twice: a warm
  // launch starts from the true residual and stops at once when that meets rtol.
  for (int restart = 0; restart < 2 && hs[DS_ERR] == DEV_OK && hs[DS_ITERS] > 0 && iters < o->maxit; ++restart) {
    FO_TRY(launch(1, o->maxit - iters));
    iters += hs[DS_ITERS];
    ++launches;
  }
  if (st) {
    memset(st, 0, sizeof *st);
    st->iterations = iters;
    st->operator_applies = iters + 1 + (o->warm_start ? 1 : 0) + 2 * (launches - 1);
    st->outer_iterations = launches;
    st->rel_residual = ctx->h_scalars[1] > 0 ? std::sqrt(ctx->h_scalars[0] / ctx->h_scalars[1]) : 0.0;
  }
  if (hs[DS_ERR] == DEV_TIMEOUT) return fo_fail(ctx, FO_ETIMEOUT, "grid barrier timed out in PCG");
  if (hs[DS_ERR] == DEV_NAN) return fo_fail(ctx, FO_ENAN, "NaN in the PCG recurrence");
  if (hs[DS_ERR] == DEV_NOCONV) return fo_fail(ctx, FO_ENOCONV, "PCG reached maxit=%d", o->maxit);
  return FO_OK;
}

extern "C" fo_status fo_state_solve_noalloc(fo_problem *p, const double *b, double *x, const fo_solve_opts *o,
                                            fo_solve_stats *st) {
  if (!p || !b || !x) return FO_EINVAL;
  fo_solve_opts def;
  fo_solve_opts_default(&def);
  if (!o) o = &def;
  if (o->precision != FO_FP64)
    return fo_fail(p->ctx, FO_EINVAL, "fo_state_solve_noalloc runs the FP64 solve only");
  if (p->batch) return fo_fail(p->ctx, FO_EINVAL, "fo_state_solve_noalloc takes a single problem");
  if (p->mesh->um) return fo_fail(p->ctx, FO_EINVAL, "fo_state_solve_noalloc takes a box mesh");
  if (p->ndof > (long long)FO_NOALLOC_MAX_DOFS)
    return fo_fail(p->ctx, FO_EINVAL, "%lld DOFs exceed the no-allocation limit of %d (a %d MiB device array)",
                   p->ndof, (int)FO_NOALLOC_MAX_DOFS, FO_NOALLOC_SCRATCH_BYTES >> 20);
  if (!p->coef_valid) FO_TRY(fo_coefficients(p));   // launches kernels, allocates nothing
  const Grid &g = p->mesh->g;
  if (p->desc.kind == FO_ELASTIC) {
    if (g.dim == 2) return noalloc_pcg<2>(p, make_elastic_stencil<2, double>(p), b, x, o, st);
    return noalloc_pcg<3>(p, make_elastic_stencil<3, double>(p), b, x, o, st);
  }
  if (g.dim == 2) return noalloc_pcg<2>(p, make_scalar_stencil<2, double>(p), b, x, o, st);
  return noalloc_pcg<3>(p, make_scalar_stencil<3, double>(p), b, x, o, st);
}
