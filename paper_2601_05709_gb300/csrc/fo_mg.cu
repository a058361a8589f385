// Geometric multigrid for the single-problem state and velocity solves: the hierarchies (level
// planning, coarse coefficients and masks, stencil rows, the coarsest level's inverse, BF16
// row copies), the solve drivers (FP64 CG, FP64 refinement around the FP32 CG) and their
// launches.  The persistent CG kernel and the V-cycle are in fo_mg.cuh.
#include "fo_mg.cuh"

FO_MG_INSTANCES(FO_MG_EXTERN)

// ===================================================================================== host
template <int D>
__global__ void k_mg_restrict_coef(Grid gc, Grid gf, const double *coef_f, double *coef_c) {
  constexpr int P = KP<D>::P;
  for (long long ec = blockIdx.x * (long long)blockDim.x + threadIdx.x; ec < gc.num_elems;
       ec += (long long)gridDim.x * blockDim.x) {
    const long long cell = ec / P;
    const int pc = (int)(ec % P);
    int ci[3];
    ci[0] = (int)(cell % gc.n[0]);
    const long long t = cell / gc.n[0];
    ci[1] = (int)(t % gc.n[1]);
    ci[2] = (int)(t / gc.n[1]);
    double sum = 0.0;
    for (int o = 0; o < (1 << D); ++o) {
      int fi[3] = {2 * ci[0] + (o & 1), 2 * ci[1] + ((o >> 1) & 1), D == 3 ? 2 * ci[2] + ((o >> 2) & 1) : 0};
      const long long fcell = fi[0] + gf.cstride[1] * fi[1] + (D == 3 ? gf.cstride[2] * fi[2] : 0);
      for (int pf = 0; pf < P; ++pf) {
        // the coarse simplex holding fine simplex pf of the fine cell at offset o: axes sorted
        // by offset (descending), ties in the fine simplex's own axis order
        int order[3], n = 0;
        for (int ob = 1; ob >= 0; --ob)
          for (int l = 0; l < D; ++l) {
            const int ax = kperm<D>(pf, l);
            if (((o >> ax) & 1) == ob) order[n++] = ax;
          }
        int q = -1;
        for (int cand = 0; cand < P && q < 0; ++cand) {
          bool same = true;
          for (int l = 0; l < D; ++l) same = same && kperm<D>(cand, l) == order[l];
          if (same) q = cand;
        }
        if (q == pc) sum += coef_f[(long long)P * fcell + pf];
      }
    }
    coef_c[ec] = sum / (double)(1 << D);
  }
}

// Non-nested pair: the coarse element's coefficient is the mean over the fine elements whose
// centroid lies in it (in integer coordinates: exact), or, should none, the coefficient of the
// fine element holding the coarse element's centroid.  A Kuhn simplex's centroid has local
// coordinate (D - j) / (D + 1) along axis pi_j.
template <int D>
__device__ __forceinline__ int mg_simplex_of(const long long rem[3], const long long den[3]) {
  int ax[3] = {0, 1, 2};
  for (int i = 1; i < D; ++i)
    for (int j = i; j > 0; --j) {
      const int a = ax[j], b = ax[j - 1];
      if (rem[a] * den[b] > rem[b] * den[a]) {
        ax[j] = b;
        ax[j - 1] = a;
      } else {
        break;
      }
    }
  for (int cand = 0; cand < KP<D>::P; ++cand) {
    bool same = true;
    for (int l = 0; l < D; ++l) same = same && kperm<D>(cand, l) == ax[l];
    if (same) return cand;
  }
  return 0;
}

template <int D>
__global__ void k_mg_restrict_coef_general(Grid gc, Grid gf, const double *coef_f, double *coef_c) {
  constexpr int P = KP<D>::P;
  for (long long ec = blockIdx.x * (long long)blockDim.x + threadIdx.x; ec < gc.num_elems;
       ec += (long long)gridDim.x * blockDim.x) {
    const long long cellc = ec / P;
    const int pc = (int)(ec % P);
    int ci[3];
    ci[0] = (int)(cellc % gc.n[0]);
    long long tt = cellc / gc.n[0];
    ci[1] = (int)(tt % gc.n[1]);
    ci[2] = (int)(tt / gc.n[1]);
    int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int k = 0; k < D; ++k) {
      lo[k] = (int)(((long long)ci[k] * gf.n[k]) / gc.n[k]);
      hi[k] = (int)std::min<long long>(gf.n[k] - 1, ((long long)(ci[k] + 1) * gf.n[k] + gc.n[k] - 1) / gc.n[k] - 1);
    }
    double sum = 0.0;
    int cnt = 0;
    for (int i2 = lo[2]; i2 <= (D == 3 ? hi[2] : 0); ++i2)
      for (int i1 = lo[1]; i1 <= hi[1]; ++i1)
        for (int i0 = lo[0]; i0 <= hi[0]; ++i0) {
          const int fi[3] = {i0, i1, i2};
          const long long fcell = i0 + gf.cstride[1] * i1 + (D == 3 ? gf.cstride[2] * i2 : 0);
          for (int pf = 0; pf < P; ++pf) {
            long long rem[3] = {0, 0, 0}, den[3] = {1, 1, 1};
            bool in = true;
            for (int j = 0; j < D; ++j) {
              const int k = kperm<D>(pf, j);
              const long long num = ((long long)fi[k] * (D + 1) + (D - j)) * gc.n[k];
              den[k] = (long long)gf.n[k] * (D + 1);
              in = in && num / den[k] == ci[k];
              rem[k] = num % den[k];
            }
            if (in && mg_simplex_of<D>(rem, den) == pc) {
              sum += coef_f[(long long)P * fcell + pf];
              ++cnt;
            }
          }
        }
    if (cnt == 0) {   // the fine element holding the coarse centroid
      int fi[3] = {0, 0, 0};
      long long rem[3] = {0, 0, 0}, den[3] = {1, 1, 1};
      for (int j = 0; j < D; ++j) {
        const int k = kperm<D>(pc, j);
        const long long num = ((long long)ci[k] * (D + 1) + (D - j)) * gf.n[k];
        den[k] = (long long)gc.n[k] * (D + 1);
        fi[k] = (int)std::min<long long>(gf.n[k] - 1, num / den[k]);
        rem[k] = num % den[k];
      }
      const long long fcell = fi[0] + gf.cstride[1] * fi[1] + (D == 3 ? gf.cstride[2] * fi[2] : 0);
      sum = coef_f[(long long)P * fcell + mg_simplex_of<D>(rem, den)];
      cnt = 1;
    }
    coef_c[ec] = sum / (double)cnt;
  }
}

// Non-nested pair: a coarse node takes the Dirichlet flags of the fine node nearest to it
// (boundary nodes map to boundary nodes of the same faces).
__global__ void k_mg_coarse_dir_general(Grid gc, Grid gf, int npn, const uint8_t *dir_f, uint8_t *dir_c) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < gc.num_nodes;
       c += (long long)gridDim.x * blockDim.x) {
    int ic[3];
    node_ijk(gc, c, ic);
    long long f = 0;
    for (int k = 0; k < gc.dim; ++k) {
      const long long i = (2LL * ic[k] * gf.n[k] + gc.n[k]) / (2LL * gc.n[k]);   // round(ic n_f / n_c)
      f += i * gf.stride[k];
    }
    for (int j = 0; j < npn; ++j) dir_c[c * npn + j] = dir_f[f * npn + j];
  }
}

__global__ void k_mg_coarse_dir(Grid gc, Grid gf, int npn, const uint8_t *dir_f, uint8_t *dir_c) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < gc.num_nodes;
       c += (long long)gridDim.x * blockDim.x) {
    int ic[3];
    node_ijk(gc, c, ic);
    const long long f = 2LL * ic[0] + gf.stride[1] * 2LL * ic[1] + (gc.dim == 3 ? gf.stride[2] * 2LL * ic[2] : 0);
    for (int j = 0; j < npn; ++j) dir_c[c * npn + j] = dir_f[f * npn + j];
  }
}

// Inverse of the coarsest level's operator, for the exact coarse solve.  One block: the dense
// n x n matrix (n = nodes x components <= MG_DIRECT_MAX) is assembled in shared memory from
// the level's FP64 difference-form rows -- A[(a,c),(a,k)] = R_ck - sum_s W_s,ck and
// A[(a,c),(nb_s,k)] = W_s,ck, a thread per node -- and inverted in place by Gauss-Jordan
// elimination without pivoting (the matrix is symmetric positive definite: Dirichlet rows are
// identity rows and their columns eliminated), in FP64; the inverse is stored in FP32.
template <int D, int NPN, bool FULL>
__global__ void k_mg_coarse_inverse(Grid g, const double *W, int n, float *ainv) {
  constexpr int S = ST<D>::S, BLK = FULL ? NPN * NPN : NPN;
  extern __shared__ __align__(16) double A[];   // [n][n]
  __shared__ double piv;
  const long long N = g.num_nodes;
  for (int k = threadIdx.x; k < n * n; k += blockDim.x) A[k] = 0.0;
  __syncthreads();
  for (long long a = threadIdx.x; a < N; a += blockDim.x) {   // rows of node a only
    int idx[3];
    node_ijk(g, a, idx);
    for (int c = 0; c < NPN; ++c)
      for (int k = 0; k < NPN; ++k) {
        if (!FULL && k != c) continue;
        const int e = FULL ? c * NPN + k : c;
        const long long r = a * NPN + c;
        double diag = W[(long long)e * N + a];
        for (int s = 1; s < S; ++s) {
          const long long nb = slot_node<D>(g, idx, a, s);
          if (nb < 0) continue;
          const double w = *slot_weight<D, NPN, FULL>(W, N, a, nb, s, e);
          diag -= w;
          A[r * n + nb * NPN + k] += w;
        }
        A[r * n + a * NPN + k] += diag;
      }
  }
  for (int p = 0; p < n; ++p) {
    __syncthreads();
    if (threadIdx.x == 0) piv = 1.0 / A[p * n + p];
    __syncthreads();
    const double q = piv;
    for (int k = threadIdx.x; k < n * n; k += blockDim.x) {   // outside row and column p
      const int i = k / n, j = k - i * n;
      if (i != p && j != p) A[k] -= A[i * n + p] * A[p * n + j] * q;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < n; k += blockDim.x)
      if (k != p) {
        A[p * n + k] *= q;
        A[k * n + p] *= -q;
      }
    if (threadIdx.x == 0) A[p * n + p] = q;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < n * n; k += blockDim.x) ainv[k] = (float)A[k];
}

// The inverse of a coarsest level too large for one block's shared memory (MG_DIRECT_MAX < n
// <= MG_DIRECT_GRID_MAX): the same FP64 Gauss-Jordan elimination on a dense matrix in global
// memory, each pivot's update spread over the whole (cooperative) grid with a grid barrier after
// the update and after the pivot row and column are scaled.  The hierarchy rebuild pays 2n
// barriers; the V-cycle then solves the coarsest level exactly instead of with nuc sweeps.
template <int D, int NPN, bool FULL>
__global__ void k_mg_coarse_inverse_grid(Grid g, const double *W, int n, double *A, float *ainv, GridBar bar) {
  constexpr int S = ST<D>::S;
  const long long N = g.num_nodes, nn = (long long)n * n;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long gs = (long long)gridDim.x * blockDim.x;
  for (long long k = tid; k < nn; k += gs) A[k] = 0.0;
  if (!grid_sync(bar)) return;
  for (long long a = tid; a < N; a += gs) {   // rows of node a: each entry written by one thread
    int idx[3];
    node_ijk(g, a, idx);
    for (int c = 0; c < NPN; ++c)
      for (int k = 0; k < NPN; ++k) {
        if (!FULL && k != c) continue;
        const int e = FULL ? c * NPN + k : c;
        const long long r = a * NPN + c;
        double diag = W[(long long)e * N + a];
        for (int s = 1; s < S; ++s) {
          const long long nb = slot_node<D>(g, idx, a, s);
          if (nb < 0) continue;
          const double w = *slot_weight<D, NPN, FULL>(W, N, a, nb, s, e);
          diag -= w;
          A[r * n + nb * NPN + k] += w;
        }
        A[r * n + a * NPN + k] += diag;
      }
  }
  if (!grid_sync(bar)) return;
  for (int p = 0; p < n; ++p) {
    const double q = 1.0 / A[(long long)p * n + p];
    for (long long k = tid; k < nn; k += gs) {   // outside row and column p
      const long long i = k / n, j = k - i * n;
      if (i != p && j != p) A[k] -= A[i * n + p] * A[(long long)p * n + j] * q;
    }
    if (!grid_sync(bar)) return;
    for (long long k = tid; k < n; k += gs)
      if (k != p) {
        A[(long long)p * n + k] *= q;
        A[k * n + p] *= -q;
      }
    if (tid == 0) A[(long long)p * n + p] = q;
    if (!grid_sync(bar)) return;
  }
  for (long long k = tid; k < nn; k += gs) ainv[k] = (float)A[k];
}

static fo_status mg_build_inverse_grid(fo_ctx *ctx, fo_mg *mg) {
  const Grid &gc = mg->g[mg->L - 1];
  const double *W = mg->W64[mg->L - 1];
  const int n = mg->nd;
  double *tail = mg->adense + (size_t)n * n;   // barrier counter and status word
  GridBar bar{reinterpret_cast<unsigned *>(tail), reinterpret_cast<int *>(tail + 8), 2000000000ull};
  auto run = [&](auto kern) -> fo_status {
    int per_sm = 0;
    FO_CU(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)kern, FO_BLOCK, 0));
    if (per_sm < 1) return fo_fail(ctx, FO_ECUDA, "coarse inverse kernel does not fit on an SM");
    long long cap = (long long)per_sm * ctx->num_sms;
    if (ctx->grid_share > 1) cap = std::max(1LL, cap / ctx->grid_share);
    // one block per SM at most: the 2n barriers, not the n^3 flops, set the time
    const int grid = (int)std::min<long long>(std::min<long long>(cap, ctx->num_sms),
                                              ((long long)n * n + FO_BLOCK - 1) / FO_BLOCK);
    FO_CU(ctx, cudaMemsetAsync(tail, 0, 16 * sizeof(double), ctx->stream));
    void *argv[] = {(void *)&gc, (void *)&W, (void *)&n, (void *)&mg->adense, (void *)&mg->ainv, (void *)&bar};
    {
      std::lock_guard<std::mutex> lk(fo_launch_mutex());
      FO_CU(ctx, cudaLaunchCooperativeKernel((const void *)kern, grid, FO_BLOCK, argv, 0, ctx->stream));
    }
    fo_note_launch(1);
    FO_CU(ctx, cudaGetLastError());
    FO_CU(ctx, cudaMemcpyAsync(ctx->h_scalars + 48, tail + 8, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    FO_CU(ctx, cudaStreamSynchronize(ctx->stream));
    if (*reinterpret_cast<const int *>(ctx->h_scalars + 48) == DEV_TIMEOUT)
      return fo_fail(ctx, FO_ETIMEOUT, "grid barrier timed out in the coarse inverse");
    return FO_OK;
  };
  if (gc.dim == 2) {
    if (mg->npn == 1) return run(k_mg_coarse_inverse_grid<2, 1, true>);
    if (mg->blk == 4) return run(k_mg_coarse_inverse_grid<2, 2, true>);
    return run(k_mg_coarse_inverse_grid<2, 2, false>);
  }
  if (mg->npn == 1) return run(k_mg_coarse_inverse_grid<3, 1, true>);
  if (mg->blk == 9) return run(k_mg_coarse_inverse_grid<3, 3, true>);
  return run(k_mg_coarse_inverse_grid<3, 3, false>);
}

static fo_status mg_build_inverse(fo_ctx *ctx, fo_mg *mg) {
  if (mg->nd == 0) return FO_OK;
  if (mg->nd > MG_DIRECT_MAX) return mg_build_inverse_grid(ctx, mg);
  const Grid &gc = mg->g[mg->L - 1];
  const double *W = mg->W64[mg->L - 1];
  cudaStream_t s = ctx->stream;
  const size_t smem = sizeof(double) * mg->nd * mg->nd;
  auto run = [&](auto kern) -> fo_status {
    std::lock_guard<std::mutex> lk(fo_launch_mutex());
    FO_TRY(fo_smem_limit(ctx, (const void *)kern, smem));
    kern<<<1, 256, smem, s>>>(gc, W, mg->nd, mg->ainv);
    fo_note_launch(1);
    FO_CU(ctx, cudaGetLastError());
    return FO_OK;
  };
  if (gc.dim == 2) {
    if (mg->npn == 1) return run(k_mg_coarse_inverse<2, 1, true>);
    if (mg->blk == 4) return run(k_mg_coarse_inverse<2, 2, true>);
    return run(k_mg_coarse_inverse<2, 2, false>);
  }
  if (mg->npn == 1) return run(k_mg_coarse_inverse<3, 1, true>);
  if (mg->blk == 9) return run(k_mg_coarse_inverse<3, 3, true>);
  return run(k_mg_coarse_inverse<3, 3, false>);
}

// The single-problem hierarchy ends at the first level small enough to be solved directly.
static int mg_plan_single(const Grid &g0, Grid *g, int npn) {
  return fo_mg_plan(g0, g, MG_MAX_LEVELS, MG_DIRECT_MAX, npn, true);
}

static int mg_direct_unknowns(const Grid *g, int L, int npn) {
  if (L < 2) return 0;
  const long long n = g[L - 1].num_nodes * npn;
  return n <= MG_DIRECT_GRID_MAX ? (int)n : 0;
}


// ------------------------------------------------------------------------- hierarchies
// Levels: halve every axis while all are even and the coarse grid keeps >= 2 cells per axis;
// with stop_unknowns > 0, also stop at the first level of at most that many unknowns (npn per
// node).
int fo_mg_plan(const Grid &g0, Grid *g, int max_levels, long long stop_unknowns, int npn, bool general) {
  g[0] = g0;
  int L = 1;
  bool halved = false;
  while (L < max_levels) {
    const Grid &f = g[L - 1];
    if (stop_unknowns > 0 && f.num_nodes * npn <= stop_unknowns) break;
    int n[3] = {1, 1, 1};
    bool ok = true, even = true;
    for (int a = 0; a < f.dim; ++a) even = even && f.n[a] % 2 == 0 && f.n[a] / 2 >= 2;
    // halve while every axis halves; otherwise (general) ceil(n/2) cells per axis -- except
    // below a hierarchy that already reached the block-run size by halving: there the block's
    // smoothing sweeps on its coarsest level cost less than the non-nested transfers' point
    // location (3D cantilever 96x48x48: 6x3x3 -> 3x2x2 made each CG iteration 50 % slower)
    if (!even && general && halved && f.num_nodes * npn <= MG_BLOCK_DOFS) ok = false;
    for (int a = 0; a < f.dim; ++a) {
      n[a] = even ? f.n[a] / 2 : (f.n[a] + 1) / 2;
      // (non-nested transfers locate points in 32-bit integers: axes below 2^15 cells)
      if (!even && (!general || f.n[a] < 3 || f.n[a] >= 32768)) ok = false;
    }
    if (!ok) break;
    if (!fo_grid_make(f.dim, n, f.lo, f.hi, g[L])) break;
    halved = halved || even;
    ++L;
  }
  return L;
}

// Byte sizes of level l's arrays, in the order b, z0, z1, t, coef, W64, W32, dinv64, dinv32, dir
// (coarse levels own all; level 0 owns coef, W32, dinv32 and dir only when own0).
static void mg_sizes(const Grid &g, int npn, int blk, bool coarse, bool own0, size_t sz[10]) {
  const size_t N = (size_t)g.num_nodes, S = (size_t)fo_row_slots(g.dim);
  for (int i = 0; i < 4; ++i) sz[i] = sizeof(float) * N * npn;
  sz[4] = (coarse || own0) ? sizeof(double) * g.num_elems : 0;
  sz[5] = coarse ? sizeof(double) * S * blk * N : 0;
  sz[6] = (coarse || own0) ? sizeof(float) * S * blk * N : 0;
  sz[7] = coarse ? sizeof(double) * N * npn : 0;
  sz[8] = (coarse || own0) ? sizeof(float) * N * npn : 0;
  sz[9] = (coarse || own0) ? N * npn : 0;
}

static void **mg_slot(fo_mg *mg, int l, int i) {
  switch (i) {
    case 0: return (void **)&mg->b[l];
    case 1: return (void **)&mg->z0[l];
    case 2: return (void **)&mg->z1[l];
    case 3: return (void **)&mg->t[l];
    case 4: return (void **)&mg->coef[l];
    case 5: return (void **)&mg->W64[l];
    case 6: return (void **)&mg->W32[l];
    case 7: return (void **)&mg->dinv64[l];
    case 8: return (void **)&mg->dinv32[l];
    default: return (void **)&mg->dir[l];
  }
}

// Bytes of a level's BF16 rows.
static size_t mg_bf16_bytes(const Grid &g, int blk) {
  return sizeof(__nv_bfloat16) * (size_t)fo_row_slots(g.dim) * blk * (size_t)g.num_nodes;
}
// Shared memory block 0 needs to stage levels from..L-1 (the layout of mg_stage_layout: rows,
// inverse diagonal, b, z[2], t and mask per level, each array 16-byte aligned, and the
// coarsest inverse).
static size_t mg_stage_bytes_from(const Grid *g, int L, int npn, int blk, int from, int nd) {
  auto al = [](size_t b) { return (b + 15) / 16 * 16; };
  size_t b = nd > 0 && nd <= MG_DIRECT_MAX ? al(sizeof(float) * (size_t)nd * nd) : 0;
  for (int l = from; l < L; ++l) {
    const size_t n = (size_t)g[l].num_nodes;
    b += al(sizeof(float) * fo_row_slots(g[l].dim) * blk * n) + 5 * al(sizeof(float) * npn * n) + al(npn * n);
  }
  return b;
}
// Staging budget that keeps the multigrid CG's co-resident grid: one block per SM in 2D (the
// launch bounds), two in 3D (each with its static shared memory beside the staged levels).
static size_t mg_stage_budget(int dim) { return dim == 2 ? (size_t)MG_STAGE_MAX_BYTES : (size_t)88 * 1024; }
// The first level that block 0 runs alone: at most MG_BLOCK_DOFS unknowns and, where some such
// level allows it, every level from it down staged in block 0's shared memory.  A level that
// is small but too large to stage stays with the grid: block 0 sweeping it from L2 took longer
// than the grid phases it saves (the 3D cantilever's 12x6x6 level: 166 us of a 556 us CG
// iteration in block 0).  Where no small level can be staged, the first small one (run from
// global memory).
static int mg_block_level(const Grid *g, int L, int npn, int blk) {
  int first = L;
  for (int l = 0; l < L; ++l)
    if ((long long)g[l].num_nodes * npn <= MG_BLOCK_DOFS) {
      first = l;
      break;
    }
  const int nd = mg_direct_unknowns(g, L, npn);
  for (int l = first; l < L; ++l)
    if (mg_stage_bytes_from(g, L, npn, blk, l, nd) <= mg_stage_budget(g[0].dim)) return l;
  return first;
}

static void mg_release(fo_ctx *ctx, fo_mg *&mg) {
  if (!mg) return;
  for (int l = 0; l < mg->L; ++l) {
    size_t sz[10];
    mg_sizes(mg->g[l], mg->npn, mg->blk, l > 0, mg->own0, sz);
    for (int i = 0; i < 10; ++i)
      if (sz[i]) fo_free(ctx, *mg_slot(mg, l, i), sz[i]);
  }
  if (mg->nd > 0) {
    fo_free(ctx, mg->ainv, sizeof(float) * mg->nd * mg->nd);
    if (mg->adense) fo_free(ctx, mg->adense, sizeof(double) * ((size_t)mg->nd * mg->nd + 16));
  }
  for (int l = 0; l < mg->L; ++l)
    if (mg->Wh[l]) fo_free(ctx, mg->Wh[l], mg_bf16_bytes(mg->g[l], mg->blk));
  fo_free(ctx, mg->dev, sizeof(MgDev));
  delete mg;
  mg = nullptr;
}

void fo_mg_release(fo_ctx *ctx, fo_mg *&mg) { mg_release(ctx, mg); }

void fo_mg_destroy(fo_problem *p) {
  mg_release(p->ctx, p->mg);
  mg_release(p->ctx, p->mgv);
}

// Multigrid pays when the hierarchy reaches a small coarsest level.  Single problems coarsen
// any grid (non-nested levels where an axis does not halve); the batched multigrid needs nested
// levels (general = false), so grids not divisible by enough powers of two keep its Jacobi
// solver.
#define MG_COARSEST_MAX_DOFS 8192
bool fo_mg_applicable(const Grid &g0, int npn, bool general) {
  Grid g[MG_MAX_LEVELS];
  const int L = fo_mg_plan(g0, g, MG_MAX_LEVELS, MG_DIRECT_MAX, npn, general);
  return L >= 2 && g[L - 1].num_nodes * npn <= MG_COARSEST_MAX_DOFS;
}

size_t fo_mg_bytes(int dim, const int n[3], int npn, int blk, bool own0, bool bf16) {
  Grid g0;
  const double lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1};
  if (!fo_grid_make(dim, n, lo, hi, g0)) return 0;
  Grid g[MG_MAX_LEVELS];
  const int L = mg_plan_single(g0, g, npn);
  size_t b = sizeof(MgDev);
  for (int l = 0; l < L; ++l) {
    size_t sz[10];
    mg_sizes(g[l], npn, blk, l > 0, own0, sz);
    for (int i = 0; i < 10; ++i) b += sz[i];
  }
  if (bf16)
    for (int l = 0; l < mg_block_level(g, L, npn, blk); ++l) b += mg_bf16_bytes(g[l], blk);
  const size_t nd = (size_t)mg_direct_unknowns(g, L, npn);
  return b + nd * nd * sizeof(float) + (nd > MG_DIRECT_MAX ? sizeof(double) * (nd * nd + 16) : 0);
}

static fo_status mg_alloc(fo_ctx *ctx, fo_mg *&out, const Grid &g0, int npn, int blk, bool own0) {
  fo_mg *mg = new fo_mg();
  out = mg;
  mg->npn = npn;
  mg->blk = blk;
  mg->own0 = own0;
  mg->L = mg_plan_single(g0, mg->g, npn);
  for (int l = 0; l < mg->L; ++l) {
    size_t sz[10];
    mg_sizes(mg->g[l], npn, blk, l > 0, own0, sz);
    for (int i = 0; i < 10; ++i)
      if (sz[i]) FO_TRY(fo_alloc(ctx, mg_slot(mg, l, i), sz[i]));
  }
  mg->nd = mg_direct_unknowns(mg->g, mg->L, npn);
  if (mg->nd > 0) {
    FO_TRY(fo_alloc(ctx, (void **)&mg->ainv, sizeof(float) * mg->nd * mg->nd));
    if (mg->nd > MG_DIRECT_MAX)
      FO_TRY(fo_alloc(ctx, (void **)&mg->adense, sizeof(double) * ((size_t)mg->nd * mg->nd + 16)));
  }
  FO_TRY(fo_alloc(ctx, (void **)&mg->dev, sizeof(MgDev)));
  return FO_OK;
}

__global__ void k_mg_rows_bf16(const float *w, __nv_bfloat16 *h, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    h[i] = __float2bfloat16_rn(w[i]);
}

// Level table to the device; level 0's FP32 rows, FP32 inverse diagonal and Dirichlet mask.
// With bf16, the grid-run levels (those above the block-run ones) get BF16 copies of their
// rows, rounded to nearest from the FP32 rows just built, and the table points their sweeps
// and residuals at them; the block-run levels keep FP32 rows (read from shared memory).
static fo_status mg_upload(fo_ctx *ctx, fo_mg *mg, const float *W0, const float *dinv0, const uint8_t *dir0,
                           float omega, bool bf16) {
  MgDev h;
  memset(&h, 0, sizeof h);
  h.L = mg->L;
  h.Lg = mg_block_level(mg->g, mg->L, mg->npn, mg->blk);
  mg->Lg = h.Lg;
  h.omega = omega;
  h.om[0] = omega;
  h.om[1] = omega;
  h.nu = 2;
  h.nuc = 16;
  h.nd = mg->nd;
  h.ainv = mg->ainv;
  for (int l = 0; l < mg->L; ++l) {
    MgLevelDev &d = h.lv[l];
    d.g = mg->g[l];
    d.W = l == 0 ? W0 : mg->W32[l];
    d.dinv = l == 0 ? dinv0 : mg->dinv32[l];
    d.dir = l == 0 ? dir0 : mg->dir[l];
    d.b = mg->b[l];
    d.z[0] = mg->z0[l];
    d.z[1] = mg->z1[l];
    d.t = mg->t[l];
    d.Wh = nullptr;
    if (bf16 && l < h.Lg) {
      const size_t bytes = mg_bf16_bytes(mg->g[l], mg->blk);
      if (!mg->Wh[l]) FO_TRY(fo_alloc(ctx, (void **)&mg->Wh[l], bytes));
      const long long n = (long long)(bytes / sizeof(__nv_bfloat16));
      k_mg_rows_bf16<<<fo_blocks_for(n, FO_BLOCK, 65536), FO_BLOCK, 0, ctx->stream>>>(d.W, mg->Wh[l], n);
      fo_note_launch(1);
      FO_CU(ctx, cudaGetLastError());
      d.Wh = mg->Wh[l];
    }
  }
  mg->rows_bf16 = bf16 ? 1 : 0;
  mg->host.resize(sizeof(MgDev));
  memcpy(mg->host.data(), &h, sizeof(MgDev));
  FO_CU(ctx, cudaMemcpyAsync(mg->dev, mg->host.data(), sizeof(MgDev), cudaMemcpyHostToDevice, ctx->stream));
  FO_CU(ctx, cudaGetLastError());
  return FO_OK;
}

// Coarse per-element coefficient (children means) and per-DOF Dirichlet mask of grid gc from
// those of the grid gf it halves.
void fo_mg_restrict(fo_ctx *ctx, const Grid &gc, const Grid &gf, int npn, const double *coef_f, const uint8_t *dir_f,
                    double *coef_c, uint8_t *dir_c) {
  cudaStream_t s = ctx->stream;
  const int blocks = fo_blocks_for(gc.num_elems, FO_BLOCK, 65536);
  if (!mg_nested(gf, gc)) {
    if (gc.dim == 2) k_mg_restrict_coef_general<2><<<blocks, FO_BLOCK, 0, s>>>(gc, gf, coef_f, coef_c);
    else k_mg_restrict_coef_general<3><<<blocks, FO_BLOCK, 0, s>>>(gc, gf, coef_f, coef_c);
    k_mg_coarse_dir_general<<<fo_blocks_for(gc.num_nodes, FO_BLOCK, 65536), FO_BLOCK, 0, s>>>(gc, gf, npn, dir_f,
                                                                                              dir_c);
    fo_note_launch(2);
    return;
  }
  if (gc.dim == 2) k_mg_restrict_coef<2><<<blocks, FO_BLOCK, 0, s>>>(gc, gf, coef_f, coef_c);
  else k_mg_restrict_coef<3><<<blocks, FO_BLOCK, 0, s>>>(gc, gf, coef_f, coef_c);
  k_mg_coarse_dir<<<fo_blocks_for(gc.num_nodes, FO_BLOCK, 65536), FO_BLOCK, 0, s>>>(gc, gf, npn, dir_f, dir_c);
  fo_note_launch(2);
}

// restrict a per-element coefficient and the per-DOF Dirichlet mask from level l-1 to level l
static void mg_restrict_level(fo_ctx *ctx, fo_mg *mg, int l, const double *coef_f, const uint8_t *dir_f) {
  fo_mg_restrict(ctx, mg->g[l], mg->g[l - 1], mg->npn, coef_f, dir_f, mg->coef[l], mg->dir[l]);
}

// State hierarchy: rebuilt after every coefficient update (coarse coefficients are the
// children means of the current A_e).
static fo_status mg_prepare_state(fo_problem *p, bool bf16) {
  fo_ctx *ctx = p->ctx;
  if (!p->mg) {
    FO_TRY(mg_alloc(ctx, p->mg, p->mesh->g, p->ncomp, p->ncomp * p->ncomp, false));
    p->mg->built_epoch = -1;
  }
  fo_mg *mg = p->mg;
  if (mg->built_epoch == p->coef_epoch) {
    if ((mg->rows_bf16 != 0) == bf16) return FO_OK;
    return mg_upload(ctx, mg, p->Wst32, p->dinv_state32, p->dir, p->ncomp == 1 ? 0.8f : 0.6f, bf16);
  }
  // coefficients and masks level by level, then every coarse level's rows in one launch
  StencilLevels sl;
  sl.first_block[0] = 0;
  for (int l = 1; l < mg->L; ++l) {
    mg_restrict_level(ctx, mg, l, l == 1 ? p->coef : mg->coef[l - 1], l == 1 ? p->dir : mg->dir[l - 1]);
    const int k = sl.n++;
    sl.g[k] = mg->g[l];
    sl.coef[k] = mg->coef[l];
    sl.dir[k] = mg->dir[l];
    sl.W[k] = mg->W64[l];
    sl.W32[k] = mg->W32[l];
    sl.di[k] = mg->dinv64[l];
    sl.di32[k] = mg->dinv32[l];
    sl.first_block[k + 1] = sl.first_block[k] + (int)((mg->g[l].num_nodes + FO_BLOCK - 1) / FO_BLOCK);
  }
  FO_CU(ctx, cudaGetLastError());
  FO_TRY(fo_launch_stencil_levels(p, sl));
  FO_TRY(mg_build_inverse(ctx, mg));
  FO_TRY(mg_upload(ctx, mg, p->Wst32, p->dinv_state32, p->dir, p->ncomp == 1 ? 0.8f : 0.6f, bf16));
  mg->built_epoch = p->coef_epoch;
  return FO_OK;
}

__global__ void k_vel_mass_coef(long long ne, const uint8_t *omega0, double alpha, double gamma0, double *mc) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ne; e += (long long)gridDim.x * blockDim.x)
    mc[e] = alpha + (omega0[e] ? gamma0 : 0.0);
}
__global__ void k_vel_dof_mask(long long nn, int d, const uint8_t *vdir, int on, uint8_t *mask) {
  for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < nn; a += (long long)gridDim.x * blockDim.x)
    for (int c = 0; c < d; ++c) mask[a * d + c] = on && vdir[a];
}
// -b on the velocity DOFs, zero on H^1_0 rows
__global__ void k_vel_rhs(long long nn, int d, const double *b, const uint8_t *mask, double *out) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nn * d; k += (long long)gridDim.x * blockDim.x)
    out[k] = mask[k] ? 0.0 : -b[k];
}

// Velocity hierarchy: the form does not depend on phi, so it is built once.  Level 0's rows
// are the problem's velocity rows; coarse levels carry the children mean of the mass-type
// coefficient alpha + gamma_0 chi_Omega0 and the same normal penalty on their faces.
static fo_status mg_prepare_velocity(fo_problem *p, bool bf16) {
  if (p->mgv) {
    if ((p->mgv->rows_bf16 != 0) == bf16) return FO_OK;
    return mg_upload(p->ctx, p->mgv, p->mgv->W32[0], p->mgv->dinv32[0], p->mgv->dir[0], 0.8f, bf16);
  }
  fo_ctx *ctx = p->ctx;
  const Grid &g0 = p->mesh->g;
  const int d = g0.dim;
  FO_TRY(mg_alloc(ctx, p->mgv, g0, d, d, true));
  fo_mg *mg = p->mgv;
  cudaStream_t s = ctx->stream;
  const double al = p->desc.alpha_mass, ga0 = p->desc.omega0_weight;
  k_vel_mass_coef<<<fo_blocks_for(g0.num_elems, FO_BLOCK, 65536), FO_BLOCK, 0, s>>>(g0.num_elems, p->omega0, al, ga0,
                                                                                   mg->coef[0]);
  k_vel_dof_mask<<<fo_blocks_for(g0.num_nodes, FO_BLOCK, 65536), FO_BLOCK, 0, s>>>(
      g0.num_nodes, d, p->vdir, p->desc.velocity_dirichlet ? 1 : 0, mg->dir[0]);
  fo_note_launch(2);
  // level 0 again with FP32 copies (same rows as the problem's FP64 ones)
  FO_TRY(fo_launch_velocity_stencil_on(p, g0, mg->coef[0], mg->dir[0], p->Wvel, mg->W32[0], p->dinv_vel,
                                       mg->dinv32[0]));
  for (int l = 1; l < mg->L; ++l) {
    mg_restrict_level(ctx, mg, l, mg->coef[l - 1], mg->dir[l - 1]);
    FO_TRY(fo_launch_velocity_stencil_on(p, mg->g[l], mg->coef[l], mg->dir[l], mg->W64[l], mg->W32[l], mg->dinv64[l],
                                         mg->dinv32[l]));
  }
  FO_TRY(mg_build_inverse(ctx, mg));
  FO_TRY(mg_upload(ctx, mg, mg->W32[0], mg->dinv32[0], mg->dir[0], 0.8f, bf16));
  return FO_OK;
}

// ------------------------------------------------------------------------------ solves
template <int D, int NPN, bool FULL, int NC>
static fo_status mg_run(fo_problem *p, fo_mg *mg, const double *W64, const double *b, double *x, long long n,
                        const fo_solve_opts *o, fo_solve_stats *st, double *bx) {
  double *buf;
  FO_TRY(fo_scratch(p, sizeof(double) * 6 * n, (void **)&buf));
  MgCg C{};
  C.W = W64;
  C.b = b;
  C.x = x;
  C.r = buf;
  C.p[0] = buf + n;
  C.p[1] = buf + 2 * n;
  C.s = buf + 3 * n;
  C.z = buf + 4 * n;
  return mg_launch<D, NPN, FULL, NC, double>(p, mg, C, o, o->rtol, o->maxit, o->warm_start, st, bx);
}

// ---- mixed: FP64 iterative refinement around the FP32 multigrid CG
// r = b - A x with the FP64 rows; ||r||^2 and ||b||^2 as per-block partials
__global__ void k_mg_ir_residual(const double *b, const double *ax, double *r, long long n, double *partials) {
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
// the two sums in a fixed order (deterministic)
__global__ void k_mg_ir_total(const double *partials, int nblocks, double *out) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (w >= 2) return;
  double t = 0;
  for (int b = lane; b < nblocks; b += 32) t += partials[(size_t)b * 2 + w];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  if (lane == 0) out[w] = t;
}
// the inner right-hand side: the residual scaled to unit norm, in FP32
__global__ void k_mg_ir_scale(const double *r, double inv, float *b32, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b32[i] = (float)(r[i] * inv);
}
// x += scale * d (the correction accumulated in FP64)
__global__ void k_mg_ir_update(double *x, const float *d, double scale, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] = fma(scale, (double)d[i], x[i]);
}

// Each refinement step forms the true residual r = b - A x in FP64, solves A d = r / ||r|| with
// the FP32 CG (FP32 rows and vectors, FP64 dot products) preconditioned by the same FP32
// V-cycle to the relative reduction inner_rtol, and adds ||r|| d to x in FP64.  It stops when
// ||r|| <= rtol ||b||, or when two consecutive steps fail to halve ||r|| (the FP64 residual's
// own rounding floor is reached).
template <int D, int NPN>
static fo_status mg_state_mixed(fo_problem *p, const double *b, double *x, const fo_solve_opts *o, fo_solve_stats *st) {
  fo_ctx *ctx = p->ctx;
  const long long n = p->ndof;
  double *buf;
  FO_TRY(fo_scratch(p, sizeof(double) * 2 * n + sizeof(float) * 7 * n + 256, (void **)&buf));
  double *r64 = buf, *ax64 = buf + n;
  float *f = reinterpret_cast<float *>(buf + 2 * n);
  MgCgT<float> C{};
  C.W = p->Wst32;
  C.b = f;
  C.x = f + n;
  C.r = f + 2 * n;
  C.p[0] = f + 3 * n;
  C.p[1] = f + 4 * n;
  C.s = f + 5 * n;
  C.z = f + 6 * n;
  const int blocks = fo_blocks_for(n, FO_BLOCK, 1024);
  double *sums = p->red + (FO_RED_DOUBLES - 128);
  if (!o->warm_start) FO_CU(ctx, cudaMemsetAsync(x, 0, sizeof(double) * n, ctx->stream));
  fo_solve_stats s;
  memset(&s, 0, sizeof s);
  double bnorm2 = -1, prev_rn2 = INFINITY, prev2_rn2 = INFINITY;
  const int max_outer = 60;
  for (int outer = 0;; ++outer) {
    FO_TRY(fo_launch_state_apply(p, x, ax64, true));
    k_mg_ir_residual<<<blocks, FO_BLOCK, 0, ctx->stream>>>(b, ax64, r64, n, p->red);
    k_mg_ir_total<<<1, 64, 0, ctx->stream>>>(p->red, blocks, sums);
    fo_note_launch(2);
    FO_CU(ctx, cudaGetLastError());
    FO_CU(ctx, cudaMemcpyAsync(ctx->h_scalars, sums, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    FO_CU(ctx, cudaStreamSynchronize(ctx->stream));
    const double rn2 = ctx->h_scalars[0];
    if (bnorm2 < 0) bnorm2 = ctx->h_scalars[1];
    s.operator_applies += 1;
    s.rel_residual = bnorm2 > 0 ? std::sqrt(rn2 / bnorm2) : 0.0;
    if (!std::isfinite(rn2)) return fo_fail(ctx, FO_ENAN, "NaN in the refinement residual");
    if (rn2 <= o->rtol * o->rtol * bnorm2 || bnorm2 == 0 || rn2 == 0) break;
    if (outer >= 2 && rn2 > 0.25 * prev_rn2 && prev_rn2 > 0.25 * prev2_rn2) break;
    prev2_rn2 = prev_rn2;
    prev_rn2 = rn2;
    if (outer >= max_outer || s.iterations >= o->maxit) {
      if (st) *st = s;
      return fo_fail(ctx, FO_ENOCONV, "iterative refinement stalled at %.3e", s.rel_residual);
    }
    const double rn = std::sqrt(rn2);
    k_mg_ir_scale<<<blocks, FO_BLOCK, 0, ctx->stream>>>(r64, 1.0 / rn, f, n);
    fo_note_launch(1);
    fo_solve_stats in;
    const fo_status r = mg_launch<D, NPN, true, 1, float>(p, p->mg, C, o, o->inner_rtol, o->inner_maxit, 0, &in,
                                                          nullptr);
    if (r != FO_OK && r != FO_ENOCONV) return r;   // an inner cap only ends that step
    s.iterations += in.iterations;
    s.operator_applies += in.operator_applies;
    s.outer_iterations = outer + 1;
    k_mg_ir_update<<<blocks, FO_BLOCK, 0, ctx->stream>>>(x, C.x, rn, n);
    fo_note_launch(1);
    FO_CU(ctx, cudaGetLastError());
  }
  if (st) *st = s;
  return FO_OK;
}

fo_status fo_state_pcg_mg(fo_problem *p, const double *b, double *x, const fo_solve_opts *o, fo_solve_stats *st) {
  FO_TRY(mg_prepare_state(p, o->mg_bf16 != 0));
  const int d = p->mesh->g.dim;
  const long long n = p->ndof;
  if (o->precision == FO_MIXED) {
    if (p->desc.kind == FO_ELASTIC) return d == 2 ? mg_state_mixed<2, 2>(p, b, x, o, st) : mg_state_mixed<3, 3>(p, b, x, o, st);
    return d == 2 ? mg_state_mixed<2, 1>(p, b, x, o, st) : mg_state_mixed<3, 1>(p, b, x, o, st);
  }
  if (p->desc.kind == FO_ELASTIC)
    return d == 2 ? mg_run<2, 2, true, 1>(p, p->mg, p->Wst, b, x, n, o, st, nullptr)
                  : mg_run<3, 3, true, 1>(p, p->mg, p->Wst, b, x, n, o, st, nullptr);
  return d == 2 ? mg_run<2, 1, true, 1>(p, p->mg, p->Wst, b, x, n, o, st, nullptr)
                : mg_run<3, 1, true, 1>(p, p->mg, p->Wst, b, x, n, o, st, nullptr);
}

// Velocity solve B theta = -b with multigrid: the d component systems share one launch.
fo_status fo_velocity_pcg_mg(fo_problem *p, const fo_solve_opts *o, double *Btt, fo_solve_stats *st) {
  FO_TRY(mg_prepare_velocity(p, o->mg_bf16 != 0));
  const Grid &g = p->mesh->g;
  const int d = g.dim;
  const long long n = (long long)d * g.num_nodes;
  double *rhs;
  FO_TRY(fo_scratch(p, sizeof(double) * 7 * n, (void **)&rhs));
  rhs += 6 * n;   // after the solver's six vectors
  k_vel_rhs<<<fo_blocks_for(n, FO_BLOCK, 65536), FO_BLOCK, 0, p->ctx->stream>>>(g.num_nodes, d, p->rhs, p->mgv->dir[0],
                                                                               rhs);
  fo_note_launch(1);
  double bx = 0.0;
  fo_status r = d == 2 ? mg_run<2, 2, false, 2>(p, p->mgv, p->Wvel, rhs, p->theta, n, o, st, &bx)
                       : mg_run<3, 3, false, 3>(p, p->mgv, p->Wvel, rhs, p->theta, n, o, st, &bx);
  if (Btt) *Btt = bx;   // B(theta, theta) = -b . theta
  return r;
}
