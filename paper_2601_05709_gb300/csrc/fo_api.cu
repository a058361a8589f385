// Host side of the C ABI: contexts, meshes, problems, field I/O, the host-only PPL and
// adaptive-time helpers, and the orchestration of one Algorithm-1 iteration.
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <algorithm>
#include <atomic>

#include "fo_internal.cuh"
#include "fo_umesh.cuh"

// ----------------------------------------------------------------------- launch counter
static std::atomic<unsigned long long> g_launches{0};
void fo_note_launch(int n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }
extern "C" fo_status fo_launch_count(unsigned long long *out) {
  if (!out) return FO_EINVAL;
  *out = g_launches.load(std::memory_order_relaxed);
  return FO_OK;
}

// ------------------------------------------------------------------------- status helpers
fo_status fo_fail(fo_ctx *ctx, fo_status st, const char *fmt, ...) {
  if (ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    ctx->err = buf;
  }
  return st;
}

fo_status fo_cuda_check(fo_ctx *ctx, cudaError_t e, const char *what) {
  if (e == cudaSuccess) return FO_OK;
  // a failed call leaves its error as the host thread's last error: clear it, so that the
  // thread's next call (another request, on the server's executors) does not report it again
  // (a sticky error stays, as it should)
  (void)cudaGetLastError();
  if (e == cudaErrorMemoryAllocation) return fo_fail(ctx, FO_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
  return fo_fail(ctx, FO_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

fo_status fo_alloc(fo_ctx *ctx, void **p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return FO_OK;
  if (ctx->budget && ctx->in_use + bytes > ctx->budget)
    return fo_fail(ctx, FO_ENOMEM_BUDGET, "allocation of %zu bytes exceeds the budget (%zu of %zu in use)",
                   bytes, ctx->in_use, ctx->budget);
  // stream-ordered: neither the allocation nor the matching free synchronises the device,
  // so contexts on other streams (the request server's executors) are not stalled; all of a
  // context's work runs on its stream, where the memory is valid from this point on
  cudaError_t e = cudaMallocAsync(p, bytes, ctx->stream);
  if (e != cudaSuccess) {
    *p = nullptr;
    return fo_cuda_check(ctx, e, "cudaMallocAsync");
  }
  ctx->in_use += bytes;
  return FO_OK;
}

void fo_free(fo_ctx *ctx, void *p, size_t bytes) {
  if (!p) return;
  cudaFreeAsync(p, ctx->stream);
  ctx->in_use -= std::min(ctx->in_use, bytes);
}

// ------------------------------------------------------------------------------- context
extern "C" fo_status fo_ctx_create(int device, void *cuda_stream, size_t mem_budget_bytes, fo_ctx **out) {
  if (!out) return FO_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return FO_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return FO_ECUDA;
  fo_ctx *c = new fo_ctx();
  c->device = device;
  c->budget = mem_budget_bytes;
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (cuda_stream) {
    c->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return FO_ECUDA;
    }
    c->own_stream = true;
  }
  if (cudaMallocHost(&c->h_scalars, 64 * sizeof(double)) != cudaSuccess) {
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return FO_ENOMEM;
  }
  *out = c;
  return FO_OK;
}

extern "C" fo_status fo_ctx_destroy(fo_ctx *ctx) {
  if (!ctx) return FO_EINVAL;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  while (!ctx->problems.empty()) fo_problem_destroy(ctx->problems.back());
  while (!ctx->meshes.empty()) fo_mesh_destroy(ctx->meshes.back());
  if (ctx->h_scalars) cudaFreeHost(ctx->h_scalars);
  for (auto &e : ctx->ev)
    if (e) cudaEventDestroy(e);
  for (auto &e : ctx->ev_solve)
    if (e) cudaEventDestroy(e);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return FO_OK;
}

// One grid barrier; block `skip` never arrives, so the others run out their wait limit.
__global__ void k_barrier_selftest(GridBar bar, int skip, int *gave_up) {
  if ((int)blockIdx.x == skip) return;
  const bool ok = grid_sync(bar);
  if (threadIdx.x == 0 && !ok) atomicAdd(gave_up, 1);
}

extern "C" fo_status fo_selftest_barrier(fo_ctx *ctx, int blocks, int skip, double limit_ms, int *gave_up) {
  if (!ctx || !gave_up || !(limit_ms > 0.0 && limit_ms <= 10000.0)) return FO_EINVAL;
  const int G = std::max(2, std::min(blocks, ctx->num_sms));
  if (skip >= G) return fo_fail(ctx, FO_EINVAL, "skip must be < the number of blocks (%d)", G);
  int *words;   // [0] barrier counter, [1] error word, [2] blocks that gave up
  FO_TRY(fo_alloc(ctx, (void **)&words, 64));
  fo_status st = FO_OK;
  int h[3] = {0, 0, 0};
  if (cudaMemsetAsync(words, 0, 64, ctx->stream) != cudaSuccess) st = fo_fail(ctx, FO_ECUDA, "memset");
  if (st == FO_OK) {
    GridBar bar{reinterpret_cast<unsigned *>(words), words + 1, (unsigned long long)(limit_ms * 1e6)};
    int *out = words + 2;
    void *argv[] = {(void *)&bar, (void *)&skip, (void *)&out};
    cudaError_t e = cudaLaunchCooperativeKernel((const void *)k_barrier_selftest, G, 32, argv, 0, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, words, sizeof h, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) st = fo_cuda_check(ctx, e, "barrier self-test");
    fo_note_launch(1);
  }
  fo_free(ctx, words, 64);
  if (st != FO_OK) return st;
  *gave_up = h[2];
  if (h[1] == DEV_TIMEOUT) return fo_fail(ctx, FO_ETIMEOUT, "grid barrier gave up after %.1f ms", limit_ms);
  return FO_OK;
}

extern "C" fo_status fo_ctx_set_timing(fo_ctx *ctx, int on) {
  if (!ctx) return FO_EINVAL;
  if (on && !ctx->ev[0]) {
    for (auto &e : ctx->ev) FO_CU(ctx, cudaEventCreate(&e));
    for (auto &e : ctx->ev_solve) FO_CU(ctx, cudaEventCreate(&e));
  }
  ctx->timing = on ? 1 : 0;
  return FO_OK;
}

extern "C" fo_status fo_ctx_set_grid_share(fo_ctx *ctx, int share) {
  if (!ctx) return FO_EINVAL;
  if (share < 1 || share > 16) return fo_fail(ctx, FO_EINVAL, "grid share must be in [1, 16]");
  ctx->grid_share = share;
  return FO_OK;
}

extern "C" fo_status fo_ctx_solve_kernel_ms(const fo_ctx *ctx, double *ms) {
  if (!ctx || !ms) return FO_EINVAL;
  *ms = ctx->last_solve_ms;
  return FO_OK;
}

extern "C" const char *fo_last_error(const fo_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

extern "C" fo_status fo_ctx_memory(const fo_ctx *ctx, size_t *bytes) {
  if (!ctx || !bytes) return FO_EINVAL;
  *bytes = ctx->in_use;
  return FO_OK;
}

extern "C" fo_status fo_ctx_sync(fo_ctx *ctx) {
  if (!ctx) return FO_EINVAL;
  FO_CU(ctx, cudaStreamSynchronize(ctx->stream));
  return FO_OK;
}

// ---------------------------------------------------------------------------------- mesh
static double mesh_diameter(const Grid &g) {
  double D = 1.0;
  for (int a = 0; a < g.dim; ++a) D *= g.hi[a] - g.lo[a];
  double NT = (double)g.num_elems;
  if (g.dim == 2) return std::sqrt(4.0 * D / (NT * std::sqrt(3.0)));
  return std::sqrt(std::pow(6.0 * std::sqrt(2.0) * D / NT, 2.0 / 3.0));
}

// The structured Kuhn grid of the box (lo, hi) with n cells per axis; false on bad extents or
// more nodes than int32 connectivity allows.
bool fo_grid_make(int dim, const int n[3], const double lo[3], const double hi[3], Grid &g) {
  g = Grid{};
  g.dim = dim;
  long long nodes = 1, cells = 1;
  for (int a = 0; a < 3; ++a) {
    if (a < dim) {
      if (n[a] < 1 || !(hi[a] > lo[a])) return false;
      g.n[a] = n[a];
      g.lo[a] = lo[a];
      g.hi[a] = hi[a];
    } else {
      g.n[a] = 1;
      g.lo[a] = 0;
      g.hi[a] = 1;
    }
    g.nn[a] = (a < dim) ? (long long)g.n[a] + 1 : 1;
    g.h[a] = (g.hi[a] - g.lo[a]) / g.n[a];
    g.inv_h[a] = 1.0 / g.h[a];
  }
  g.stride[0] = 1;
  g.stride[1] = g.nn[0];
  g.stride[2] = g.nn[0] * g.nn[1];
  g.cstride[0] = 1;
  g.cstride[1] = g.n[0];
  g.cstride[2] = (long long)g.n[0] * g.n[1];
  for (int a = 0; a < dim; ++a) {
    nodes *= g.nn[a];
    cells *= g.n[a];
  }
  if (nodes > (1ll << 31) - 1) return false;
  g.num_nodes = nodes;
  g.num_cells = cells;
  g.num_elems = cells * (dim == 2 ? 2 : 6);
  g.vol_e = (dim == 2) ? g.h[0] * g.h[1] / 2.0 : g.h[0] * g.h[1] * g.h[2] / 6.0;
  for (int a = 0; a < 3; ++a) {
    if (dim == 2) g.facet_area[a] = g.h[1 - (a & 1)];
    else {
      int o1 = (a + 1) % 3, o2 = (a + 2) % 3;
      g.facet_area[a] = g.h[o1] * g.h[o2] / 2.0;
    }
  }
  return true;
}

extern "C" fo_status fo_mesh_box(fo_ctx *ctx, int dim, const int n[3], const double lo[3], const double hi[3],
                                 fo_mesh **out) {
  if (!ctx || !out || !n || !lo || !hi) return FO_EINVAL;
  *out = nullptr;
  if (dim != 2 && dim != 3) return fo_fail(ctx, FO_EINVAL, "dim must be 2 or 3");
  Grid g{};
  if (!fo_grid_make(dim, n, lo, hi, g)) return fo_fail(ctx, FO_EINVAL, "bad extents or mesh too large");
  fo_mesh *m = new fo_mesh();
  m->ctx = ctx;
  m->g = g;
  m->h_diam = mesh_diameter(g);
  fo_status st = fo_alloc(ctx, (void **)&m->d_cells, sizeof(int32_t) * g.num_elems * (dim + 1));
  if (st == FO_OK) st = fo_alloc(ctx, (void **)&m->d_coords, sizeof(double) * g.num_nodes * dim);
  if (st == FO_OK) st = fo_launch_mesh_build(m);
  if (st != FO_OK) {
    fo_free(ctx, m->d_cells, sizeof(int32_t) * g.num_elems * (dim + 1));
    fo_free(ctx, m->d_coords, sizeof(double) * g.num_nodes * dim);
    delete m;
    return st;
  }
  ctx->meshes.push_back(m);
  *out = m;
  return FO_OK;
}

extern "C" fo_status fo_mesh_from_arrays(fo_ctx *ctx, int dim, int64_t nn, const double *coords, int64_t nt,
                                        const int32_t *cells, fo_mesh **out) {
  if (!ctx || !out || !coords || !cells) return FO_EINVAL;
  *out = nullptr;
  if (dim != 2 && dim != 3) return fo_fail(ctx, FO_EINVAL, "dim must be 2 or 3");
  if (nn < dim + 1 || nt < 1 || nn > (1ll << 31) - 1 || nt * (dim + 1) > (1ll << 31) - 1)
    return fo_fail(ctx, FO_EINVAL, "bad node or element count");
  for (int64_t i = 0; i < nt * (dim + 1); ++i)
    if (cells[i] < 0 || cells[i] >= nn) return fo_fail(ctx, FO_EINVAL, "vertex id %d out of range", (int)cells[i]);
  for (int64_t i = 0; i < nn * dim; ++i)
    if (!std::isfinite(coords[i])) return fo_fail(ctx, FO_ENAN, "non-finite coordinate");
  fo_mesh *m = new fo_mesh();
  m->ctx = ctx;
  Grid &g = m->g;
  g = Grid{};
  g.dim = dim;
  g.num_nodes = nn;
  g.num_elems = nt;
  g.num_cells = 0;
  m->um = new fo_umesh();
  m->um->dim = dim;
  m->um->nn = nn;
  m->um->nt = nt;
  fo_status st = fo_alloc(ctx, (void **)&m->d_cells, sizeof(int32_t) * nt * (dim + 1));
  if (st == FO_OK) st = fo_alloc(ctx, (void **)&m->d_coords, sizeof(double) * nn * dim);
  if (st == FO_OK)
    st = fo_cuda_check(ctx, cudaMemcpyAsync(m->d_cells, cells, sizeof(int32_t) * nt * (dim + 1), cudaMemcpyHostToDevice,
                                            ctx->stream), "copy cells");
  if (st == FO_OK)
    st = fo_cuda_check(ctx, cudaMemcpyAsync(m->d_coords, coords, sizeof(double) * nn * dim, cudaMemcpyHostToDevice,
                                            ctx->stream), "copy coords");
  if (st == FO_OK) st = fo_umesh_build(m, coords, cells);
  if (st == FO_OK) st = fo_cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "mesh setup");
  if (st != FO_OK) {
    fo_umesh_release(m);
    fo_free(ctx, m->d_cells, sizeof(int32_t) * nt * (dim + 1));
    fo_free(ctx, m->d_coords, sizeof(double) * nn * dim);
    delete m;
    return st;
  }
  for (int a = 0; a < 3; ++a) {
    g.lo[a] = a < dim ? m->um->lo[a] : 0.0;
    g.hi[a] = a < dim ? m->um->hi[a] : 0.0;
    g.n[a] = 0;
  }
  const double D = m->um->volume;
  m->h_diam = dim == 2 ? std::sqrt(4.0 * D / ((double)nt * std::sqrt(3.0)))
                       : std::sqrt(std::pow(6.0 * std::sqrt(2.0) * D / (double)nt, 2.0 / 3.0));
  ctx->meshes.push_back(m);
  *out = m;
  return FO_OK;
}

extern "C" fo_status fo_mesh_destroy(fo_mesh *m) {
  if (!m) return FO_EINVAL;
  fo_ctx *ctx = m->ctx;
  cudaStreamSynchronize(ctx->stream);
  for (size_t i = 0; i < ctx->problems.size();) {
    if (ctx->problems[i]->mesh == m) fo_problem_destroy(ctx->problems[i]);
    else ++i;
  }
  const Grid &g = m->g;
  fo_umesh_release(m);
  fo_free(ctx, m->d_cells, sizeof(int32_t) * g.num_elems * (g.dim + 1));
  fo_free(ctx, m->d_coords, sizeof(double) * g.num_nodes * g.dim);
  ctx->meshes.erase(std::remove(ctx->meshes.begin(), ctx->meshes.end(), m), ctx->meshes.end());
  delete m;
  return FO_OK;
}

extern "C" fo_status fo_mesh_query(const fo_mesh *m, fo_mesh_info *out) {
  if (!m || !out) return FO_EINVAL;
  const Grid &g = m->g;
  memset(out, 0, sizeof *out);
  out->dim = g.dim;
  double D = 1;
  for (int a = 0; a < 3; ++a) {
    out->n[a] = a < g.dim ? g.n[a] : 0;
    out->lo[a] = a < g.dim ? g.lo[a] : 0;
    out->hi[a] = a < g.dim ? g.hi[a] : 0;
    if (a < g.dim) D *= g.hi[a] - g.lo[a];
  }
  out->num_nodes = g.num_nodes;
  out->num_cells = g.num_cells;
  out->num_elems = g.num_elems;
  out->volume = m->um ? m->um->volume : D;
  out->h = m->h_diam;
  return FO_OK;
}

extern "C" fo_status fo_mesh_copy_out(const fo_mesh *m, int32_t *cells, double *coords) {
  if (!m) return FO_EINVAL;
  fo_ctx *ctx = m->ctx;
  const Grid &g = m->g;
  if (cells)
    FO_CU(ctx, cudaMemcpyAsync(cells, m->d_cells, sizeof(int32_t) * g.num_elems * (g.dim + 1),
                               cudaMemcpyDeviceToHost, ctx->stream));
  if (coords)
    FO_CU(ctx, cudaMemcpyAsync(coords, m->d_coords, sizeof(double) * g.num_nodes * g.dim, cudaMemcpyDeviceToHost,
                               ctx->stream));
  FO_CU(ctx, cudaStreamSynchronize(ctx->stream));
  return FO_OK;
}

// ------------------------------------------------------------------------------- problem
// Sizes of a problem's device fields, in the order of prob_bytes_fields.
// `entries`: stored operator entries per block slot -- S N_n on the structured grid (S stencil
// slots per node), the node graph's nonzeros on a general mesh; `vel_blk`: entries per velocity
// block (d: component-diagonal on the box grid; d^2 on a general mesh).
// entries: stencil entries of the transport rows (all slots, or the general mesh's CSR);
// rows: those of the stored symmetric state and velocity rows (the stored slots, or the CSR).
static std::vector<size_t> problem_field_sizes(int d, long long NN, long long NT, long long ND, bool with_f,
                                               long long entries, long long rows, int vel_blk, int ncases = 1) {
  const size_t E = (size_t)entries, ER = (size_t)rows;
  const size_t npn = (size_t)(ND / NN);   // state components per node
  std::vector<size_t> v = {
      sizeof(double) * ER * npn * npn, sizeof(float) * ER * npn * npn, sizeof(double) * ER * vel_blk,
      sizeof(double) * NN,     sizeof(double) * NT,     sizeof(float) * NT,       (size_t)NT,
      (size_t)NT,              (size_t)ND,              (size_t)NN,               sizeof(double) * ND * ncases,
      sizeof(double) * ND * ncases, sizeof(double) * ND * ncases, sizeof(double) * d * NN, sizeof(double) * d * NN,
      sizeof(double) * ND,     sizeof(float) * ND,      sizeof(double) * d * NN,  sizeof(double) * E,
      sizeof(double) * E,      sizeof(double) * NN,     sizeof(double) * FO_RED_DOUBLES,
      64,                      sizeof(int) * DS_COUNT,  sizeof(double) * NT,     (size_t)NT,
  };
  if (with_f) v.push_back(sizeof(double) * NN);
  return v;
}

static size_t prob_bytes_fields(const fo_problem *p, std::vector<std::pair<void **, size_t>> &list) {
  const Grid &g = p->mesh->g;
  const long long entries = p->mesh->um ? p->mesh->um->nnz : (long long)(g.dim == 2 ? 7 : 15) * g.num_nodes;
  const long long rows = p->mesh->um ? p->mesh->um->nnz : (long long)fo_row_slots(g.dim) * g.num_nodes;
  const std::vector<size_t> sz = problem_field_sizes(g.dim, g.num_nodes, g.num_elems, p->ndof,
                                                     p->f || p->desc.kind != FO_ELASTIC, entries, rows,
                                                     p->mesh->um ? g.dim * g.dim : g.dim, p->ncases);
  std::vector<void **> ptr = {
      (void **)&p->Wst,        (void **)&p->Wst32,        (void **)&p->Wvel,
      (void **)&p->phi,        (void **)&p->coef,         (void **)&p->coef32,       (void **)&p->chi,
      (void **)&p->omega0,     (void **)&p->dir,          (void **)&p->vdir,         (void **)&p->load,
      (void **)&p->u,          (void **)&p->p,            (void **)&p->rhs,          (void **)&p->theta,
      (void **)&p->dinv_state, (void **)&p->dinv_state32, (void **)&p->dinv_vel,     (void **)&p->L,
      (void **)&p->R,          (void **)&p->dinvL,        (void **)&p->red,
      (void **)&p->bar,        (void **)&p->dev_status,   (void **)&p->chif,         (void **)&p->regmask,
  };
  if (sz.size() > ptr.size()) ptr.push_back((void **)&p->f);
  list.clear();
  size_t s = 0;
  for (size_t i = 0; i < sz.size(); ++i) {
    list.push_back({ptr[i], sz[i]});
    s += sz[i];
  }
  return s;
}

// Device bytes allocated for a box mesh and a single (non-batch) problem on it, with the
// largest solver scratch of its state / adjoint and velocity solves (state_vecs, vel_vecs
// FP64 vectors of their systems) and the transient bump-centre array; what a served request
// holds at most, multigrid hierarchies aside.
size_t fo_problem_footprint(int dim, const int n[3], int kind, int state_vecs, int vel_vecs, int n_bumps) {
  long long NN = 1, cells = 1;
  for (int a = 0; a < dim; ++a) {
    NN *= (long long)n[a] + 1;
    cells *= n[a];
  }
  const long long NT = cells * (dim == 2 ? 2 : 6);
  const long long ND = NN * (kind == FO_ELASTIC ? dim : 1);
  size_t total = sizeof(int32_t) * NT * (dim + 1) + sizeof(double) * NN * dim;   // mesh
  for (size_t b : problem_field_sizes(dim, NN, NT, ND, kind != FO_ELASTIC, (dim == 2 ? 7 : 15) * NN,
                                      (long long)fo_row_slots(dim) * NN, dim))
    total += b;
  const size_t state = sizeof(double) * state_vecs * (size_t)ND;
  const size_t vel = sizeof(double) * vel_vecs * (size_t)dim * NN;
  const size_t bumps = sizeof(double) * (size_t)std::max(n_bumps, 0) * dim;
  return total + std::max(std::max(state, vel), bumps);
}

extern "C" fo_status fo_problem_destroy(fo_problem *p) {
  if (!p) return FO_EINVAL;
  fo_ctx *ctx = p->ctx;
  cudaStreamSynchronize(ctx->stream);
  fo_batch_destroy(p);
  fo_inverse_destroy(p);
  fo_mg_destroy(p);
  std::vector<std::pair<void **, size_t>> list;
  prob_bytes_fields(p, list);
  for (auto &e : list) {
    fo_free(ctx, *e.first, e.second);
    *e.first = nullptr;
  }
  fo_free(ctx, p->scratch.buf, p->scratch.bytes);
  ctx->problems.erase(std::remove(ctx->problems.begin(), ctx->problems.end(), p), ctx->problems.end());
  delete p;
  return FO_OK;
}

extern "C" fo_status fo_problem_create(fo_mesh *m, const fo_model_desc *desc, fo_problem **out) {
  if (!m || !desc || !out) return FO_EINVAL;
  fo_ctx *ctx = m->ctx;
  *out = nullptr;
  if (desc->kind < FO_HEAT || desc->kind > FO_LOGISTIC) return fo_fail(ctx, FO_EINVAL, "bad model kind");
  if (desc->kind == FO_LOGISTIC &&
      (m->um || desc->n_inst > 0 || desc->n_cases > 1 || desc->n_volume > 0 || desc->coef_rule != FO_COEF_CENTROID ||
       !(desc->growth_rate > 0) || !(desc->a_in > 0) || !(desc->a_out > 0)))
    return fo_fail(ctx, FO_EINVAL,
                   "the logistic model runs on box meshes with one load case, the one-point coefficient rule, at "
                   "most one volume constraint, r > 0 and positive carrying capacities");
  if (desc->n_point_loads < 0 || desc->n_point_loads > 4 || desc->n_tractions < 0 || desc->n_tractions > 4 ||
      desc->n_omega0 < 0 || desc->n_omega0 > 4)
    return fo_fail(ctx, FO_EINVAL, "too many loads / subdomain boxes");
  const Grid &g = m->g;
  for (int i = 0; i < desc->n_point_loads; ++i)
    if (desc->point_node[i] < 0 || desc->point_node[i] >= g.num_nodes)
      return fo_fail(ctx, FO_EINVAL, "point load node out of range");
  for (int i = 0; i < desc->n_tractions; ++i)
    if (desc->traction_face[i] < 0 || desc->traction_face[i] >= 2 * g.dim)
      return fo_fail(ctx, FO_EINVAL, "bad traction face");
  if (desc->kind == FO_ELASTIC && !(desc->nu > -1.0 && desc->nu < 0.5 && desc->E > 0))
    return fo_fail(ctx, FO_EINVAL, "bad elastic parameters");
  if (desc->n_inst < 0 || (desc->n_inst > 0 && desc->kind != FO_HELMHOLTZ))
    return fo_fail(ctx, FO_EINVAL, "a task-parallel batch (n_inst > 0) is a FO_HELMHOLTZ family");
  if (desc->coef_rule != FO_COEF_CENTROID && desc->coef_rule != FO_COEF_CUT)
    return fo_fail(ctx, FO_EINVAL, "bad coefficient rule");
  if (desc->n_cases < 0 || desc->n_cases > 4 || desc->n_volume < 0 || desc->n_volume > 4)
    return fo_fail(ctx, FO_EINVAL, "at most 4 load cases and 4 volume constraints");
  for (int i = 0; i < desc->n_point_loads; ++i)
    if (desc->point_case[i] < 0 || desc->point_case[i] >= std::max(desc->n_cases, 1))
      return fo_fail(ctx, FO_EINVAL, "point load case out of range");
  for (int i = 0; i < desc->n_tractions; ++i)
    if (desc->traction_case[i] < 0 || desc->traction_case[i] >= std::max(desc->n_cases, 1))
      return fo_fail(ctx, FO_EINVAL, "traction case out of range");
  for (int j = 0; j < desc->n_volume; ++j)
    if (!(desc->volume_V[j] > 0)) return fo_fail(ctx, FO_EINVAL, "volume targets must be positive");
  if (desc->n_inst > 0 && (desc->n_cases > 1 || desc->n_volume > 0))
    return fo_fail(ctx, FO_EINVAL, "task-parallel batches take one load and at most one volume constraint");
  if (desc->n_inst > 0 && desc->coef_rule != FO_COEF_CENTROID)
    return fo_fail(ctx, FO_EINVAL, "task-parallel batches take the one-point coefficient rule");
  if (m->um && desc->n_inst > 0)
    return fo_fail(ctx, FO_EINVAL, "task-parallel batches run on box meshes (fo_mesh_box)");
  if (desc->inverse &&
      (desc->kind != FO_ELASTIC || m->um || desc->n_inst > 0 || desc->coef_rule != FO_COEF_CENTROID ||
       desc->n_volume > 0 || desc->volume_target > 0 || !desc->meas || !(desc->kv_alpha >= 0) || !(desc->kv_beta >= 0)))
    return fo_fail(ctx, FO_EINVAL,
                   "inverse elasticity: FO_ELASTIC on a box mesh, one-point rule, no constraint, measurements given, "
                   "alpha, beta >= 0");
  fo_problem *p = new fo_problem();
  p->ctx = ctx;
  p->mesh = m;
  p->desc = *desc;
  p->desc.f_nodal = nullptr;
  p->ncomp = desc->kind == FO_ELASTIC ? g.dim : 1;
  p->ndof = g.num_nodes * p->ncomp;
  p->ncases = std::max(desc->n_cases, 1);
  p->nvol = desc->n_volume;
  if (desc->kind == FO_ELASTIC) {
    p->lame_lambda = desc->E * desc->nu / ((1.0 + desc->nu) * (1.0 - 2.0 * desc->nu));
    p->lame_mu = desc->E / (2.0 * (1.0 + desc->nu));
  }
  if (desc->kind == FO_HELMHOLTZ && !(desc->k > 0)) p->desc.k = 1.0;
  if (desc->kind == FO_HEAT || desc->kind == FO_LOGISTIC) p->desc.k = 1.0;
  p->desc.u_init = nullptr;
  p->desc.inst_k = p->desc.inst_omega = p->desc.inst_f = nullptr;
  p->desc.meas = nullptr;   // copied by fo_inverse_create
  if (desc->n_inst > 0) {   // batch: A_e alone in coef; k_i, omega_i, f_i per instance
    p->desc.k = 1.0;
    p->desc.omega = 0.0;
  }
  std::vector<std::pair<void **, size_t>> list;
  prob_bytes_fields(p, list);
  fo_status st = FO_OK;
  for (auto &e : list) {
    st = fo_alloc(ctx, e.first, e.second);
    if (st != FO_OK) break;
  }
  ctx->problems.push_back(p);
  if (st == FO_OK && p->f && desc->kind == FO_LOGISTIC) {   // f holds the initial Newton guess
    std::vector<double> u0;
    const double *src = desc->u_init;
    if (!src) {
      u0.assign((size_t)g.num_nodes, desc->a_in);
      src = u0.data();
    }
    st = fo_cuda_check(ctx, cudaMemcpyAsync(p->f, src, sizeof(double) * g.num_nodes, cudaMemcpyHostToDevice,
                                            ctx->stream), "copy u_init");
    if (st == FO_OK) st = fo_cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "copy u_init");
  } else if (st == FO_OK && p->f) {
    if (desc->f_nodal)
      st = fo_cuda_check(ctx, cudaMemcpyAsync(p->f, desc->f_nodal, sizeof(double) * g.num_nodes,
                                              cudaMemcpyHostToDevice, ctx->stream), "copy f");
    else
      st = fo_cuda_check(ctx, cudaMemsetAsync(p->f, 0, sizeof(double) * g.num_nodes, ctx->stream), "zero f");
  }
  if (st == FO_OK) st = fo_cuda_check(ctx, cudaMemsetAsync(p->phi, 0, sizeof(double) * g.num_nodes, ctx->stream), "phi");
  if (st == FO_OK)
    st = fo_cuda_check(ctx, cudaMemsetAsync(p->u, 0, sizeof(double) * p->ndof * p->ncases, ctx->stream), "u");
  if (st == FO_OK) st = fo_cuda_check(ctx, cudaMemsetAsync(p->theta, 0, sizeof(double) * g.dim * g.num_nodes, ctx->stream), "theta");
  if (m->um) {
    if (st == FO_OK) st = fo_umesh_masks(p);
    if (st == FO_OK) st = fo_umesh_loads(p);
    if (st == FO_OK) st = fo_umesh_velocity_setup(p);
  } else {
    if (st == FO_OK) st = fo_launch_masks(p);
    if (st == FO_OK) st = fo_launch_loads(p);
    if (st == FO_OK) st = fo_launch_velocity_diag(p);
  }
  if (st == FO_OK && desc->n_inst > 0) st = fo_batch_create(p, desc);
  if (st == FO_OK && desc->inverse) st = fo_inverse_create(p, desc);
  if (st == FO_OK) st = fo_cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "problem setup");
  if (st != FO_OK) {
    fo_problem_destroy(p);
    return st;
  }
  *out = p;
  return FO_OK;
}

static fo_status copy_in(fo_problem *p, double *dst, const double *src, size_t n, int on_device) {
  fo_ctx *ctx = p->ctx;
  if (!src) return fo_fail(ctx, FO_EINVAL, "null input");
  FO_CU(ctx, cudaMemcpyAsync(dst, src, sizeof(double) * n,
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream));
  if (!on_device) FO_CU(ctx, cudaStreamSynchronize(ctx->stream));   // host buffer may be reused
  return FO_OK;
}

extern "C" fo_status fo_set_levelset(fo_problem *p, const double *phi, int on_device) {
  if (!p) return FO_EINVAL;
  FO_TRY(copy_in(p, p->phi, phi, p->mesh->g.num_nodes, on_device));
  p->coef_valid = false;
  return FO_OK;
}

extern "C" fo_status fo_initial_level(fo_problem *p, int count, const double *centers, const double *radii,
                                      double factor, int ord) {
  if (!p || count < 1 || !centers || !radii || (ord != 2 && ord != 0)) return FO_EINVAL;
  p->coef_valid = false;
  return fo_launch_initial_level(p, count, centers, radii, factor, ord);
}

extern "C" fo_status fo_levelset_bumps(fo_problem *p, int count, const double *centers, double width,
                                       double offset) {
  if (!p || count < 1 || !centers || !(width > 0)) return FO_EINVAL;
  p->coef_valid = false;
  return fo_launch_phi_bumps(p, count, centers, width, offset);
}

extern "C" fo_status fo_coefficients(fo_problem *p) {
  if (!p) return FO_EINVAL;
  if (p->mesh->um) {   // general mesh: coefficients and the assembled state operator
    FO_TRY(fo_umesh_coefficients(p));
    p->coef_valid = true;
    p->coef_epoch += 1;
    return FO_OK;
  }
  FO_TRY(fo_launch_coefficients(p));
  if (p->batch) FO_TRY(fo_batch_prepare(p));
  else if (p->desc.kind != FO_LOGISTIC) FO_TRY(fo_launch_state_diag(p));   // logistic: rows per Newton step
  p->coef_valid = true;
  p->coef_epoch += 1;
  return FO_OK;
}

extern "C" fo_status fo_state_solve(fo_problem *p, const fo_solve_opts *o, fo_solve_stats *st) {
  if (!p) return FO_EINVAL;
  fo_solve_opts def;
  fo_solve_opts_default(&def);
  if (!o) o = &def;
  if (!p->coef_valid) FO_TRY(fo_coefficients(p));
  p->ctx->last_solve_ms = 0.0;
  fo_status s;
  if (p->batch) s = fo_batch_state(p, false, o, st);
  else if (p->desc.kind == FO_LOGISTIC) s = fo_logistic_state(p, o, st, &p->newton_steps);
  else if (p->inv) s = fo_inverse_states(p, o, st);
  else if (p->ncases == 1) s = fo_state_pcg(p, p->load, p->u, o, st);
  else {   // one solve per load case (eq. compli_plus); statistics summed, worst residual kept
    fo_solve_stats tot;
    memset(&tot, 0, sizeof tot);
    s = FO_OK;
    for (int k = 0; k < p->ncases && (s == FO_OK || s == FO_ENOCONV); ++k) {
      fo_solve_stats sk;
      memset(&sk, 0, sizeof sk);
      const fo_status sk_st = fo_state_pcg(p, p->load + (size_t)k * p->ndof, p->u + (size_t)k * p->ndof, o, &sk);
      if (sk_st != FO_OK) s = sk_st;
      tot.iterations += sk.iterations;
      tot.outer_iterations += sk.outer_iterations;
      tot.operator_applies += sk.operator_applies;
      tot.rel_residual = std::max(tot.rel_residual, sk.rel_residual);
    }
    if (st) *st = tot;
  }
  if (s == FO_OK || s == FO_ENOCONV) p->u_valid = true;
  return s;
}

__global__ void k_scale(const double *__restrict__ x, double *__restrict__ y, double c, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = c * x[i];
}

extern "C" fo_status fo_adjoint_solve(fo_problem *p, const fo_solve_opts *o, fo_solve_stats *st) {
  if (!p) return FO_EINVAL;
  fo_solve_opts def;
  fo_solve_opts_default(&def);
  if (!o) o = &def;
  if (!p->coef_valid) FO_TRY(fo_coefficients(p));
  if (p->batch) return fo_batch_state(p, true, o, st);
  if (p->desc.kind == FO_LOGISTIC) return fo_logistic_adjoint(p, o, st);
  if (p->inv) return fo_inverse_adjoints(p, o, st);
  double c = p->desc.kind == FO_ELASTIC ? -2.0 : -1.0;
  double *b = p->rhs;   // reuse the RHS buffer as the adjoint load (d*N_n >= N_dof)
  fo_solve_opts oo = *o;
  oo.warm_start = 0;
  fo_status s = FO_OK;
  for (int k = 0; k < p->ncases && s == FO_OK; ++k) {   // one adjoint per load case
    k_scale<<<fo_blocks_for(p->ndof), FO_BLOCK, 0, p->ctx->stream>>>(p->load + (size_t)k * p->ndof, b, c, p->ndof);
    fo_note_launch(1);
    FO_CU(p->ctx, cudaGetLastError());
    s = fo_state_pcg(p, b, p->p + (size_t)k * p->ndof, &oo, st);
  }
  p->rhs_valid = false;
  return s;
}

// Number of constraints of a problem: the region constraints, else |Omega| / V when V > 0.
static int problem_nc(const fo_problem *p) { return p->nvol > 0 ? p->nvol : (p->desc.volume_target > 0 ? 1 : 0); }

// J summed over the load cases and |Omega|.
static fo_status cost_and_volume(fo_problem *p, double *J, double *vol) {
  if (!p->coef_valid) FO_TRY(fo_coefficients(p));
  double j = 0, v = 0;
  if (p->batch) FO_TRY(fo_batch_functionals(p, &j, &v, nullptr));
  else
    for (int k = 0; k < p->ncases; ++k) {
      double jk = 0;
      const double *u = p->u + (size_t)k * p->ndof, *F = p->load + (size_t)k * p->ndof;
      if (p->mesh->um) FO_TRY(fo_umesh_functionals_on(p, u, F, &jk, &v));
      else FO_TRY(fo_launch_functionals_on(p, u, F, &jk, &v));
      j += jk;
    }
  if (p->inv) FO_TRY(fo_inverse_cost(p, &j));   // the Kohn-Vogelius cost (|Omega| as computed)
  if (!std::isfinite(j) || !std::isfinite(v)) return fo_fail(p->ctx, FO_ENAN, "non-finite functional");
  *J = j;
  *vol = v;
  return FO_OK;
}

extern "C" fo_status fo_functionals(fo_problem *p, double *J, double *C) {
  if (!p) return FO_EINVAL;
  double j = 0, vol = 0;
  FO_TRY(cost_and_volume(p, &j, &vol));
  if (J) *J = j;
  if (C) {
    if (p->nvol > 0) {
      double c[4];
      FO_TRY(fo_functionals_v(p, nullptr, c, p->nvol));
      *C = c[0];
    } else {
      *C = p->desc.volume_target > 0 ? vol / p->desc.volume_target : vol;
    }
  }
  return FO_OK;
}

extern "C" fo_status fo_functionals_v(fo_problem *p, double *J, double *C, int nc) {
  if (!p) return FO_EINVAL;
  if (nc != problem_nc(p) || (nc > 0 && !C))
    return fo_fail(p->ctx, FO_EINVAL, "the problem has %d constraints", problem_nc(p));
  double j = 0, vol = 0;
  FO_TRY(cost_and_volume(p, &j, &vol));
  if (J) *J = j;
  if (p->nvol > 0) {
    double rv[4];
    FO_TRY(fo_region_volumes(p, p->mesh->um ? p->mesh->um->vol : nullptr, rv));
    for (int q = 0; q < p->nvol; ++q) C[q] = rv[q] / p->desc.volume_V[q];
  } else if (nc == 1) {
    C[0] = vol / p->desc.volume_target;
  }
  return FO_OK;
}

extern "C" fo_status fo_shape_derivative_v(fo_problem *p, const double *lambda, int nc, double *rhs_out) {
  if (!p) return FO_EINVAL;
  if (nc != problem_nc(p) || (nc > 0 && !lambda))
    return fo_fail(p->ctx, FO_EINVAL, "the problem has %d constraints", problem_nc(p));
  if (p->batch || p->inv || (p->ncases == 1 && p->nvol == 0)) return fo_shape_derivative(p, nc ? lambda[0] : 0.0, rhs_out);
  if (!p->coef_valid) FO_TRY(fo_coefficients(p));
  fo_ctx *ctx = p->ctx;
  const Grid &g = p->mesh->g;
  const long long NN = g.num_nodes, NT = g.num_elems;
  // zero state and source (for the constraint terms and the source-free cases) and one weight array
  double *z;
  FO_TRY(fo_scratch(p, sizeof(double) * (std::max<long long>(p->ndof, NN) + NT), (void **)&z));
  double *w = z + std::max<long long>(p->ndof, NN);
  FO_CU(ctx, cudaMemsetAsync(z, 0, sizeof(double) * std::max<long long>(p->ndof, NN), ctx->stream));
  const double *chif = p->desc.coef_rule == FO_COEF_CUT ? p->chif : nullptr;
  const double invV = p->desc.volume_target > 0 ? 1.0 / p->desc.volume_target : 1.0;
  auto shape = [&](const double *u, const double *f, double lam, const double *wt, double iv, int add) {
    return p->mesh->um ? fo_umesh_shape_rhs_ex(p, u, f, lam, wt, iv, add) : fo_launch_shape_rhs_ex(p, u, f, lam, wt, iv, add);
  };
  for (int k = 0; k < p->ncases; ++k) {   // sum_k b^J(u_k) (+ lambda b^C with one constraint)
    const double lam = (p->nvol == 0 && k == 0 && nc == 1) ? lambda[0] : 0.0;
    const double *f = (k == 0) ? p->f : z;
    FO_TRY(shape(p->u + (size_t)k * p->ndof, f ? f : z, lam, chif, invV, k > 0));
  }
  for (int q = 0; q < p->nvol; ++q) {     // + lambda_j b^C_j: S1 = chi chi_Rj / V_j I (u = 0)
    if (lambda[q] == 0.0) continue;
    FO_TRY(fo_region_weight(p, q, w));
    FO_TRY(shape(z, z, lambda[q], w, 1.0 / p->desc.volume_V[q], 1));
  }
  p->rhs_valid = true;
  p->last_lambda = nc ? lambda[0] : 0.0;
  if (rhs_out) {
    FO_CU(ctx, cudaMemcpyAsync(rhs_out, p->rhs, sizeof(double) * g.dim * NN, cudaMemcpyDeviceToHost, ctx->stream));
    FO_CU(ctx, cudaStreamSynchronize(ctx->stream));
  }
  return FO_OK;
}

extern "C" fo_status fo_shape_derivative(fo_problem *p, double lambda, double *rhs_out) {
  if (!p) return FO_EINVAL;
  if (!p->batch && !p->inv && (p->ncases > 1 || p->nvol > 0)) {   // one multiplier: the first constraint's
    double lv[4] = {lambda, 0, 0, 0};
    return fo_shape_derivative_v(p, lv, problem_nc(p), rhs_out);
  }
  if (!p->coef_valid) FO_TRY(fo_coefficients(p));
  if (p->batch) FO_TRY(fo_batch_shape_rhs(p, lambda));
  else if (p->inv) FO_TRY(fo_inverse_shape(p));
  else if (p->desc.kind == FO_LOGISTIC)
    FO_TRY(fo_launch_logistic_shape(p, lambda, nullptr, p->desc.volume_target > 0 ? 1.0 / p->desc.volume_target : 1.0, 0));
  else if (p->mesh->um) FO_TRY(fo_umesh_shape_rhs(p, lambda));
  else FO_TRY(fo_launch_shape_rhs(p, lambda));
  p->rhs_valid = true;
  p->last_lambda = lambda;
  if (rhs_out) {
    const Grid &g = p->mesh->g;
    FO_CU(p->ctx, cudaMemcpyAsync(rhs_out, p->rhs, sizeof(double) * g.dim * g.num_nodes, cudaMemcpyDeviceToHost,
                                  p->ctx->stream));
    FO_CU(p->ctx, cudaStreamSynchronize(p->ctx->stream));
  }
  return FO_OK;
}

extern "C" fo_status fo_descent(fo_problem *p, const fo_solve_opts *o, double *Btt, fo_solve_stats *st) {
  if (!p) return FO_EINVAL;
  if (!p->rhs_valid) return fo_fail(p->ctx, FO_ESTATE, "fo_descent needs fo_shape_derivative first");
  fo_solve_opts def;
  fo_solve_opts_default(&def);
  if (!o) o = &def;
  double btt = 0;
  fo_status s = fo_velocity_pcg(p, o, &btt, st);
  if (Btt) *Btt = btt;
  if (s == FO_OK || s == FO_ENOCONV) p->theta_valid = true;
  p->transport_valid = false;
  return s;
}

extern "C" fo_status fo_transport_assemble(fo_problem *p, double dt, double h, int smooth) {
  if (!p || !(dt > 0) || !(h > 0)) return FO_EINVAL;
  if (p->mesh->um) FO_TRY(fo_umesh_transport_assemble(p, dt, h, smooth));
  else FO_TRY(fo_launch_transport_assemble(p, dt, h, smooth));
  p->transport_valid = true;
  p->transport_dt = dt;
  p->transport_h = h;
  p->transport_smooth = smooth;
  return FO_OK;
}

extern "C" fo_status fo_levelset_step(fo_problem *p, double t_end, int nsteps, double h, int smooth,
                                      const fo_solve_opts *o, fo_solve_stats *st) {
  if (!p || nsteps < 1 || !(t_end > 0) || !(h > 0)) return FO_EINVAL;
  fo_solve_opts def;
  fo_solve_opts_default(&def);
  if (!o) o = &def;
  double dt = t_end / nsteps;
  if (p->mesh->um) {   // general mesh: assembly and all substeps' BiCGStab solves
    fo_status s = fo_umesh_levelset_step(p, t_end, nsteps, h, smooth, o, st);
    p->transport_valid = true;
    p->transport_dt = dt;
    p->transport_h = h;
    p->transport_smooth = smooth;
    p->coef_valid = false;
    return s;
  }
  if (!(p->transport_valid && p->transport_dt == dt && p->transport_h == h && p->transport_smooth == smooth))
    FO_TRY(fo_transport_assemble(p, dt, h, smooth));
  fo_status s = fo_transport_run(p, nsteps, o, st);
  p->coef_valid = false;
  return s;
}

extern "C" fo_status fo_reinit(fo_problem *p, int nsteps, double t_final, double h, const fo_solve_opts *o,
                               fo_solve_stats *st) {
  if (!p || nsteps < 1 || !(t_final > 0) || !(h > 0)) return FO_EINVAL;
  fo_solve_opts def;
  fo_solve_opts_default(&def);
  if (!o) o = &def;
  fo_status s = p->mesh->um ? fo_umesh_reinit(p, nsteps, t_final, h, o, st)
                            : fo_reinit_run(p, nsteps, t_final / nsteps, h, o, st);
  p->coef_valid = false;
  return s;
}

// Batched fields (U, P, LOAD of a task-parallel batch) are [N_n][nip] on the device, with
// instance i in lane lane_of[i], and [N_n][n_inst] in the caller's order at the interface.
static double *batch_field(fo_problem *p, int field) {
  if (!p->batch) return nullptr;
  switch (field) {
    case FO_FIELD_U: return p->batch->U;
    case FO_FIELD_P: return p->batch->P;
    case FO_FIELD_LOAD: return p->batch->B;
    default: return nullptr;
  }
}

static fo_status batch_to_host(fo_problem *p, const double *dev, double *out, int on_device) {
  fo_ctx *ctx = p->ctx;
  const size_t NN = (size_t)p->mesh->g.num_nodes, nip = p->batch->nip, n = p->batch->n_inst;
  std::vector<double> tmp(NN * nip), outv;
  FO_CU(ctx, cudaMemcpyAsync(tmp.data(), dev, sizeof(double) * NN * nip, cudaMemcpyDeviceToHost, ctx->stream));
  FO_CU(ctx, cudaStreamSynchronize(ctx->stream));
  double *dst = out;
  if (on_device) {
    outv.resize(NN * n);
    dst = outv.data();
  }
  const std::vector<int> &lane = p->batch->lane_of;
  for (size_t a = 0; a < NN; ++a)
    for (size_t i = 0; i < n; ++i) dst[a * n + i] = tmp[a * nip + lane[i]];
  if (on_device) {
    FO_CU(ctx, cudaMemcpyAsync(out, dst, sizeof(double) * NN * n, cudaMemcpyHostToDevice, ctx->stream));
    FO_CU(ctx, cudaStreamSynchronize(ctx->stream));
  }
  return FO_OK;
}

static fo_status batch_from_host(fo_problem *p, double *dev, const double *v, int on_device) {
  fo_ctx *ctx = p->ctx;
  const size_t NN = (size_t)p->mesh->g.num_nodes, nip = p->batch->nip, n = p->batch->n_inst;
  std::vector<double> in, tmp(NN * nip, 0.0);
  const double *src = v;
  if (on_device) {
    in.resize(NN * n);
    FO_CU(ctx, cudaMemcpyAsync(in.data(), v, sizeof(double) * NN * n, cudaMemcpyDeviceToHost, ctx->stream));
    FO_CU(ctx, cudaStreamSynchronize(ctx->stream));
    src = in.data();
  }
  const std::vector<int> &lane = p->batch->lane_of;
  for (size_t a = 0; a < NN; ++a)
    for (size_t i = 0; i < n; ++i) tmp[a * nip + lane[i]] = src[a * n + i];
  FO_CU(ctx, cudaMemcpyAsync(dev, tmp.data(), sizeof(double) * NN * nip, cudaMemcpyHostToDevice, ctx->stream));
  FO_CU(ctx, cudaStreamSynchronize(ctx->stream));
  return FO_OK;
}

static double *field_ptr(fo_problem *p, int field, size_t *n, bool *is_u8) {
  const Grid &g = p->mesh->g;
  *is_u8 = false;
  switch (field) {
    case FO_FIELD_PHI: *n = g.num_nodes; return p->phi;
    case FO_FIELD_U: *n = p->ndof * p->ncases; return p->u;
    case FO_FIELD_P: *n = p->ndof * p->ncases; return p->p;
    case FO_FIELD_THETA: *n = g.dim * g.num_nodes; return p->theta;
    case FO_FIELD_RHS: *n = g.dim * g.num_nodes; return p->rhs;
    case FO_FIELD_COEF: *n = g.num_elems; return p->coef;
    case FO_FIELD_CHI:
      *n = g.num_elems;
      *is_u8 = p->desc.coef_rule != FO_COEF_CUT;
      return p->desc.coef_rule == FO_COEF_CUT ? p->chif : (double *)p->chi;
    case FO_FIELD_LOAD: *n = p->ndof * p->ncases; return p->load;
    case FO_FIELD_OMEGA0: *n = g.num_elems; *is_u8 = true; return (double *)p->omega0;
    case FO_FIELD_V: *n = p->ndof * p->ncases; return p->inv ? p->inv->v : nullptr;
    case FO_FIELD_Q: *n = p->ndof * p->ncases; return p->inv ? p->inv->q : nullptr;
    case FO_FIELD_MEAS: *n = p->ndof * p->ncases; return p->inv ? p->inv->g : nullptr;
    default: return nullptr;
  }
}

extern "C" fo_status fo_get(fo_problem *p, int field, double *out) {
  if (!p || !out) return FO_EINVAL;
  if (double *bf = batch_field(p, field)) return batch_to_host(p, bf, out, 0);
  size_t n;
  bool u8;
  double *src = field_ptr(p, field, &n, &u8);
  if (!src) return fo_fail(p->ctx, FO_EINVAL, "unknown field %d", field);
  fo_ctx *ctx = p->ctx;
  if (field == FO_FIELD_COEF && p->desc.kind == FO_HELMHOLTZ) {
    // stored as A_e * k; report A_e
  }
  if (u8) {
    std::vector<uint8_t> tmp(n);
    FO_CU(ctx, cudaMemcpyAsync(tmp.data(), src, n, cudaMemcpyDeviceToHost, ctx->stream));
    FO_CU(ctx, cudaStreamSynchronize(ctx->stream));
    for (size_t i = 0; i < n; ++i) out[i] = tmp[i];
    return FO_OK;
  }
  FO_CU(ctx, cudaMemcpyAsync(out, src, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream));
  FO_CU(ctx, cudaStreamSynchronize(ctx->stream));
  if (field == FO_FIELD_COEF && p->desc.kind == FO_HELMHOLTZ)
    for (size_t i = 0; i < n; ++i) out[i] /= p->desc.k;
  return FO_OK;
}

extern "C" fo_status fo_set(fo_problem *p, int field, const double *v, int on_device) {
  if (!p || !v) return FO_EINVAL;
  if (p->batch && field == FO_FIELD_U) {
    FO_TRY(batch_from_host(p, p->batch->U, v, on_device));
    p->u_valid = true;
    return FO_OK;
  }
  if (p->batch && (field == FO_FIELD_P || field == FO_FIELD_LOAD))
    return fo_fail(p->ctx, FO_EINVAL, "field %d cannot be set", field);
  size_t n;
  bool u8;
  double *dst = field_ptr(p, field, &n, &u8);
  if (!dst || u8 || field == FO_FIELD_COEF || field == FO_FIELD_LOAD)
    return fo_fail(p->ctx, FO_EINVAL, "field %d cannot be set", field);
  FO_TRY(copy_in(p, dst, v, n, on_device));
  if (field == FO_FIELD_PHI) p->coef_valid = false;
  if (field == FO_FIELD_U) p->u_valid = true;
  if (field == FO_FIELD_RHS) p->rhs_valid = true;
  if (field == FO_FIELD_THETA) {
    p->theta_valid = true;
    p->transport_valid = false;
  }
  return FO_OK;
}

extern "C" fo_status fo_apply(fo_problem *p, int op, const double *x, double *y, int on_device) {
  if (!p || !x || !y) return FO_EINVAL;
  fo_ctx *ctx = p->ctx;
  const Grid &g = p->mesh->g;
  size_t n;
  switch (op) {
    case FO_OP_STATE: case FO_OP_STATE_FP32: n = p->ndof; break;
    case FO_OP_VELOCITY: n = g.dim * g.num_nodes; break;
    case FO_OP_TRANSPORT_L: case FO_OP_TRANSPORT_R:
      if (!p->transport_valid) return fo_fail(ctx, FO_ESTATE, "transport matrices not assembled");
      n = g.num_nodes;
      break;
    default: return fo_fail(ctx, FO_EINVAL, "unknown operator %d", op);
  }
  if ((op == FO_OP_STATE || op == FO_OP_STATE_FP32) && !p->coef_valid) FO_TRY(fo_coefficients(p));
  if (p->batch && (op == FO_OP_STATE || op == FO_OP_STATE_FP32)) {   // all instances, [N_n][n_inst]
    const size_t nx = (size_t)g.num_nodes * p->batch->nip;
    double *bx, *by;
    FO_TRY(fo_alloc(ctx, (void **)&bx, sizeof(double) * 2 * nx));
    by = bx + nx;
    fo_status r = batch_from_host(p, bx, x, on_device);
    if (r == FO_OK) r = fo_batch_apply(p, bx, by, op == FO_OP_STATE_FP32);
    if (r == FO_OK) r = batch_to_host(p, by, y, on_device);
    fo_free(ctx, bx, sizeof(double) * 2 * nx);
    return r;
  }
  double *dx, *dy;
  FO_TRY(fo_alloc(ctx, (void **)&dx, sizeof(double) * n));
  fo_status st = fo_alloc(ctx, (void **)&dy, sizeof(double) * n);
  if (st != FO_OK) {
    fo_free(ctx, dx, sizeof(double) * n);
    return st;
  }
  cudaMemcpyKind kin = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cudaMemcpyKind kout = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  st = fo_cuda_check(ctx, cudaMemcpyAsync(dx, x, sizeof(double) * n, kin, ctx->stream), "apply in");
  if (st == FO_OK) {
    if (p->mesh->um) {
      if (op == FO_OP_STATE || op == FO_OP_STATE_FP32) st = fo_umesh_state_apply(p, dx, dy, op == FO_OP_STATE_FP32);
      else if (op == FO_OP_VELOCITY) st = fo_umesh_velocity_apply(p, dx, dy);
      else st = fo_umesh_transport_apply(p, op == FO_OP_TRANSPORT_L ? 0 : 1, dx, dy);
    } else if (op == FO_OP_STATE) st = fo_launch_state_apply(p, dx, dy, true);
    else if (op == FO_OP_STATE_FP32) st = fo_launch_state_apply32(p, dx, dy);
    else if (op == FO_OP_VELOCITY) st = fo_launch_velocity_apply(p, dx, dy);
    else st = fo_launch_stencil_apply(p, op == FO_OP_TRANSPORT_L ? p->L : p->R, dx, dy);
  }
  if (st == FO_OK) st = fo_cuda_check(ctx, cudaMemcpyAsync(y, dy, sizeof(double) * n, kout, ctx->stream), "apply out");
  if (st == FO_OK) st = fo_cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "apply sync");
  fo_free(ctx, dx, sizeof(double) * n);
  fo_free(ctx, dy, sizeof(double) * n);
  return st;
}

// ------------------------------------------------------------------------- host helpers
extern "C" void fo_ppl_init(fo_ppl *s, int nc) {
  if (!s) return;
  memset(s, 0, sizeof *s);
  s->nc = nc < 0 ? 0 : (nc > 4 ? 4 : nc);
  s->r = 0.999;
  s->delta = 0.5;
  s->alpha = 2000.0;
  s->beta = 0.5;
}

extern "C" void fo_ppl_update(fo_ppl *s, const double *C, double J, double *lambda_out, double *L_out) {
  if (!s) return;
  const int nc = s->nc;
  double dd = 0;
  for (int i = 0; i < nc; ++i) dd += (s->lambda[i] - s->mu[i]) * (s->lambda[i] - s->mu[i]);
  for (int i = 0; i < nc; ++i) s->mu[i] = s->mu[i] + s->delta * (s->lambda[i] - s->mu[i]) / (dd + 1.0);
  for (int i = 0; i < nc; ++i) {
    s->lambda[i] = s->mu[i] + s->alpha / (1.0 + s->alpha * s->beta) * (C[i] - 1.0);
    s->z[i] = (s->lambda[i] - s->mu[i]) / s->alpha;
  }
  s->delta = s->r * s->delta;
  double L = J, zz = 0, lm = 0;
  for (int i = 0; i < nc; ++i) {
    L += s->lambda[i] * (C[i] - 1.0) + s->mu[i] * s->z[i];
    zz += s->z[i] * s->z[i];
    lm += (s->lambda[i] - s->mu[i]) * (s->lambda[i] - s->mu[i]);
  }
  L += 0.5 * s->alpha * zz + 0.5 * s->beta * lm;
  if (lambda_out)
    for (int i = 0; i < nc; ++i) lambda_out[i] = s->lambda[i];
  if (L_out) *L_out = L;
}

extern "C" void fo_adaptime(double Btt, const fo_run_options *o, double *t_end, int *nsteps) {
  fo_run_options def;
  fo_run_options_default(&def);
  if (!o) o = &def;
  double t = o->dfactor / std::max(Btt, 1e-12);
  t = std::min(std::max(t, o->t_min), o->t_max);
  double s = (o->s_max - o->s_min) * std::pow((t - o->t_min) / (o->t_max - o->t_min), 1.0 / 6.0) + o->s_min;
  s = std::min(std::max(s, (double)o->s_min), (double)o->s_max);
  if (t_end) *t_end = t;
  if (nsteps) *nsteps = (int)std::floor(s + 0.5);
}

extern "C" void fo_stop_opts_default(fo_stop_opts *o) {
  if (!o) return;
  o->start_to_check = 30;
  o->tol = 1e-2;
  o->ctrn_tol = 1e-2;
  o->prev = 10;
}

// Stopping criterion (Sec. 5.7): at i = n - 1 > start_to_check, the largest difference of
// values[i] from the previous `prev` values below tol |values[i]|, and max |C_j - 1| below
// ctrn_tol when there are constraints.
extern "C" void fo_stop_check(const double *values, int n, const double *C, int nc, const fo_stop_opts *o, int *stop) {
  if (!stop) return;
  *stop = 0;
  fo_stop_opts def;
  fo_stop_opts_default(&def);
  if (!o) o = &def;
  const int i = n - 1;
  if (!values || i <= o->start_to_check || i < o->prev || o->prev < 1) return;
  double spread = 0;
  for (int j = i - o->prev; j < i; ++j) spread = std::max(spread, std::fabs(values[i] - values[j]));
  if (!(spread < o->tol * std::fabs(values[i]))) return;
  if (nc > 0 && C) {
    double err = 0;
    for (int q = 0; q < nc; ++q) err = std::max(err, std::fabs(C[q] - 1.0));
    if (!(err < o->ctrn_tol)) return;
  }
  *stop = 1;
}

extern "C" void fo_solve_opts_default(fo_solve_opts *o) {
  if (!o) return;
  memset(o, 0, sizeof *o);
  o->precision = FO_FP64;
  o->rtol = 1e-12;
  o->maxit = 200000;
  o->warm_start = 0;
  o->inner_rtol = 1e-3;
  o->inner_maxit = 20000;
  o->grid_blocks = 0;
}

extern "C" void fo_run_options_default(fo_run_options *o) {
  if (!o) return;
  memset(o, 0, sizeof *o);
  o->dfactor = 1e-2;
  o->t_min = 1e-3;
  o->t_max = 1e-1;
  o->s_min = 8;
  o->s_max = 16;
  o->smooth = 0;
  o->reinit_step = 0;
  o->reinit_steps = 8;
  o->reinit_time = 1e-1;
  o->h = 0;
  fo_solve_opts_default(&o->state);
  fo_solve_opts_default(&o->velocity);
  fo_solve_opts_default(&o->transport);
  o->state.warm_start = 1;
}

// ----------------------------------------------------------------- one Algorithm-1 step
extern "C" fo_status fo_opt_step(fo_problem *p, int iter, const fo_run_options *o, fo_ppl *ppl, fo_iter_log *log) {
  if (!p || !o) return FO_EINVAL;
  fo_iter_log lg;
  memset(&lg, 0, sizeof lg);
  fo_ctx *ctx = p->ctx;
  const bool tm = ctx->timing != 0;
  auto mark = [&](int i) -> fo_status {
    if (tm) FO_CU(ctx, cudaEventRecord(ctx->ev[i], ctx->stream));
    return FO_OK;
  };
  const double h = o->h > 0 ? o->h : p->mesh->h_diam;
  FO_TRY(mark(0));
  FO_TRY(fo_coefficients(p));
  ctx->last_solve_ms = 0.0;
  fo_status s = fo_state_solve(p, &o->state, &lg.state);
  if (s != FO_OK) return s;
  lg.ms_state_kernel = ctx->last_solve_ms;
  if (p->desc.kind == FO_LOGISTIC || p->inv) {   // the adjoints are solves of their own (Sec. 6.4, Sec. 3)
    lg.newton_steps = p->desc.kind == FO_LOGISTIC ? p->newton_steps : 0;
    s = fo_adjoint_solve(p, &o->state, &lg.adjoint);
    if (s != FO_OK && s != FO_ENOCONV) return s;
  }
  FO_TRY(mark(1));
  const int nc = problem_nc(p);
  double J = 0, Cv[4] = {0, 0, 0, 0}, lv[4] = {0, 0, 0, 0};
  FO_TRY(fo_functionals_v(p, &J, Cv, nc));
  FO_TRY(mark(2));
  lg.J = J;
  lg.L = J;
  lg.nc = nc;
  if (nc > 0) {
    lg.C = Cv[0];
    if (ppl) {   // one PPL update of the whole constraint vector (Sec. 5.4)
      if (ppl->nc != nc) return fo_fail(ctx, FO_EINVAL, "the PPL state has %d constraints, the problem %d", ppl->nc, nc);
      fo_ppl_update(ppl, Cv, J, lv, &lg.L);
    }
  }
  for (int q = 0; q < 4; ++q) {
    lg.Cv[q] = Cv[q];
    lg.lambdav[q] = lv[q];
  }
  lg.lambda = lv[0];
  FO_TRY(mark(3));
  FO_TRY(fo_shape_derivative_v(p, lv, nc, nullptr));
  FO_TRY(mark(4));
  double Btt = 0;
  s = fo_descent(p, &o->velocity, &Btt, &lg.velocity);
  if (s != FO_OK) return s;
  FO_TRY(mark(5));
  lg.Btt = Btt;
  double t_end;
  int ns;
  fo_adaptime(Btt, o, &t_end, &ns);
  lg.t_end = t_end;
  lg.nsteps = ns;
  s = fo_levelset_step(p, t_end, ns, h, o->smooth, &o->transport, &lg.transport);
  if (s != FO_OK) return s;
  FO_TRY(mark(6));
  if (o->reinit_step > 0 && iter > 0 && iter % o->reinit_step == 0) {
    s = fo_reinit(p, o->reinit_steps, o->reinit_time, h, &o->transport, &lg.reinit_stats);
    if (s != FO_OK) return s;
    lg.reinit = 1;
  }
  FO_TRY(mark(7));
  if (tm) {
    FO_CU(ctx, cudaEventSynchronize(ctx->ev[7]));
    float ms[7];
    for (int i = 0; i < 7; ++i) FO_CU(ctx, cudaEventElapsedTime(&ms[i], ctx->ev[i], ctx->ev[i + 1]));
    lg.ms_state = ms[0];
    lg.ms_functionals = ms[1] + ms[2];   // functionals + host PPL update
    lg.ms_shape = ms[3];
    lg.ms_velocity = ms[4];
    lg.ms_transport = ms[5];
    lg.ms_reinit = ms[6];
  }
  if (log) *log = lg;
  return FO_OK;
}
