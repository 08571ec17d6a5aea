// C ABI of the reciprocal incoherent-light evaluator (declarations and contracts in
// include/rci.h).  Host code here only validates arguments, sequences kernels on the
// grid's stream and moves scalars; every numerical step runs in the kernels.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <complex>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <atomic>

#include "bcr.cuh"
#include "kernels.cuh"
#include "tc_gemm.cuh"

static std::atomic<uint64_t> g_launches{0};
void rci_note_launch(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

struct rci_grid {
  rci_grid_desc d{};
  GridGeom g{};
  cudaStream_t s = nullptr;
  int device = 0;
  int64_t N = 0;
  // problem
  double* widths = nullptr;
  double* eps = nullptr;
  double2 *dg = nullptr, *cx = nullptr, *cy = nullptr;
  double2 *dg0 = nullptr, *kss = nullptr;  // design-independent parts of the diagonal
  BcrHandle* bcr = nullptr;
  bool has_design = false, factored = false;
  // single right-hand-side vectors (FP64) and FP32 shadows
  double2 *b1 = nullptr, *x1 = nullptr, *r1 = nullptr;
  void *r32 = nullptr, *d32 = nullptr;
  // objective row, source-plane field, lags, scalars
  double2* crow = nullptr;
  double2* vsrc = nullptr;
  double* lags = nullptr;
  double* qpart = nullptr;
  double* dscal = nullptr;  // [0] qform, [1..] misc
  double* part_r = nullptr;
  double* part_b = nullptr;
  double* ratio = nullptr;  // per-RHS residual ratio (up to MAXQ)
  double* vf_scratch = nullptr;
  int32_t* dstatus = nullptr;
  // multi right-hand side buffers (grown on demand)
  int mq_cap = 0;
  double2 *mb = nullptr, *mx = nullptr, *mr = nullptr;
  void *m32a = nullptr, *m32b = nullptr;
  double *th_d = nullptr, *wq_d = nullptr, *f_d = nullptr;
  int th_cap = 0;
  // FP64 fallback of an FP32 grid: an FP64 factorisation made when refinement on the FP32
  // one fails (non-finite, stagnating or out of steps), used until the next design
  BcrHandle* bcr64 = nullptr;
  bool use64 = false;
  double2* corr64 = nullptr;
  int64_t corr64_n = 0;
  DevMem mem64;  // where the fallback's buffers came from (cudaMalloc when the grid's own
                 // memory source, e.g. a serving arena, had no room left for them)
  // Krylov refinement (allocated the first time plain refinement stalls): basis V
  // (KR_M + 1 vectors), preconditioned directions Z (KR_M), a zero vector, dot scratch
  double2* kbuf = nullptr;
  double2* kpart = nullptr;
  DevMem memk;
  // correlated-light inputs (theta, weights, C, alpha) and multi-output results (grown on demand)
  void* cbuf = nullptr;
  size_t cbuf_bytes = 0;
  double* mF = nullptr;
  int mF_cap = 0;
  // gradient buffers (allocated by the first gradient call)
  double2 *mu = nullptr, *gsrc = nullptr, *tpart = nullptr;
  double* dgrad = nullptr;
  // light cache
  bool lags_valid = false;
  rci_light lags_key{};
  std::vector<double> tab_key;    // TABULATED light of the cached lags: theta then rho
  void* tabbuf = nullptr;         // device: theta, rho, sub-panel table, rule, nodes
  size_t tabbuf_bytes = 0;
  // settings
  double tol32 = 1e-10, tol64 = 1e-13;
  int max_refine32 = 31, max_refine64 = 2;  // FP32: solves, the first one included
  size_t bytes = 0;
  double growth = 0.0, growth64 = 0.0;  // growth estimates of the factorisations (FP32/FP64)
  cudaEvent_t ev[6] = {};
  Profiler prof;
  std::string err;
  DevMem mem;  // device memory source (cudaMalloc unless a serving arena supplies one)
};

namespace {

constexpr int MAXQ = 256;  // right-hand sides per multi-RHS chunk

rci_status fail(rci_grid* g, rci_status st, const std::string& msg) {
  if (g) g->err = msg;
  return st;
}

rci_status cuda_fail(rci_grid* g, cudaError_t e, const char* where) {
  if (e == cudaErrorMemoryAllocation)
    return fail(g, RCI_ENOMEM, std::string(where) + ": device allocation failed");
  return fail(g, RCI_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(expr, where)                                  \
  do {                                                   \
    cudaError_t _e = (expr);                             \
    if (_e != cudaSuccess) return cuda_fail(g, _e, where); \
  } while (0)

template <typename P>
cudaError_t dalloc(rci_grid* g, P** p, size_t bytes) {
  cudaError_t e = g->mem.alloc((void**)p, bytes);
  if (e == cudaSuccess) g->bytes += bytes;
  return e;
}

void dfree(rci_grid* g, void* p) { g->mem.release(p); }

bool desc_ok(const rci_grid_desc* d, std::string& why) {
  if (d->n_cells < 1 || d->cell_px < 1 || d->ppl < 2 || d->npml < 1 || d->ny < 4) {
    why = "counts must be positive (n_cells, cell_px, npml >= 1, ppl >= 2, ny >= 4)";
    return false;
  }
  if (d->rows_sub < 1 || d->rows_pillar < 1 || d->src_offset < 0 || d->src_offset >= d->rows_sub) {
    why = "rows_sub, rows_pillar >= 1 and 0 <= src_offset < rows_sub required";
    return false;
  }
  if (d->ny - 2 * d->npml - d->rows_sub - d->rows_pillar < 1) {
    why = "ny leaves no air rows above the pillars";
    return false;
  }
  if (d->ny > 256) {
    // the single-right-hand-side solve holds the row vectors of the stored blocks in
    // registers (ny / 32 16-byte vectors per lane and row in FP64, the FP32 grid's fallback)
    why = "ny > 256 is not supported";
    return false;
  }
  if (d->prec == RCI_FP32_REFINE && (d->ny & 1)) {
    why = "FP32_REFINE grids need an even ny (rows are read as pairs of complex64)";
    return false;
  }
  if (!(d->eps_pillar > 0 && d->eps_sub > 0 && d->eps_air > 0) || !(d->pml_R0 > 0 && d->pml_R0 < 1) ||
      d->pml_m < 0) {
    why = "permittivities must be positive, 0 < pml_R0 < 1, pml_m >= 0";
    return false;
  }
  if (d->prec != RCI_FP64 && d->prec != RCI_FP32_REFINE) {
    why = "unknown precision";
    return false;
  }
  int64_t nx = (int64_t)d->n_cells * d->cell_px + 2 * (int64_t)d->npml;
  if (nx > (1 << 22)) {
    why = "grid too wide";
    return false;
  }
  return true;
}

GridGeom make_geom(const rci_grid_desc& d) {
  GridGeom g{};
  g.nx = d.n_cells * d.cell_px + 2 * d.npml;
  g.ny = d.ny;
  g.npml = d.npml;
  g.n_src = g.nx - 2 * d.npml;
  g.j_src = d.npml + d.src_offset;
  g.j_p0 = d.npml + d.rows_sub;
  g.j_p1 = g.j_p0 + d.rows_pillar;
  g.n_cells = d.n_cells;
  g.cell_px = d.cell_px;
  g.h = 1.0 / d.ppl;
  g.k0 = 2.0 * M_PI;
  g.k_sub = g.k0 * std::sqrt(d.eps_sub);
  g.eps_pillar = d.eps_pillar;
  g.eps_sub = d.eps_sub;
  g.eps_air = d.eps_air;
  double dd = d.npml * g.h;
  g.sigma_max = -(d.pml_m + 1) * std::log(d.pml_R0) / (2.0 * dd);
  g.width = g.n_src * g.h;
  g.pml_m = d.pml_m;
  return g;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

bool light_eq(const rci_light& a, const rci_light& b) {
  return a.kind == b.kind && a.c == b.c && a.th1 == b.th1 && a.th2 == b.th2 && a.lags == b.lags;
}

constexpr int64_t TAB_MAX = 65536;

rci_status check_light(rci_grid* g, const rci_light* L) {
  if (!L) return fail(g, RCI_EINVAL, "light is NULL");
  if (L->kind == RCI_LIGHT_CONE) {
    if (!(L->c > 0 && L->c < M_PI / 2)) return fail(g, RCI_EINVAL, "cone half-angle must be in (0, pi/2)");
  } else if (L->kind == RCI_LIGHT_ANNULUS) {
    if (!(L->th1 >= 0 && L->th1 < L->th2 && L->th2 < M_PI / 2))
      return fail(g, RCI_EINVAL, "annulus needs 0 <= th1 < th2 < pi/2");
  } else if (L->kind == RCI_LIGHT_USER_LAGS) {
    if (!L->lags) return fail(g, RCI_EINVAL, "user lags pointer is NULL");
  } else if (L->kind == RCI_LIGHT_TABULATED) {
    if (!L->tab_theta || !L->tab_rho || L->n_tab < 2 || L->n_tab > TAB_MAX)
      return fail(g, RCI_EINVAL, "tabulated light needs 2 <= n_tab <= 65536 angles and densities");
    for (int64_t q = 0; q < L->n_tab; ++q) {
      const double t = L->tab_theta[q], r = L->tab_rho[q];
      if (!(t >= 0.0 && t < M_PI / 2) || (q > 0 && !(t > L->tab_theta[q - 1])))
        return fail(g, RCI_EINVAL, "tabulated angles must ascend strictly within [0, pi/2)");
      if (!(r >= 0.0) || !std::isfinite(r))
        return fail(g, RCI_EINVAL, "tabulated densities must be finite and >= 0");
    }
  } else {
    return fail(g, RCI_EINVAL, "unknown light kind");
  }
  return RCI_OK;
}

rci_status ensure_lags(rci_grid* g, const rci_light* L) {
  rci_status st = check_light(g, L);
  if (st != RCI_OK) return st;
  if (L->kind == RCI_LIGHT_USER_LAGS) {
    CK(cudaMemcpyAsync(g->lags, L->lags, sizeof(double) * g->g.n_src, cudaMemcpyHostToDevice, g->s),
       "copy lags");
    g->lags_valid = false;
    return RCI_OK;
  }
  if (L->kind == RCI_LIGHT_TABULATED) {
    const int64_t nt = L->n_tab;
    std::vector<double> key(L->tab_theta, L->tab_theta + nt);
    key.insert(key.end(), L->tab_rho, L->tab_rho + nt);
    if (g->lags_valid && g->lags_key.kind == RCI_LIGHT_TABULATED && g->tab_key == key)
      return RCI_OK;
    // sub-panels: each segment split into equal parts in u = sin(theta) no wider than half
    // the shortest period of cos(k_s u D) over the source plane (D <= (n_src - 1) h)
    const double dmax = (double)(g->g.n_src - 1) * g->g.h;
    const double umax = M_PI / (g->g.k_sub * (dmax > 0.0 ? dmax : g->g.h));
    std::vector<int4> seg;
    for (int64_t q = 0; q + 1 < nt; ++q) {
      const double du = std::sin(L->tab_theta[q + 1]) - std::sin(L->tab_theta[q]);
      const int S = (int)std::max(1.0, std::ceil(du / umax));
      for (int i = 0; i < S; ++i) seg.push_back(make_int4((int)q, i, S, 0));
    }
    const int P = (int)seg.size();
    if ((int64_t)P * TAB_ORDER > (1 << 26)) return fail(g, RCI_EINVAL, "tabulated light too fine");
    const size_t need = sizeof(double) * 2 * nt + sizeof(int4) * P + sizeof(double) * 2 * TAB_ORDER +
                        sizeof(double2) * (size_t)P * TAB_ORDER + 64 * 5;
    if (g->tabbuf_bytes < need) {
      dfree(g, g->tabbuf);
      g->tabbuf = nullptr;
      g->tabbuf_bytes = 0;
      CK(dalloc(g, (char**)&g->tabbuf, need), "tabulated light");
      g->tabbuf_bytes = need;
    }
    auto carve = [](char*& p, size_t b) { char* r = p; p += (b + 63) & ~(size_t)63; return r; };
    char* p = (char*)g->tabbuf;
    double* th_d = (double*)carve(p, sizeof(double) * nt);
    double* rho_d = (double*)carve(p, sizeof(double) * nt);
    int4* seg_d = (int4*)carve(p, sizeof(int4) * P);
    double* glx = (double*)carve(p, sizeof(double) * TAB_ORDER);
    double* glw = (double*)carve(p, sizeof(double) * TAB_ORDER);
    double2* node = (double2*)carve(p, sizeof(double2) * (size_t)P * TAB_ORDER);
    g->tab_key = std::move(key);
    CK(cudaMemcpyAsync(th_d, g->tab_key.data(), sizeof(double) * nt, cudaMemcpyHostToDevice, g->s),
       "tabulated light");
    CK(cudaMemcpyAsync(rho_d, g->tab_key.data() + nt, sizeof(double) * nt, cudaMemcpyHostToDevice,
                       g->s),
       "tabulated light");
    CK(cudaMemcpyAsync(seg_d, seg.data(), sizeof(int4) * P, cudaMemcpyHostToDevice, g->s),
       "tabulated light");
    CK(launch_w_lags_tabulated(th_d, rho_d, seg_d, P, glx, glw, node, g->g.k_sub, g->g.h,
                               g->g.n_src, g->lags, g->s),
       "W lags (tabulated)");
    // the sub-panel table is a local vector: its copy must be done before it goes away
    CK(cudaStreamSynchronize(g->s), "tabulated light");
    g->lags_key = *L;
    g->lags_valid = true;
    return RCI_OK;
  }
  if (g->lags_valid && light_eq(g->lags_key, *L)) return RCI_OK;
  CK(launch_w_lags(L->kind, L->c, L->th1, L->th2, g->g.k_sub, g->g.h, g->g.n_src, g->lags, g->s),
     "W lags");
  g->lags_key = *L;
  g->lags_valid = true;
  return RCI_OK;
}

// conj(w) as a full-grid right-hand side in b (zeroed first).  The objective row is kept
// in g->crow for the brute-force projection.
rci_status build_objective(rci_grid* g, const rci_objective* o, double2* b) {
  const GridGeom& G = g->g;
  if (!o) return fail(g, RCI_EINVAL, "objective is NULL");
  CK(cudaMemsetAsync(b, 0, sizeof(double2) * g->N, g->s), "zero rhs");
  if (o->kind == RCI_OBJ_POINT) {
    if (o->i_f < 0 || o->i_f >= G.nx || o->j_f < 0 || o->j_f >= G.ny)
      return fail(g, RCI_EINVAL, "focus node outside the grid");
    double2 one = make_double2(1.0, 0.0);
    CK(cudaMemcpyAsync(b + (int64_t)o->i_f * G.ny + o->j_f, &one, sizeof(double2),
                       cudaMemcpyHostToDevice, g->s),
       "point source");
    CK(cudaStreamSynchronize(g->s), "point source");
    return RCI_OK;
  }
  if (o->monitor_row < 0 || o->monitor_row >= G.ny)
    return fail(g, RCI_EINVAL, "monitor row outside the grid");
  if (o->kind == RCI_OBJ_PLANEWAVE) {
    if (!(std::fabs(o->theta_out) < M_PI / 2)) return fail(g, RCI_EINVAL, "theta_out out of range");
    CK(launch_planewave_row(G, o->theta_out, g->crow, g->s), "planewave objective");
  } else if (o->kind == RCI_OBJ_VIRTUAL_FOCUS) {
    if (o->d_rows < 0) return fail(g, RCI_EINVAL, "d_rows must be >= 0");
    CK(launch_virtual_focus_row(G, o->x_f, o->d_rows, g->crow, g->vf_scratch, g->s),
       "virtual focus objective");
  } else if (o->kind == RCI_OBJ_USER_ROW) {
    if (!o->w_row) return fail(g, RCI_EINVAL, "w_row is NULL");
    CK(cudaMemcpyAsync(g->crow, o->w_row, sizeof(double2) * G.n_src, cudaMemcpyHostToDevice, g->s),
       "user objective");
    CK(launch_conj(g->crow, G.n_src, g->s), "user objective");
  } else {
    return fail(g, RCI_EINVAL, "unknown objective kind");
  }
  CK(launch_scatter_row(G, g->crow, o->monitor_row, b, g->s), "objective rhs");
  return RCI_OK;
}

rci_status ensure_multi(rci_grid* g, int nq) {
  if (g->mq_cap >= nq) return RCI_OK;
  dfree(g, g->mb);
  dfree(g, g->mx);
  dfree(g, g->mr);
  dfree(g, g->m32a);
  dfree(g, g->m32b);
  g->mb = g->mx = g->mr = nullptr;
  g->m32a = g->m32b = nullptr;
  size_t n = (size_t)g->N * nq;
  CK(dalloc(g, &g->mb, n * sizeof(double2)), "multi-rhs buffers");
  CK(dalloc(g, &g->mx, n * sizeof(double2)), "multi-rhs buffers");
  CK(dalloc(g, &g->mr, n * sizeof(double2)), "multi-rhs buffers");
  if (g->d.prec == RCI_FP32_REFINE) {
    CK(dalloc(g, &g->m32a, n * sizeof(float2)), "multi-rhs buffers");
    CK(dalloc(g, &g->m32b, n * sizeof(float2)), "multi-rhs buffers");
  } else {
    CK(dalloc(g, &g->m32a, n * sizeof(double2)), "multi-rhs buffers");  // FP64 corrections
  }
  g->mq_cap = nq;
  return RCI_OK;
}

// Residual r = b - A x (FP64 stencil) and the largest ||r||/||b|| over the columns.
rci_status residual_ratio(rci_grid* g, const double2* b, const double2* x, double2* r, int nrhs,
                          double* worst) {
  int nblk = residual_blocks(g->g);
  {
    ProfScope ps(&g->prof, PF_RESIDUAL, g->s, 18.0 * g->N * nrhs,
                 (double)g->N * (48.0 + 48.0 * nrhs), 2);
    CK(launch_residual(g->g, g->dg, g->cx, g->cy, b, x, r, nrhs, g->part_r, g->part_b, g->s),
       "residual");
    CK(launch_ratio_norms(g->part_r, g->part_b, nblk, nrhs, g->ratio, g->s), "residual norms");
  }
  std::vector<double> h(nrhs);
  CK(cudaMemcpyAsync(h.data(), g->ratio, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, g->s),
     "residual norms");
  CK(cudaStreamSynchronize(g->s), "residual norms");
  double w = 0.0;
  for (double v : h) {
    if (!std::isfinite(v)) {
      *worst = v;
      return fail(g, RCI_ENUMERIC, "non-finite residual");
    }
    w = v > w ? v : w;
  }
  *worst = w;
  return RCI_OK;
}

// FP64 refinement on an FP64 factorisation h: x = A^-1 b, then corrections d while the
// FP64 stencil residual is above tol64 (at most max_refine64 steps).
rci_status solve64(rci_grid* g, BcrHandle* h, const double2* b, double2* x, double2* r, double2* d,
                   int nrhs, int* it, double* worst) {
  const int64_t n = g->N * nrhs;
  CK(bcr_solve(h, g->cx, b, x, nrhs, g->s), "solve");
  rci_status st = residual_ratio(g, b, x, r, nrhs, worst);
  if (st != RCI_OK) return st;
  while (*worst > g->tol64 && *it < g->max_refine64) {
    CK(bcr_solve(h, g->cx, r, d, nrhs, g->s), "refine solve");
    CK(launch_axpy64(x, d, n, g->s), "refine update");
    ++*it;
    st = residual_ratio(g, b, x, r, nrhs, worst);
    if (st != RCI_OK) return st;
  }
  return RCI_OK;
}

// Factor the current design in FP64 for an FP32 grid whose refinement failed (the
// classic fallback of mixed-precision solvers, e.g. LAPACK's single/double refinement
// driver): the FP64 factor store is allocated the first time and kept for later designs.
rci_status fp64_fallback(rci_grid* g) {
  if (g->use64) return RCI_OK;
  if (!g->bcr64) {
    // The fallback is not part of a grid's admitted footprint: when the grid's memory source
    // (a serving arena) is full, the FP64 store comes from cudaMalloc instead.
    cudaError_t e = bcr_create(g->g.nx, g->g.ny, RCI_FP64, &g->mem, &g->bcr64, nullptr);
    if (e == cudaErrorMemoryAllocation && g->mem.alloc_fn) {
      (void)cudaGetLastError();
      e = bcr_create(g->g.nx, g->g.ny, RCI_FP64, nullptr, &g->bcr64, nullptr);
    }
    CK(e, "FP64 fallback store");
    bcr_set_profiler(g->bcr64, &g->prof);
  }
  CK(bcr_factor(g->bcr64, g->dg, g->cx, g->cy, g->s), "FP64 fallback factor");
  int32_t st = 0;
  CK(bcr_read_status(g->bcr64, &st, g->s, &g->growth64), "FP64 fallback status");
  if (st == DEV_SINGULAR) return fail(g, RCI_ESINGULAR, "zero pivot in a diagonal block (FP64)");
  g->use64 = true;
  return RCI_OK;
}

rci_status ensure_corr64(rci_grid* g, int64_t n) {
  if (g->corr64_n >= n) return RCI_OK;
  g->mem64.release(g->corr64);
  g->corr64 = nullptr;
  g->corr64_n = 0;
  g->mem64 = g->mem;
  cudaError_t e = g->mem64.alloc((void**)&g->corr64, sizeof(double2) * n);
  if (e == cudaErrorMemoryAllocation && g->mem.alloc_fn) {
    (void)cudaGetLastError();
    g->mem64 = DevMem{};
    e = g->mem64.alloc((void**)&g->corr64, sizeof(double2) * n);
  }
  CK(e, "FP64 fallback correction");
  g->corr64_n = n;
  return RCI_OK;
}

// Krylov refinement of one right-hand side: flexible GMRES on the FP64 stencil operator A,
// right-preconditioned by the FP32 factorisation (z = M^-1 v by one FP32 solve; flexible,
// since the FP32 solve is linear only up to rounding), restarted every KR_M steps, Gram-
// Schmidt applied twice per step.  Used when plain refinement stalls: the Krylov space
// corrects the few error directions the FP32 factorisation resolves poorly, at one FP32
// solve per step, where the alternative is an FP64 factorisation.  Starts from x, takes at
// most max_steps preconditioned steps; *worst is the true residual ratio at the end.
constexpr int KR_M = 16;
static_assert(KR_M + 1 <= KV_MAX_VECTORS, "basis fits one multi-dot");

rci_status ensure_krylov(rci_grid* g) {
  if (g->kbuf) return RCI_OK;
  const size_t nvec = (size_t)(2 * KR_M + 2);  // V (KR_M + 1), Z (KR_M), zero
  const size_t bytes = nvec * (size_t)g->N * sizeof(double2);
  const size_t pbytes = ((size_t)KV_DOT_BLOCKS * KV_MAX_VECTORS + KV_MAX_VECTORS) * sizeof(double2);
  g->memk = g->mem;
  cudaError_t e = g->memk.alloc((void**)&g->kbuf, bytes);
  if (e == cudaSuccess) e = g->memk.alloc((void**)&g->kpart, pbytes);
  if (e == cudaErrorMemoryAllocation && g->mem.alloc_fn) {  // arena full: cudaMalloc
    (void)cudaGetLastError();
    g->memk.release(g->kbuf);
    g->memk.release(g->kpart);
    g->kbuf = g->kpart = nullptr;
    g->memk = DevMem{};
    e = g->memk.alloc((void**)&g->kbuf, bytes);
    if (e == cudaSuccess) e = g->memk.alloc((void**)&g->kpart, pbytes);
  }
  if (e != cudaSuccess) {
    g->memk.release(g->kbuf);
    g->memk.release(g->kpart);
    g->kbuf = g->kpart = nullptr;
  }
  CK(e, "Krylov refinement buffers");
  double2* zero = g->kbuf + (size_t)(2 * KR_M + 1) * g->N;
  CK(cudaMemsetAsync(zero, 0, sizeof(double2) * g->N, g->s), "Krylov zero vector");
  return RCI_OK;
}

rci_status krylov_refine(rci_grid* g, const double2* b, double2* x, double2* r, void* a32,
                         void* b32, int max_steps, int* steps, double* worst) {
  using cd = std::complex<double>;
  rci_status st = ensure_krylov(g);
  if (st != RCI_OK) return st;
  const int64_t N = g->N;
  double2* V = g->kbuf;
  double2* Z = V + (size_t)(KR_M + 1) * N;
  double2* zero = Z + (size_t)KR_M * N;
  double2* part = g->kpart;
  double2* hdev = g->kpart + (size_t)KV_DOT_BLOCKS * KV_MAX_VECTORS;
  // out[i] = (V_i, w) for i < nv, read back to the host
  auto dots = [&](const double2* Vb, int nv, const double2* w, std::vector<cd>& out) -> rci_status {
    std::vector<double2> h(nv);
    CK(launch_cdot_multi(Vb, N, nv, w, N, part, hdev, g->s), "Krylov inner products");
    CK(cudaMemcpyAsync(h.data(), hdev, sizeof(double2) * nv, cudaMemcpyDeviceToHost, g->s),
       "Krylov inner products");
    CK(cudaStreamSynchronize(g->s), "Krylov inner products");
    out.assign(nv, cd());
    for (int i = 0; i < nv; ++i) out[i] = cd(h[i].x, h[i].y);
    return RCI_OK;
  };
  // w += sign sum_i c[i] V_i
  auto combine = [&](double2* w, const double2* Vb, const std::vector<cd>& c, int nv,
                     double sign) -> rci_status {
    std::vector<double2> h(nv);
    for (int i = 0; i < nv; ++i) h[i] = make_double2(c[i].real(), c[i].imag());
    CK(cudaMemcpyAsync(hdev, h.data(), sizeof(double2) * nv, cudaMemcpyHostToDevice, g->s),
       "Krylov coefficients");
    CK(launch_caxpy_multi(w, Vb, N, nv, hdev, sign, N, g->s), "Krylov combination");
    return RCI_OK;
  };
  std::vector<cd> t1;
  if ((st = dots(b, 1, b, t1)) != RCI_OK) return st;
  const double bnorm = std::sqrt(std::max(t1[0].real(), 0.0));
  if (!(bnorm > 0.0)) return residual_ratio(g, b, x, r, 1, worst);
  int used = 0;
  double prev = 0.0;
  for (int restart = 0; used < max_steps; ++restart) {
    if ((st = residual_ratio(g, b, x, r, 1, worst)) != RCI_OK) return st;
    if (*worst <= g->tol32) break;
    if (restart > 0 && *worst > 0.5 * prev) break;  // a cycle that barely helps: give up
    prev = *worst;
    const double beta = *worst * bnorm;
    CK(launch_cscale(V, r, 1.0 / beta, N, g->s), "Krylov basis");
    std::vector<cd> H((size_t)(KR_M + 1) * KR_M, cd()), gv(KR_M + 1, cd()), sn(KR_M, cd());
    std::vector<double> cs(KR_M, 0.0);
    auto Hij = [&](int i, int j) -> cd& { return H[(size_t)i * KR_M + j]; };
    gv[0] = beta;
    int k = 0;
    for (int j = 0; j < KR_M && used < max_steps; ++j) {
      double2* vj = V + (size_t)j * N;
      double2* zj = Z + (size_t)j * N;
      double2* w = V + (size_t)(j + 1) * N;
      // z_j = M^-1 v_j (one FP32 solve), w = A z_j (FP64 stencil: r = 0 - A z_j)
      CK(launch_to_f32(vj, (float2*)a32, N, g->s), "Krylov to fp32");
      CK(bcr_solve(g->bcr, g->cx, a32, b32, 1, g->s), "Krylov preconditioner");
      CK(launch_to_f64((const float2*)b32, zj, N, g->s), "Krylov to fp64");
      ++used;
      CK(launch_residual(g->g, g->dg, g->cx, g->cy, zero, zj, r, 1, g->part_r, g->part_b, g->s),
         "Krylov operator");
      CK(launch_cscale(w, r, -1.0, N, g->s), "Krylov operator");
      // w -= V h, twice (classical Gram-Schmidt with one reorthogonalisation)
      std::vector<cd> h1, h2, nw;
      if ((st = dots(V, j + 1, w, h1)) != RCI_OK) return st;
      if ((st = combine(w, V, h1, j + 1, -1.0)) != RCI_OK) return st;
      if ((st = dots(V, j + 1, w, h2)) != RCI_OK) return st;
      if ((st = combine(w, V, h2, j + 1, -1.0)) != RCI_OK) return st;
      if ((st = dots(w, 1, w, nw)) != RCI_OK) return st;
      const double hn = std::sqrt(std::max(nw[0].real(), 0.0));
      if (!std::isfinite(hn)) return fail(g, RCI_ENUMERIC, "non-finite Krylov step");
      for (int i = 0; i <= j; ++i) Hij(i, j) = h1[i] + h2[i];
      Hij(j + 1, j) = hn;
      // earlier Givens rotations on the new column, then the one that zeroes H(j+1, j)
      for (int i = 0; i < j; ++i) {
        const cd a = Hij(i, j), c = Hij(i + 1, j);
        Hij(i, j) = cs[i] * a + sn[i] * c;
        Hij(i + 1, j) = -std::conj(sn[i]) * a + cs[i] * c;
      }
      {
        const cd a = Hij(j, j), c = Hij(j + 1, j);
        const double nu = std::sqrt(std::norm(a) + std::norm(c));
        if (std::abs(a) == 0.0) {
          cs[j] = 0.0;
          sn[j] = 1.0;
          Hij(j, j) = c;
        } else {
          const cd ph = a / std::abs(a);
          cs[j] = std::abs(a) / nu;
          sn[j] = ph * std::conj(c) / nu;
          Hij(j, j) = ph * nu;
        }
        Hij(j + 1, j) = 0.0;
        gv[j + 1] = -std::conj(sn[j]) * gv[j];
        gv[j] = cs[j] * gv[j];
      }
      k = j + 1;
      if (hn > 0.0) CK(launch_cscale(w, w, 1.0 / hn, N, g->s), "Krylov basis");
      if (std::abs(gv[j + 1]) <= 0.5 * g->tol32 * bnorm || hn == 0.0) break;
    }
    // x += Z y with R y = g (R: the rotated Hessenberg matrix)
    std::vector<cd> y(k, cd());
    for (int i = k - 1; i >= 0; --i) {
      cd t = gv[i];
      for (int l = i + 1; l < k; ++l) t -= Hij(i, l) * y[l];
      y[i] = Hij(i, i) != 0.0 ? t / Hij(i, i) : cd();
    }
    if (k > 0 && (st = combine(x, Z, y, k, 1.0)) != RCI_OK) return st;
  }
  *steps = used;
  return residual_ratio(g, b, x, r, 1, worst);
}

// Solve A x = b (FP64 in/out, device, nrhs columns) with the grid's factorisation and
// iterative refinement on the FP64 stencil residual.  r, a32, b32 are scratch buffers of
// the same length: complex64 for FP32 grids; for FP64 grids a32 is complex128 (the
// correction) and b32 is unused.  An FP32 grid refines while each step reduces the
// residual at least 0.7-fold, up to max_refine32 steps; a non-finite residual, stagnation
// or running out of steps switches it to its FP64 fallback factorisation.
// FP32 refinement on the grid's FP32 factorisation: x = M^-1 b, then corrections while the
// FP64 stencil residual is above tol32; a single right-hand side whose plain refinement
// stalls continues with the Krylov refinement within the same step budget.  *need64: the
// factorisation could not resolve the system (non-finite residual, or refinement stalled
// or out of steps); *it: refinement steps (the first solve not counted), *kry: Krylov steps.
rci_status fp32_refine(rci_grid* g, const double2* b, double2* x, double2* r, void* a32,
                       void* b32, int nrhs, int* it_out, int* kry_out, double* worst,
                       bool* need64) {
  const int64_t n = g->N * nrhs;
  int it = 0, kry = 0;
  *need64 = false;
  CK(cudaMemsetAsync(x, 0, sizeof(double2) * n, g->s), "zero x");
  CK(cudaMemcpyAsync(r, b, sizeof(double2) * n, cudaMemcpyDeviceToDevice, g->s), "copy b");
  double prev = 1.0;
  while (true) {
    CK(launch_to_f32(r, (float2*)a32, n, g->s), "to fp32");
    CK(bcr_solve(g->bcr, g->cx, a32, b32, nrhs, g->s), "fp32 solve");
    CK(launch_add_f32(x, (const float2*)b32, n, g->s), "update");
    ++it;
    rci_status st = residual_ratio(g, b, x, r, nrhs, worst);
    if (st == RCI_ENUMERIC) {
      *need64 = true;
      break;
    }
    if (st != RCI_OK) return st;
    if (*worst <= g->tol32) break;
    if (it >= g->max_refine32 || (it >= 3 && *worst > 0.7 * prev)) {
      // plain refinement stalled: one right-hand side continues with the Krylov
      // refinement within the remaining step budget
      if (nrhs == 1 && it < g->max_refine32) {
        int ks = 0;
        st = krylov_refine(g, b, x, r, a32, b32, g->max_refine32 - it, &ks, worst);
        it += ks;
        kry = ks;
        if (st == RCI_OK && *worst <= g->tol32) break;
        if (st != RCI_OK && st != RCI_ENUMERIC) return st;
      }
      *need64 = true;
      break;
    }
    prev = *worst;
  }
  *it_out = it - 1;  // the first FP32 solve is not a refinement step
  *kry_out = kry;
  return RCI_OK;
}

// Factor the current design again with the FP32 factorisation on the SIMT pipe, after its
// tensor-core factorisation (3xTF32 products) could not resolve the system: one rounding per
// FMA is enough for designs that the 3.5-fold larger product error tips over, at a fraction
// of the cost of the FP64 factorisation.  *ok: the factorisation met no zero pivot.
rci_status simt_refactor(rci_grid* g, bool* ok) {
  *ok = false;
  bcr_set_simt(g->bcr, true);
  CK(bcr_factor(g->bcr, g->dg, g->cx, g->cy, g->s), "FP32 SIMT factor");
  int32_t st = 0;
  CK(bcr_read_status(g->bcr, &st, g->s, &g->growth), "FP32 SIMT factor status");
  *ok = st == DEV_OK;
  return RCI_OK;
}

rci_status refined_solve(rci_grid* g, const double2* b, double2* x, double2* r, void* a32,
                         void* b32, int nrhs, rci_info* info) {
  const int64_t n = g->N * nrhs;
  double worst = 0.0;
  int it = 0, kry = 0;
  bool fell_back = false;
  rci_status st = RCI_OK;
  if (g->d.prec == RCI_FP64) {
    st = solve64(g, g->bcr, b, x, r, (double2*)a32, nrhs, &it, &worst);
    if (st != RCI_OK) return st;
  } else {
    bool need64 = g->use64;
    if (!need64) {
      st = fp32_refine(g, b, x, r, a32, b32, nrhs, &it, &kry, &worst, &need64);
      if (st != RCI_OK) return st;
      if (need64 && !bcr_simt(g->bcr)) {
        // precision ladder: the FP32 SIMT factorisation before the FP64 one
        bool ok = false;
        st = simt_refactor(g, &ok);
        if (st != RCI_OK) return st;
        if (ok) {
          st = fp32_refine(g, b, x, r, a32, b32, nrhs, &it, &kry, &worst, &need64);
          if (st != RCI_OK) return st;
        }
      }
    }
    if (need64) {
      st = fp64_fallback(g);
      if (st != RCI_OK) return st;
      st = ensure_corr64(g, n);
      if (st != RCI_OK) return st;
      it = 0;
      st = solve64(g, g->bcr64, b, x, r, g->corr64, nrhs, &it, &worst);
      if (st != RCI_OK) return st;
      fell_back = true;
    }
  }
  if (info) {
    info->refine_iters = it;
    info->rel_residual = worst;
    info->fallback = fell_back ? 1 : 0;
    info->growth_est = fell_back ? g->growth64 : g->growth;
    info->krylov_steps = kry;
    info->simt_refactor = bcr_simt(g->bcr) ? 1 : 0;
  }
  if (nrhs > 1) {  // the multi-RHS solve runs tensor-core GEMMs with bounded waits
    int32_t dst = 0;
    CK(bcr_read_status(g->bcr, &dst, g->s), "solve status");
    if (dst == DEV_TIMEOUT) return fail(g, RCI_ETIMEOUT, "a bounded tensor-core wait expired");
  }
  double tol = (g->d.prec == RCI_FP64 || fell_back) ? 1e-9 : g->tol32;
  if (worst > tol) return fail(g, RCI_ENOCONV, "iterative refinement did not converge");
  return RCI_OK;
}

rci_status reciprocal_solve(rci_grid* g, const rci_objective* o, rci_info* info) {
  if (!g->factored) return fail(g, RCI_ESTATE, "grid is not factored");
  rci_status st = build_objective(g, o, g->b1);
  if (st != RCI_OK) return st;
  CK(cudaEventRecord(g->ev[2], g->s), "event");
  st = refined_solve(g, g->b1, g->x1, g->r1, g->r32, g->d32, 1, info);
  CK(cudaEventRecord(g->ev[3], g->s), "event");
  if (st != RCI_OK && st != RCI_ENOCONV) return st;
  CK(launch_gather_source_row(g->g, g->x1, g->vsrc, g->s), "gather v");
  if (info) {
    float ms = 0;
    cudaEventSynchronize(g->ev[3]);
    cudaEventElapsedTime(&ms, g->ev[2], g->ev[3]);
    info->ms_solve = ms;
  }
  return st;
}

rci_status run_angles(rci_grid* g, const rci_objective* o, const double* th_dev,
                      const double* wq_dev, int nq, double* f_dev, rci_info* info) {
  const GridGeom& G = g->g;
  // objective row / point (reuses the reciprocal builder for validation and crow)
  rci_status st = build_objective(g, o, g->b1);
  if (st != RCI_OK) return st;
  int chunk = nq < MAXQ ? nq : MAXQ;
  st = ensure_multi(g, chunk);
  if (st != RCI_OK) return st;
  int worst_it = 0, fb = 0, sr = 0;
  double worst_res = 0.0;
  rci_status agg = RCI_OK;
  for (int q0 = 0; q0 < nq; q0 += chunk) {
    int c = nq - q0 < chunk ? nq - q0 : chunk;
    CK(cudaMemsetAsync(g->mb, 0, sizeof(double2) * g->N * c, g->s), "zero sources");
    CK(launch_sources(G, th_dev + q0, c, c, g->mb, g->s), "sources");
    rci_info ci{};
    st = refined_solve(g, g->mb, g->mx, g->mr, g->m32a, g->m32b, c, &ci);
    if (st != RCI_OK && st != RCI_ENOCONV) return st;
    if (st == RCI_ENOCONV) agg = st;
    worst_it = ci.refine_iters > worst_it ? ci.refine_iters : worst_it;
    worst_res = ci.rel_residual > worst_res ? ci.rel_residual : worst_res;
    fb |= ci.fallback;
    sr |= ci.simt_refactor;
    if (o->kind == RCI_OBJ_POINT) {
      CK(launch_project_point(G, o->i_f, o->j_f, g->mx, c, c, f_dev + q0, g->s), "project");
    } else {
      CK(launch_project_row(G, g->crow, o->monitor_row, g->mx, c, c, f_dev + q0, g->s), "project");
    }
  }
  (void)wq_dev;
  if (info) {
    info->refine_iters = worst_it;
    info->rel_residual = worst_res;
    info->fallback = fb;
    info->simt_refactor = sr;
    info->growth_est = g->use64 ? g->growth64 : g->growth;
  }
  return agg;
}

rci_status ensure_theta(rci_grid* g, int nq) {
  if (g->th_cap >= nq) return RCI_OK;
  dfree(g, g->th_d);
  dfree(g, g->wq_d);
  dfree(g, g->f_d);
  g->th_d = g->wq_d = g->f_d = nullptr;
  CK(dalloc(g, &g->th_d, sizeof(double) * nq), "angles");
  CK(dalloc(g, &g->wq_d, sizeof(double) * nq), "angles");
  CK(dalloc(g, &g->f_d, sizeof(double) * nq), "angles");
  g->th_cap = nq;
  return RCI_OK;
}

rci_status finish_angles(rci_grid* g, int nq, double* fom, double* avg) {
  if (fom)
    CK(cudaMemcpyAsync(fom, g->f_d, sizeof(double) * nq, cudaMemcpyDeviceToHost, g->s), "fom copy");
  CK(launch_weighted_sum(g->wq_d, g->f_d, nq, g->dscal + 1, g->s), "weighted sum");
  double a = 0.0;
  CK(cudaMemcpyAsync(&a, g->dscal + 1, sizeof(double), cudaMemcpyDeviceToHost, g->s), "avg copy");
  CK(cudaStreamSynchronize(g->s), "avg copy");
  if (g->prof.on) g->prof.collect();
  if (!std::isfinite(a)) return fail(g, RCI_ENUMERIC, "non-finite brute-force average");
  if (avg) *avg = a;
  return RCI_OK;
}

}  // namespace

extern "C" {

const char* rci_status_str(rci_status s) {
  switch (s) {
    case RCI_OK: return "ok";
    case RCI_EINVAL: return "invalid argument";
    case RCI_ENOMEM: return "out of device memory";
    case RCI_ECUDA: return "CUDA error";
    case RCI_ESTATE: return "call out of order";
    case RCI_ESINGULAR: return "singular diagonal block";
    case RCI_ENOCONV: return "iterative refinement did not converge";
    case RCI_ENUMERIC: return "non-finite value";
    case RCI_ETIMEOUT: return "device wait timed out";
  }
  return "unknown status";
}

const char* rci_last_error(const rci_grid* g) { return g ? g->err.c_str() : ""; }

}  // extern "C"

namespace {
// Release a grid's memory and events; with sync, after draining the grid's stream.
void destroy_grid(rci_grid* g, bool sync) {
  DeviceGuard dg(g->device);
  if (sync && g->s) cudaStreamSynchronize(g->s);
  void* ps[] = {g->widths, g->eps, g->dg, g->cx, g->cy, g->dg0, g->kss, g->b1, g->x1, g->r1, g->r32, g->d32,
                g->crow, g->vsrc, g->lags, g->qpart, g->dscal, g->part_r, g->part_b, g->ratio,
                g->vf_scratch, g->dstatus, g->mb, g->mx, g->mr, g->m32a, g->m32b, g->th_d,
                g->wq_d, g->f_d, g->mu, g->gsrc, g->tpart, g->dgrad, g->cbuf, g->mF,
                g->tabbuf};
  for (void* p : ps) dfree(g, p);
  g->mem64.release(g->corr64);
  g->memk.release(g->kbuf);
  g->memk.release(g->kpart);
  bcr_destroy(g->bcr);
  bcr_destroy(g->bcr64);
  if (g->prof.pool) {
    for (int i = 0; i < g->prof.cap; ++i) cudaEventDestroy(g->prof.pool[i]);
    delete[] g->prof.pool;
    delete[] g->prof.recs;
  }
  for (cudaEvent_t e : g->ev)
    if (e) cudaEventDestroy(e);
  delete g;
}
}  // namespace

// A grid with no device work pending (its stream drained by the caller after its last
// call): released without waiting on the stream, which may since carry other work.
void rci_grid_destroy_idle(rci_grid* g) {
  if (g) destroy_grid(g, false);
}

extern "C" {

rci_status rci_destroy_grid(rci_grid* g) {
  if (!g) return RCI_OK;
  destroy_grid(g, true);
  return RCI_OK;
}

}  // extern "C"

namespace {

// Gradient buffers: the adjoint field, W v on the source plane and its partials, dF/dw.
cudaError_t alloc_grad_buffers(rci_grid* g) {
  if (g->mu) return cudaSuccess;
  const int64_t ns = g->g.n_src;
  RCI_CUDA_TRY(dalloc(g, &g->mu, sizeof(double2) * g->N));
  RCI_CUDA_TRY(dalloc(g, &g->gsrc, sizeof(double2) * ns));
  RCI_CUDA_TRY(dalloc(g, &g->tpart, sizeof(double2) * ns * toeplitz_mv_chunks(ns)));
  RCI_CUDA_TRY(dalloc(g, &g->dgrad, sizeof(double) * g->d.n_cells));
  return cudaSuccess;
}

// Every device buffer a single-RHS evaluation needs (and the gradient's when asked), from
// g->mem.  No kernel launch, no event, no synchronisation: with a counting allocator this
// is the exact footprint of the grid.
cudaError_t grid_alloc(rci_grid* g, bool with_grad) {
  const int64_t N = g->N, ns = g->g.n_src;
  const rci_grid_desc* desc = &g->d;
  RCI_CUDA_TRY(dalloc(g, &g->widths, sizeof(double) * desc->n_cells));
  RCI_CUDA_TRY(dalloc(g, &g->eps, sizeof(double) * N));
  RCI_CUDA_TRY(dalloc(g, &g->dg, sizeof(double2) * N));
  RCI_CUDA_TRY(dalloc(g, &g->cx, sizeof(double2) * N));
  RCI_CUDA_TRY(dalloc(g, &g->cy, sizeof(double2) * N));
  RCI_CUDA_TRY(dalloc(g, &g->dg0, sizeof(double2) * N));
  RCI_CUDA_TRY(dalloc(g, &g->kss, sizeof(double2) * N));
  RCI_CUDA_TRY(dalloc(g, &g->b1, sizeof(double2) * N));
  RCI_CUDA_TRY(dalloc(g, &g->x1, sizeof(double2) * N));
  RCI_CUDA_TRY(dalloc(g, &g->r1, sizeof(double2) * N));
  if (desc->prec == RCI_FP32_REFINE) {
    RCI_CUDA_TRY(dalloc(g, &g->r32, sizeof(float2) * N));
    RCI_CUDA_TRY(dalloc(g, &g->d32, sizeof(float2) * N));
  } else {
    RCI_CUDA_TRY(dalloc(g, &g->r32, sizeof(double2) * N));  // FP64 refinement corrections
  }
  RCI_CUDA_TRY(dalloc(g, &g->crow, sizeof(double2) * ns));
  RCI_CUDA_TRY(dalloc(g, &g->vsrc, sizeof(double2) * ns));
  RCI_CUDA_TRY(dalloc(g, &g->lags, sizeof(double) * ns));
  RCI_CUDA_TRY(dalloc(g, &g->qpart, sizeof(double) * qform_num_partials(ns)));
  RCI_CUDA_TRY(dalloc(g, &g->dscal, sizeof(double) * 8));
  RCI_CUDA_TRY(dalloc(g, &g->part_r, sizeof(double) * residual_blocks(g->g) * MAXQ));
  RCI_CUDA_TRY(dalloc(g, &g->part_b, sizeof(double) * residual_blocks(g->g) * MAXQ));
  RCI_CUDA_TRY(dalloc(g, &g->ratio, sizeof(double) * MAXQ));
  RCI_CUDA_TRY(dalloc(g, &g->vf_scratch, sizeof(double) * (2 * VF_ORDER + 6 * VF_NODES)));
  RCI_CUDA_TRY(dalloc(g, &g->dstatus, sizeof(int32_t)));
  RCI_CUDA_TRY(bcr_create(g->g.nx, g->g.ny, desc->prec, &g->mem, &g->bcr, nullptr));
  RCI_CUDA_TRY(bcr_reserve_ws(g->bcr, 1));
  if (with_grad) RCI_CUDA_TRY(alloc_grad_buffers(g));
  return cudaSuccess;
}

rci_grid* grid_shell(const rci_grid_desc* desc, cudaStream_t s, const DevMem* mem) {
  rci_grid* g = new (std::nothrow) rci_grid();
  if (!g) return nullptr;
  g->d = *desc;
  g->g = make_geom(*desc);
  g->s = s;
  g->device = desc->device;
  g->N = (int64_t)g->g.nx * g->g.ny;
  if (mem) g->mem = *mem;
  return g;
}

struct CountingArena {
  size_t total = 0;
  uintptr_t next = 4096;
};
cudaError_t counting_alloc(void* ctx, void** p, size_t bytes) {
  auto* c = static_cast<CountingArena*>(ctx);
  const size_t b = (bytes + 255) & ~(size_t)255;
  c->total += b;
  *p = reinterpret_cast<void*>(c->next);
  c->next += b;
  return cudaSuccess;
}
void counting_free(void*, void*) {}

}  // namespace

// Allocate a grid whose device memory comes from mem (nullptr: cudaMalloc), with the
// gradient buffers up front when asked.  Host bookkeeping and allocations only: no kernel,
// no event, no synchronisation (the serving runtime calls this under its admission lock).
rci_status rci_grid_alloc_with(const rci_grid_desc* desc, cudaStream_t stream, const DevMem* mem,
                               int with_grad, rci_grid** out) {
  if (!desc || !out) return RCI_EINVAL;
  *out = nullptr;
  std::string why;
  if (!desc_ok(desc, why)) return RCI_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || desc->device < 0 || desc->device >= ndev)
    return RCI_ECUDA;
  rci_grid* g = grid_shell(desc, stream, mem);
  if (!g) return RCI_ENOMEM;
  DeviceGuard guard(g->device);
  cudaError_t e = grid_alloc(g, with_grad != 0);
  if (e != cudaSuccess) {
    rci_destroy_grid(g);
    return e == cudaErrorMemoryAllocation ? RCI_ENOMEM : RCI_ECUDA;
  }
  *out = g;
  return RCI_OK;
}

// Second half of grid creation: the design-independent stencil coefficients and the
// events, then a synchronisation of the grid's stream.  On failure the caller destroys g.
rci_status rci_grid_init(rci_grid* g) {
  DeviceGuard guard(g->device);
  cudaError_t e;
  if ((e = cudaMemsetAsync(g->cx, 0, sizeof(double2) * g->N, g->s)) != cudaSuccess ||
      (e = launch_pml_coefficients(g->g, g->dg0, g->kss, g->cx, g->cy, g->b1, g->s)) != cudaSuccess)
    return cuda_fail(g, e, "grid setup");
  for (auto& ev : g->ev)
    if (!ev && (e = cudaEventCreateWithFlags(&ev, cudaEventDefault)) != cudaSuccess)
      return cuda_fail(g, e, "events");
  if ((e = cudaStreamSynchronize(g->s)) != cudaSuccess) return cuda_fail(g, e, "grid setup");
  return RCI_OK;
}

rci_status rci_grid_create_with(const rci_grid_desc* desc, cudaStream_t stream, const DevMem* mem,
                                int with_grad, rci_grid** out) {
  rci_status st = rci_grid_alloc_with(desc, stream, mem, with_grad, out);
  if (st != RCI_OK) return st;
  st = rci_grid_init(*out);
  if (st != RCI_OK) {
    rci_destroy_grid(*out);
    *out = nullptr;
  }
  return st;
}

// Point the grid's work at another stream (the grid must be idle: every call of the ABI
// returns with its stream drained or its results still to be read on that stream).
void rci_grid_rebind_stream(rci_grid* g, cudaStream_t s) {
  if (g) g->s = s;
}

extern "C" {

rci_status rci_create_grid(const rci_grid_desc* desc, void* stream, rci_grid** out) {
  return rci_grid_create_with(desc, (cudaStream_t)stream, nullptr, 0, out);
}

rci_status rci_grid_footprint(const rci_grid_desc* desc, int with_gradient, size_t* bytes) {
  if (!desc || !bytes) return RCI_EINVAL;
  std::string why;
  if (!desc_ok(desc, why)) return RCI_EINVAL;
  CountingArena c;
  DevMem m;
  m.ctx = &c;
  m.alloc_fn = counting_alloc;
  m.free_fn = counting_free;
  rci_grid* g = grid_shell(desc, nullptr, &m);
  if (!g) return RCI_ENOMEM;
  cudaError_t e = grid_alloc(g, with_gradient != 0);
  bcr_destroy(g->bcr);
  delete g;
  if (e != cudaSuccess) return RCI_EINVAL;
  *bytes = c.total;
  return RCI_OK;
}

rci_status rci_grid_query(const rci_grid* g, int64_t* nx, int64_t* ny, int64_t* n_src,
                          size_t* device_bytes) {
  if (!g) return RCI_EINVAL;
  if (nx) *nx = g->g.nx;
  if (ny) *ny = g->g.ny;
  if (n_src) *n_src = g->g.n_src;
  if (device_bytes) *device_bytes = g->bytes + (g->bcr ? bcr_bytes(g->bcr) : 0);
  return RCI_OK;
}

rci_status rci_set_design(rci_grid* g, const double* widths, int64_t n_cells, int on_device) {
  if (!g) return RCI_EINVAL;
  if (!widths) return fail(g, RCI_EINVAL, "widths is NULL");
  if (n_cells != g->d.n_cells) return fail(g, RCI_EINVAL, "need one width per cell");
  DeviceGuard dg(g->device);
  if (!on_device) {
    // host widths are checked here; device widths are checked by the raster kernel and
    // reported by the next rci_factor (no device-to-host round trip on that path)
    const double period = g->d.cell_px * g->g.h;
    for (int64_t m = 0; m < n_cells; ++m)
      if (!(widths[m] > 0.0 && widths[m] < period))
        return fail(g, RCI_EINVAL, "each width must lie in (0, period)");
  }
  CK(cudaMemsetAsync(g->dstatus, 0, sizeof(int32_t), g->s), "status");
  CK(cudaMemcpyAsync(g->widths, widths, sizeof(double) * n_cells,
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, g->s),
     "widths");
  {
    ProfScope ps(&g->prof, PF_SETUP, g->s, 0.0, 56.0 * g->N, 1);
    CK(launch_raster_eps(g->g, g->widths, g->eps, g->dg0, g->kss, g->dg, g->dstatus, g->s),
       "raster");
  }
  g->has_design = true;
  g->factored = false;
  g->use64 = false;
  bcr_set_simt(g->bcr, false);  // a new design starts on the tensor-core factorisation
  return RCI_OK;
}

rci_status rci_factor(rci_grid* g) {
  if (!g) return RCI_EINVAL;
  if (!g->has_design) return fail(g, RCI_ESTATE, "no design set");
  DeviceGuard dg(g->device);
  CK(cudaEventRecord(g->ev[0], g->s), "event");
  CK(bcr_factor(g->bcr, g->dg, g->cx, g->cy, g->s), "factor");
  CK(cudaEventRecord(g->ev[1], g->s), "event");
  int32_t st = 0, sd = 0;
  CK(cudaMemcpyAsync(&sd, g->dstatus, sizeof(int32_t), cudaMemcpyDeviceToHost, g->s), "status");
  CK(bcr_read_status(g->bcr, &st, g->s, &g->growth), "factor status");
  if (g->prof.on) g->prof.collect();
  if (sd == DEV_BADINPUT) {
    g->has_design = false;
    return fail(g, RCI_EINVAL, "a device width lies outside (0, period)");
  }
  if (st == DEV_TIMEOUT) return fail(g, RCI_ETIMEOUT, "a bounded tensor-core wait expired");
  if (st == DEV_SINGULAR) {
    if (g->d.prec == RCI_FP64) return fail(g, RCI_ESINGULAR, "zero pivot in a diagonal block");
    // an FP32 pivot vanished: factor this design again on the FP32 SIMT pipe and, if a pivot
    // vanishes there too, in FP64
    bool ok = false;
    if (!bcr_simt(g->bcr)) {
      rci_status ss = simt_refactor(g, &ok);
      if (ss != RCI_OK) return ss;
    }
    if (!ok) {
      rci_status fs = fp64_fallback(g);
      if (fs != RCI_OK) return fs;
    }
  }
  g->factored = true;
  return RCI_OK;
}

rci_status rci_solve(rci_grid* g, const double* b, double* x, int64_t nrhs, rci_info* info) {
  if (!g) return RCI_EINVAL;
  if (!b || !x || nrhs < 1 || nrhs > MAXQ) return fail(g, RCI_EINVAL, "bad solve arguments (1 <= nrhs <= 256)");
  if (!g->factored) return fail(g, RCI_ESTATE, "grid is not factored");
  DeviceGuard dg(g->device);
  rci_status st;
  if (nrhs == 1) {
    CK(cudaMemcpyAsync(g->b1, b, sizeof(double2) * g->N, cudaMemcpyDeviceToDevice, g->s), "copy b");
    st = refined_solve(g, g->b1, g->x1, g->r1, g->r32, g->d32, 1, info);
    CK(cudaMemcpyAsync(x, g->x1, sizeof(double2) * g->N, cudaMemcpyDeviceToDevice, g->s), "copy x");
  } else {
    st = ensure_multi(g, (int)nrhs);
    if (st != RCI_OK) return st;
    CK(cudaMemcpyAsync(g->mb, b, sizeof(double2) * g->N * nrhs, cudaMemcpyDeviceToDevice, g->s),
       "copy b");
    st = refined_solve(g, g->mb, g->mx, g->mr, g->m32a, g->m32b, (int)nrhs, info);
    CK(cudaMemcpyAsync(x, g->mx, sizeof(double2) * g->N * nrhs, cudaMemcpyDeviceToDevice, g->s),
       "copy x");
  }
  CK(cudaStreamSynchronize(g->s), "solve");
  if (g->prof.on) g->prof.collect();
  return st;
}

rci_status rci_solve_reciprocal(rci_grid* g, const rci_objective* obj, double* v_src_out,
                                double* v_full_out, rci_info* info) {
  if (!g) return RCI_EINVAL;
  DeviceGuard dg(g->device);
  rci_status st = reciprocal_solve(g, obj, info);
  if (st != RCI_OK && st != RCI_ENOCONV) return st;
  if (v_src_out)
    CK(cudaMemcpyAsync(v_src_out, g->vsrc, sizeof(double2) * g->g.n_src, cudaMemcpyDeviceToDevice,
                       g->s),
       "copy v");
  if (v_full_out) {
    CK(cudaMemcpyAsync(v_full_out, g->x1, sizeof(double2) * g->N, cudaMemcpyDeviceToDevice, g->s),
       "copy v");
    CK(launch_conj((double2*)v_full_out, g->N, g->s), "conj v");
  }
  CK(cudaStreamSynchronize(g->s), "reciprocal");
  return st;
}

rci_status rci_avg_intensity(rci_grid* g, const rci_objective* obj, const rci_light* light,
                             double* out, rci_info* info) {
  if (!g) return RCI_EINVAL;
  if (!out) return fail(g, RCI_EINVAL, "out is NULL");
  DeviceGuard dg(g->device);
  rci_status st = check_light(g, light);
  if (st != RCI_OK) return st;
  rci_status sst = reciprocal_solve(g, obj, info);
  if (sst != RCI_OK && sst != RCI_ENOCONV) return sst;
  st = ensure_lags(g, light);
  if (st != RCI_OK) return st;
  CK(cudaEventRecord(g->ev[4], g->s), "event");
  {
    const double n = (double)g->g.n_src;
    ProfScope ps(&g->prof, PF_QFORM, g->s, 2.0 * n * n, 24.0 * n, 2);
    CK(launch_qform(g->vsrc, g->lags, g->g.n_src, g->qpart, g->dscal, g->s), "qform");
  }
  CK(cudaEventRecord(g->ev[5], g->s), "event");
  double F = 0.0;
  CK(cudaMemcpyAsync(&F, g->dscal, sizeof(double), cudaMemcpyDeviceToHost, g->s), "qform copy");
  CK(cudaStreamSynchronize(g->s), "qform");
  if (g->prof.on) g->prof.collect();
  if (!std::isfinite(F)) return fail(g, RCI_ENUMERIC, "non-finite averaged intensity");
  *out = F;
  if (info) {
    float ms = 0;
    cudaEventElapsedTime(&ms, g->ev[4], g->ev[5]);
    info->ms_qform = ms;
    cudaEventElapsedTime(&ms, g->ev[0], g->ev[1]);
    info->ms_factor = ms;
  }
  return sst;
}

rci_status rci_avg_intensity_grad(rci_grid* g, const rci_objective* obj, const rci_light* light,
                                  double* value, double* dF_dwidths, rci_info* info) {
  if (!g) return RCI_EINVAL;
  DeviceGuard dg(g->device);
  rci_status st = check_light(g, light);
  if (st != RCI_OK) return st;
  const GridGeom& G = g->g;
  const int64_t ns = G.n_src;
  CK(alloc_grad_buffers(g), "gradient buffers");
  // forward: z = A^{-1} conj(w) in x1, v on the source plane, F = v^dag W v
  rci_info i1{};
  rci_status s1 = reciprocal_solve(g, obj, &i1);
  if (s1 != RCI_OK && s1 != RCI_ENOCONV) return s1;
  st = ensure_lags(g, light);
  if (st != RCI_OK) return st;
  {
    const double n = (double)ns;
    ProfScope ps(&g->prof, PF_QFORM, g->s, 2.0 * n * n, 24.0 * n, 2);
    CK(launch_qform(g->vsrc, g->lags, ns, g->qpart, g->dscal, g->s), "qform");
  }
  // adjoint right-hand side P_S^T (W v) and mu = A^{-1} P_S^T (W v)
  {
    const double n = (double)ns;
    ProfScope ps(&g->prof, PF_GRAD, g->s, 4.0 * n * n, 40.0 * n, 2);
    CK(launch_toeplitz_mv(g->vsrc, g->lags, ns, g->tpart, g->gsrc, g->s), "W v");
  }
  CK(cudaMemsetAsync(g->b1, 0, sizeof(double2) * g->N, g->s), "zero rhs");
  CK(launch_scatter_row(G, g->gsrc, G.j_src, g->b1, g->s), "adjoint rhs");
  rci_info i2{};
  CK(cudaEventRecord(g->ev[2], g->s), "event");
  rci_status s2 = refined_solve(g, g->b1, g->mu, g->r1, g->r32, g->d32, 1, &i2);
  CK(cudaEventRecord(g->ev[3], g->s), "event");
  if (s2 != RCI_OK && s2 != RCI_ENOCONV) return s2;
  {
    const double rows = (double)(G.j_p1 - G.j_p0);
    ProfScope ps(&g->prof, PF_GRAD, g->s, 2.0 * 20.0 * rows * g->d.n_cells,
                 2.0 * 48.0 * rows * g->d.n_cells, 1);
    CK(launch_width_grad(G, g->widths, g->mu, g->x1, g->kss, g->dgrad, g->s), "width gradient");
  }
  double F = 0.0;
  CK(cudaMemcpyAsync(&F, g->dscal, sizeof(double), cudaMemcpyDeviceToHost, g->s), "qform copy");
  std::vector<double> grad(dF_dwidths ? g->d.n_cells : 0);
  if (dF_dwidths)
    CK(cudaMemcpyAsync(grad.data(), g->dgrad, sizeof(double) * g->d.n_cells,
                       cudaMemcpyDeviceToHost, g->s),
       "gradient copy");
  CK(cudaStreamSynchronize(g->s), "gradient");
  if (g->prof.on) g->prof.collect();
  if (!std::isfinite(F)) return fail(g, RCI_ENUMERIC, "non-finite averaged intensity");
  for (double x : grad)
    if (!std::isfinite(x)) return fail(g, RCI_ENUMERIC, "non-finite gradient");
  if (value) *value = F;
  if (dF_dwidths) std::memcpy(dF_dwidths, grad.data(), sizeof(double) * grad.size());
  if (info) {
    info->refine_iters = i1.refine_iters > i2.refine_iters ? i1.refine_iters : i2.refine_iters;
    info->rel_residual = i1.rel_residual > i2.rel_residual ? i1.rel_residual : i2.rel_residual;
    info->fallback = i1.fallback | i2.fallback;
    info->growth_est = i2.growth_est > i1.growth_est ? i2.growth_est : i1.growth_est;
    info->krylov_steps = i1.krylov_steps + i2.krylov_steps;
    info->simt_refactor = i1.simt_refactor | i2.simt_refactor;
    float ms = 0;
    cudaEventElapsedTime(&ms, g->ev[2], g->ev[3]);
    info->ms_solve = i1.ms_solve + ms;
    cudaEventElapsedTime(&ms, g->ev[0], g->ev[1]);
    info->ms_factor = ms;
  }
  return s1 != RCI_OK ? s1 : s2;
}

rci_status rci_avg_intensity_correlated(rci_grid* g, const rci_objective* obj, const double* theta,
                                        const double* weight, int64_t nq, const double* C,
                                        double* out, rci_info* info) {
  if (!g) return RCI_EINVAL;
  if (!theta || !weight || !C || !out || nq < 1 || nq > 8192)
    return fail(g, RCI_EINVAL, "bad correlated-light arguments (1 <= nq <= 8192)");
  for (int64_t q = 0; q < nq; ++q)
    if (!(std::fabs(theta[q]) < M_PI / 2)) return fail(g, RCI_EINVAL, "angles must lie in (-pi/2, pi/2)");
  DeviceGuard dg(g->device);
  const size_t need = sizeof(double) * 2 * nq + sizeof(double2) * (nq * nq + nq) + 256;
  if (g->cbuf_bytes < need) {
    dfree(g, g->cbuf);
    g->cbuf = nullptr;
    g->cbuf_bytes = 0;
    CK(dalloc(g, &g->cbuf, need), "correlated-light buffers");
    g->cbuf_bytes = need;
  }
  double* th_d = (double*)g->cbuf;
  double* om_d = th_d + nq;
  double2* C_d = (double2*)(((uintptr_t)(om_d + nq) + 15) & ~(uintptr_t)15);
  double2* al_d = C_d + nq * nq;
  rci_status sst = reciprocal_solve(g, obj, info);
  if (sst != RCI_OK && sst != RCI_ENOCONV) return sst;
  CK(cudaMemcpyAsync(th_d, theta, sizeof(double) * nq, cudaMemcpyHostToDevice, g->s), "angles");
  CK(cudaMemcpyAsync(om_d, weight, sizeof(double) * nq, cudaMemcpyHostToDevice, g->s), "weights");
  CK(cudaMemcpyAsync(C_d, C, sizeof(double2) * nq * nq, cudaMemcpyHostToDevice, g->s), "correlation");
  {
    const double n = (double)g->g.n_src;
    ProfScope ps(&g->prof, PF_QFORM, g->s, 8.0 * n * nq + 8.0 * nq * (double)nq,
                 16.0 * n + 16.0 * nq * (double)nq, 2);
    CK(launch_correlated_form(g->g, g->vsrc, th_d, om_d, C_d, (int)nq, al_d, g->dscal, g->s),
       "correlated form");
  }
  double F = 0.0;
  CK(cudaMemcpyAsync(&F, g->dscal, sizeof(double), cudaMemcpyDeviceToHost, g->s), "form copy");
  CK(cudaStreamSynchronize(g->s), "correlated form");
  if (g->prof.on) g->prof.collect();
  if (!std::isfinite(F)) return fail(g, RCI_ENUMERIC, "non-finite averaged intensity");
  *out = F;
  return sst;
}

rci_status rci_avg_intensity_dense(rci_grid* g, const rci_objective* obj, const double* W,
                                   double* out, rci_info* info) {
  if (!g) return RCI_EINVAL;
  if (!W || !out) return fail(g, RCI_EINVAL, "W or out is NULL");
  DeviceGuard dg(g->device);
  rci_status sst = reciprocal_solve(g, obj, info);
  if (sst != RCI_OK && sst != RCI_ENOCONV) return sst;
  {
    const double n = (double)g->g.n_src;
    ProfScope ps(&g->prof, PF_QFORM, g->s, 8.0 * n * n, 16.0 * n * n, 2);
    // r1 (N complex) is free after the solve: the per-row partials
    CK(launch_dense_form(g->vsrc, (const double2*)W, g->g.n_src, (double*)g->r1, g->dscal, g->s),
       "dense form");
  }
  double F = 0.0;
  CK(cudaMemcpyAsync(&F, g->dscal, sizeof(double), cudaMemcpyDeviceToHost, g->s), "form copy");
  CK(cudaStreamSynchronize(g->s), "dense form");
  if (g->prof.on) g->prof.collect();
  if (!std::isfinite(F)) return fail(g, RCI_ENUMERIC, "non-finite averaged intensity");
  *out = F;
  return sst;
}

rci_status rci_avg_intensity_multi(rci_grid* g, const rci_objective* objs, int64_t K,
                                   const rci_light* light, double* F_out, double* total,
                                   rci_info* info) {
  if (!g) return RCI_EINVAL;
  if (!objs || K < 1 || K > (1 << 16)) return fail(g, RCI_EINVAL, "bad objective list");
  if (!g->factored) return fail(g, RCI_ESTATE, "grid is not factored");
  rci_status st = check_light(g, light);
  if (st != RCI_OK) return st;
  DeviceGuard dg(g->device);
  st = ensure_lags(g, light);
  if (st != RCI_OK) return st;
  if (g->mF_cap < K) {
    dfree(g, g->mF);
    g->mF = nullptr;
    g->mF_cap = 0;
    CK(dalloc(g, &g->mF, sizeof(double) * K), "multi-output results");
    g->mF_cap = (int)K;
  }
  const int chunk = K < MAXQ ? (int)K : MAXQ;
  st = ensure_multi(g, chunk);
  if (st != RCI_OK) return st;
  const GridGeom& G = g->g;
  int worst_it = 0, fb = 0, sr = 0;
  double worst_res = 0.0;
  rci_status agg = RCI_OK;
  for (int64_t o0 = 0; o0 < K; o0 += chunk) {
    const int c = K - o0 < chunk ? (int)(K - o0) : chunk;
    // conj(w_o) for the chunk's objectives, one column each
    for (int q = 0; q < c; ++q) {
      st = build_objective(g, &objs[o0 + q], g->b1);
      if (st != RCI_OK) return st;
      CK(launch_put_column(g->b1, g->N, c, q, g->mb, g->s), "objective column");
    }
    rci_info ci{};
    st = refined_solve(g, g->mb, g->mx, g->mr, g->m32a, g->m32b, c, &ci);
    if (st != RCI_OK && st != RCI_ENOCONV) return st;
    if (st == RCI_ENOCONV) agg = st;
    worst_it = ci.refine_iters > worst_it ? ci.refine_iters : worst_it;
    worst_res = ci.rel_residual > worst_res ? ci.rel_residual : worst_res;
    fb |= ci.fallback;
    sr |= ci.simt_refactor;
    for (int q = 0; q < c; ++q) {
      CK(launch_gather_source_col(G, g->mx, c, q, g->vsrc, g->s), "gather v");
      const double n = (double)G.n_src;
      ProfScope ps(&g->prof, PF_QFORM, g->s, 2.0 * n * n, 24.0 * n, 2);
      CK(launch_qform(g->vsrc, g->lags, G.n_src, g->qpart, g->mF + o0 + q, g->s), "qform");
    }
  }
  std::vector<double> h(K);
  CK(cudaMemcpyAsync(h.data(), g->mF, sizeof(double) * K, cudaMemcpyDeviceToHost, g->s), "results");
  CK(cudaStreamSynchronize(g->s), "multi-output");
  if (g->prof.on) g->prof.collect();
  double tot = 0.0;
  for (double x : h) {
    if (!std::isfinite(x)) return fail(g, RCI_ENUMERIC, "non-finite averaged intensity");
    tot += x;
  }
  if (F_out) std::memcpy(F_out, h.data(), sizeof(double) * K);
  if (total) *total = tot;
  if (info) {
    info->refine_iters = worst_it;
    info->rel_residual = worst_res;
    info->fallback = fb;
    info->simt_refactor = sr;
    info->growth_est = g->use64 ? g->growth64 : g->growth;
  }
  return agg;
}

rci_status rci_solve_angles(rci_grid* g, const rci_objective* obj, const double* theta,
                            const double* weight, int64_t nq, double* fom_per_angle,
                            double* avg_out, rci_info* info) {
  if (!g) return RCI_EINVAL;
  if (!theta || !weight || nq < 1 || nq > (1 << 20)) return fail(g, RCI_EINVAL, "bad angle arguments");
  if (!g->factored) return fail(g, RCI_ESTATE, "grid is not factored");
  for (int64_t q = 0; q < nq; ++q)
    if (!(std::fabs(theta[q]) < M_PI / 2)) return fail(g, RCI_EINVAL, "angles must lie in (-pi/2, pi/2)");
  DeviceGuard dg(g->device);
  rci_status st = ensure_theta(g, (int)nq);
  if (st != RCI_OK) return st;
  CK(cudaMemcpyAsync(g->th_d, theta, sizeof(double) * nq, cudaMemcpyHostToDevice, g->s), "angles");
  CK(cudaMemcpyAsync(g->wq_d, weight, sizeof(double) * nq, cudaMemcpyHostToDevice, g->s), "angles");
  rci_status rs = run_angles(g, obj, g->th_d, g->wq_d, (int)nq, g->f_d, info);
  if (rs != RCI_OK && rs != RCI_ENOCONV) return rs;
  st = finish_angles(g, (int)nq, fom_per_angle, avg_out);
  return st != RCI_OK ? st : rs;
}

rci_status rci_avg_bruteforce(rci_grid* g, const rci_objective* obj, const rci_light* light,
                              int64_t nq, double* fom_per_angle, double* avg_out, rci_info* info) {
  if (!g) return RCI_EINVAL;
  if (!g->factored) return fail(g, RCI_ESTATE, "grid is not factored");
  rci_status st = check_light(g, light);
  if (st != RCI_OK) return st;
  if (light->kind == RCI_LIGHT_USER_LAGS) return fail(g, RCI_EINVAL, "brute force needs a cone or an annulus");
  if (nq < 1 || nq > (1 << 20) || (light->kind == RCI_LIGHT_ANNULUS && nq % 2))
    return fail(g, RCI_EINVAL, "bad number of angles (even for an annulus)");
  DeviceGuard dg(g->device);
  st = ensure_theta(g, (int)nq);
  if (st != RCI_OK) return st;
  CK(launch_light_rule(light->kind, light->c, light->th1, light->th2, (int)nq, g->th_d, g->wq_d,
                       g->s),
     "quadrature rule");
  rci_status rs = run_angles(g, obj, g->th_d, g->wq_d, (int)nq, g->f_d, info);
  if (rs != RCI_OK && rs != RCI_ENOCONV) return rs;
  st = finish_angles(g, (int)nq, fom_per_angle, avg_out);
  return st != RCI_OK ? st : rs;
}

rci_status rci_qform_toeplitz(const double* v, const double* lags, int64_t n, double* out,
                              void* stream) {
  if (!v || !lags || !out || n < 1 || n > (1LL << 31)) return RCI_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  double* part = nullptr;
  double* dout = nullptr;
  size_t np = (size_t)qform_num_partials(n);
  if (cudaMalloc(&part, sizeof(double) * np) != cudaSuccess) return RCI_ENOMEM;
  if (cudaMalloc(&dout, sizeof(double)) != cudaSuccess) {
    cudaFree(part);
    return RCI_ENOMEM;
  }
  rci_status st = RCI_OK;
  double F = 0.0;
  if (launch_qform((const double2*)v, lags, n, part, dout, s) != cudaSuccess ||
      cudaMemcpyAsync(&F, dout, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    st = RCI_ECUDA;
  cudaFree(part);
  cudaFree(dout);
  if (st == RCI_OK) {
    if (!std::isfinite(F)) return RCI_ENUMERIC;
    *out = F;
  }
  return st;
}

rci_status rci_gauss_legendre(int64_t n, double a, double b, double* nodes, double* weights,
                              void* stream) {
  if (n < 1 || n > (1 << 20) || !nodes || !weights) return RCI_EINVAL;
  cudaError_t e = launch_gauss_legendre((int)n, a, b, nodes, weights, (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  return e == cudaSuccess ? RCI_OK : RCI_ECUDA;
}

rci_status rci_get_eps(rci_grid* g, double* eps_out) {
  if (!g) return RCI_EINVAL;
  if (!eps_out) return fail(g, RCI_EINVAL, "eps_out is NULL");
  if (!g->has_design) return fail(g, RCI_ESTATE, "no design set");
  DeviceGuard dg(g->device);
  CK(cudaMemcpyAsync(eps_out, g->eps, sizeof(double) * g->N, cudaMemcpyDeviceToDevice, g->s), "eps");
  CK(cudaStreamSynchronize(g->s), "eps");
  return RCI_OK;
}

rci_status rci_apply_operator(rci_grid* g, const double* x, double* y) {
  if (!g) return RCI_EINVAL;
  if (!x || !y) return fail(g, RCI_EINVAL, "NULL vector");
  if (!g->has_design) return fail(g, RCI_ESTATE, "no design set");
  DeviceGuard dg(g->device);
  CK(launch_apply_A(g->g, g->dg, g->cx, g->cy, (const double2*)x, (double2*)y, 1, g->s), "apply A");
  CK(cudaStreamSynchronize(g->s), "apply A");
  return RCI_OK;
}

rci_status rci_set_refinement(rci_grid* g, double tol, int32_t max_steps) {
  if (!g) return RCI_EINVAL;
  if (!(tol > 0.0) || max_steps < 0 || max_steps > 100)
    return fail(g, RCI_EINVAL, "need tol > 0 and 0 <= max_steps <= 100");
  if (g->d.prec == RCI_FP64) {
    g->tol64 = tol;
    g->max_refine64 = max_steps;
  } else {
    g->tol32 = tol;
    g->max_refine32 = max_steps + 1;  // counts the first FP32 solve
  }
  return RCI_OK;
}

uint64_t rci_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

rci_status rci_block_inverse(const void* src, void* out, int64_t n, int64_t batch, int32_t prec,
                             int32_t kernel, void* stream) {
  if (!src || !out || n < 1 || n > 1024 || batch < 1 || batch > (1 << 24) || kernel < 0 ||
      kernel > 2 || (prec != RCI_FP64 && prec != RCI_FP32_REFINE))
    return RCI_EINVAL;
  if (kernel == 2 && (prec != RCI_FP32_REFINE || n > 160)) return RCI_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int32_t* st = nullptr;
  int32_t h = 0;
  cudaError_t e = cudaMalloc((void**)&st, sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemsetAsync(st, 0, sizeof(int32_t), s);
  if (e == cudaSuccess) e = bcr_block_inverse(src, out, (int)n, (int)batch, prec, kernel, st, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, st, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(st);
  if (e == cudaErrorInvalidValue) return RCI_EINVAL;
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? RCI_ENOMEM : RCI_ECUDA;
  if (h == DEV_SINGULAR) return RCI_ESINGULAR;
  if (h == DEV_TIMEOUT) return RCI_ETIMEOUT;
  return RCI_OK;
}

rci_status rci_cgemm_batched(int64_t M, int64_t N, int64_t K, int32_t ta, int32_t tb,
                             double alpha, const void* A, int64_t lda, int64_t sA, const void* B,
                             int64_t ldb, int64_t sB, double beta, const void* C0, int64_t ldc0,
                             int64_t sC0, void* C, int64_t ldc, int64_t sC, int64_t batch,
                             int32_t prec, int32_t kernel, void* stream) {
  const int64_t lim = 1 << 20;
  if (!A || !B || !C || M < 1 || N < 1 || K < 1 || M > lim || N > lim || K > lim || batch < 1 ||
      batch > 65535 || kernel < 0 || kernel > 3 || (prec != RCI_FP64 && prec != RCI_FP32_REFINE))
    return RCI_EINVAL;
  if (!std::isfinite(alpha) || !std::isfinite(beta)) return RCI_EINVAL;
  const int64_t am = ta ? K : M, ak = ta ? M : K, bk = tb ? N : K, bn = tb ? K : N;
  if (lda < ak || ldb < bn || ldc < N || sA < 0 || sB < 0 || sC < 0 || (C0 && (ldc0 < N || sC0 < 0)))
    return RCI_EINVAL;
  (void)am;
  (void)bk;
  if (prec == RCI_FP64 && (kernel == 1 || kernel == 2)) return RCI_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int32_t* st = nullptr;
  int32_t h = 0;
  cudaError_t e = cudaMalloc((void**)&st, sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemsetAsync(st, 0, sizeof(int32_t), s);
  if (e == cudaSuccess)
    e = bcr_gemm((int)M, (int)N, (int)K, ta != 0, tb != 0, alpha, A, lda, sA, B, ldb, sB,
                 C0 ? beta : 0.0, C0, ldc0, sC0, C, ldc, sC, (int)batch, prec, kernel, st, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, st, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(st);
  if (e == cudaErrorInvalidValue) return RCI_EINVAL;
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? RCI_ENOMEM : RCI_ECUDA;
  if (h == DEV_TIMEOUT) return RCI_ETIMEOUT;
  return h == DEV_OK ? RCI_OK : RCI_ECUDA;
}

int64_t rci_set_wait_limit(int64_t cycles) {
  const long long old = tc_wait_limit();
  tc_set_wait_limit((long long)cycles);
  return (int64_t)old;
}

rci_status rci_profile_enable(rci_grid* g, int on) {
  if (!g) return RCI_EINVAL;
  DeviceGuard dg(g->device);
  Profiler& p = g->prof;
  if (on && !p.pool) {
    const int cap = 1 << 14;
    p.pool = new (std::nothrow) cudaEvent_t[cap];
    p.recs = new (std::nothrow) Profiler::Rec[cap];
    if (!p.pool || !p.recs) return fail(g, RCI_ENOMEM, "profiler allocation failed");
    for (int i = 0; i < cap; ++i) CK(cudaEventCreate(&p.pool[i]), "profiler events");
    p.cap = cap;
  }
  CK(cudaStreamSynchronize(g->s), "profiler");
  p.reset();
  p.on = on != 0;
  bcr_set_profiler(g->bcr, p.on ? &p : nullptr);
  return RCI_OK;
}

rci_status rci_profile_read(rci_grid* g, rci_profile* out) {
  if (!g || !out) return RCI_EINVAL;
  DeviceGuard dg(g->device);
  CK(cudaStreamSynchronize(g->s), "profiler");
  if (g->prof.on) g->prof.collect();
  std::memset(out, 0, sizeof(*out));
  for (int f = 0; f < PF_COUNT && f < RCI_PROFILE_FAMILIES; ++f) {
    out->ms[f] = g->prof.ms[f];
    out->flops[f] = g->prof.flops[f];
    out->bytes[f] = g->prof.bytes[f];
    out->launches[f] = g->prof.launches[f];
  }
  return RCI_OK;
}

}  // extern "C"
