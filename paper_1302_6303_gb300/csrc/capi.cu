// C ABI entry points (include/nrd.h): argument checks, context state, and the
// kernel sequences behind each call.
#include <cmath>
#include <cstdio>
#include <cstring>

#include "nrd_internal.h"

int step_pending_check(nrd_ctx* c, bool pending_ok, cudaStream_t s) {
  if (!c->pend) return NRD_OK;
  if (!pending_ok) {
    c->err = "a step is pending: call nrd_step_end first";
    return NRD_ESTATE;
  }
  if (s != c->pend_s) {
    c->err = "a step is pending: use the stream of nrd_step_begin";
    return NRD_ESTATE;
  }
  return NRD_OK;
}

namespace {

const char* kNullCtx = "null context";

// tile shapes with compiled stencil instances (32x8x8 is not one: the
// tangent stencil's five halo fields and face fluxes would need 243 KB of
// shared memory per CTA)
const int kShapes[][3] = {{32, 4, 4}, {32, 8, 4}, {32, 4, 8}, {32, 2, 4}, {16, 8, 4},
                          {16, 4, 8}, {16, 8, 8}, {16, 4, 4}, {8, 8, 8}, {8, 8, 4}};
const int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);

int fail(nrd_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

int check_launch(nrd_ctx* c) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(c, NRD_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  return NRD_OK;
}

// hierarchy and material present; with pending_ok, a step begun by
// nrd_step_begin may be in flight (the call must then use its stream),
// otherwise none may be
int need_ready(nrd_ctx* c, bool pending_ok = false, cudaStream_t s = nullptr) {
  if (!c->have_hier) return fail(c, NRD_ESTATE, "no hierarchy: call nrd_set_hierarchy first");
  if (!c->have_mat) return fail(c, NRD_ESTATE, "no material: call nrd_set_material first");
  return step_pending_check(c, pending_ok, s);
}

int check_params(const nrd_params* p, std::string& err) {
  if (!(p->k > 0.0)) { err = "k must be positive"; return NRD_EINVAL; }
  if (p->limiter != NRD_LIM_WILSON && p->limiter != NRD_LIM_PAPER_LITERAL) { err = "bad limiter"; return NRD_EINVAL; }
  if (p->restart < 1 || p->restart > 31) { err = "restart must be in [1, 31]"; return NRD_EINVAL; }
  if (p->max_krylov < 1) { err = "max_krylov must be >= 1"; return NRD_EINVAL; }
  if (p->jv_mode != NRD_JV_FD && p->jv_mode != NRD_JV_ANALYTIC) { err = "bad jv_mode"; return NRD_EINVAL; }
  if (p->pc_precision != NRD_PC_F64 && p->pc_precision != NRD_PC_F32) { err = "bad pc_precision"; return NRD_EINVAL; }
  if (p->nu1 < 0 || p->nu2 < 0 || p->coarse_sweeps < 0) { err = "sweep counts must be >= 0"; return NRD_EINVAL; }
  if (p->nmg < 1 || p->nmg > NRD_MAX_MG) { err = "nmg must be in [1, 12]"; return NRD_EINVAL; }
  if (!(p->rtol >= 0.0) || !(p->atol >= 0.0)) { err = "tolerances must be >= 0"; return NRD_EINVAL; }
  if (p->max_newton < 1) { err = "max_newton must be >= 1"; return NRD_EINVAL; }
  if (p->graph != 0 && p->graph != 1) { err = "graph must be 0 or 1"; return NRD_EINVAL; }
  if (p->smoother != NRD_SMOOTH_RBGS && p->smoother != NRD_SMOOTH_JACOBI &&
      p->smoother != NRD_SMOOTH_LINE) { err = "bad smoother"; return NRD_EINVAL; }
  if (!(p->omega > 0.0 && p->omega <= 1.0)) { err = "omega must be in (0, 1]"; return NRD_EINVAL; }
  if (!(p->eta_max > 0.0 && p->eta_max < 1.0)) { err = "eta_max must be in (0, 1)"; return NRD_EINVAL; }
  if (!(p->eta0 > 0.0 && p->eta0 <= p->eta_max)) { err = "eta0 must be in (0, eta_max]"; return NRD_EINVAL; }
  bool ok = (p->tile_x == 0 && p->tile_y == 0 && p->tile_z == 0);
  for (int t = 0; t < kNumShapes && !ok; t++)
    ok = (p->tile_x == kShapes[t][0] && p->tile_y == kShapes[t][1] && p->tile_z == kShapes[t][2]);
  if (!ok) { err = "unsupported tile shape"; return NRD_EINVAL; }
  return NRD_OK;
}

void set_model(nrd_ctx* c) {
  c->mp.k = c->p.k;
  c->mp.limiter = c->p.limiter;
  for (int f = 0; f < 6; f++) {
    c->mp.bc_R[f] = c->have_hier ? c->H.bc_R[f] : 0.0;
    c->mp.bc_type[f] = c->have_hier ? c->H.bc_type[f] : 0;
  }
}

void free_fields(nrd_ctx* c) {
  auto F = [](void* p) { if (p) cudaFree(p); };
  F(c->d_z); F(c->d_gz); F(c->d_gu); F(c->d_gv); F(c->d_cf); F(c->d_tmp); F(c->d_jc); F(c->d_pef); F(c->d_cc);
  F(c->d_lam); F(c->d_gam); F(c->d_z3);
  c->d_z3 = nullptr;
  c->d_z = nullptr; c->d_gz = nullptr; c->d_gu = nullptr; c->d_gv = nullptr; c->d_cf = nullptr;
  c->d_tmp = nullptr; c->d_jc = nullptr; c->d_pef = nullptr; c->d_cc = nullptr; c->d_lam = nullptr; c->d_gam = nullptr;
  c->lin_ready = false;
  reducer_free(c->R);
  if (c->pc) pc_free(c->pc);
  c->pc = nullptr;
  c->pc_ready = false;
  solver_free(c);
}

}  // namespace

int ctx_residual(nrd_ctx* c, const double* u, const double* b, double a0, double dt, double* F,
                 bool fill_ghosts, cudaStream_t s, const double* par) {
  Hier& H = c->H;
  if (fill_ghosts) launch_ghost_fill(H, c->mp, c->d_z, u, c->d_gu, 1, s);
  StencilIO io{};
  io.u = u;
  io.gu = c->d_gu;
  io.b = b;
  io.a0 = a0;
  io.dt = dt;
  io.par = par;
  io.out = F;
  io.cfflux = c->d_cf;
  io.pef = c->d_pef;   // the split form (every face once)
  c->timer.begin(NRD_TK_RESIDUAL, s);
  launch_stencil(H, c->mp, c->d_z, c->d_gz, ST_RESIDUAL, io, s, c->d_z3);
  c->timer.end(NRD_TK_RESIDUAL, s);
  launch_reflux(H, io, ST_RESIDUAL, s);
  return check_launch(c);
}

int ctx_linearise(nrd_ctx* c, const double* u, const double* b, double a0, double dt, double* F,
                  cudaStream_t s, const double* par, bool with_dz) {
  Hier& H = c->H;
  launch_ghost_fill(H, c->mp, c->d_z, u, c->d_gu, 1, s);
  StencilIO io{};
  io.u = u;
  io.gu = c->d_gu;
  io.b = b;
  io.a0 = a0;
  io.dt = dt;
  io.out = F;
  io.cfflux = c->d_cf;
  io.jc = c->d_jc;
  io.craw = pc_craw(c->pc);
  io.cc = c->d_cc;
  io.beta = dt / a0;
  io.par = par;
  pc_lin_targets(c->pc, &io.a32, &io.a64, &io.p2, &io.p2f);
  c->timer.begin(NRD_TK_LINEARISE, s);
  io.pef = with_dz ? nullptr : c->d_pef;   // the split form (every face once)
  launch_stencil(H, c->mp, c->d_z, c->d_gz, with_dz ? ST_LINZ : ST_LIN, io, s, c->d_z3);
  c->timer.end(NRD_TK_LINEARISE, s);
  launch_reflux(H, io, ST_RESIDUAL, s);
  c->timer.begin(NRD_TK_PC_SETUP, s);
  int rc = pc_finish(c->pc, H, u, c->d_z, a0, dt, true, s, par != nullptr);
  c->timer.end(NRD_TK_PC_SETUP, s);
  if (rc != NRD_OK) return fail(c, rc, "preconditioner set-up failed");
  c->lin_ready = true;
  c->lin_dz = with_dz;
  c->pc_ready = true;
  return check_launch(c);
}

int ctx_jv(nrd_ctx* c, const double* u, const double* v, const double* b, const double* F0,
           double a0, double dt, int mode, double* Jv, bool fill_u_ghosts, cudaStream_t s,
           const double* par) {
  Hier& H = c->H;
  if (mode == NRD_JV_FROZEN) {
    c->timer.begin(NRD_TK_GHOST, s);
    launch_ghost_fill(H, c->mp, c->d_z, v, c->d_gv, 0, s);
    c->timer.end(NRD_TK_GHOST, s);
    StencilIO io{};
    io.v = v;
    io.gv = c->d_gv;
    io.a0 = a0;
    io.dt = dt;
    io.par = par;
    io.out = Jv;
    io.cfflux = c->d_cf;
    c->timer.begin(NRD_TK_JV, s);
    launch_jv_frozen(H, c->mp, c->d_jc, c->d_cc, io, s);
    c->timer.end(NRD_TK_JV, s);
    launch_reflux(H, io, ST_JV, s);
    return check_launch(c);
  }
  if (fill_u_ghosts) launch_ghost_fill(H, c->mp, c->d_z, u, c->d_gu, 1, s);
  c->timer.begin(NRD_TK_GHOST, s);
  launch_ghost_fill(H, c->mp, c->d_z, v, c->d_gv, 0, s);
  c->timer.end(NRD_TK_GHOST, s);
  StencilIO io{};
  io.u = u;
  io.v = v;
  io.gu = c->d_gu;
  io.gv = c->d_gv;
  io.a0 = a0;
  io.dt = dt;
  io.out = Jv;
  io.cfflux = c->d_cf;
  if (mode == NRD_JV_FD) {
    c->timer.begin(NRD_TK_JV_FD, s);
    launch_fd_eps(H, c->R, u, v, c->p.u_min, 0, s);
    io.b = b;
    io.F0 = F0;
    io.eps = c->R.d_res + 0;
    launch_stencil(H, c->mp, c->d_z, c->d_gz, ST_FD, io, s, c->d_z3);
    c->timer.end(NRD_TK_JV_FD, s);
    launch_reflux(H, io, ST_FD, s);
  } else {
    c->timer.begin(NRD_TK_JV, s);
    launch_stencil(H, c->mp, c->d_z, c->d_gz, ST_JV, io, s, c->d_z3);
    c->timer.end(NRD_TK_JV, s);
    launch_reflux(H, io, ST_JV, s);
  }
  return check_launch(c);
}

extern "C" {

int nrd_params_default(nrd_params* p) {
  if (!p) return NRD_EINVAL;
  std::memset(p, 0, sizeof(*p));
  p->k = 0.01;
  p->limiter = NRD_LIM_WILSON;
  p->u_min = 1e-6;
  p->restart = 30;
  p->max_krylov = 300;
  p->jv_mode = NRD_JV_ANALYTIC;
  p->pc_precision = NRD_PC_F32;
  p->nu1 = 2;
  p->nu2 = 2;
  p->nmg = 4;
  p->coarse_sweeps = 4;
  p->rtol = 1e-8;
  p->atol = 0.0;
  p->max_newton = 20;
  p->eta_max = 0.9;
  p->ew_gamma = 0.9;
  p->tile_x = 0;
  p->tile_y = 0;
  p->tile_z = 0;
  p->graph = 1;
  p->smoother = NRD_SMOOTH_RBGS;
  p->omega = 6.0 / 7.0;
  p->eta0 = 0.3;
  return NRD_OK;
}

int nrd_create(const nrd_params* p, nrd_ctx** out) {
  if (!out) return NRD_EINVAL;
  *out = nullptr;
  nrd_params def;
  nrd_params_default(&def);
  std::string err;
  if (p && check_params(p, err) != NRD_OK) return NRD_EINVAL;
  nrd_ctx* c = new (std::nothrow) nrd_ctx();
  if (!c) return NRD_ENOMEM;
  c->p = p ? *p : def;
  set_model(c);
  *out = c;
  return NRD_OK;
}

int nrd_destroy(nrd_ctx* c) {
  if (!c) return NRD_EINVAL;
  if (c->pend) cudaStreamSynchronize(c->pend_s);   // nothing in flight may outlive the buffers
  c->timer.destroy();
  free_fields(c);
  if (c->have_hier) hier_free(c->H);
  delete c;
  return NRD_OK;
}

const char* nrd_last_error(const nrd_ctx* c) {
  if (!c) return kNullCtx;
  return c->err.c_str();
}

int nrd_set_params(nrd_ctx* c, const nrd_params* p) {
  if (!c || !p) return NRD_EINVAL;
  if (step_pending_check(c, false, nullptr)) return NRD_ESTATE;
  std::string err;
  if (check_params(p, err) != NRD_OK) return fail(c, NRD_EINVAL, err);
  bool retile = (p->tile_x != c->p.tile_x || p->tile_y != c->p.tile_y ||
                 p->tile_z != c->p.tile_z);
  bool repc = (p->nmg != c->p.nmg || p->pc_precision != c->p.pc_precision ||
               p->restart != c->p.restart);
  c->p = *p;
  c->gen++;
  set_model(c);
  if (c->pc) {
    pc_set_sweeps(c->pc, p->nu1, p->nu2, p->coarse_sweeps);
    pc_set_smoother(c->pc, p->smoother, p->omega);
  }
  if (c->have_hier && retile) {
    c->H.tile_x = p->tile_x ? p->tile_x : 32;
    c->H.tile_y = p->tile_y ? p->tile_y : 4;
    c->H.tile_z = p->tile_z ? p->tile_z : 4;
    std::string err;
    int rc = hier_tiles(c->H, err);
    if (rc != NRD_OK) return fail(c, rc, err);
    if (c->pc) pc_drop_graphs(c->pc);
  }
  if (c->have_hier && repc) {
    return fail(c, NRD_ESTATE, "nmg, precision or restart changed: call nrd_set_hierarchy "
                               "again");
  }
  return NRD_OK;
}

int nrd_set_hierarchy(nrd_ctx* c, int nlevels, const int* nboxes, const int* boxes,
                      const int* bc_type, const double* bc_R) {
  if (!c) return NRD_EINVAL;
  if (step_pending_check(c, false, nullptr)) return NRD_ESTATE;
  if (!nboxes || !boxes || !bc_type || !bc_R) return fail(c, NRD_EINVAL, "null argument");
  free_fields(c);
  if (c->have_hier) hier_free(c->H);
  c->have_hier = false;
  c->have_mat = false;
  c->H = Hier();
  c->H.tile_x = c->p.tile_x ? c->p.tile_x : 32;
  c->H.tile_y = c->p.tile_y ? c->p.tile_y : 4;
  c->H.tile_z = c->p.tile_z ? c->p.tile_z : 4;
  std::string err;
  int rc = hier_build(c->H, nlevels, nboxes, boxes, bc_type, bc_R, err);
  if (rc != NRD_OK) return fail(c, rc, err);
  rc = hier_upload(c->H, err);
  if (rc != NRD_OK) {
    hier_free(c->H);
    return fail(c, rc, err);
  }
  Hier& H = c->H;
  size_t N = H.N, G = H.G;
  bool ok = cudaMalloc(&c->d_z, N * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&c->d_gz, (G ? G : 1) * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&c->d_gu, 2 * (G ? G : 1) * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&c->d_gv, 2 * (G ? G : 1) * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&c->d_cf, 2 * (G ? G : 1) * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&c->d_tmp, 2 * N * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&c->d_jc, 6 * (3 * N + G) * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&c->d_pef, 2 * (3 * N + G) * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&c->d_cc, 3 * N * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&c->d_lam, 2 * (3 * N + G) * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&c->d_gam, 3 * (G ? G : 1) * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&c->d_z3, (N + G) * sizeof(double)) == cudaSuccess &&
            reducer_init(c->R, (int)N) == NRD_OK;
  if (!ok) {
    free_fields(c);
    hier_free(c->H);
    return fail(c, NRD_ENOMEM, "device allocation failed");
  }
  cudaMemset(c->d_cf, 0, 2 * (G ? G : 1) * sizeof(double));
  rc = pc_alloc(&c->pc, H, c->p, err);
  if (rc != NRD_OK) {
    free_fields(c);
    hier_free(c->H);
    return fail(c, rc, err);
  }
  if (cudaDeviceSynchronize() != cudaSuccess) {
    free_fields(c);
    hier_free(c->H);
    return fail(c, NRD_ECUDA, "device synchronisation failed");
  }
  c->have_hier = true;
  set_model(c);
  return NRD_OK;
}

int nrd_layout(const nrd_ctx* c, int64_t* ncells, int64_t* nghosts, int64_t* nleaf) {
  if (!c) return NRD_EINVAL;
  if (!c->have_hier) return NRD_ESTATE;
  if (ncells) *ncells = c->H.N;
  if (nghosts) *nghosts = c->H.G;
  if (nleaf) *nleaf = c->H.nleaf;
  return NRD_OK;
}

int nrd_set_material(nrd_ctx* c, const float* z, cudaStream_t s) {
  if (!c) return NRD_EINVAL;
  if (step_pending_check(c, false, nullptr)) return NRD_ESTATE;
  if (!c->have_hier) return fail(c, NRD_ESTATE, "no hierarchy");
  if (!z) return fail(c, NRD_EINVAL, "null z");
  if (cudaMemcpyAsync(c->d_z, z, (size_t)c->H.N * sizeof(float), cudaMemcpyDeviceToDevice, s) !=
      cudaSuccess)
    return fail(c, NRD_ECUDA, "copy of z failed");
  launch_ghost_z(c->H, c->d_z, c->d_gz, s);
  launch_cube(c->H, c->d_z, c->d_gz, c->d_z3, s);
  c->have_mat = true;
  c->pc_ready = false;
  c->lin_ready = false;
  return check_launch(c);
}

int nrd_ghost_fill(nrd_ctx* c, const double* u, double* gE, double* gT, float* gz, cudaStream_t s) {
  if (!c) return NRD_EINVAL;
  int rc = need_ready(c);
  if (rc) return rc;
  if (!u || !gE || !gT) return fail(c, NRD_EINVAL, "null argument");
  Hier& H = c->H;
  launch_ghost_fill(H, c->mp, c->d_z, u, c->d_gu, 1, s);
  size_t G = H.G;
  if (G) {
    cudaMemcpyAsync(gE, c->d_gu, G * sizeof(double), cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(gT, c->d_gu + G, G * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (gz) cudaMemcpyAsync(gz, c->d_gz, G * sizeof(float), cudaMemcpyDeviceToDevice, s);
  }
  return check_launch(c);
}

int nrd_residual(nrd_ctx* c, const double* u, const double* b, double a0, double dt, double* F,
                 cudaStream_t s) {
  if (!c) return NRD_EINVAL;
  int rc = need_ready(c);
  if (rc) return rc;
  if (!u || !b || !F) return fail(c, NRD_EINVAL, "null argument");
  return ctx_residual(c, u, b, a0, dt, F, true, s);
}

int nrd_jv(nrd_ctx* c, const double* u, const double* v, const double* b, const double* F0,
           double a0, double dt, int mode, double* Jv, cudaStream_t s) {
  if (!c) return NRD_EINVAL;
  int rc = need_ready(c);
  if (rc) return rc;
  if (!u || !v || !Jv) return fail(c, NRD_EINVAL, "null argument");
  if (mode != NRD_JV_FD && mode != NRD_JV_ANALYTIC && mode != NRD_JV_FROZEN)
    return fail(c, NRD_EINVAL, "bad mode");
  if (mode == NRD_JV_FD && (!b || !F0)) return fail(c, NRD_EINVAL, "FD mode needs b and F0");
  if (mode == NRD_JV_FROZEN && !c->lin_ready)
    return fail(c, NRD_ESTATE, "NRD_JV_FROZEN needs nrd_linearise first");
  return ctx_jv(c, u, v, b, F0, a0, dt, mode, Jv, true, s);
}

int nrd_linearise(nrd_ctx* c, const double* u, const double* b, double a0, double dt, double* F,
                  cudaStream_t s) {
  if (!c) return NRD_EINVAL;
  int rc = need_ready(c);
  if (rc) return rc;
  if (!u || !b || !F) return fail(c, NRD_EINVAL, "null argument");
  if (!(a0 > 0.0) || !(dt > 0.0)) return fail(c, NRD_EINVAL, "a0 and dt must be positive");
  return ctx_linearise(c, u, b, a0, dt, F, s, nullptr, true);
}

int nrd_vjp(nrd_ctx* c, const double* w, double a0, double dt, double* JTw, double* dz,
            cudaStream_t s) {
  if (!c) return NRD_EINVAL;
  int rc = need_ready(c);
  if (rc) return rc;
  if (!w || !JTw) return fail(c, NRD_EINVAL, "null argument");
  if (!c->lin_ready) return fail(c, NRD_ESTATE, "nrd_vjp needs nrd_linearise first");
  if (dz && !c->lin_dz)
    return fail(c, NRD_ESTATE, "dz needs the material partials: call nrd_linearise first");
  launch_vjp(c->H, c->d_jc, c->d_cc, c->d_z, w, c->d_lam, c->d_gam, a0, dt, JTw, dz, s);
  return check_launch(c);
}

int nrd_adjoint_solve(nrd_ctx* c, const double* g, double a0, double dt, double rtol,
                      double* lam, nrd_stats* st, cudaStream_t s) {
  if (!c) return NRD_EINVAL;
  int rc = need_ready(c);
  if (rc) return rc;
  if (!g || !lam) return fail(c, NRD_EINVAL, "null argument");
  if (!c->lin_ready) return fail(c, NRD_ESTATE, "nrd_adjoint_solve needs nrd_linearise first");
  if (!(rtol > 0.0)) return fail(c, NRD_EINVAL, "rtol must be positive");
  return solver_adjoint(c, g, a0, dt, rtol, lam, st, s);
}

int nrd_fd_eps(nrd_ctx* c, const double* u, const double* v, double* eps_host, cudaStream_t s) {
  if (!c) return NRD_EINVAL;
  int rc = need_ready(c);
  if (rc) return rc;
  if (!u || !v || !eps_host) return fail(c, NRD_EINVAL, "null argument");
  launch_fd_eps(c->H, c->R, u, v, c->p.u_min, 0, s);
  cudaMemcpyAsync(c->R.h_res, c->R.d_res, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return fail(c, NRD_ECUDA, "sync failed");
  *eps_host = c->R.h_res[0];
  return check_launch(c);
}

int nrd_dot(nrd_ctx* c, const double* x, const double* y, double* out, cudaStream_t s) {
  if (!c) return NRD_EINVAL;
  if (!c->have_hier) return fail(c, NRD_ESTATE, "no hierarchy");
  if (step_pending_check(c, true, s)) return NRD_ESTATE;
  if (!x || !y || !out) return fail(c, NRD_EINVAL, "null argument");
  launch_wdot(c->H, c->R, x, y, 1, s);
  cudaMemcpyAsync(c->R.h_res + 1, c->R.d_res + 1, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return fail(c, NRD_ECUDA, "sync failed");
  *out = c->R.h_res[1];
  return check_launch(c);
}

int nrd_precond_setup(nrd_ctx* c, const double* u, double a0, double dt, cudaStream_t s) {
  if (!c) return NRD_EINVAL;
  int rc = need_ready(c);
  if (rc) return rc;
  if (!u) return fail(c, NRD_EINVAL, "null argument");
  if (!(a0 > 0.0) || !(dt > 0.0)) return fail(c, NRD_EINVAL, "a0 and dt must be positive");
  launch_ghost_fill(c->H, c->mp, c->d_z, u, c->d_gu, 1, s);
  c->timer.begin(NRD_TK_PC_SETUP, s);
  rc = pc_setup(c->pc, c->H, c->mp, u, c->d_gu, c->d_z, c->d_gz, a0, dt, s);
  c->timer.end(NRD_TK_PC_SETUP, s);
  if (rc != NRD_OK) return fail(c, rc, "preconditioner set-up failed");
  c->pc_ready = true;
  return check_launch(c);
}

int nrd_precond_apply(nrd_ctx* c, const double* w, double* y, cudaStream_t s) {
  if (!c) return NRD_EINVAL;
  int rc = need_ready(c);
  if (rc) return rc;
  if (!c->pc_ready) return fail(c, NRD_ESTATE, "call nrd_precond_setup first");
  if (!w || !y) return fail(c, NRD_EINVAL, "null argument");
  c->timer.begin(NRD_TK_PC_APPLY, s);
  rc = pc_apply(c->pc, c->H, w, y, s);
  c->timer.end(NRD_TK_PC_APPLY, s);
  if (rc != NRD_OK) return fail(c, rc, "preconditioner apply failed");
  return check_launch(c);
}

int nrd_newton(nrd_ctx* c, double* u, const double* b, double a0, double dt, nrd_stats* st,
               cudaStream_t s) {
  if (!c) return NRD_EINVAL;
  int rc = need_ready(c);
  if (rc) return rc;
  if (!u || !b) return fail(c, NRD_EINVAL, "null argument");
  if (!(a0 > 0.0) || !(dt > 0.0)) return fail(c, NRD_EINVAL, "a0 and dt must be positive");
  return solver_newton(c, u, b, a0, dt, st, s);
}

// checks and the history combination of a step:
// b = (1+alpha) u_n - alpha^2/(1+alpha) u_{n-1}, a0 = (1+2 alpha)/(1+alpha)
// (Eq. bdf2); backward Euler (Eq. be): b = u_n, a0 = 1.
static int step_prepare(nrd_ctx* c, double* u, const double* u_n, const double* u_nm1,
                        double dt, double dt_prev, double* a0, cudaStream_t s) {
  int rc = need_ready(c);
  if (rc) return rc;
  if (!u || !u_n) return fail(c, NRD_EINVAL, "null argument");
  if (!(dt > 0.0)) return fail(c, NRD_EINVAL, "dt must be positive");
  if (u_nm1 && !(dt_prev > 0.0)) return fail(c, NRD_EINVAL, "dt_prev must be positive for BDF2");
  rc = solver_alloc(c);
  if (rc != NRD_OK) return rc;
  const int n2 = 2 * c->H.N;
  cudaMemcpyAsync(c->d_b, u_n, n2 * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (u_nm1) {
    const double al = dt / dt_prev;
    *a0 = (1.0 + 2.0 * al) / (1.0 + al);
    launch_axpy(n2, al, u_n, c->d_b, s);                       // (1 + al) u_n
    launch_axpy(n2, -al * al / (1.0 + al), u_nm1, c->d_b, s);
  } else {
    *a0 = 1.0;
  }
  return NRD_OK;
}

int nrd_step(nrd_ctx* c, double* u, const double* u_n, const double* u_nm1, double dt,
             double dt_prev, nrd_stats* st, cudaStream_t s) {
  if (!c) return NRD_EINVAL;
  double a0 = 1.0;
  const int rc = step_prepare(c, u, u_n, u_nm1, dt, dt_prev, &a0, s);
  if (rc) return rc;
  return solver_newton(c, u, c->d_b, a0, dt, st, s);
}

int nrd_step_begin(nrd_ctx* c, double* u, const double* u_n, const double* u_nm1, double dt,
                   double dt_prev, cudaStream_t s) {
  if (!c) return NRD_EINVAL;
  double a0 = 1.0;
  const int rc = step_prepare(c, u, u_n, u_nm1, dt, dt_prev, &a0, s);
  if (rc) return rc;
  return solver_newton_begin(c, u, c->d_b, a0, dt, s);
}

int nrd_step_end(nrd_ctx* c, nrd_stats* st) {
  if (!c) return NRD_EINVAL;
  return solver_newton_end(c, st);
}

int nrd_tag(nrd_ctx* c, const double* u, double thr_c, double thr_g, double thr_r, uint8_t* tags,
            cudaStream_t s) {
  if (!c) return NRD_EINVAL;
  int rc = need_ready(c, true, s);
  if (rc) return rc;
  if (!u || !tags) return fail(c, NRD_EINVAL, "null argument");
  Hier& H = c->H;
  size_t N = H.N;
  // composite values: covered cells := mean of their children
  cudaMemcpyAsync(c->d_tmp, u, 2 * N * sizeof(double), cudaMemcpyDeviceToDevice, s);
  launch_average_down(H, c->d_tmp, 2, (int)N, s);
  launch_ghost_fill(H, c->mp, c->d_z, c->d_tmp, c->d_gu, 1, s);
  launch_emax(H, c->R, u, 2, s);
  launch_tag(H, c->d_tmp, c->d_gu, thr_c, thr_g, thr_r, c->R.d_res + 2, tags, s);
  return check_launch(c);
}

int nrd_autotune(nrd_ctx* c, const double* u, const double* b, double a0, double dt,
                 int* tile_out, double* ms_out, cudaStream_t s) {
  if (!c) return NRD_EINVAL;
  int rc = need_ready(c);
  if (rc) return rc;
  if (!u || !b) return fail(c, NRD_EINVAL, "null argument");
  if (!(a0 > 0.0) || !(dt > 0.0)) return fail(c, NRD_EINVAL, "a0 and dt must be positive");
  rc = solver_alloc(c);
  if (rc != NRD_OK) return rc;
  Hier& H = c->H;
  const size_t n2 = 2 * (size_t)H.N;
  bool timer_on = c->timer.on;
  c->timer.on = false;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int best = -1;
  float best_ms = 1e30f;
  std::string err;
  for (int t = 0; t < kNumShapes; t++) {
    H.tile_x = kShapes[t][0];
    H.tile_y = kShapes[t][1];
    H.tile_z = kShapes[t][2];
    c->gen++;
    if (hier_tiles(H, err) != NRD_OK) continue;
    pc_drop_graphs(c->pc);
    float ms = 0.0f;
    for (int rep = 0; rep < 4; rep++) {
      cudaEventRecord(e0, s);
      ctx_linearise(c, u, b, a0, dt, c->d_F, s);
      pc_apply(c->pc, H, c->d_F, c->d_w, s);
      ctx_jv(c, u, c->d_w, nullptr, nullptr, a0, dt, NRD_JV_FROZEN, c->d_r, false, s);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        c->timer.on = timer_on;
        return fail(c, NRD_ECUDA, "autotune synchronisation failed");
      }
      float m = 0.0f;
      cudaEventElapsedTime(&m, e0, e1);
      if (rep > 0) ms += m;
    }
    if (ms < best_ms) {
      best_ms = ms;
      best = t;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->timer.on = timer_on;
  if (best < 0) return fail(c, NRD_ECUDA, "no tile shape could be timed");
  H.tile_x = c->p.tile_x = kShapes[best][0];
  H.tile_y = c->p.tile_y = kShapes[best][1];
  H.tile_z = c->p.tile_z = kShapes[best][2];
  c->gen++;
  if (hier_tiles(H, err) != NRD_OK) return fail(c, NRD_ECUDA, err);
  pc_drop_graphs(c->pc);
  c->lin_ready = false;
  (void)n2;
  if (tile_out) {
    tile_out[0] = H.tile_x;
    tile_out[1] = H.tile_y;
    tile_out[2] = H.tile_z;
  }
  if (ms_out) *ms_out = best_ms / 3.0;
  return check_launch(c);
}

int nrd_autotune_sweeps(nrd_ctx* c, const double* u_n, const double* u_nm1, double dt,
                        double dt_prev, int* nu_out, double* ms_out, cudaStream_t s) {
  if (!c) return NRD_EINVAL;
  int rc = need_ready(c);
  if (rc) return rc;
  if (!u_n || !(dt > 0.0)) return fail(c, NRD_EINVAL, "bad argument");
  // candidates (nu1, nu2, coarse sweeps, smoother): the paper's V(1,0) up to
  // V(3,3), with red-black Gauss-Seidel and with damped Jacobi (Sec. 4.3)
  const int sched[][3] = {{1, 0, 2}, {1, 1, 2}, {2, 1, 3}, {2, 2, 4}, {3, 3, 6}};
  const int nsched = sizeof(sched) / sizeof(sched[0]);
  int cand[2 * nsched][4];
  for (int q = 0; q < 2 * nsched; q++) {
    for (int t = 0; t < 3; t++) cand[q][t] = sched[q % nsched][t];
    cand[q][3] = (q < nsched) ? NRD_SMOOTH_RBGS : NRD_SMOOTH_JACOBI;
  }
  const int ncand = 2 * nsched;
  const size_t n2 = 2 * (size_t)c->H.N;
  bool timer_on = c->timer.on;
  c->timer.on = false;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int best = -1;
  float best_ms = 1e30f;
  for (int q = 0; q < ncand; q++) {
    c->p.nu1 = cand[q][0];
    c->p.nu2 = cand[q][1];
    c->p.coarse_sweeps = cand[q][2];
    c->p.smoother = cand[q][3];
    pc_set_sweeps(c->pc, cand[q][0], cand[q][1], cand[q][2]);
    pc_set_smoother(c->pc, cand[q][3], c->p.omega);
    c->gen++;
    float ms = 0.0f;
    bool ok = true;
    for (int rep = 0; rep < 2; rep++) {
      cudaMemcpyAsync(c->d_tmp, u_n, n2 * sizeof(double), cudaMemcpyDeviceToDevice, s);
      nrd_stats st;
      cudaEventRecord(e0, s);
      int r = nrd_step(c, c->d_tmp, u_n, u_nm1, dt, dt_prev, &st, s);
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      if (r != NRD_OK) { ok = false; break; }
      if (rep == 1) cudaEventElapsedTime(&ms, e0, e1);
    }
    if (ok && ms < best_ms) {
      best_ms = ms;
      best = q;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->timer.on = timer_on;
  if (best < 0) return fail(c, NRD_ENONCONV, "no sweep schedule converged");
  c->p.nu1 = cand[best][0];
  c->p.nu2 = cand[best][1];
  c->p.coarse_sweeps = cand[best][2];
  c->p.smoother = cand[best][3];
  pc_set_sweeps(c->pc, cand[best][0], cand[best][1], cand[best][2]);
  pc_set_smoother(c->pc, cand[best][3], c->p.omega);
  c->gen++;
  if (nu_out) {
    nu_out[0] = cand[best][0];
    nu_out[1] = cand[best][1];
    nu_out[2] = cand[best][2];
    nu_out[3] = cand[best][3];
  }
  if (ms_out) *ms_out = best_ms;
  return check_launch(c);
}

int nrd_timing_enable(nrd_ctx* c, int enable) {
  if (!c) return NRD_EINVAL;
  if (step_pending_check(c, false, nullptr)) return NRD_ESTATE;
  c->timer.on = enable != 0;
  c->timer.reset();
  return NRD_OK;
}

int nrd_timing_read(nrd_ctx* c, int group, double* ms, int64_t* launches) {
  if (!c) return NRD_EINVAL;
  if (group < 0 || group >= NRD_TK_COUNT || !ms || !launches)
    return fail(c, NRD_EINVAL, "bad timing group or null output");
  double tot = 0.0;
  size_t n = c->timer.used[group];
  for (size_t i = 0; i + 1 < n; i += 2) {
    if (cudaEventSynchronize(c->timer.ev[group][i + 1]) != cudaSuccess)
      return fail(c, NRD_ECUDA, "event synchronisation failed");
    float t = 0.0f;
    cudaEventElapsedTime(&t, c->timer.ev[group][i], c->timer.ev[group][i + 1]);
    tot += t;
  }
  *ms = tot;
  *launches = (int64_t)(n / 2);
  return NRD_OK;
}

}  // extern "C"
