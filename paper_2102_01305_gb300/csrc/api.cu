// C ABI of libibl (declared in include/ibl.h): validation, device memory,
// the per-step launch sequence and host<->device copies.  No arithmetic of
// the method runs on the host; every step of the path is a kernel.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "ibl_internal.cuh"

static std::string g_create_err;

namespace ibl {

ibl_status fail(ibl_ctx* c, ibl_status s, const std::string& msg) {
  if (c) c->err = msg;
  else g_create_err = msg;
  return s;
}

ibl_status cuda_check(ibl_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return IBL_OK;
  const std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) return fail(c, IBL_ENOMEM, m);
  return fail(c, IBL_ECUDA, m);
}

}  // namespace ibl

using namespace ibl;

#define CK(expr, what)                                         \
  do {                                                         \
    ibl_status s_ = cuda_check(c, (expr), what);               \
    if (s_ != IBL_OK) return s_;                               \
  } while (0)

// Map device status bits to the ABI's error codes (most severe first).
static ibl_status status_code(ibl_ctx* c) {
  const int s = c->sticky;
  if (s & ST_DIVERGED) return fail(c, IBL_EDIVERGED, "non-finite or runaway density detected");
  if (s & ST_TIMEOUT) return fail(c, IBL_ETIMEOUT, "a bounded device wait gave up");
  if (s & ST_OVERFLOW)
    return fail(c, IBL_EINVAL,
                "marker stencil leaves a non-periodic axis or an IB capacity (band slots, tile "
                "marker list, system row) was exceeded");
  if (s & ST_NOTCONV) return fail(c, IBL_ENOTCONV, "implicit IB solve did not converge");
  return IBL_OK;
}

namespace ibl {
ibl_status sync_and_collect(ibl_ctx* c);
}
ibl_status ibl::sync_and_collect(ibl_ctx* c) {
  CK(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
  int s = 0;
  CK(to_host(c, &s, c->d_status, sizeof(int)), "status read");
  // non-convergence is reported once per occurrence; the others are sticky
  c->sticky |= s;
  ibl_status r = status_code(c);
  if (s & ST_NOTCONV) {
    const int keep = s & ~ST_NOTCONV;
    CK(to_device(c, c->d_status, &keep, sizeof(int)), "status reset");
    CK(cudaStreamSynchronize(c->stream), "status reset");
    c->sticky &= ~ST_NOTCONV;
  }
  return r;
}

static bool is_zh(int b) { return b == IBL_VEL_INLET || b == IBL_PRESS_OUTLET; }

extern "C" {

ibl_status ibl_create(const ibl_grid* grid, double tau, int32_t lattice, ibl_ctx** out) {
  if (!out) return fail(nullptr, IBL_EINVAL, "out is NULL");
  *out = nullptr;
  if (!grid) return fail(nullptr, IBL_EINVAL, "grid is NULL");
  if (lattice != IBL_D2Q9 && lattice != IBL_D3Q19) return fail(nullptr, IBL_EINVAL, "unknown lattice");
  if (grid->nx <= 0 || grid->ny <= 0 || grid->nz <= 0) return fail(nullptr, IBL_EINVAL, "grid sizes must be > 0");
  if (lattice == IBL_D2Q9 && grid->nz != 1) return fail(nullptr, IBL_EINVAL, "D2Q9 needs nz == 1");
  if ((long long)grid->nx * grid->ny * grid->nz >= (1LL << 31))
    return fail(nullptr, IBL_EINVAL, "at most 2^31 - 1 cells per context");
  if (!(tau > 0.5) || !std::isfinite(tau)) return fail(nullptr, IBL_EINVAL, "tau must be > 1/2");
  if (grid->precision < IBL_FP64 || grid->precision > IBL_BF16DEV)
    return fail(nullptr, IBL_EINVAL, "unknown precision");
  const int D = lattice == IBL_D2Q9 ? 2 : 3;
  int bc[6];
  for (int i = 0; i < 6; ++i) {
    bc[i] = grid->bc[i];
    if (bc[i] < IBL_PERIODIC || bc[i] > IBL_PRESS_OUTLET) return fail(nullptr, IBL_EINVAL, "unknown face condition");
  }
  if (D == 2) bc[4] = bc[5] = IBL_PERIODIC;
  int zh_axis = -1;
  for (int a = 0; a < D; ++a) {
    if ((bc[2 * a] == IBL_PERIODIC) != (bc[2 * a + 1] == IBL_PERIODIC))
      return fail(nullptr, IBL_EINVAL, "periodic faces must come in pairs");
    if (is_zh(bc[2 * a]) || is_zh(bc[2 * a + 1])) zh_axis = a;
  }
  if (zh_axis >= 0)
    for (int b = 0; b < D; ++b)
      if (b != zh_axis && bc[2 * b] != IBL_PERIODIC)
        return fail(nullptr, IBL_EINVAL, "a Zou-He face needs periodic lateral axes");
  ibl_ctx* c = new ibl_ctx();
  c->Q = lattice;
  c->D = D;
  c->nx = grid->nx; c->ny = grid->ny; c->nz = grid->nz;
  c->N = (long long)grid->nx * grid->ny * grid->nz;
  for (int i = 0; i < 6; ++i) c->bc[i] = bc[i];
  for (int a = 0; a < 3; ++a) {
    c->u_in[a] = grid->u_in[a];
    c->G[a] = a < D ? grid->body_force[a] : 0.0;
  }
  c->rho_out = grid->rho_out;
  c->prec = grid->precision;
  c->tau = tau;
  c->elem = c->prec == IBL_FP64 ? 8 : (c->prec == IBL_FP32 ? 4 : 2);
  // band tiles: 16 x 4 x 4 in 3D, 16 x 16 in 2D (256 cells)
  c->tg.tx = TILE_X;
  c->tg.ty = D == 3 ? TILE_Y : TILE_CELLS / TILE_X;
  c->tg.tz = D == 3 ? TILE_Z3 : 1;
  c->tg.ntx = (c->nx + c->tg.tx - 1) / c->tg.tx;
  c->tg.nty = (c->ny + c->tg.ty - 1) / c->tg.ty;
  c->tg.ntz = (c->nz + c->tg.tz - 1) / c->tg.tz;
  c->tg.n_tiles = c->tg.ntx * c->tg.nty * c->tg.ntz;
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
  const size_t bytes = (size_t)c->Q * (size_t)c->N * c->elem;
  if (e == cudaSuccess) e = cudaMalloc(&c->f[0], bytes);
  if (e == cudaSuccess) e = cudaMalloc(&c->f[1], bytes);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_status, 2 * sizeof(int));
  if (e == cudaSuccess) e = fill_zero(c, c->d_status, 2 * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&c->d_mass_parts, sizeof(double) * MASS_PARTS);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_mass_ref, sizeof(double) * 3);
  if (e == cudaSuccess) e = fill_zero(c, c->d_mass_ref, sizeof(double) * 3);
  if (e != cudaSuccess) {
    ibl_status s = cuda_check(nullptr, e, "ibl_create");
    ibl_destroy(c);
    return s;
  }
  *out = c;
  return IBL_OK;
}

ibl_status ibl_destroy(ibl_ctx* c) {
  if (!c) return IBL_OK;
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->stream_bulk) {
    cudaStreamSynchronize(c->stream_bulk);
    cudaStreamDestroy(c->stream_bulk);
  }
  if (c->ev_tiles) cudaEventDestroy(c->ev_tiles);
  if (c->ev_bulk) cudaEventDestroy(c->ev_bulk);
  ib_free(c);
  if (c->f[0]) cudaFree(c->f[0]);
  if (c->f[1]) cudaFree(c->f[1]);
  if (c->d_status) cudaFree(c->d_status);
  if (c->d_mass_parts) cudaFree(c->d_mass_parts);
  if (c->d_mass_ref) cudaFree(c->d_mass_ref);
  if (c->d_pt_perm) cudaFree(c->d_pt_perm);
  if (c->d_pt_bins) cudaFree(c->d_pt_bins);
  if (c->d_pt_mom) cudaFree(c->d_pt_mom);
  if (c->d_pt_sbase) cudaFree(c->d_pt_sbase);
  if (c->d_pt_swts) cudaFree(c->d_pt_swts);
  for (auto& ev : c->stage_ev)
    if (ev) cudaEventDestroy(ev);
  for (auto& ev : c->prof_ev) cudaEventDestroy(ev);
  for (auto& ev : c->pev_pool) cudaEventDestroy(ev);
  if (c->h_stage) cudaFreeHost(c->h_stage);
  if (c->stream) cudaStreamDestroy(c->stream);
  delete c;
  return IBL_OK;
}

ibl_status ibl_init_fluid(ibl_ctx* c, const double* rho, const double* u) {
  if (!c) return IBL_EINVAL;
  double* d = nullptr;
  const size_t n1 = (size_t)c->N;
  const size_t tot = (rho ? n1 : 0) + (u ? n1 * c->D : 0);
  if (tot) CK(cudaMalloc(&d, sizeof(double) * tot), "init_fluid alloc");
  double* d_rho = rho ? d : nullptr;
  double* d_u = u ? d + (rho ? n1 : 0) : nullptr;
  ibl_status st = IBL_OK;
  cudaError_t e = cudaSuccess;
  if (rho) e = cudaMemcpyAsync(d_rho, rho, sizeof(double) * n1, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess && u)
    e = cudaMemcpyAsync(d_u, u, sizeof(double) * n1 * c->D, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = launch_init_eq(c, d_rho, d_u);
  c->poststream = true;
  if (e == cudaSuccess) e = launch_mass_check(c, 0);   // reference total of the mass check
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  st = cuda_check(c, e, "init_fluid");
  if (d) cudaFree(d);
  if (st != IBL_OK) return st;
  c->initialised = true;
  c->poststream = true;
  c->step = 0;
  c->warm = false;
  c->warm_steps = 0;
  return IBL_OK;
}

ibl_status ibl_set_populations(ibl_ctx* c, const double* f) {
  if (!c || !f) return c ? fail(c, IBL_EINVAL, "f is NULL") : IBL_EINVAL;
  double* d = nullptr;
  const size_t n = (size_t)c->N * c->Q;
  CK(cudaMalloc(&d, sizeof(double) * n), "set_populations alloc");
  cudaError_t e = cudaMemcpyAsync(d, f, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = launch_set_pop(c, d);
  c->poststream = true;
  if (e == cudaSuccess) e = launch_mass_check(c, 0);   // reference total of the mass check
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFree(d);
  ibl_status st = cuda_check(c, e, "set_populations");
  if (st != IBL_OK) return st;
  c->initialised = true;
  c->poststream = true;
  c->step = 0;
  c->warm = false;
  c->warm_steps = 0;
  return IBL_OK;
}

ibl_status ibl_set_markers(ibl_ctx* c, int32_t m, const double* X0, const double* ds,
                           const double hinge[3], const double axis[3], const double origin[3],
                           int32_t* body_id) {
  if (!c) return IBL_EINVAL;
  if (m <= 0 || !X0 || !ds || !hinge || !axis || !origin)
    return fail(c, IBL_EINVAL, "ibl_set_markers: m > 0 and non-NULL arrays required");
  if ((int)c->bodies.size() >= 16) return fail(c, IBL_EINVAL, "at most 16 bodies");
  for (int a = 0; a < c->D; ++a)
    if ((a == 0 ? c->nx : (a == 1 ? c->ny : c->nz)) < 8)
      return fail(c, IBL_EINVAL, "axes carrying markers need at least 8 nodes");
  const double en = std::sqrt(axis[0] * axis[0] + axis[1] * axis[1] + axis[2] * axis[2]);
  if (!(en > 0)) return fail(c, IBL_EINVAL, "rotation axis is zero");
  for (int l = 0; l < m; ++l)
    if (!(ds[l] > 0)) return fail(c, IBL_EINVAL, "element sizes ds must be > 0");
  Body b;
  b.offset = c->m_total;
  b.m = m;
  for (int a = 0; a < 3; ++a) {
    b.hinge[a] = hinge[a];
    b.axis[a] = axis[a] / en;
    b.origin[a] = origin[a];
  }
  if (c->D == 2) {
    b.axis[0] = b.axis[1] = 0.0;
    b.axis[2] = axis[2] >= 0 ? 1.0 : -1.0;
  }
  for (int l = 0; l < m; ++l) {
    for (int a = 0; a < 3; ++a) c->h_X0.push_back(a < c->D ? X0[(size_t)l * c->D + a] : 0.0);
    c->h_ds.push_back(ds[l]);
  }
  c->bodies.push_back(b);
  c->m_total += m;
  c->ib_ready = false;
  if (body_id) *body_id = (int32_t)c->bodies.size() - 1;
  return IBL_OK;
}

static ibl_status copy_wave(ibl_ctx* c, const ibl_wave* w, Wave& out, std::vector<double>& table) {
  out.kind = IBL_WAVE_CONST;
  out.amp = 0;
  out.offset = 0;
  table.clear();
  if (!w) return IBL_OK;
  if (w->kind < IBL_WAVE_CONST || w->kind > IBL_WAVE_TABLE) return fail(c, IBL_EINVAL, "unknown wave kind");
  out.kind = w->kind;
  out.amp = w->amp;
  out.offset = w->offset;
  if (w->kind == IBL_WAVE_TABLE) {
    if (!w->table || w->n_table <= 0) return fail(c, IBL_EINVAL, "table wave needs samples");
    table.assign(w->table, w->table + w->n_table);
  }
  return IBL_OK;
}

ibl_status ibl_set_kinematics(ibl_ctx* c, int32_t body_id, const ibl_wave* A, const ibl_wave* alpha,
                              double beta, double phi, double f, double J) {
  if (!c) return IBL_EINVAL;
  if (body_id < 0 || body_id >= (int)c->bodies.size()) return fail(c, IBL_EINVAL, "bad body id");
  if (!std::isfinite(beta) || !std::isfinite(phi) || !std::isfinite(f) || !std::isfinite(J))
    return fail(c, IBL_EINVAL, "kinematic parameters must be finite");
  Body& b = c->bodies[body_id];
  ibl_status s = copy_wave(c, A, b.A, b.hostA);
  if (s != IBL_OK) return s;
  s = copy_wave(c, alpha, b.alpha, b.hostAlpha);
  if (s != IBL_OK) return s;
  b.beta = beta;
  b.phi = phi;
  b.f = f;
  b.J = J;
  return IBL_OK;
}

// Second stream and the two events of the split step, created on first use.
static ibl_status ensure_split(ibl_ctx* c) {
  if (c->stream_bulk) return IBL_OK;
  CK(cudaStreamCreateWithFlags(&c->stream_bulk, cudaStreamNonBlocking), "bulk stream");
  CK(cudaEventCreateWithFlags(&c->ev_tiles, cudaEventDisableTiming), "event");
  CK(cudaEventCreateWithFlags(&c->ev_bulk, cudaEventDisableTiming), "event");
  return IBL_OK;
}

static ibl_status ensure_ib(ibl_ctx* c) {
  if (c->ib_ready || c->m_total == 0) return IBL_OK;
  if (c->precond_kind == 1 && !sep_all_separable(c, nullptr))
    return fail(c, IBL_EINVAL,
                "separable preconditioner: every body needs its markers on a chord x span product mesh "
                "rotating about the z axis (3D)");
  CK(cudaStreamSynchronize(c->stream), "sync");
  CK(ib_alloc(c), "IB buffers");
  const size_t m = c->m_total;
  CK(to_device(c, c->d_X0, c->h_X0.data(), sizeof(double) * 3 * m), "X0 upload");
  CK(to_device(c, c->d_ds, c->h_ds.data(), sizeof(double) * m), "ds upload");
  if (c->h_stage) cudaFreeHost(c->h_stage);
  c->h_stage = nullptr;
  c->stage_doubles = 6 * m;
  CK(cudaMallocHost(&c->h_stage, sizeof(double) * 4 * c->stage_doubles), "staging alloc");
  for (auto& ev : c->stage_ev)
    if (!ev) CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event");
  return IBL_OK;
}

ibl_status ibl_set_marker_state(ibl_ctx* c, int32_t body_id, const double* X, const double* U) {
  if (!c) return IBL_EINVAL;
  if (body_id < 0 || body_id >= (int)c->bodies.size()) return fail(c, IBL_EINVAL, "bad body id");
  if (!X || !U) return fail(c, IBL_EINVAL, "X and U are required");
  ibl_status s = ensure_ib(c);
  if (s != IBL_OK) return s;
  Body& b = c->bodies[body_id];
  const int k = c->stage_next;
  c->stage_next = (k + 1) & 3;
  CK(cudaEventSynchronize(c->stage_ev[k]), "staging wait");
  double* st = c->h_stage + (size_t)k * c->stage_doubles;
  for (int l = 0; l < b.m; ++l)
    for (int a = 0; a < 3; ++a) {
      st[3 * l + a] = a < c->D ? X[(size_t)l * c->D + a] : 0.0;
      st[3 * (size_t)b.m + 3 * l + a] = a < c->D ? U[(size_t)l * c->D + a] : 0.0;
    }
  CK(cudaMemcpyAsync(c->d_Xp + 3 * (size_t)b.offset, st, sizeof(double) * 3 * b.m, cudaMemcpyHostToDevice,
                     c->stream), "X upload");
  CK(cudaMemcpyAsync(c->d_Up + 3 * (size_t)b.offset, st + 3 * (size_t)b.m, sizeof(double) * 3 * b.m,
                     cudaMemcpyHostToDevice, c->stream), "U upload");
  CK(cudaEventRecord(c->stage_ev[k], c->stream), "staging record");
  b.prescribed = true;
  return IBL_OK;
}

ibl_status ibl_set_lift_axis(ibl_ctx* c, int32_t body_id, const double e[3]) {
  if (!c) return IBL_EINVAL;
  if (body_id < 0 || body_id >= (int)c->bodies.size() || !e) return fail(c, IBL_EINVAL, "bad body id or axis");
  const double n = std::sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
  if (!(n > 0)) return fail(c, IBL_EINVAL, "zero lift axis");
  for (int a = 0; a < 3; ++a) c->bodies[body_id].lift[a] = e[a] / n;
  return IBL_OK;
}

ibl_status ibl_set_reference(ibl_ctx* c, double U_ref, double L_or_S, double rho_ref) {
  if (!c) return IBL_EINVAL;
  if (!(U_ref > 0) || !(L_or_S > 0) || !(rho_ref > 0)) return fail(c, IBL_EINVAL, "reference values must be > 0");
  c->U_ref = U_ref;
  c->L_ref = L_or_S;
  c->rho_ref = rho_ref;
  return IBL_OK;
}

ibl_status ibl_step(ibl_ctx* c, int64_t n) {
  if (!c) return IBL_EINVAL;
  if (n < 0) return fail(c, IBL_EINVAL, "n must be >= 0");
  if (!c->initialised) return fail(c, IBL_ESTATE, "fluid not initialised");
  if (c->sticky & (ST_DIVERGED | ST_OVERFLOW)) return status_code(c);
  ibl_status s = ensure_ib(c);
  if (s != IBL_OK) return s;
  const bool with_ib = c->m_total > 0;
  // split step: the cells outside the IB band collide on a second stream
  // while the IB chain runs; the band tiles collide after the spreading
  const bool split = with_ib && (c->overlap == 1 || (c->overlap < 0 && c->N >= (1LL << 20) &&
                                                     c->m_total <= SPLIT_MAX_MARKERS));
  // serial split (on request): the IB chain on every SM, then the cells
  // outside the band (the persistent kernel without the band lookup, every
  // SM) and the band tiles.  Measured on the 512 x 384 x 320 wings: 1.66 ms
  // for the two collide kernels against 1.54 ms for the one-kernel collide.
  const bool serial = with_ib && !split && c->overlap == 2;
  if (split) {
    s = ensure_split(c);
    if (s != IBL_OK) return s;
  }
  for (int64_t k = 0; k < n; ++k) {
    cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    if (c->profiling) {
      const size_t need = 6 * (size_t)(c->prof_steps + 1);
      while (c->prof_ev.size() < need) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e), "profile event");
        c->prof_ev.push_back(e);
      }
      for (int j = 0; j < 6; ++j) ev[j] = c->prof_ev[6 * c->prof_steps + j];
      c->prof_split.push_back(split ? 1 : 0);
      c->prof_steps++;
    }
    if (ev[0]) CK(cudaEventRecord(ev[0], c->stream), "event");
    phase_mark(c, -1);
    if (split) {
      CK(ib_step_front(c), "IB step");
      CK(cudaEventRecord(c->ev_tiles, c->stream), "event");
      CK(cudaStreamWaitEvent(c->stream_bulk, c->ev_tiles, 0), "stream wait");
      if (ev[4]) CK(cudaEventRecord(ev[4], c->stream_bulk), "event");
      CK(launch_collide_bulk(c, std::max(1, num_sms() - pcg_block_count(c)), c->stream_bulk), "bulk collide");
      if (ev[5]) CK(cudaEventRecord(ev[5], c->stream_bulk), "event");
      CK(cudaEventRecord(c->ev_bulk, c->stream_bulk), "event");
      CK(ib_step_back(c), "IB step");
      if (ev[1]) CK(cudaEventRecord(ev[1], c->stream), "event");
      CK(launch_collide_band(c, std::max(1, std::min(c->cap_slots, 4 * num_sms()))), "band collide");
      phase_mark(c, 9);
      if (ev[2]) CK(cudaEventRecord(ev[2], c->stream), "event");
      CK(cudaStreamWaitEvent(c->stream, c->ev_bulk, 0), "stream wait");
    } else if (serial) {
      CK(ib_step(c), "IB step");
      if (ev[1]) CK(cudaEventRecord(ev[1], c->stream), "event");
      CK(launch_collide_bulk(c, num_sms(), c->stream), "bulk collide");
      CK(launch_collide_band(c, std::max(1, std::min(c->cap_slots, 4 * num_sms()))), "band collide");
      phase_mark(c, 9);
      if (ev[2]) CK(cudaEventRecord(ev[2], c->stream), "event");
    } else {
      if (with_ib) CK(ib_step(c), "IB step");
      if (ev[1]) CK(cudaEventRecord(ev[1], c->stream), "event");
      CK(launch_collide(c, with_ib), "collide");
      phase_mark(c, 9);
      if (ev[2]) CK(cudaEventRecord(ev[2], c->stream), "event");
    }
    if (ev[3]) CK(cudaEventRecord(ev[3], c->stream), "event");
    c->cur ^= 1;
    c->poststream = false;
    c->step++;
    if (c->mass_every > 0 && c->step % c->mass_every == 0) CK(launch_mass_check(c, 1), "mass check");
  }
  return IBL_OK;
}

ibl_status ibl_set_mass_check(ibl_ctx* c, int32_t every, double rel_tol) {
  if (!c) return IBL_EINVAL;
  if (every < 0 || !(rel_tol >= 0.0) || !std::isfinite(rel_tol))
    return fail(c, IBL_EINVAL, "mass check: every >= 0 and a finite rel_tol >= 0");
  c->mass_every = every;
  c->mass_tol = rel_tol;
  return IBL_OK;
}

ibl_status ibl_mass_check_read(ibl_ctx* c, double* m0, double* m_last, int64_t* checks) {
  if (!c) return IBL_EINVAL;
  ibl_status s = sync_and_collect(c);
  if (s != IBL_OK && s != IBL_ENOTCONV && s != IBL_EDIVERGED) return s;
  double r[3];
  CK(to_host(c, r, c->d_mass_ref, sizeof(r)), "mass check read");
  if (m0) *m0 = r[0];
  if (m_last) *m_last = r[1];
  if (checks) *checks = (int64_t)r[2];
  return s;
}

ibl_status ibl_solver_blocks(ibl_ctx* c, int32_t blocks) {
  if (!c) return IBL_EINVAL;
  if (blocks < 0 || blocks > 256) return fail(c, IBL_EINVAL, "solver blocks must be in [0, 256]");
  c->pcg_blocks = blocks;
  return IBL_OK;
}

ibl_status ibl_solver_preconditioner(ibl_ctx* c, int32_t kind, int32_t resident_rows) {
  if (!c) return IBL_EINVAL;
  if (kind < -1 || kind > 1) return fail(c, IBL_EINVAL, "preconditioner kind must be -1, 0 or 1");
  if (resident_rows < -1 || resident_rows > 0) return fail(c, IBL_EINVAL, "resident_rows must be -1 or 0");
  if (kind != c->precond_kind && c->ib_ready) {
    // the preconditioner's buffers are sized at the next step
    CK(cudaStreamSynchronize(c->stream), "sync");
    c->ib_ready = false;
  }
  c->precond_kind = kind;
  c->resident_rows = resident_rows;
  return IBL_OK;
}

ibl_status ibl_set_overlap(ibl_ctx* c, int32_t mode) {
  if (!c) return IBL_EINVAL;
  if (mode < -1 || mode > 2) return fail(c, IBL_EINVAL, "overlap mode must be -1, 0, 1 or 2");
  c->overlap = mode;
  return IBL_OK;
}

ibl_status ibl_set_collide_shape(ibl_ctx* c, int32_t bx, int32_t by, int32_t pairs) {
  if (!c) return IBL_EINVAL;
  if (!(bx == 32 || bx == 64 || bx == 128 || bx == 256) || by < 1 || bx * by > 256 || pairs < 0 || pairs > 3)
    return fail(c, IBL_EINVAL, "collide shape: bx in {32, 64, 128, 256}, by >= 1, bx * by <= 256, pairs 0 .. 3");
  c->collide_bx = bx;
  c->collide_by = by;
  c->collide_pairs = pairs;
  return IBL_OK;
}

ibl_status ibl_sync(ibl_ctx* c) {
  if (!c) return IBL_EINVAL;
  return sync_and_collect(c);
}

static void coefficients(ibl_ctx* c, int b, const double F[3], double* CL, double* CT, double* CD) {
  const double q = 0.5 * c->rho_ref * c->U_ref * c->U_ref * c->L_ref;
  const double* e = c->bodies[b].lift;
  const double drag = F[0] / q;
  double lift = 0;
  for (int a = 0; a < c->D; ++a) lift += F[a] * e[a];
  if (CL) *CL = lift / q;
  if (CD) *CD = drag;
  if (CT) *CT = -drag;
}

ibl_status ibl_forces(ibl_ctx* c, int32_t body_id, double* C_L, double* C_T, double* C_D) {
  if (!c) return IBL_EINVAL;
  if (body_id < 0 || body_id >= (int)c->bodies.size()) return fail(c, IBL_EINVAL, "bad body id");
  ibl_status s = sync_and_collect(c);
  if (s != IBL_OK && s != IBL_ENOTCONV) return s;
  if (c->step == 0 || !c->ib_ready) return fail(c, IBL_ESTATE, "no completed step");
  double F[3];
  const long long idx = ((long long)body_id * HIST_LEN + ((c->step - 1) % HIST_LEN)) * 3;
  CK(to_host(c, F, c->d_hist + idx, sizeof(F)), "force read");
  coefficients(c, body_id, F, C_L, C_T, C_D);
  return s;
}

ibl_status ibl_force_history(ibl_ctx* c, int32_t body_id, int64_t max, double* out3, int64_t* n) {
  if (!c) return IBL_EINVAL;
  if (body_id < 0 || body_id >= (int)c->bodies.size() || max < 0 || (!out3 && max > 0))
    return fail(c, IBL_EINVAL, "bad arguments");
  ibl_status s = sync_and_collect(c);
  if (s != IBL_OK && s != IBL_ENOTCONV) return s;
  long long avail = std::min<long long>(c->step, HIST_LEN);
  if (!c->ib_ready) avail = 0;
  const long long cnt = std::min<long long>(avail, max);
  std::vector<double> F(3 * (size_t)HIST_LEN);
  if (cnt > 0)
    CK(to_host(c, F.data(), c->d_hist + (size_t)body_id * HIST_LEN * 3, sizeof(double) * 3 * HIST_LEN),
       "history read");
  for (long long k = 0; k < cnt; ++k) {
    const long long stepk = c->step - cnt + k;
    const double* f = F.data() + 3 * (stepk % HIST_LEN);
    coefficients(c, body_id, f, out3 + 3 * k, out3 + 3 * k + 1, out3 + 3 * k + 2);
  }
  if (n) *n = cnt;
  return s;
}

ibl_status ibl_get_field(ibl_ctx* c, int32_t what, double* out) {
  if (!c) return IBL_EINVAL;
  if (!out) return fail(c, IBL_EINVAL, "out is NULL");
  if (!c->initialised) return fail(c, IBL_ESTATE, "fluid not initialised");
  if (what < IBL_FIELD_RHO || what > IBL_FIELD_FORCE) return fail(c, IBL_EINVAL, "unknown field");
  ibl_status s = sync_and_collect(c);
  if (s != IBL_OK && s != IBL_ENOTCONV) return s;
  const size_t n = (size_t)c->N * (what == IBL_FIELD_RHO ? 1 : c->D);
  double* d = nullptr;
  CK(cudaMalloc(&d, sizeof(double) * n), "field alloc");
  cudaError_t e;
  if (what == IBL_FIELD_FORCE) {
    if (c->m_total == 0 || !c->ib_ready) e = cudaMemsetAsync(d, 0, sizeof(double) * n, c->stream);
    else e = launch_force_field(c, d);
  } else {
    e = launch_fields(c, what == IBL_FIELD_RHO ? d : nullptr, what == IBL_FIELD_U ? d : nullptr, nullptr);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, d, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFree(d);
  CK(e, "get_field");
  return s;
}

ibl_status ibl_get_populations(ibl_ctx* c, double* f) {
  if (!c) return IBL_EINVAL;
  if (!f) return fail(c, IBL_EINVAL, "f is NULL");
  if (!c->initialised) return fail(c, IBL_ESTATE, "fluid not initialised");
  ibl_status s = sync_and_collect(c);
  if (s != IBL_OK && s != IBL_ENOTCONV) return s;
  const size_t n = (size_t)c->N * c->Q;
  double* d = nullptr;
  CK(cudaMalloc(&d, sizeof(double) * n), "population alloc");
  cudaError_t e = launch_fields(c, nullptr, nullptr, d);
  if (e == cudaSuccess) e = cudaMemcpyAsync(f, d, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFree(d);
  CK(e, "get_populations");
  return s;
}

ibl_status ibl_get_markers(ibl_ctx* c, int32_t body_id, double* X, double* U, double* F) {
  if (!c) return IBL_EINVAL;
  if (body_id < 0 || body_id >= (int)c->bodies.size()) return fail(c, IBL_EINVAL, "bad body id");
  ibl_status s = sync_and_collect(c);
  if (s != IBL_OK && s != IBL_ENOTCONV) return s;
  if (!c->ib_ready) return fail(c, IBL_ESTATE, "no completed step");
  const Body& b = c->bodies[body_id];
  std::vector<double> tmp(3 * (size_t)b.m);
  double* outs[3] = {X, U, F};
  double* srcs[3] = {c->d_X, c->d_U, c->d_mforce};
  for (int k = 0; k < 3; ++k) {
    if (!outs[k]) continue;
    CK(to_host(c, tmp.data(), srcs[k] + 3 * (size_t)b.offset, sizeof(double) * 3 * b.m), "marker read");
    for (int l = 0; l < b.m; ++l)
      for (int a = 0; a < c->D; ++a) outs[k][(size_t)l * c->D + a] = tmp[3 * l + a];
  }
  return s;
}

ibl_status ibl_mass(ibl_ctx* c, double* mass) {
  if (!c) return IBL_EINVAL;
  if (!mass) return fail(c, IBL_EINVAL, "mass is NULL");
  if (!c->initialised) return fail(c, IBL_ESTATE, "fluid not initialised");
  ibl_status s = sync_and_collect(c);
  if (s != IBL_OK && s != IBL_ENOTCONV) return s;
  const int parts = 1024;
  double* d = nullptr;
  CK(cudaMalloc(&d, sizeof(double) * parts), "mass alloc");
  cudaError_t e = launch_mass(c, d, parts, nullptr);
  std::vector<double> h(parts);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), d, sizeof(double) * parts, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFree(d);
  CK(e, "mass");
  double acc = 0;
  for (int k = 0; k < parts; ++k) acc += h[k];
  *mass = acc;
  return s;
}

ibl_status ibl_lattice_velocities(int32_t lattice, int32_t* q, int32_t* cvec, double* w) {
  if (lattice != IBL_D2Q9 && lattice != IBL_D3Q19) return IBL_EINVAL;
  if (q) *q = lattice;
  for (int i = 0; i < lattice; ++i) {
    if (lattice == 9) {
      if (cvec) { cvec[3 * i] = Lat<9>::cx(i); cvec[3 * i + 1] = Lat<9>::cy(i); cvec[3 * i + 2] = 0; }
      if (w) w[i] = Lat<9>::w(i);
    } else {
      if (cvec) { cvec[3 * i] = Lat<19>::cx(i); cvec[3 * i + 1] = Lat<19>::cy(i); cvec[3 * i + 2] = Lat<19>::cz(i); }
      if (w) w[i] = Lat<19>::w(i);
    }
  }
  return IBL_OK;
}

ibl_status ibl_solver_stats(ibl_ctx* c, int32_t* iterations, double* rel_residual, int64_t* refreshes) {
  if (!c) return IBL_EINVAL;
  ibl_status s = sync_and_collect(c);
  if (s != IBL_OK && s != IBL_ENOTCONV) return s;
  int info[4] = {0, 0, 0, 0};
  double res = 0;
  if (c->ib_ready) {
    CK(to_host(c, info, c->d_cg_info, sizeof(info)), "stats");
    CK(to_host(c, &res, c->d_cg_res, sizeof(double)), "stats");
  }
  if (iterations) *iterations = info[0];
  if (rel_residual) *rel_residual = res;
  if (refreshes) *refreshes = c->refreshes + info[3];
  return s;
}

ibl_status ibl_solver_config(ibl_ctx* c, int32_t refresh_every, double tol, int32_t extrapolate) {
  if (!c) return IBL_EINVAL;
  if (refresh_every < 1 || !(tol >= 0.0) || tol >= 1.0) return fail(c, IBL_EINVAL, "refresh_every >= 1, 0 <= tol < 1");
  c->refresh_every = refresh_every;
  c->solver_tol = tol;
  c->extrapolate = extrapolate >= 2 ? 2 : (extrapolate == 1 ? 1 : (extrapolate == 0 ? 0 : -1));
  return IBL_OK;
}

ibl_status ibl_profile(ibl_ctx* c, int32_t enable) {
  if (!c) return IBL_EINVAL;
  CK(cudaStreamSynchronize(c->stream), "sync");
  c->profiling = enable != 0;
  c->prof_level = enable;
  c->prof_steps = 0;
  c->prof_split.clear();
  c->pev_used = 0;
  c->pev_log.clear();
  return IBL_OK;
}

ibl_status ibl_profile_read(ibl_ctx* c, double* collide_ms, double* ib_ms, int64_t* steps) {
  if (!c) return IBL_EINVAL;
  CK(cudaStreamSynchronize(c->stream), "sync");
  double tc = 0, ti = 0;
  for (long long k = 0; k < c->prof_steps; ++k) {
    float a = 0, b = 0, d = 0;
    cudaEvent_t* e = &c->prof_ev[6 * k];
    CK(cudaEventElapsedTime(&a, e[0], e[1]), "elapsed");
    CK(cudaEventElapsedTime(&b, e[1], e[2]), "elapsed");
    CK(cudaEventElapsedTime(&d, e[2], e[3]), "elapsed");
    if (c->prof_split[k]) {
      float bulk = 0;
      CK(cudaEventElapsedTime(&bulk, e[4], e[5]), "elapsed");
      tc += b + bulk;
      ti += a;
    } else {
      tc += b;
      ti += a + d;
    }
  }
  if (collide_ms) *collide_ms = tc;
  if (ib_ms) *ib_ms = ti;
  if (steps) *steps = c->prof_steps;
  return IBL_OK;
}

ibl_status ibl_profile_phases(ibl_ctx* c, double* ms, int32_t n) {
  if (!c || n < 0 || (n > 0 && !ms)) return IBL_EINVAL;
  CK(cudaStreamSynchronize(c->stream), "sync");
  for (int i = 0; i < n; ++i) ms[i] = 0.0;
  cudaEvent_t prev = nullptr;
  for (auto& pe : c->pev_log) {
    if (pe.first >= 0 && prev && pe.first < n) {
      float t = 0;
      CK(cudaEventElapsedTime(&t, prev, pe.second), "elapsed");
      ms[pe.first] += t;
    }
    prev = pe.second;
  }
  return IBL_OK;
}

ibl_status ibl_solver_trace(ibl_ctx* c, int64_t* ns, int32_t max, int32_t* n) {
  if (!c || (!ns && max > 0)) return IBL_EINVAL;
  ibl_status s = sync_and_collect(c);
  if (s != IBL_OK && s != IBL_ENOTCONV) return s;
  unsigned long long t[256] = {0};
  if (c->ib_ready) CK(to_host(c, t, c->d_trace, sizeof(t)), "trace read");
  const int k = std::min<int>(max, 256);
  for (int i = 0; i < k; ++i) ns[i] = (int64_t)t[i];
  if (n) *n = k;
  return s;
}

ibl_status ibl_launch_count(const ibl_ctx* c, int64_t* n) {
  if (!c || !n) return IBL_EINVAL;
  *n = c->launches;
  return IBL_OK;
}

ibl_status ibl_stream(const ibl_ctx* c, void** stream) {
  if (!c || !stream) return IBL_EINVAL;
  *stream = (void*)c->stream;
  return IBL_OK;
}

const char* ibl_last_error(const ibl_ctx* c) {
  if (!c) return g_create_err.c_str();
  return c->err.c_str();
}

}  // extern "C"
