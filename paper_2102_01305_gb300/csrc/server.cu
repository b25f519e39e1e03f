// Serving form: continuous batching of parameter-sweep runs on one GPU.
//
// A background thread owns every run's context.  Each pass it
//   1. admits queued requests in arrival order while the active count and the
//      HBM budget allow (a run's device footprint is estimated from its grid,
//      lattice, precision and marker count before its context is created);
//   2. enqueues the next chunk of steps of every active run whose previous
//      chunk has finished (each run has its own CUDA stream, so the chunks of
//      different runs overlap on the device);
//   3. retires finished (or cancelled) runs: reads their force histories, reduces them to
//      the per-wing maxima and means of C_L and C_T (the quantities of the
//      paper's parametric study, Sec. 3.4-3.7 and Fig. 11), destroys the
//      context and returns its memory to the budget.
// Every run advances through exactly the same kernel sequence as it would
// alone, so its result does not depend on what else is running.  With
// tuning on, a run's solve block count follows from its marker count, and
// its overlap mode and collide shape (which never change results) from a
// timed first chunk, cached per run shape.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <tuple>
#include <vector>

#include "ibl_internal.cuh"

namespace {

using clock_type = std::chrono::steady_clock;

// Launch candidates of the tuning chunk: overlap mode, collide block, pairs.
struct Launch {
  int overlap, bx, by, pairs;
};
constexpr Launch CANDIDATES[] = {{1, 64, 2, 3}, {0, 64, 2, 3}, {0, 128, 1, 3}, {0, 64, 4, 1}, {0, 64, 4, 2}};
constexpr int NCAND = sizeof(CANDIDATES) / sizeof(CANDIDATES[0]);
constexpr int TUNE_MIN_STEPS = 2;          // timed steps per candidate
constexpr int MARKERS_PER_SOLVE_BLOCK = 64;

using ShapeKey = std::tuple<int, int, int, double, int, int>;   // nx, ny, nz, chord, precision, faces

struct Run {
  int64_t id = 0;
  ibl_run_request req{};
  ibl_run_result res{};          // shared: read by ibl_server_poll under the server's mutex
  ibl_ctx* ctx = nullptr;        // worker-owned
  cudaEvent_t ev = nullptr;      // worker-owned
  bool inflight = false;         // worker-owned
  int64_t steps_enqueued = 0;    // worker-owned
  std::atomic<bool> cancel{false};
  size_t bytes = 0;
  int m[2] = {0, 0};
  // tuning (worker-owned)
  bool tune_pending = false;     // the next chunk is the tuning chunk
  bool tune_inflight = false;    // the tuning chunk is on the stream
  int tune_steps = 0;            // timed steps per candidate
  cudaEvent_t tev[2 * NCAND] = {};
  Launch launch{-1, 64, 2, 3};
  int solve_blocks = 0;
  bool tuned = false;
};

ShapeKey shape_key(const ibl_run_request& r) {
  return ShapeKey(r.nx, r.ny, r.nz, r.chord, r.precision, r.faces);
}

}  // namespace

// Shared state (queue, results, budget and counters) is guarded by `mu`;
// the worker thread owns the active runs' contexts and does the slow work
// (building a context, enqueueing steps, reading results, destroying it)
// without holding `mu`, so that submit and poll never wait behind it.
struct ibl_server {
  ibl_server_config cfg{};
  int device = 0;
  clock_type::time_point t0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<std::shared_ptr<Run>> queue;
  std::map<int64_t, std::shared_ptr<Run>> all;
  int64_t next_id = 1;
  size_t in_use = 0;
  int active = 0;                                 // admitted and not yet retired
  int finished = 0;
  std::vector<std::shared_ptr<Run>> running;      // worker-owned
  std::map<ShapeKey, Launch> tuned;                // worker-owned: fastest launch per run shape
  int num_sms = 0;
  // scheduling thread's time, ns (written by the worker, read by ibl_server_load)
  std::atomic<int64_t> busy_ns{0}, enqueue_ns{0}, build_ns{0}, retire_ns{0};
  std::atomic<bool> stop{false};
  std::thread worker;
  std::string err;
};

namespace {

double now_s(const ibl_server* s) {
  return std::chrono::duration<double>(clock_type::now() - s->t0).count();
}

int64_t ns_since(clock_type::time_point t) {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(clock_type::now() - t).count();
}

ibl_status apply_launch(ibl_ctx* ctx, const Launch& l) {
  const ibl_status st = ibl_set_overlap(ctx, l.overlap);
  return st != IBL_OK ? st : ibl_set_collide_shape(ctx, l.bx, l.by, l.pairs);
}

// Flat elliptic planform (chord c, span 5c), unit-spaced cell-centred marker
// mesh clipped to the ellipse; body frame x chordwise (leading edge at -c/2),
// y normal, z spanwise.  Each marker carries its cell's area.
void planform(double chord, std::vector<double>& X0, std::vector<double>& ds) {
  const double a = 0.5 * chord, b = 2.5 * chord;
  const int ni = (int)std::ceil(a) + 1, nk = (int)std::ceil(b) + 1;
  X0.clear();
  ds.clear();
  for (int i = -ni; i < ni; ++i)
    for (int k = -nk; k < nk; ++k) {
      const double x = i + 0.5, z = k + 0.5;
      if ((x / a) * (x / a) + (z / b) * (z / b) <= 1.0) {
        X0.push_back(x);
        X0.push_back(0.0);
        X0.push_back(z);
        ds.push_back(1.0);
      }
    }
}

size_t estimate_bytes(const ibl_run_request& r, int m_total, int m_body) {
  const size_t N = (size_t)r.nx * r.ny * r.nz;
  const size_t elem = r.precision == IBL_FP64 ? 8 : (r.precision == IBL_FP32 ? 4 : 2);
  size_t b = 2 * 19 * N * elem;                                     // populations
  const size_t tiles = (N + ibl::TILE_CELLS - 1) / ibl::TILE_CELLS;
  const size_t slots = std::min<size_t>(tiles, (size_t)m_total + 4096);
  const size_t rs = r.precision == IBL_FP64 ? 8 : 4;
  b += tiles * 4 + slots * (7 * ibl::TILE_CELLS * rs + 3 * ibl::TILE_CELLS * 8 + ibl::TILE_MARKER_CAP * 4 + 16);
  b += (size_t)m_total * (ibl::G_MAXNNZ * 12 + 320 * 4 + 64 * 8 + 12 * 8);
  b += 2 * (size_t)m_body * ((m_body + 3) & ~3) * 4;                // dense preconditioners
  b += 2 * (size_t)ibl::HIST_LEN * 3 * 8;                            // force histories
  return b + (64u << 20);                                           // slack
}

// Relaxation time and the largest imposed velocities of a request (lattice
// units): U_tip = 2 Phi f c with Phi = 120 degrees (Eq. 24, Sec. 3.4),
// nu = U_tip c / Re, tau = 3 nu + 1/2 (Eq. 3), free stream U_inf = J U_tip.
void run_parameters(const ibl_run_request& r, double& tau, double& u_tip, double& u_inf) {
  const double pi = 3.14159265358979323846;
  u_tip = 2.0 * (2.0 * pi / 3.0) * (1.0 / r.period) * r.chord;
  const double nu = u_tip * r.chord / r.Re;
  tau = 3.0 * nu + 0.5;
  u_inf = r.J * u_tip;
}

// Stability screen at submission (BGK collision): requests outside it are
// refused with IBL_EUNSTABLE instead of diverging after using the GPU.
// Bounds from the 64-request sweep (Re 75-150, f 0.05 / 0.25, J 1e-3..2, on
// 96^3 .. 256 x 192 x 160 boxes): every run with tau below 0.505 or a
// uniform free stream of 0.05 lattice units or more diverged, and so did
// every run whose wings moved faster than 0.05 lattice units at the tip with
// a wall-cell Reynolds number u_tip / nu above 5; tip speeds of 0.02 were
// stable down to tau = 0.505.
constexpr double SERVE_TAU_MIN = 0.505;
constexpr double SERVE_U_FREE_MAX = 0.05;
constexpr double SERVE_U_WALL_MAX = 0.15;
constexpr double SERVE_U_WALL_FAST = 0.05;
constexpr double SERVE_RE_CELL_FAST_MAX = 5.0;

bool stable_request(double tau, double u_tip, double u_inf) {
  const double nu = (tau - 0.5) / 3.0;
  if (!(tau >= SERVE_TAU_MIN) || !(u_inf <= SERVE_U_FREE_MAX) || !(u_tip <= SERVE_U_WALL_MAX)) return false;
  return !(u_tip > SERVE_U_WALL_FAST && u_tip > SERVE_RE_CELL_FAST_MAX * nu);
}

// Build the context of a clap-and-fling wing pair (Sec. 3.3): trailing-edge
// hinges c/2 apart about the mid-plane, opening angle (pi/3)|sin(2 pi t/T)|
// per wing, Re = U_tip c / nu with U_tip = 2 Phi f c, Phi = 120 degrees
// (Eq. 24), tau = 3 nu + 1/2 (Eq. 3), free stream U_inf = J U_tip.
ibl_status build_run(ibl_server* s, Run& run) {
  const ibl_run_request& r = run.req;
  const double pi = 3.14159265358979323846;
  const double f = 1.0 / r.period;
  double tau = 0, u_tip = 0, u_inf = 0;
  run_parameters(r, tau, u_tip, u_inf);
  ibl_grid g{};
  g.nx = r.nx; g.ny = r.ny; g.nz = r.nz;
  const int xface0 = r.faces ? IBL_VEL_INLET : IBL_PERIODIC;
  const int xface1 = r.faces ? IBL_PRESS_OUTLET : IBL_PERIODIC;
  const int bc[6] = {xface0, xface1, IBL_PERIODIC, IBL_PERIODIC, IBL_PERIODIC, IBL_PERIODIC};
  for (int i = 0; i < 6; ++i) g.bc[i] = bc[i];
  g.u_in[0] = u_inf;
  g.rho_out = 1.0;
  g.precision = r.precision;
  ibl_status st = ibl_create(&g, tau, IBL_D3Q19, &run.ctx);
  if (st != IBL_OK) return st;
  std::vector<double> X0, ds;
  planform(r.chord, X0, ds);
  const int m = (int)ds.size();
  const double hx = std::round(r.nx / 3.0), ymid = 0.5 * r.ny, zc = 0.5 * r.nz, gap = 0.5 * r.chord;
  const double hinge[3] = {0.5 * r.chord, 0.0, 0.0};
  for (int w = 0; w < 2; ++w) {
    const double side = w == 0 ? -1.0 : 1.0;
    const double axis[3] = {0.0, 0.0, w == 0 ? 1.0 : -1.0};
    const double origin[3] = {hx - 0.5 * r.chord, ymid + side * 0.5 * gap, zc};
    int32_t bid = -1;
    st = ibl_set_markers(run.ctx, m, X0.data(), ds.data(), hinge, axis, origin, &bid);
    if (st != IBL_OK) return st;
    ibl_wave A{IBL_WAVE_CONST, 0.0, 0.0, nullptr, 0};
    ibl_wave al{IBL_WAVE_ABS_SIN, pi / 3.0, 0.0, nullptr, 0};
    st = ibl_set_kinematics(run.ctx, bid, &A, &al, 0.0, 0.0, f, r.J);
    if (st != IBL_OK) return st;
    const double lift[3] = {0.0, side, 0.0};
    st = ibl_set_lift_axis(run.ctx, bid, lift);
    if (st != IBL_OK) return st;
    run.m[w] = m;
  }
  st = ibl_set_reference(run.ctx, u_tip, (double)m, 1.0);
  if (st != IBL_OK) return st;
  if (s->cfg.tune) {
    // solve blocks from the marker count alone (they fix the reduction order)
    const int half = std::max(4, s->num_sms / 2);
    run.solve_blocks = std::min(half, std::max(4, (2 * m + MARKERS_PER_SOLVE_BLOCK - 1) / MARKERS_PER_SOLVE_BLOCK));
    st = ibl_solver_blocks(run.ctx, run.solve_blocks);
    if (st != IBL_OK) return st;
    const auto it = s->tuned.find(shape_key(r));
    if (it != s->tuned.end()) {
      run.launch = it->second;
      run.tuned = true;
      st = apply_launch(run.ctx, run.launch);
      if (st != IBL_OK) return st;
    } else if (r.steps >= 1 + NCAND * TUNE_MIN_STEPS) {
      int per = std::max(TUNE_MIN_STEPS, (s->cfg.chunk_steps - 1) / NCAND);
      while (1 + (int64_t)NCAND * per > r.steps) --per;
      run.tune_steps = per;
      for (auto& e : run.tev)
        if (cudaEventCreate(&e) != cudaSuccess) return IBL_ECUDA;
      run.tune_pending = true;
    }
  }
  std::vector<double> u(3 * (size_t)g.nx * g.ny * g.nz, 0.0);
  std::fill(u.begin(), u.begin() + (size_t)g.nx * g.ny * g.nz, u_inf);
  st = ibl_init_fluid(run.ctx, nullptr, u.data());
  if (st != IBL_OK) return st;
  return cudaEventCreateWithFlags(&run.ev, cudaEventDisableTiming) == cudaSuccess ? IBL_OK : IBL_ECUDA;
}

// Reduce a finished run's force histories to the per-wing statistics and
// release its context (no lock held); the caller publishes the result.
void collect(Run& run, ibl_status st, ibl_run_result& res) {
  res.status = st;
  if (st == IBL_OK || st == IBL_ENOTCONV) {
    std::vector<double> h(3 * (size_t)std::max<int64_t>(run.req.steps, 1));
    for (int w = 0; w < 2; ++w) {
      int64_t n = 0;
      const ibl_status hs = ibl_force_history(run.ctx, w, run.req.steps, h.data(), &n);
      if (hs != IBL_OK && hs != IBL_ENOTCONV) {
        res.status = hs;
        break;
      }
      double clmax = -1e300, ctmax = -1e300, clsum = 0, ctsum = 0;
      for (int64_t k = 0; k < n; ++k) {
        clmax = std::max(clmax, h[3 * k]);
        ctmax = std::max(ctmax, h[3 * k + 1]);
        clsum += h[3 * k];
        ctsum += h[3 * k + 1];
      }
      res.CL_max[w] = n ? clmax : 0;
      res.CT_max[w] = n ? ctmax : 0;
      res.CL_mean[w] = n ? clsum / n : 0;
      res.CT_mean[w] = n ? ctsum / n : 0;
      res.CL_last[w] = n ? h[3 * (n - 1)] : 0;
      res.CT_last[w] = n ? h[3 * (n - 1) + 1] : 0;
    }
  }
  if (run.ev) cudaEventDestroy(run.ev);
  run.ev = nullptr;
  for (auto& e : run.tev) {
    if (e) cudaEventDestroy(e);
    e = nullptr;
  }
  res.solve_blocks = run.solve_blocks;
  res.overlap = run.launch.overlap;
  res.collide_bx = run.launch.bx;
  res.collide_by = run.launch.by;
  res.collide_pairs = run.launch.pairs;
  res.tuned = run.tuned ? 1 : 0;
  if (run.ctx) ibl_destroy(run.ctx);
  run.ctx = nullptr;
}

// Publish a finished (or failed, or cancelled) run and, if it was admitted,
// return its memory to the budget; `mu` must be held.
void publish(ibl_server* s, Run& run, const ibl_run_result& res, bool admitted) {
  const double submit = run.res.submit_s, start = run.res.start_s;
  const int64_t done = run.steps_enqueued;
  run.res = res;
  run.res.submit_s = submit;
  run.res.start_s = start;
  run.res.steps_done = done;
  run.res.finish_s = now_s(s);
  run.res.done = 1;
  if (admitted) {
    s->in_use -= run.bytes;
    s->active--;
  }
  s->finished++;
  s->cv.notify_all();
}

// The tuning chunk: one untimed step (the first solve builds the
// preconditioner), then tune_steps steps under each candidate launch between
// a pair of timing events on the run's stream.  Every candidate computes the
// same populations, so the run advances exactly as it would untuned.
ibl_status enqueue_tuning(Run& r, int64_t& steps) {
  void* stream = nullptr;
  ibl_stream(r.ctx, &stream);
  steps = 0;
  ibl_status st = ibl_step(r.ctx, 1);
  if (st != IBL_OK) return st;
  steps = 1;
  for (int k = 0; k < NCAND; ++k) {
    st = apply_launch(r.ctx, CANDIDATES[k]);
    if (st != IBL_OK) return st;
    cudaEventRecord(r.tev[2 * k], (cudaStream_t)stream);
    st = ibl_step(r.ctx, r.tune_steps);
    if (st != IBL_OK) return st;
    cudaEventRecord(r.tev[2 * k + 1], (cudaStream_t)stream);
    steps += r.tune_steps;
  }
  return IBL_OK;
}

// After the tuning chunk: keep the fastest candidate for this run and for
// every later run of the same shape.
ibl_status finish_tuning(ibl_server* s, Run& r) {
  int best = 0;
  float best_ms = 0.0f;
  for (int k = 0; k < NCAND; ++k) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, r.tev[2 * k], r.tev[2 * k + 1]) != cudaSuccess) return IBL_ECUDA;
    if (k == 0 || ms < best_ms) {
      best = k;
      best_ms = ms;
    }
  }
  r.launch = CANDIDATES[best];
  r.tuned = true;
  s->tuned.emplace(shape_key(r.req), r.launch);
  return apply_launch(r.ctx, r.launch);
}

void worker_loop(ibl_server* s) {
  cudaSetDevice(s->device);
  while (!s->stop.load()) {
    const auto t_pass = clock_type::now();
    bool busy = false;
    // 1. admission by arrival order, active count and HBM budget; the
    // contexts are built after the lock is released
    std::vector<std::shared_ptr<Run>> admit;
    {
      std::lock_guard<std::mutex> lock(s->mu);
      while (!s->queue.empty() && s->active < s->cfg.max_active) {
        auto run = s->queue.front();
        if (run->cancel.load()) {
          s->queue.pop_front();
          ibl_run_result res = run->res;
          res.status = IBL_ECANCELED;
          publish(s, *run, res, false);
          continue;
        }
        if (s->in_use + run->bytes > (size_t)s->cfg.hbm_budget_bytes && s->active > 0) break;
        s->queue.pop_front();
        s->in_use += run->bytes;
        s->active++;
        admit.push_back(run);
      }
    }
    for (auto& run : admit) {
      const double t_start = now_s(s);
      const auto t0 = clock_type::now();
      const ibl_status st = build_run(s, *run);
      s->build_ns += ns_since(t0);
      busy = true;
      if (st != IBL_OK) {
        ibl_run_result res{};
        collect(*run, st, res);
        std::lock_guard<std::mutex> lock(s->mu);
        run->res.start_s = t_start;
        publish(s, *run, res, true);
        continue;
      }
      {
        std::lock_guard<std::mutex> lock(s->mu);
        run->res.start_s = t_start;
      }
      s->running.push_back(run);
    }
    // 2. next chunk of every run whose previous chunk finished; 3. retire
    for (size_t i = 0; i < s->running.size();) {
      Run& r = *s->running[i];
      ibl_status st = IBL_OK;
      if (r.inflight) {
        if (cudaEventQuery(r.ev) == cudaErrorNotReady) {
          ++i;
          continue;
        }
        r.inflight = false;
        busy = true;
        // the run's stream is idle: reading its status bits costs one small
        // copy, and a divergence stops the run here instead of at its end
        st = ibl_sync(r.ctx);
        if (st == IBL_ENOTCONV) st = IBL_OK;   // reported, not fatal
        if (st == IBL_OK && r.tune_inflight) {
          r.tune_inflight = false;
          st = finish_tuning(s, r);
        }
      }
      const bool cancelled = r.cancel.load();
      bool finish = cancelled || st != IBL_OK || r.steps_enqueued >= r.req.steps;
      if (!finish) {
        const auto t0 = clock_type::now();
        int64_t n = 0;
        if (r.tune_pending) {
          r.tune_pending = false;
          st = enqueue_tuning(r, n);
          r.tune_inflight = st == IBL_OK;
        } else {
          n = std::min<int64_t>(s->cfg.chunk_steps, r.req.steps - r.steps_enqueued);
          st = ibl_step(r.ctx, n);
        }
        if (st == IBL_OK) {
          void* stream = nullptr;
          ibl_stream(r.ctx, &stream);
          cudaEventRecord(r.ev, (cudaStream_t)stream);
          r.inflight = true;
          r.steps_enqueued += n;
        }
        s->enqueue_ns += ns_since(t0);
        if (st == IBL_OK) {
          std::lock_guard<std::mutex> lock(s->mu);
          r.res.steps_done = r.steps_enqueued;
        } else {
          finish = true;
        }
      }
      if (!finish) {
        busy = true;
        ++i;
        continue;
      }
      const auto t0 = clock_type::now();
      if (cancelled && st == IBL_OK) st = IBL_ECANCELED;
      else if (st == IBL_OK) st = ibl_sync(r.ctx);
      ibl_run_result res{};
      collect(r, st, res);
      s->retire_ns += ns_since(t0);
      {
        std::lock_guard<std::mutex> lock(s->mu);
        publish(s, r, res, true);
      }
      s->running.erase(s->running.begin() + i);
      busy = true;
    }
    if (busy) s->busy_ns += ns_since(t_pass);
    else std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

}  // namespace

extern "C" {

ibl_status ibl_server_create(const ibl_server_config* cfg, ibl_server** out) {
  if (!out || !cfg) return IBL_EINVAL;
  *out = nullptr;
  if (cfg->max_active < 1 || cfg->chunk_steps < 1 || cfg->hbm_budget_bytes <= 0 || cfg->tune < 0 || cfg->tune > 1)
    return IBL_EINVAL;
  ibl_server* s = new ibl_server();
  s->cfg = *cfg;
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    return IBL_ECUDA;
  }
  cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device);
  s->t0 = clock_type::now();
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return IBL_OK;
}

ibl_status ibl_server_submit(ibl_server* s, const ibl_run_request* req, int64_t* run_id) {
  if (!s || !req) return IBL_EINVAL;
  const double submit_s = now_s(s);   // before any lock: the wait for it counts as latency
  if (req->nx < 16 || req->ny < 16 || req->nz < 16 || !(req->chord >= 4.0) || !(req->Re > 0) ||
      !(req->period > 0) || !(req->J >= 0) || req->steps < 1 || req->steps > ibl::HIST_LEN ||
      req->precision < IBL_FP64 || req->precision > IBL_BF16DEV)
    return IBL_EINVAL;
  // the wings must fit: chord and span within the box with stencil margins
  if (req->chord * 5.0 + 8 > req->nz || std::round(req->nx / 3.0) - req->chord < 4 ||
      0.5 * req->ny - 0.25 * req->chord - req->chord < 4)
    return IBL_EINVAL;
  double tau = 0, u_tip = 0, u_inf = 0;
  run_parameters(*req, tau, u_tip, u_inf);
  if (!stable_request(tau, u_tip, u_inf)) return IBL_EUNSTABLE;
  auto run = std::make_shared<Run>();
  run->req = *req;
  std::vector<double> X0, ds;
  planform(req->chord, X0, ds);
  const int m = (int)ds.size();
  run->bytes = estimate_bytes(*req, 2 * m, m);
  if (run->bytes > (size_t)s->cfg.hbm_budget_bytes) return IBL_ENOMEM;
  run->res.submit_s = submit_s;
  run->res.status = IBL_OK;
  std::lock_guard<std::mutex> lock(s->mu);
  run->id = s->next_id++;
  s->queue.push_back(run);
  s->all[run->id] = run;
  if (run_id) *run_id = run->id;
  return IBL_OK;
}

ibl_status ibl_server_cancel(ibl_server* s, int64_t run_id) {
  if (!s) return IBL_EINVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->all.find(run_id);
  if (it == s->all.end()) return IBL_EINVAL;
  if (!it->second->res.done) it->second->cancel.store(true);
  return IBL_OK;
}

ibl_status ibl_server_poll(ibl_server* s, int64_t run_id, ibl_run_result* out) {
  if (!s || !out) return IBL_EINVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->all.find(run_id);
  if (it == s->all.end()) return IBL_EINVAL;
  *out = it->second->res;
  return IBL_OK;
}

ibl_status ibl_server_wait_all(ibl_server* s, double timeout_s) {
  if (!s) return IBL_EINVAL;
  std::unique_lock<std::mutex> lock(s->mu);
  const auto deadline = clock_type::now() + std::chrono::duration<double>(timeout_s);
  while (!(s->queue.empty() && s->active == 0)) {
    if (s->cv.wait_until(lock, deadline) == std::cv_status::timeout && !(s->queue.empty() && s->active == 0))
      return IBL_ETIMEOUT;
  }
  return IBL_OK;
}

ibl_status ibl_server_load(ibl_server* s, double* wall_s, double* busy_s, double* enqueue_s, double* build_s,
                           double* retire_s) {
  if (!s) return IBL_EINVAL;
  if (wall_s) *wall_s = now_s(s);
  if (busy_s) *busy_s = 1e-9 * (double)s->busy_ns.load();
  if (enqueue_s) *enqueue_s = 1e-9 * (double)s->enqueue_ns.load();
  if (build_s) *build_s = 1e-9 * (double)s->build_ns.load();
  if (retire_s) *retire_s = 1e-9 * (double)s->retire_ns.load();
  return IBL_OK;
}

ibl_status ibl_server_stats(ibl_server* s, int32_t* queued, int32_t* active, int32_t* finished,
                            int64_t* hbm_in_use) {
  if (!s) return IBL_EINVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  if (queued) *queued = (int32_t)s->queue.size();
  if (active) *active = (int32_t)s->active;
  if (finished) *finished = s->finished;
  if (hbm_in_use) *hbm_in_use = (int64_t)s->in_use;
  return IBL_OK;
}

ibl_status ibl_server_destroy(ibl_server* s) {
  if (!s) return IBL_OK;
  s->stop.store(true);
  if (s->worker.joinable()) s->worker.join();
  for (auto& r : s->running) {
    if (r->ev) cudaEventDestroy(r->ev);
    if (r->ctx) ibl_destroy(r->ctx);
  }
  delete s;
  return IBL_OK;
}

}  // extern "C"
