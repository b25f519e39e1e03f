// Internal definitions shared by the CUDA translation units of libibl.
//
// Data layout in HBM (one context):
//   populations  two buffers f[2], each Q x N of the storage type, direction
//                major (SoA), cell index (z*ny + y)*nx + x, x contiguous.  The
//                stored value is the deviation g_i = f_i - w_i (rho_0 = 1),
//                which keeps FP32 / FP16 / BF16 rounding relative to the small
//                non-rest part of f.
//   between steps the "current" buffer holds POST-COLLISION populations of
//                the previous step; a step pulls them along -c_i (streaming,
//                left side of Eq. 1), applies the face conditions, recovers
//                the moments, collides (Eq. 7) and writes the next buffer at
//                the same cell (pull scheme).  After ibl_init_fluid the buffer
//                holds post-streaming populations; the first step then
//                collides without pulling.
//   IB band      grid tiles of TILE_X x TILE_Y x TILE_Z cells touched by a
//                marker stencil get a slot; per slot the band moments
//                (rho, u*) and the force density F, each TILE_CELLS wide.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "ibl.h"

#include "lattice.cuh"

namespace ibl {

struct SepBody;   // separable preconditioner of one body (sep.cuh)

// ----------------------------------------------------------------- bodies
struct Wave {
  int kind;
  double amp, offset;
};

struct BodyDev {
  int offset, m;
  double hinge[3], axis[3], origin[3];
  double st[8];          // motion state of the step (A, A', alpha', cos, sin, e_s, alpha)
  int prescribed;        // 1: use the uploaded X/U for this step
};

struct Body {
  int offset = 0, m = 0;
  double hinge[3] = {0, 0, 0}, axis[3] = {0, 0, 1}, origin[3] = {0, 0, 0};
  double beta = 0, phi = 0, f = 0, J = 0;
  Wave A{0, 0, 0}, alpha{0, 0, 0};
  std::vector<double> hostA, hostAlpha;   // TABLE samples
  double lift[3] = {0, 1, 0};
  bool prescribed = false;
  int precond_offset = 0;   // offset of this body's dense preconditioner (floats)
};

}  // namespace ibl

// ----------------------------------------------------------------- the context
struct ibl_ctx {
  int Q = 0, D = 0;
  int nx = 0, ny = 0, nz = 0;
  long long N = 0;
  int bc[6] = {0, 0, 0, 0, 0, 0};
  double u_in[3] = {0, 0, 0}, rho_out = 1.0, G[3] = {0, 0, 0};
  int prec = IBL_FP32;
  double tau = 1.0;
  int device = 0;
  cudaStream_t stream = nullptr;
  // collide of the cells outside the IB band, concurrent with the IB chain
  cudaStream_t stream_bulk = nullptr;
  cudaEvent_t ev_tiles = nullptr;   // band tiles of the step assigned (stream)
  cudaEvent_t ev_bulk = nullptr;    // bulk collide done (stream_bulk)
  int overlap = -1;                 // -1 automatic, 0 off, 1 on
  int collide_bx = 64, collide_by = 2;   // thread block of the one-kernel collide
  int collide_pairs = 3;             // 16-bit storage: 3 two cells and ZP planes per thread, 1 two cells,
                                     // 2 staged planes, 0 one cell per thread
  size_t elem = 4;               // bytes per stored population
  void* f[2] = {nullptr, nullptr};
  int cur = 0;
  bool initialised = false;
  bool poststream = true;        // current buffer holds post-streaming populations
  long long step = 0;
  long long launches = 0;
  int* d_status = nullptr;       // [0] step status bits, [1] point-operator flag
  double* d_mass_parts = nullptr;  // MASS_PARTS partial sums of the periodic mass check
  double* d_mass_ref = nullptr;    // [0] total at initialisation, [1] last total, [2] checks
  int mass_every = 500;            // steps between mass checks (0: off)
  double mass_tol = 0.0;           // relative drift bound (0: default for the precision)
  int* d_pt_perm = nullptr;      // point operators: sorted point order (pt_cap ints)
  int* d_pt_bins = nullptr;      // point operators: per-tile counters / offsets (n_tiles ints)
  size_t pt_cap = 0;
  void* d_pt_mom = nullptr;       // point operators: drho and u* of every cell (4 N values)
  void* d_pt_sbase = nullptr;     // point operators: stencil bases (3 per point)
  void* d_pt_swts = nullptr;      // point operators: double-float stencil weights (12 per point)
  size_t pt_st_cap = 0;
  size_t pt_mom_bytes = 0;
  int sticky = 0;                // host copy of status bits seen so far
  std::string err;

  // ---- IB state
  std::vector<ibl::Body> bodies;
  int m_total = 0;
  ibl::TileGeom tg{};
  bool ib_ready = false;         // device IB buffers sized for m_total
  int cap_slots = 0;
  double U_ref = 1.0, L_ref = 1.0, rho_ref = 1.0;
  // device arrays (doubles unless noted)
  double* d_X0 = nullptr;        // m x 3 body frame
  double* d_ds = nullptr;        // m
  int* d_body = nullptr;         // m body index
  double* d_X = nullptr;         // m x 3 world positions of the step
  double* d_U = nullptr;         // m x 3 wall velocities
  double* d_Xp = nullptr;        // m x 3 prescribed positions (ibl_set_marker_state)
  double* d_Up = nullptr;
  ibl::BodyDev* d_bodies = nullptr;
  int* d_tile_slot = nullptr;    // n_tiles
  int* d_slot_tile = nullptr;    // cap_slots
  int* d_band_count = nullptr;   // 1 int: used slots
  int* d_tile_mcount = nullptr;  // cap_slots
  int* d_tile_markers = nullptr; // cap_slots x TILE_MARKER_CAP
  void* d_band_F = nullptr;      // cap_slots x 3 x TILE_CELLS (real)
  int* d_base = nullptr;         // m x 3 stencil base nodes (unwrapped)
  double* d_wts = nullptr;       // m x 3 x 4 delta weights per axis (double-float pairs, 8 B each)
  double* d_rho_l = nullptr;     // m interpolated density
  double* d_B = nullptr;         // m x 3 right-hand side
  double* d_w = nullptr;         // m x 3 solution (du_B * ds)
  double* d_r = nullptr;         // m x 3
  double* d_p = nullptr;         // 2 x m x 3 (ping-pong)
  double* d_Ap = nullptr;        // m x 3
  double* d_z = nullptr;         // m x 3
  float* d_xf = nullptr;         // 3 padded FP32 vectors feeding the preconditioner
  size_t xf_floats = 0;          // floats per padded vector
  unsigned long long* d_trace = nullptr;   // 256 PCG phase timestamps
  unsigned long long* d_acc = nullptr;     // cap_slots x 3 x TILE_CELLS fixed-point spread sums
  int* d_slot_body = nullptr;              // body that first touched each band slot
  int* d_mixed = nullptr;                  // 1: use the tile-based assembly this step
  int* d_cand = nullptr;                   // m x CAND_MAX rigid-body partner candidates
  int* d_ncand = nullptr;
  bool cand_ready = false;
  int* d_Gcol = nullptr;         // m x G_MAXNNZ
  double* d_Gval = nullptr;      // m x G_MAXNNZ
  int* d_Gnnz = nullptr;         // m
  double* d_Gdiag_max = nullptr; // per body, for the shift
  float* d_M = nullptr;          // sum_b m_b^2 dense preconditioners
  size_t M_floats = 0;
  double* d_red = nullptr;       // reduction scratch
  int* d_cg_info = nullptr;      // [iterations, refresh request]
  double* d_cg_res = nullptr;    // final relative residual
  double* d_hist = nullptr;      // bodies x HIST_LEN x 3 force vectors
  double* d_mforce = nullptr;    // m x 3 marker forces 2 rho_l w
  int* d_boff = nullptr;         // bodies + 1 marker offsets
  long long refreshes = 0;
  long long last_refresh_step = -1000000;
  bool precond_valid = false;
  bool warm = false;             // d_w holds the previous solution
  long long warm_steps = 0;      // consecutive solves behind d_w (2+: extrapolate)
  int extrapolate = 1;            // initial guess: 2 quadratic, 1 linear extrapolation, 0 last solution, -1 zero
  int refresh_every = 384;       // steps between scheduled preconditioner rebuilds
  double solver_tol = 0.0;       // 0: default for the storage precision
  int pcg_blocks = 0;            // blocks of the cooperative solve (0: half the SMs)
  int precond_kind = -1;         // -1 automatic, 0 dense per-body inverse, 1 separable
  bool sep_on = false;           // the separable preconditioner is in use (sep.cu)
  ibl::SepBody* d_sep = nullptr; // per body: sizes, index maps, factors, scratch
  std::vector<void*> sep_allocs; // device buffers behind d_sep
  bool sep_eigen_ready = false;  // span factors decomposed
  int sep_blocks = 0;            // blocks of the cooperative rebuild
  size_t sep_smem = 0;           // dynamic shared memory the solve's separable stages need
  int resident_rows = -1;        // -1 preconditioner rows in shared memory when they fit, 0 never
  size_t pcg_smem = 0;           // dynamic shared memory of the last solve launch
  double* d_wprev = nullptr;     // m x 3 solution of the previous step
  double* d_wprev2 = nullptr;    // m x 3 solution of the step before that
  // optional per-step event timing (ibl_profile)
  bool profiling = false;
  // 6 events per step: [0] start, [1] IB chain done, [2] collide done,
  // [3] end (stream); [4], [5] bulk collide start/end (stream_bulk, when split)
  std::vector<cudaEvent_t> prof_ev;
  std::vector<char> prof_split;
  long long prof_steps = 0;
  // ibl_profile(ctx, 2): an event after every kernel of the step on the
  // main stream, logged as (phase, event); phase -1 opens a step
  int prof_level = 0;
  std::vector<cudaEvent_t> pev_pool;
  size_t pev_used = 0;
  std::vector<std::pair<int, cudaEvent_t>> pev_log;
  // host copies of the bodies' marker sets (uploaded when the IB buffers are sized)
  std::vector<double> h_X0;      // m x 3
  std::vector<double> h_ds;      // m
  // pinned staging ring for ibl_set_marker_state
  double* h_stage = nullptr;
  cudaEvent_t stage_ev[4] = {nullptr, nullptr, nullptr, nullptr};
  int stage_next = 0;
  size_t stage_doubles = 0;
};

namespace ibl {

// error helpers (api.cu)
// Host <-> device copies and fills ordered on the context's stream.  The
// stream is non-blocking, so the legacy-stream forms (cudaMemcpy,
// cudaMemset) are not ordered against the context's kernels: with other
// contexts loading the GPU a fill could land after a kernel that had
// already written the same buffer.
inline cudaError_t to_device(ibl_ctx* c, void* dst, const void* src, size_t bytes) {
  return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->stream);
}
inline cudaError_t to_host(ibl_ctx* c, void* dst, const void* src, size_t bytes) {
  const cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, c->stream);
  return e != cudaSuccess ? e : cudaStreamSynchronize(c->stream);
}
inline cudaError_t fill_zero(ibl_ctx* c, void* dst, size_t bytes) {
  return cudaMemsetAsync(dst, 0, bytes, c->stream);
}
ibl_status fail(ibl_ctx* c, ibl_status s, const std::string& msg);
ibl_status cuda_check(ibl_ctx* c, cudaError_t e, const char* what);
ibl_status sync_and_collect(ibl_ctx* c);   // drain the stream, fold device status bits

// fluid launches (lbm.cu)
cudaError_t launch_init_eq(ibl_ctx* c, const double* d_rho, const double* d_u);
cudaError_t launch_set_pop(ibl_ctx* c, const double* d_f);
cudaError_t launch_collide(ibl_ctx* c, bool with_ib);
cudaError_t launch_collide_bulk(ibl_ctx* c, int blocks, cudaStream_t st);
cudaError_t launch_collide_band(ibl_ctx* c, int blocks);
cudaError_t launch_fields(ibl_ctx* c, double* d_rho, double* d_u, double* d_pop);
cudaError_t launch_mass(ibl_ctx* c, double* d_partials, int nparts, double* d_out);
constexpr int MASS_PARTS = 1024;
cudaError_t launch_mass_check(ibl_ctx* c, int mode);   // 0: store the reference, 1: check

// IB launches (ib.cu)
cudaError_t ib_alloc(ibl_ctx* c);
void ib_free(ibl_ctx* c);
cudaError_t ib_step(ibl_ctx* c);          // kinematics .. spreading, before the collision
cudaError_t ib_step_front(ibl_ctx* c);    // kinematics and the band tiles of the step
cudaError_t ib_step_back(ibl_ctx* c);     // interpolation .. solve .. spreading
int num_sms();
void phase_mark(ibl_ctx* c, int phase);   // ibl_profile level 2 only
int pcg_block_count(const ibl_ctx* c);
// Marker count up to which the step is split automatically: beyond it the
// solve (dense per-body preconditioner, m^2 per iteration) dominates and
// gets every SM.
constexpr int SPLIT_MAX_MARKERS = 8192;
cudaError_t launch_force_field(ibl_ctx* c, double* d_out);

// separable preconditioner (sep.cu)
// Bodies with at least this many markers (the largest body counts) use the
// separable preconditioner automatically when every body is separable: the
// dense inverse costs m_b^2 FP32 per iteration and m_b^3 per rebuild.
constexpr int SEP_AUTO_MIN_MARKERS = 4096;
bool sep_all_separable(const ibl_ctx* c, int* max_markers);
cudaError_t sep_alloc(ibl_ctx* c);
void sep_free(ibl_ctx* c);
size_t sep_smem_bytes(const ibl_ctx* c);
cudaError_t sep_launch(ibl_ctx* c, const int geo_n[3], const int geo_per[3]);

}  // namespace ibl
