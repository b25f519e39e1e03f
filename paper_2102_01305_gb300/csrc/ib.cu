// Immersed-boundary kernels: the implicit velocity-correction exchange of
// Sec. 2.2 (Wu and Shu's formulation) between the fluid and the markers.
//
// Per step, in the paper's order:
//   k_kinematics     marker positions X and wall velocities U_B (Eqs. 20-23,
//                    rotational velocity of Sec. 3.3; the per-body motion
//                    state comes from the host), stencil base nodes and the
//                    4-point cosine weights (Eq. 14, FP64, stored as FP32 pairs);
//   k_mark/assign/append
//                    grid tiles touched by a stencil get a band slot and a
//                    list of the markers that touch them;
//   k_interp_assemble
//                    one launch, two block ranges: rho_l and u*_l (Eq. 17)
//                    from the populations of the stencil nodes (moments of
//                    Eq. 11), B = U_B - u*_l (Eq. 19); and the sparse
//                    G_lk = sum_x D(x-X_l) D(x-X_k) (Eq. 18 without ds_k: the
//                    solve is run on w = ds * du_B, G w = B);
//   k_pcg            preconditioned conjugate gradients for the three velocity
//                    components at once in double-float arithmetic, an FP32
//                    dense per-body approximate inverse as preconditioner,
//                    rebuilt in-kernel (blocked Gauss-Jordan) every few hundred
//                    steps;
//   (end of k_pcg)   du(x) = sum_l w_l D(x - X_l) (Eq. 15) into 64-bit
//                    fixed-point band accumulators (order-independent sums);
//                    the collide kernel forms F = 2 rho du (Eq. 26) from them;
//   (end of k_pcg)   F_w = -sum_l 2 rho_l w_l per body in FP64, fixed order.
#include <cooperative_groups.h>

#include <cmath>

#include "df.cuh"
#include "ib_stencil.cuh"
#include "sep.cuh"

namespace cg = cooperative_groups;

namespace ibl {

constexpr int MAX_BODIES = 16;
constexpr int GJ_NB = 64;          // Gauss-Jordan pivot block
constexpr int PCG_MAX_ITERS = 200;
// relative preconditioned residual (the spread field's A-norm error) per
// storage precision, under the field error the storage itself accumulates:
// FP32 runs sit at field errors of ~2e-6 against the FP64 reference after
// hundreds of steps whether the solve stops at 1e-6 or 1e-7 (measured on
// every FP32 parity case), so FP32 stops at 1e-6 like FP16 / BF16
constexpr double PCG_TOL = 1e-10;       // FP64
constexpr double PCG_TOL_FP32 = 1e-6;   // FP32 deviations
constexpr double PCG_TOL_HALF = 1e-6;   // FP16 / BF16 deviations

// Early rebuilds follow a rent-or-buy rule.  Since the last rebuild, every
// solve adds to a running excess the iterations it needed beyond both the
// first solve after that rebuild and REBUILD_ITERS_OK.  Below that count a
// rebuild does not pay: on the 256 x 192 x 160 wings the count climbs from
// 11 to 20 within 380 steps as the markers leave the rebuild's pose, and
// rebuilding on that excess (every 60-100 steps) left the step time
// unchanged.  When the excess passes the rebuild's cost in
// iterations, the next solve rebuilds first.  That cost is the ratio of the
// operation counts: 2 m_b^3 for an inverse, and 6 m_b^2 for one iteration's
// preconditioner product over three right-hand sides.  Each is summed over
// the bodies, and the ratio is floored at REBUILD_MIN_EXCESS.  Only
// iteration counts enter the rule, so runs stay reproducible bit for bit.
// A solve that does not converge asks for a rebuild directly.
constexpr int REBUILD_MIN_EXCESS = 64;
constexpr int REBUILD_ITERS_OK = 40;

struct BodyTable {
  int n;
  BodyDev b[MAX_BODIES];
};

struct Geo {
  int D;
  int n[3];
  int per[3];     // periodic axis flags
  TileGeom tg;
};

__device__ __forceinline__ int wrap(int v, int n) {
  // stencil offsets stay within one period of the axis (n >= 8 is enforced)
  if (v < 0) v += n;
  else if (v >= n) v -= n;
  return v;
}

// One thread per (marker, axis): the axis's position, wall velocity, stencil
// base and weights (the rotation is recomputed by each of the three threads,
// which is cheaper than serialising the three stencils on one thread).
__global__ void k_kinematics(BodyTable bt, int m_total, const int* __restrict__ body_of,
                             const double* __restrict__ X0, const double* __restrict__ Xp,
                             const double* __restrict__ Up, double* __restrict__ X,
                             double* __restrict__ U, int* __restrict__ base,
                             df* __restrict__ wts, double t, Geo geo, int* status) {
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  const int l = gid / 3, a = gid - 3 * (gid / 3);
  if (l >= m_total) return;
  const BodyDev& B = bt.b[body_of[l]];
  double x, u;
  if (B.prescribed) {
    x = Xp[3 * l + a];
    u = Up[3 * l + a];
  } else {
    // per-body motion state of this step (formed on the host): A, A', alpha', cos, sin, e_s
    const double* st = B.st;
    const double A = st[0], Ad = st[1], ald = st[2], c = st[3], s = st[4];
    const double es[3] = {st[5], st[6], 0.0};
    const double* e = B.axis;
    double d[3];
    for (int k = 0; k < 3; ++k) d[k] = X0[3 * l + k] - B.hinge[k];
    // Rodrigues: r = d cos + (e x d) sin + e (e.d)(1 - cos)
    const double ed = e[0] * d[0] + e[1] * d[1] + e[2] * d[2];
    const double exd[3] = {e[1] * d[2] - e[2] * d[1], e[2] * d[0] - e[0] * d[2],
                           e[0] * d[1] - e[1] * d[0]};
    double r[3];
    for (int k = 0; k < 3; ++k) r[k] = d[k] * c + exd[k] * s + e[k] * ed * (1.0 - c);
    const int a1 = a == 2 ? 0 : a + 1, a2 = a == 0 ? 2 : a - 1;
    const double exr = e[a1] * r[a2] - e[a2] * r[a1];
    x = B.origin[a] + B.hinge[a] + r[a] + A * es[a];
    u = Ad * es[a] + ald * exr;
  }
  if (a >= geo.D) {
    X[3 * l + a] = 0.0;
    U[3 * l + a] = 0.0;
    base[3 * l + a] = 0;
    wts[12 * l + 4 * a + 0] = df_make(1.f, 0.f);
    wts[12 * l + 4 * a + 1] = df_make(0.f, 0.f);
    wts[12 * l + 4 * a + 2] = df_make(0.f, 0.f);
    wts[12 * l + 4 * a + 3] = df_make(0.f, 0.f);
    return;
  }
  X[3 * l + a] = x;
  U[3 * l + a] = u;
  int b0;
  double w[4];
  if (!stencil_axis(x, geo.n[a], geo.per[a] != 0, b0, w)) atomicOr(status, ST_OVERFLOW);
  for (int k = 0; k < 4; ++k) wts[12 * l + 4 * a + k] = df_from_double(w[k]);
  base[3 * l + a] = b0;
}

// ------------------------------------------------------------------ band tiles
__device__ __forceinline__ int tile_of(const Geo& g, int nx, int ny, int nz) {
  return ((nz / g.tg.tz) * g.tg.nty + (ny / g.tg.ty)) * g.tg.ntx + (nx / g.tg.tx);
}

// Tiles touched by marker l's stencil (at most 2 per axis); returns the count.
__device__ int touched_tiles(const Geo& g, const int* b, int out[8]) {
  int tl[3][2], cnt[3];
  for (int a = 0; a < 3; ++a) {
    if (a >= g.D) { tl[a][0] = 0; cnt[a] = 1; continue; }
    const int ext = a == 0 ? g.tg.tx : (a == 1 ? g.tg.ty : g.tg.tz);
    cnt[a] = 0;
    for (int k = 0; k < 4; ++k) {
      const int node = g.per[a] ? wrap(b[a] + k, g.n[a]) : b[a] + k;
      const int t = node / ext;
      bool seen = false;
      for (int j = 0; j < cnt[a]; ++j) seen |= (tl[a][j] == t);
      if (!seen && cnt[a] < 2) tl[a][cnt[a]++] = t;
    }
  }
  int n = 0;
  for (int i = 0; i < cnt[2]; ++i)
    for (int j = 0; j < cnt[1]; ++j)
      for (int k = 0; k < cnt[0]; ++k)
        out[n++] = (tl[2][i] * g.tg.nty + tl[1][j]) * g.tg.ntx + tl[0][k];
  return n;
}


__global__ void k_mark_tiles(int m_total, const int* __restrict__ base, Geo g,
                             int* __restrict__ tile_slot) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= m_total) return;
  int t[8];
  const int n = touched_tiles(g, base + 3 * l, t);
  for (int i = 0; i < n; ++i) tile_slot[t[i]] = -2;
}

// Every tile: marked (-2) ones get a band slot with cleared per-slot state;
// all others, including the last step's band, get -1.  (No separate reset of
// the last band is needed.)
__global__ void k_assign_slots(int n_tiles, int* __restrict__ tile_slot, int* __restrict__ slot_tile,
                               int* __restrict__ band_count, int cap, int* __restrict__ tile_mcount,
                               int* __restrict__ slot_body, int* status) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n_tiles; t += gridDim.x * blockDim.x) {
    if (tile_slot[t] == -2) {
      const int s = atomicAdd(band_count, 1);
      if (s < cap) {
        tile_slot[t] = s;
        slot_tile[s] = t;
        tile_mcount[s] = 0;
        slot_body[s] = -1;
      } else {
        tile_slot[t] = -1;
        atomicOr(status, ST_OVERFLOW);
      }
    } else {
      tile_slot[t] = -1;
    }
  }
}

// One thread per (marker, touched tile): the appends of a marker are
// independent, so none waits on another's atomics.
__global__ void k_append_markers(int m_total, const int* __restrict__ base, Geo g,
                                 const int* __restrict__ tile_slot, int* __restrict__ tile_mcount,
                                 int* __restrict__ tile_markers, int* status, const int* __restrict__ body_of,
                                 int* __restrict__ slot_body, int* __restrict__ mixed) {
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  const int l = gid >> 3, i = gid & 7;
  if (l >= m_total) return;
  int t[8];
  const int n = touched_tiles(g, base + 3 * l, t);
  if (i >= n) return;
  const int s = tile_slot[t[i]];
  if (s < 0) return;
  const int bl = body_of[l];
  const int prev = atomicCAS(&slot_body[s], -1, bl);
  if (prev != -1 && prev != bl) *mixed = 1;   // two bodies' stencils share a tile
  const int pos = atomicAdd(&tile_mcount[s], 1);
  if (pos < TILE_MARKER_CAP) tile_markers[s * TILE_MARKER_CAP + pos] = l;
  else atomicOr(status, ST_OVERFLOW);
}

// rho_l and u*_l (Eq. 17) gathered straight from the populations of each
// stencil node (the same pull, face rules and moment arithmetic as the
// collision), FP64 accumulation; B = U_B - u*_l (Eq. 19).  One warp per
// marker, 64 (3D) or 16 (2D) nodes over its lanes.
template <int Q, class T, bool PULL>
__device__ __forceinline__ void interpolate_body(int vblock, int m_total, const int* __restrict__ base, const df* __restrict__ wts,
                              const T* __restrict__ src, FluidParams<typename Store<T>::R> p, Geo g,
                              const double* __restrict__ U, double* __restrict__ rho_l,
                              double* __restrict__ B) {
  using R = typename Store<T>::R;
  const int warp = (vblock * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= m_total) return;
  const int l = warp;
  const int* b = base + 3 * l;
  const df* w = wts + 12 * l;
  const int nnodes = g.D == 3 ? 64 : 16;
  // double-float accumulation of sum_x D(x - X_l) (1 + drho, u*): the weight
  // products and sums stay on the FP32 pipes
  dfacc acc[4] = {acc_zero(), acc_zero(), acc_zero(), acc_zero()};
  for (int k = lane; k < nnodes; k += 32) {
    const int i = k & 3, j = (k >> 2) & 3, q = k >> 4;
    int node[3] = {b[0] + i, b[1] + j, g.D == 3 ? b[2] + q : 0};
    for (int a = 0; a < g.D; ++a)
      if (g.per[a]) node[a] = wrap(node[a], g.n[a]);
    df wt = df_mul(w[i], w[4 + j]);
    if (g.D == 3) wt = df_mul(wt, w[8 + q]);
    const long long cell = ((long long)node[2] * p.ny + node[1]) * p.nx + node[0];
    R drho, u[3];
    node_moments<Q, T, PULL>(src, node[0], node[1], node[2], cell, p, drho, u);
    acc_fma(acc[0], wt, df_from_float(1.f));
    acc_fma(acc[0], wt, to_df(drho));
    for (int c = 0; c < 3; ++c) acc_fma(acc[1 + c], wt, to_df(u[c]));
  }
  df v[4];
  for (int c = 0; c < 4; ++c) v[c] = df_warp_sum(acc_value(acc[c]));
  if (lane == 0) {
    rho_l[l] = df_to_double(v[0]);
    for (int a = 0; a < 3; ++a) B[3 * l + a] = (a < g.D) ? U[3 * l + a] - df_to_double(v[1 + a]) : 0.0;
  }
}

// ------------------------------------------------------------------ system assembly
// Markers of one rigid body keep their mutual distances.  Two stencils
// overlap only if every coordinate differs by less than 4, hence only if the
// Euclidean distance is below 4 sqrt(D): that set, computed once from the
// body-frame coordinates, holds every possible partner of a marker forever.
constexpr int CAND_MAX = 320;

__global__ void k_build_candidates(int m_total, const double* __restrict__ X0, const int* __restrict__ body_of,
                                   const int* __restrict__ boff, int D, int* __restrict__ cand,
                                   int* __restrict__ ncand, int* __restrict__ status) {
  const int l = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (l >= m_total) return;
  const int b = body_of[l];
  const int o = boff[b], e = boff[b + 1];
  const double r2 = 16.0 * D * (1.0 + 1e-12);
  int count = 0;
  for (int k0 = o; k0 < e; k0 += 32) {
    const int k = k0 + lane;
    bool take = false;
    if (k < e) {
      double d2 = 0.0;
      for (int a = 0; a < 3; ++a) {
        const double d = X0[3 * k + a] - X0[3 * l + a];
        d2 += d * d;
      }
      take = d2 < r2;
    }
    const unsigned mask = __ballot_sync(0xffffffffu, take);
    const int pos = count + __popc(mask & ((1u << lane) - 1));
    if (take && pos < CAND_MAX) cand[(long long)l * CAND_MAX + pos] = k;
    count += __popc(mask);
  }
  if (lane == 0) {
    ncand[l] = min(count, CAND_MAX);
    if (count > CAND_MAX) *status = 1;   // too dense for the lists: always use the tile search
  }
}

// Minimal-image difference of stencil bases along an axis.
__device__ __forceinline__ int base_diff(int bk, int bl, int n, int per) {
  int d = bk - bl;
  if (per) {
    d = wrap(d, n);
    if (d > n / 2) d -= n;
  }
  return d;
}

// One warp per row l: candidates are the markers listed in l's touched tiles;
// a pair is counted in the tile holding the lowest node of the two stencils'
// overlap box, so every k appears once.  Rows are sorted by column so that
// the SpMV sums in a fixed order.
// Overlap product of the two stencils of markers l and k (Eq. 18 entry
// without ds_k); false if the stencils do not share a node.
__device__ __forceinline__ bool pair_entry(const Geo& g, const int* bl, const df* wl, const int* bk,
                                           const df* wk, df& val, int lo[3]) {
  df prod = df_make(1.f, 0.f);
  for (int a = 0; a < 3; ++a) {
    if (a >= g.D) { lo[a] = 0; continue; }
    const int d = base_diff(bk[a], bl[a], g.n[a], g.per[a]);   // base_k - base_l
    if (d < -3 || d > 3) return false;
    const int o0 = d > 0 ? d : 0, o1 = d < 0 ? 3 + d : 3;
    dfacc s1 = acc_zero();
    for (int o = o0; o <= o1; ++o) acc_fma(s1, wl[4 * a + o], wk[4 * a + (o - d)]);
    prod = df_mul(prod, acc_value(s1));
    const int node = bl[a] + o0;
    lo[a] = g.per[a] ? wrap(node, g.n[a]) : node;
  }
  val = prod;
  return true;
}

__device__ __forceinline__ void assemble_body(int vblock, int m_total, const int* __restrict__ base, const df* __restrict__ wts,
                           const int* __restrict__ tile_slot, const int* __restrict__ tile_mcount,
                           const int* __restrict__ tile_markers, Geo g, const int* __restrict__ body_of,
                           int* __restrict__ Gcol, df* __restrict__ Gval, int* __restrict__ Gnnz,
                           unsigned long long* __restrict__ rowsum_max, int* status,
                           const int* __restrict__ cand, const int* __restrict__ ncand,
                           const int* __restrict__ use_tiles, const int* __restrict__ cand_bad) {
  __shared__ int s_col[8][G_MAXNNZ];
  __shared__ df s_val[8][G_MAXNNZ];
  const int wib = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int l = vblock * 8 + wib;
  if (l >= m_total) return;
  const int* bl = base + 3 * l;
  const df* wl = wts + 12 * l;
  if (cand && !*use_tiles && !*cand_bad) {
    // rigid-body path: precomputed candidates, already in ascending order
    const int nc = ncand[l];
    int count = 0;
    float rowsum = 0.f;
    for (int j0 = 0; j0 < nc; j0 += 32) {
      const int j = j0 + lane;
      bool take = false;
      df val = df_make(0.f, 0.f);
      int k = -1;
      if (j < nc) {
        k = cand[(long long)l * CAND_MAX + j];
        int lo[3];
        take = pair_entry(g, bl, wl, base + 3 * k, wts + 12 * k, val, lo);
      }
      const unsigned mask = __ballot_sync(0xffffffffu, take);
      const int pos = count + __popc(mask & ((1u << lane) - 1));
      if (take) {
        if (pos < G_MAXNNZ) {
          Gcol[(long long)l * G_MAXNNZ + pos] = k;
          Gval[(long long)l * G_MAXNNZ + pos] = val;
        } else {
          atomicOr(status, ST_OVERFLOW);
        }
        rowsum += fabsf(val.hi);
      }
      count += __popc(mask);
    }
    for (int o = 16; o > 0; o >>= 1) rowsum += __shfl_xor_sync(0xffffffffu, rowsum, o);
    if (lane == 0) {
      Gnnz[l] = min(count, G_MAXNNZ);
      atomicMax(&rowsum_max[body_of[l]], (unsigned long long)__double_as_longlong((double)rowsum));
    }
    return;
  }
  int tiles[8];
  const int nt = touched_tiles(g, bl, tiles);
  int count = 0;
  float rowsum = 0.f;
  for (int ti = 0; ti < nt; ++ti) {
    const int t = tiles[ti];
    const int s = tile_slot[t];
    if (s < 0) continue;
    const int cnt = min(tile_mcount[s], TILE_MARKER_CAP);
    for (int j0 = 0; j0 < cnt; j0 += 32) {
      const int j = j0 + lane;
      bool take = false;
      df val = df_make(0.f, 0.f);
      int k = -1;
      if (j < cnt) {
        k = tile_markers[s * TILE_MARKER_CAP + j];
        int lo[3];
        take = pair_entry(g, bl, wl, base + 3 * k, wts + 12 * k, val, lo);
        // count the pair only in the tile of the lowest node both stencils share
        if (take && tile_of(g, lo[0], lo[1], g.D == 3 ? lo[2] : 0) != t) take = false;
      }
      const unsigned mask = __ballot_sync(0xffffffffu, take);
      const int pos = count + __popc(mask & ((1u << lane) - 1));
      if (take) {
        if (pos < G_MAXNNZ) {
          s_col[wib][pos] = k;
          s_val[wib][pos] = val;
        } else {
          atomicOr(status, ST_OVERFLOW);
        }
        rowsum += fabsf(val.hi);
      }
      count += __popc(mask);
    }
  }
  __syncwarp();
  count = min(count, G_MAXNNZ);
  // rank sort by column (keys are distinct)
  for (int i = lane; i < count; i += 32) {
    const int key = s_col[wib][i];
    int rank = 0;
    for (int j = 0; j < count; ++j) rank += s_col[wib][j] < key;
    Gcol[(long long)l * G_MAXNNZ + rank] = key;
    Gval[(long long)l * G_MAXNNZ + rank] = s_val[wib][i];
  }
  for (int o = 16; o > 0; o >>= 1) rowsum += __shfl_xor_sync(0xffffffffu, rowsum, o);
  if (lane == 0) {
    Gnnz[l] = count;
    atomicMax(&rowsum_max[body_of[l]], (unsigned long long)__double_as_longlong((double)rowsum));
  }
}

// Interpolation (blocks [0, nb_interp): one warp per marker) and system
// assembly (the remaining blocks: one warp per row) in one launch: both
// need only the step's marker lists, and their latencies overlap.
struct AssembleArgs {
  const int* tile_slot;
  const int* tile_mcount;
  const int* tile_markers;
  const int* body_of;
  int* Gcol;
  df* Gval;
  int* Gnnz;
  unsigned long long* rowsum_max;
  int* status;
  const int* cand;
  const int* ncand;
  const int* use_tiles;
  const int* cand_bad;
};

template <int Q, class T, bool PULL>
__global__ void __launch_bounds__(256) k_interp_assemble(int nb_interp, int m_total, const int* __restrict__ base,
                                                         const df* __restrict__ wts, const T* __restrict__ src,
                                                         FluidParams<typename Store<T>::R> p, Geo g,
                                                         const double* __restrict__ U, double* __restrict__ rho_l,
                                                         double* __restrict__ B, AssembleArgs aa) {
  if ((int)blockIdx.x < nb_interp) {
    interpolate_body<Q, T, PULL>(blockIdx.x, m_total, base, wts, src, p, g, U, rho_l, B);
  } else {
    assemble_body(blockIdx.x - nb_interp, m_total, base, wts, aa.tile_slot, aa.tile_mcount, aa.tile_markers, g,
                  aa.body_of, aa.Gcol, aa.Gval, aa.Gnnz, aa.rowsum_max, aa.status, aa.cand, aa.ncand,
                  aa.use_tiles, aa.cand_bad);
  }
}

// ------------------------------------------------------------------ PCG with in-kernel preconditioner rebuild
// One (marker, stencil node) term of the spreading du(x) = sum_l w_l D(x - X_l)
// (Eq. 15) into 64-bit fixed-point band accumulators: integer addition is
// associative, so the sums are bitwise independent of the order the atomics
// land in.  Item gid = marker * nodes + node.
constexpr double FIX_LIMIT = 9.0e18 / FIX_SCALE;   // |sum| < 1.3e5 at 2^46, resolution 1.4e-14
__device__ __forceinline__ void spread_node(long long gid, int m_total, const int* __restrict__ base,
                                            const df* __restrict__ wts, const df* __restrict__ wsol,
                                            const int* __restrict__ tile_slot, const Geo& g,
                                            unsigned long long* __restrict__ acc, int* status) {
  const int nn = g.D == 3 ? 64 : 16;
  const int l = (int)(gid / nn), k = (int)(gid % nn);
  if (l >= m_total) return;
  const int* b = base + 3 * l;
  const df* w = wts + 12 * l;
  const int i = k & 3, j = (k >> 2) & 3, q = k >> 4;
  int node[3] = {b[0] + i, b[1] + j, g.D == 3 ? b[2] + q : 0};
  for (int a = 0; a < g.D; ++a)
    if (g.per[a]) node[a] = wrap(node[a], g.n[a]);
  df wt = df_mul(w[i], w[4 + j]);
  if (g.D == 3) wt = df_mul(wt, w[8 + q]);
  const int s = tile_slot[tile_of(g, node[0], node[1], node[2])];
  if (s < 0) return;
  const int local = ((node[2] % g.tg.tz) * g.tg.ty + (node[1] % g.tg.ty)) * g.tg.tx + (node[0] % g.tg.tx);
  unsigned long long* a3 = acc + (long long)s * 3 * TILE_CELLS + local;
  for (int c = 0; c < g.D; ++c) {
    // the double-float product in fixed point: both parts scale exactly by
    // 2^46 and round to integers separately (error <= 1 unit of 2^-46)
    const df v = df_mul(wt, wsol[3 * l + c]);
    if (!(fabsf(v.hi) < (float)FIX_LIMIT)) { atomicOr(status, ST_OVERFLOW); continue; }
    const long long fx = __float2ll_rn(v.hi * (float)FIX_SCALE) + __float2ll_rn(v.lo * (float)FIX_SCALE);
    atomicAdd(a3 + c * TILE_CELLS, (unsigned long long)fx);
  }
}

constexpr int PCG_THREADS = 1024;
constexpr int TRACE_SLOTS = 256;
constexpr int TRACE_PER_IT = 9;   // phase marks per traced iteration, from slot 8
constexpr int PCG_WARPS = PCG_THREADS / 32;

struct PcgArgs {
  int m_total;
  int D;
  int nbodies;
  int boff[MAX_BODIES + 1];     // marker offsets
  long long poff[MAX_BODIES];   // preconditioner offsets (floats, 16-byte aligned)
  int voff[MAX_BODIES];         // offset of each body's slice in the padded FP32 vectors
  int vtotal;                   // floats of one padded FP32 vector (all bodies), multiple of 12
  int smem_floats;              // dynamic shared memory available for staging, in floats
  int row_slot;                 // floats per resident preconditioner row (0: rows read from L2)
  const int* body_of;
  const int* Gcol;
  const df* Gv;     // system matrix entries (double-float)
  const int* Gnnz;
  const unsigned long long* rowsum_max;
  const double* B;
  double* w;        // solution, FP64 copy for the spreading
  // double-float vectors of the recurrence (m x 3)
  df* wd;           // solution
  df* wprevd;       // solution of the step before (extrapolated warm start)
  df* wprev2d;      // and of the step before that (quadratic extrapolation)
  df* rd;
  df* pd;
  df* Apd;
  float* zf;        // preconditioned residual M r (FP32: the preconditioner's output)
  float* rf;        // FP32 copies feeding the preconditioner: r, A p, B
  float* Apf;
  float* Bf;
  float* M;
  df* red;          // [gridDim][8] partials
  int* info;        // [0] iterations, [1] rebuild request, [2] converged flag, [3] early rebuilds,
                    // [4] iterations of the first solve after the last rebuild, [5] excess since
  int rebuild_excess;   // rebuild cost in iterations (early-rebuild threshold)
  double* res;      // final relative residual
  double tol;
  int warm;
  int refresh;      // host-scheduled rebuild
  int* status;
  unsigned long long* trace;   // optional phase timestamps (ns), see ibl_solver_trace
  // spreading of the solution at the end of the solve (Eq. 15)
  const int* base;
  const df* wts;
  const int* tile_slot;
  unsigned long long* acc;
  Geo geo;
  // body-force reduction after the solve (Sec. 3.7)
  const double* rho_l;
  double* mforce;
  double* hist;
  long long step;
  // separable preconditioner (all bodies) instead of the dense inverses
  const SepBody* sep;
  int sep_on;
};

__device__ __forceinline__ void trace_mark(const PcgArgs& A, int slot) {
  if (A.trace && blockIdx.x == 0 && threadIdx.x == 0 && slot < TRACE_SLOTS) {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    A.trace[slot] = t;
  }
}

// Fixed-order block sum of three doubles per warp (lane 0 holds them); the
// totals are returned to every thread.
__device__ void block_total3(double v[3], double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0)
    for (int c = 0; c < 3; ++c) sh[3 * wid + c] = v[c];
  __syncthreads();
  if (threadIdx.x < 32) {
    for (int c = 0; c < 3; ++c) {
      double t = threadIdx.x < PCG_WARPS ? sh[3 * threadIdx.x + c] : 0.0;
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      v[c] = t;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int c = 0; c < 3; ++c) sh[3 * PCG_WARPS + c] = v[c];
  __syncthreads();
  for (int c = 0; c < 3; ++c) v[c] = sh[3 * PCG_WARPS + c];
}

// Fixed-order block sum of one double per warp (lane 0 holds it); the total
// is returned to every thread.
__device__ double block_total(double v, double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < PCG_WARPS ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) sh[PCG_WARPS] = t;
  }
  __syncthreads();
  t = sh[PCG_WARPS];
  return t;
}

// Sum of the per-block partials in a fixed order by warp 0; every block
// computes bitwise the same totals, returned to all threads.  Each lane
// issues all of its loads before adding (one memory round trip).
constexpr int MAX_PCG_BLOCKS = 256;
template <int NV>
__device__ void grid_total(const double* red, int slot, double out[NV], double* sh) {
  __syncthreads();
  if (threadIdx.x < 32) {
    double buf[MAX_PCG_BLOCKS / 32][NV];
#pragma unroll
    for (int u = 0; u < MAX_PCG_BLOCKS / 32; ++u) {
      const int b = threadIdx.x + 32 * u;
#pragma unroll
      for (int c = 0; c < NV; ++c) buf[u][c] = b < (int)gridDim.x ? __ldcg(red + b * 8 + slot + c) : 0.0;
    }
    double v[NV];
#pragma unroll
    for (int c = 0; c < NV; ++c) {
      v[c] = 0.0;
#pragma unroll
      for (int u = 0; u < MAX_PCG_BLOCKS / 32; ++u) v[c] += buf[u][c];
    }
    for (int o = 16; o > 0; o >>= 1)
      for (int c = 0; c < NV; ++c) v[c] += __shfl_xor_sync(0xffffffffu, v[c], o);
    if (threadIdx.x == 0)
      for (int c = 0; c < NV; ++c) sh[c] = v[c];
  }
  __syncthreads();
  for (int c = 0; c < NV; ++c) out[c] = sh[c];
}

// Block partial of three double-float sums: lane c < 3 of every warp holds
// component c; warp c adds the warps in a fixed order and writes out[c].
__device__ void block_partial3(df v, df* sh, df* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane < 3) sh[3 * wid + lane] = v;
  __syncthreads();
  if (wid < 3) {
    df t = lane < PCG_WARPS ? sh[3 * lane + wid] : df_make(0.f, 0.f);
    t = df_warp_sum(t);
    if (lane == 0) out[wid] = t;
  }
}

// Grid total of one double-float partial (slot `slot` of every block), for
// one warp: each lane issues all of its loads at once (one memory round
// trip), adds its blocks in a fixed pairwise tree, then a butterfly; every
// lane ends with the total.
__device__ __forceinline__ df grid_total_df(const df* red, int slot) {
  constexpr int U = MAX_PCG_BLOCKS / 32;
  const int lane = threadIdx.x & 31;
  float2 v[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int b = lane + 32 * u;
    v[u] = b < (int)gridDim.x ? __ldcg(reinterpret_cast<const float2*>(red + b * 8 + slot)) : make_float2(0.f, 0.f);
  }
  // pairwise tree over the lane's blocks (depth log2 U instead of U)
  df t[U];
#pragma unroll
  for (int u = 0; u < U; ++u) t[u] = df_make(v[u].x, v[u].y);
#pragma unroll
  for (int w = U / 2; w >= 1; w >>= 1)
#pragma unroll
    for (int u = 0; u < w; ++u) t[u] = df_add(t[u], t[u + w]);
  return df_warp_sum(t[0]);
}

// Row stride of a body's dense preconditioner: padded to 4 floats so rows
// start 16-byte aligned for 128-bit loads.
__host__ __device__ __forceinline__ int precond_ld(int mb) { return (mb + 3) & ~3; }

// x = a - s b (FP32, all bodies' padded slices) into shared memory, or null
// when the vectors do not fit (then precond_row forms x from global memory).
// Slices start at multiples of 12 floats, so entry i is component i % 3 and
// the 128-bit group q holds components (4q, 4q+1, 4q+2, 4q+3) mod 3.
__device__ float* stage_x(const PcgArgs& A, const float* __restrict__ a, const float* __restrict__ b,
                          const float s[3], float* sm) {
  if (A.vtotal > A.smem_floats) return nullptr;
  __syncthreads();
  const int nq = A.vtotal >> 2;
  const float4* a4 = reinterpret_cast<const float4*>(a);
  const float4* b4 = reinterpret_cast<const float4*>(b);
  float4* o4 = reinterpret_cast<float4*>(sm);
#pragma unroll 4
  for (int q = threadIdx.x; q < nq; q += blockDim.x) {
    float4 v = __ldcg(a4 + q);
    if (b) {
      const float4 w = __ldcg(b4 + q);
      const int c0 = (4 * q) % 3;
      const float s0 = s[c0], s1 = s[(c0 + 1) % 3], s2 = s[(c0 + 2) % 3];
      v.x = fmaf(-s0, w.x, v.x);
      v.y = fmaf(-s1, w.y, v.y);
      v.z = fmaf(-s2, w.z, v.z);
      v.w = fmaf(-s0, w.w, v.w);
    }
    o4[q] = v;
  }
  __syncthreads();
  return sm;
}

// One row of the preconditioner: sum_j M_lj x_j with x_j = a_j - s * b_j
// (FP32).  x comes from shared memory (xs, already formed) or is formed here
// from global memory; 128-bit loads of M and x, lane-parallel over the row;
// the result is returned in every lane.
__device__ __forceinline__ void precond_row(const PcgArgs& A, int l, const float* __restrict__ xs,
                                            const float* __restrict__ a, const float* __restrict__ b,
                                            const float s[3], float out[3], int lane,
                                            const float* __restrict__ rs) {
  const int bd = A.body_of[l];
  const int o = A.boff[bd], mb = A.boff[bd + 1] - o;
  const int ld = precond_ld(mb);
  const float* row = A.M + A.poff[bd] + (long long)(l - o) * ld;
  float s0 = 0.f, s1 = 0.f, s2 = 0.f;
  const int nq = ld >> 2;
  if (xs && rs) {
    // the row is resident in shared memory (rs) for the whole solve
    const float* xb = xs + A.voff[bd];
#pragma unroll 4
    for (int q = lane; q < nq; q += 32) {
      const float4 mv = reinterpret_cast<const float4*>(rs)[q];
      const float4* xv = reinterpret_cast<const float4*>(xb + 12 * q);
      const float4 x0 = xv[0], x1 = xv[1], x2 = xv[2];
      s0 = fmaf(mv.x, x0.x, s0); s1 = fmaf(mv.x, x0.y, s1); s2 = fmaf(mv.x, x0.z, s2);
      s0 = fmaf(mv.y, x0.w, s0); s1 = fmaf(mv.y, x1.x, s1); s2 = fmaf(mv.y, x1.y, s2);
      s0 = fmaf(mv.z, x1.z, s0); s1 = fmaf(mv.z, x1.w, s1); s2 = fmaf(mv.z, x2.x, s2);
      s0 = fmaf(mv.w, x2.y, s0); s1 = fmaf(mv.w, x2.z, s1); s2 = fmaf(mv.w, x2.w, s2);
    }
  } else if (xs) {
    const float* xb = xs + A.voff[bd];
#pragma unroll 4
    for (int q = lane; q < nq; q += 32) {
      const float4 mv = __ldcg(reinterpret_cast<const float4*>(row) + q);
      const float4* xv = reinterpret_cast<const float4*>(xb + 12 * q);
      const float4 x0 = xv[0], x1 = xv[1], x2 = xv[2];
      s0 = fmaf(mv.x, x0.x, s0); s1 = fmaf(mv.x, x0.y, s1); s2 = fmaf(mv.x, x0.z, s2);
      s0 = fmaf(mv.y, x0.w, s0); s1 = fmaf(mv.y, x1.x, s1); s2 = fmaf(mv.y, x1.y, s2);
      s0 = fmaf(mv.z, x1.z, s0); s1 = fmaf(mv.z, x1.w, s1); s2 = fmaf(mv.z, x2.x, s2);
      s0 = fmaf(mv.w, x2.y, s0); s1 = fmaf(mv.w, x2.z, s1); s2 = fmaf(mv.w, x2.w, s2);
    }
  } else {
    const float* ab = a + A.voff[bd];
    const float* bb = b ? b + A.voff[bd] : nullptr;
#pragma unroll 2
    for (int q = lane; q < nq; q += 32) {
      const float4 mv = __ldcg(reinterpret_cast<const float4*>(row) + q);
      const float4* av = reinterpret_cast<const float4*>(ab + 12 * q);
      float4 x0 = av[0], x1 = av[1], x2 = av[2];
      if (bb) {
        const float4* bv = reinterpret_cast<const float4*>(bb + 12 * q);
        const float4 y0 = bv[0], y1 = bv[1], y2 = bv[2];
        x0.x = fmaf(-s[0], y0.x, x0.x); x0.y = fmaf(-s[1], y0.y, x0.y); x0.z = fmaf(-s[2], y0.z, x0.z);
        x0.w = fmaf(-s[0], y0.w, x0.w); x1.x = fmaf(-s[1], y1.x, x1.x); x1.y = fmaf(-s[2], y1.y, x1.y);
        x1.z = fmaf(-s[0], y1.z, x1.z); x1.w = fmaf(-s[1], y1.w, x1.w); x2.x = fmaf(-s[2], y2.x, x2.x);
        x2.y = fmaf(-s[0], y2.y, x2.y); x2.z = fmaf(-s[1], y2.z, x2.z); x2.w = fmaf(-s[2], y2.w, x2.w);
      }
      s0 = fmaf(mv.x, x0.x, s0); s1 = fmaf(mv.x, x0.y, s1); s2 = fmaf(mv.x, x0.z, s2);
      s0 = fmaf(mv.y, x0.w, s0); s1 = fmaf(mv.y, x1.x, s1); s2 = fmaf(mv.y, x1.y, s2);
      s0 = fmaf(mv.z, x1.z, s0); s1 = fmaf(mv.z, x1.w, s1); s2 = fmaf(mv.z, x2.x, s2);
      s0 = fmaf(mv.w, x2.y, s0); s1 = fmaf(mv.w, x2.z, s1); s2 = fmaf(mv.w, x2.w, s2);
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, off);
    s1 += __shfl_xor_sync(0xffffffffu, s1, off);
    s2 += __shfl_xor_sync(0xffffffffu, s2, off);
  }
  out[0] = s0; out[1] = s1; out[2] = s2;
}

// Rows l0 = 2p and l1 = 2p + 1 of the preconditioner in one pass when they
// belong to the same body (the usual case): each staged x group is read once
// for both rows, halving the shared-memory traffic that bounds this product.
// rs0 / rs1: the rows' resident copies or nullptr.  z1 is untouched when
// l1 >= m.
__device__ __forceinline__ void precond_pair(const PcgArgs& A, int p, const float* __restrict__ xs,
                                             const float* __restrict__ a, const float* __restrict__ b,
                                             const float s[3], float z0[3], float z1[3], int lane,
                                             const float* __restrict__ rs0, const float* __restrict__ rs1) {
  const int m = A.m_total;
  const int l0 = 2 * p, l1 = 2 * p + 1;
  const int bd = A.body_of[l0];
  if (!xs || l1 >= m || A.body_of[l1] != bd) {
    precond_row(A, l0, xs, a, b, s, z0, lane, rs0);
    if (l1 < m) precond_row(A, l1, xs, a, b, s, z1, lane, rs1);
    return;
  }
  const int o = A.boff[bd], ld = precond_ld(A.boff[bd + 1] - o), nq = ld >> 2;
  const float4* r0 = reinterpret_cast<const float4*>(rs0 ? rs0 : A.M + A.poff[bd] + (long long)(l0 - o) * ld);
  const float4* r1 = reinterpret_cast<const float4*>(rs1 ? rs1 : A.M + A.poff[bd] + (long long)(l1 - o) * ld);
  const float* xb = xs + A.voff[bd];
  float a0 = 0.f, a1 = 0.f, a2 = 0.f, b0 = 0.f, b1 = 0.f, b2 = 0.f;
#pragma unroll 2
  for (int q = lane; q < nq; q += 32) {
    const float4 m0 = rs0 ? r0[q] : __ldcg(r0 + q);
    const float4 m1 = rs1 ? r1[q] : __ldcg(r1 + q);
    const float4* xv = reinterpret_cast<const float4*>(xb + 12 * q);
    const float4 x0 = xv[0], x1 = xv[1], x2 = xv[2];
    a0 = fmaf(m0.x, x0.x, a0); a1 = fmaf(m0.x, x0.y, a1); a2 = fmaf(m0.x, x0.z, a2);
    a0 = fmaf(m0.y, x0.w, a0); a1 = fmaf(m0.y, x1.x, a1); a2 = fmaf(m0.y, x1.y, a2);
    a0 = fmaf(m0.z, x1.z, a0); a1 = fmaf(m0.z, x1.w, a1); a2 = fmaf(m0.z, x2.x, a2);
    a0 = fmaf(m0.w, x2.y, a0); a1 = fmaf(m0.w, x2.z, a1); a2 = fmaf(m0.w, x2.w, a2);
    b0 = fmaf(m1.x, x0.x, b0); b1 = fmaf(m1.x, x0.y, b1); b2 = fmaf(m1.x, x0.z, b2);
    b0 = fmaf(m1.y, x0.w, b0); b1 = fmaf(m1.y, x1.x, b1); b2 = fmaf(m1.y, x1.y, b2);
    b0 = fmaf(m1.z, x1.z, b0); b1 = fmaf(m1.z, x1.w, b1); b2 = fmaf(m1.z, x2.x, b2);
    b0 = fmaf(m1.w, x2.y, b0); b1 = fmaf(m1.w, x2.z, b1); b2 = fmaf(m1.w, x2.w, b2);
  }
  for (int off = 16; off > 0; off >>= 1) {
    a0 += __shfl_xor_sync(0xffffffffu, a0, off);
    a1 += __shfl_xor_sync(0xffffffffu, a1, off);
    a2 += __shfl_xor_sync(0xffffffffu, a2, off);
    b0 += __shfl_xor_sync(0xffffffffu, b0, off);
    b1 += __shfl_xor_sync(0xffffffffu, b1, off);
    b2 += __shfl_xor_sync(0xffffffffu, b2, off);
  }
  z0[0] = a0; z0[1] = a1; z0[2] = a2;
  z1[0] = b0; z1[1] = b1; z1[2] = b2;
}

// ---------------------------------------------------------------- dense rebuild
// In-place blocked Gauss-Jordan inverse of every body's dense SPD matrix
// (no pivoting; the matrix is G_b + sigma I, row stride precond_ld(m_b)).
// For the pivot block P (GJ_NB wide):
//   P <- P^-1;  row panel R <- P^-1 R;  rest S <- S - C R;  column panel C <- -C P^-1.
// The three panel products run through one register-tiled shared-memory
// routine (128 x 128 output tiles, 4 x 4 outputs per thread, K <= GJ_NB).
constexpr int GT = 128;                 // output tile edge (GT x GJ_NB = 2048 float4 groups)
constexpr int GS = GT + 4;              // padded shared-memory row
constexpr size_t GJ_SMEM = sizeof(float) * 2 * GJ_NB * GS;
// dynamic shared memory of the solve kernel: the rebuild's tiles, then one
// staged FP32 vector of all bodies (up to ~19k markers) and, when they fit,
// the block's preconditioner rows; at most 224 KB (227 KB per block, less
// the kernel's static shared memory)
constexpr size_t PCG_SMEM_MAX = 224 * 1024;

// Both routines below are compiled as separate functions: inlined into the
// solve kernel, which runs at 64 registers a thread, the tile product's
// accumulators spilled to local memory.
// out[i0+r][j0+c] = (acc ? out : 0) + alpha * sum_q A[r][q] B[q][j0+c] over one
// tile (r < nr, c < nc), skipping output rows in [sk0, sk1) and columns in
// [ck0, ck1).  Ag points at the tile's first A row; Bg at B's row 0 (its
// columns are absolute).  Inputs are staged in shared memory before any
// output is written, so out may alias A or B within the tile.
__device__ __noinline__ void tile_gemm(float* out, int ldo, const float* Ag, int lda, const float* Bg, int ldb, int i0,
                          int j0, int nr, int nc, int K, float alpha, bool acc, int sk0, int sk1, int ck0,
                          int ck1, float* sm) {
  float* As = sm;               // [q][r], GJ_NB x GS
  float* Bs = sm + GJ_NB * GS;  // [q][c], GJ_NB x GS
  __syncthreads();
  // 128-bit staging of 2048 float4 groups per operand, two per thread and
  // operand in flight at a time (rows, columns and K are multiples of 4
  // except at ragged edges, where the group falls back to masked scalar
  // loads); lda, ldb and the tile origins are multiples of 4 floats, so full
  // groups are 16-byte aligned.
  for (int u0 = 0; u0 < 2048 / PCG_THREADS; u0 += 2) {
    float4 av[2], bv[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int f = threadIdx.x + (u0 + u) * PCG_THREADS;
      const int r = f >> 4, q4 = (f & 15) << 2;
      if (r < nr && q4 + 3 < K) {
        av[u] = __ldcg(reinterpret_cast<const float4*>(Ag + (long long)r * lda + q4));
      } else {
        float t[4];
        for (int i = 0; i < 4; ++i) t[i] = (r < nr && q4 + i < K) ? Ag[(long long)r * lda + q4 + i] : 0.f;
        av[u] = make_float4(t[0], t[1], t[2], t[3]);
      }
      const int q = f >> 5, c4 = (f & 31) << 2;
      if (q < K && c4 + 3 < nc) {
        bv[u] = __ldcg(reinterpret_cast<const float4*>(Bg + (long long)q * ldb + j0 + c4));
      } else {
        float t[4];
        for (int i = 0; i < 4; ++i) t[i] = (q < K && c4 + i < nc) ? Bg[(long long)q * ldb + j0 + c4 + i] : 0.f;
        bv[u] = make_float4(t[0], t[1], t[2], t[3]);
      }
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int f = threadIdx.x + (u0 + u) * PCG_THREADS;
      const int r = f >> 4, q4 = (f & 15) << 2;
      As[(q4 + 0) * GS + r] = av[u].x;
      As[(q4 + 1) * GS + r] = av[u].y;
      As[(q4 + 2) * GS + r] = av[u].z;
      As[(q4 + 3) * GS + r] = av[u].w;
      const int q = f >> 5, c4 = (f & 31) << 2;
      *reinterpret_cast<float4*>(Bs + q * GS + c4) = bv[u];
    }
  }
  __syncthreads();
  // 32 x 32 groups of 4 x 4 outputs, PCG_THREADS / 32 row groups at a time
  const int tx = threadIdx.x & 31;
  for (int ty = threadIdx.x >> 5; ty < 32; ty += PCG_THREADS / 32) {
    float a4[4][4];
    for (int u = 0; u < 4; ++u)
      for (int v = 0; v < 4; ++v) a4[u][v] = 0.f;
    for (int q = 0; q < K; ++q) {
      const float4 av = *reinterpret_cast<const float4*>(As + q * GS + 4 * ty);
      const float4 bv = *reinterpret_cast<const float4*>(Bs + q * GS + 4 * tx);
      const float ar[4] = {av.x, av.y, av.z, av.w};
      const float br[4] = {bv.x, bv.y, bv.z, bv.w};
      for (int u = 0; u < 4; ++u)
        for (int v = 0; v < 4; ++v) a4[u][v] = fmaf(ar[u], br[v], a4[u][v]);
    }
    // the thread's four output groups: when they are whole columns outside
    // the skipped range, all four are read before any is written (the
    // compiler cannot reorder loads and stores through the same pointer)
    const int c0 = 4 * tx, jj = j0 + c0;
    const bool whole = c0 + 3 < nc && (jj + 3 < ck0 || jj >= ck1);
    float4 prev[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int r = 4 * ty + u, i = i0 + r;
      prev[u] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (acc && whole && r < nr && !(i >= sk0 && i < sk1))
        prev[u] = *reinterpret_cast<const float4*>(out + (long long)i * ldo + jj);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int r = 4 * ty + u, i = i0 + r;
      if (r >= nr || (i >= sk0 && i < sk1)) continue;
      float* o = out + (long long)i * ldo + jj;
      // four whole columns outside the skipped range: one 128-bit access
      // (ldo and the tile origins are multiples of 4 floats)
      if (whole) {
        float4 ov = prev[u];
        ov.x += alpha * a4[u][0];
        ov.y += alpha * a4[u][1];
        ov.z += alpha * a4[u][2];
        ov.w += alpha * a4[u][3];
        *reinterpret_cast<float4*>(o) = ov;
        continue;
      }
      for (int v = 0; v < 4; ++v) {
        const int c = c0 + v, j = jj + v;
        if (c >= nc || (j >= ck0 && j < ck1)) continue;
        o[v] = (acc ? o[v] : 0.f) + alpha * a4[u][v];
      }
    }
  }
}

// In-place inverse of the kn x kn pivot block at (k0, k0) of Mb (row stride
// ld) by threads 0..127 of the block; buf holds 2 x GJ_NB floats of shared
// memory.
__device__ __noinline__ void pivot_block_invert(float* Mb, int ld, int k0, int kn, float* buf) {
  const int i = threadIdx.x >> 1, h = threadIdx.x & 1, lane = threadIdx.x & 31;
  float a[32];
#pragma unroll
  for (int jj = 0; jj < 32; ++jj) {
    const int j = 32 * h + jj;
    a[jj] = (i < kn && j < kn) ? Mb[(long long)(k0 + i) * ld + k0 + j] : (i == j ? 1.f : 0.f);
  }
#pragma unroll
  for (int k = 0; k < GJ_NB; ++k) {
    float* rowk = buf + (k & 1) * GJ_NB;
    if (i == k) {
#pragma unroll
      for (int jj = 0; jj < 32; ++jj) rowk[32 * h + jj] = a[jj];
    }
    asm volatile("bar.sync 1, 128;" ::: "memory");
    const float pk = 1.0f / rowk[k];
    // element (i, k) lives in the thread of half k / 32 of row i
    const float ci = __shfl_sync(0xffffffffu, a[k & 31], (lane & ~1) | (k >> 5));
    const float* rh = rowk + 32 * h;
    if (i == k) {
#pragma unroll
      for (int jj = 0; jj < 32; ++jj) a[jj] = rh[jj] * pk;
    } else {
#pragma unroll
      for (int jj = 0; jj < 32; ++jj) a[jj] = fmaf(-ci, rh[jj] * pk, a[jj]);
    }
    if (h == (k >> 5)) a[k & 31] = i == k ? pk : -ci * pk;
  }
#pragma unroll
  for (int jj = 0; jj < 32; ++jj) {
    const int j = 32 * h + jj;
    if (i < kn && j < kn) Mb[(long long)(k0 + i) * ld + k0 + j] = a[jj];
  }
}

// Tiles of all bodies are dealt to the blocks round-robin in body order:
// with `done` tiles of earlier bodies dealt, this block's first tile of the
// next body is the smallest t >= 0 with (done + t) mod gridDim = blockIdx
// (t may exceed the body's count).
__device__ __forceinline__ int first_tile(int done) {
  const int t = (int)blockIdx.x - done % (int)gridDim.x;
  return t < 0 ? t + (int)gridDim.x : t;
}

__device__ __noinline__ void gj_invert(const PcgArgs& A, cg::grid_group& grid, float* sm) {
  int maxnb = 0;
  for (int b = 0; b < A.nbodies; ++b) {
    const int mb = A.boff[b + 1] - A.boff[b];
    maxnb = max(maxnb, (mb + GJ_NB - 1) / GJ_NB);
  }
  for (int kb = 0; kb < maxnb; ++kb) {
    const int k0 = kb * GJ_NB;
    // phase 1: invert the pivot block of body b in block b by Gauss-Jordan:
    // 64 sequential pivots, so 4 warps with a named barrier do it (a
    // block-wide barrier over 32 warps per pivot costs more than the
    // arithmetic).  Thread t holds half a row in registers (row t / 2,
    // columns 32 (t % 2) ...), the pivot loop is unrolled so that every
    // register index is static, and the pivot row goes through one of two
    // shared-memory buffers (one barrier per pivot).  A ragged last block is
    // padded with the identity, whose pivots leave the kn x kn part alone.
    for (int b = blockIdx.x; b < A.nbodies; b += gridDim.x) {
      const int mb = A.boff[b + 1] - A.boff[b];
      if (k0 >= mb) continue;
      const int kn = min(GJ_NB, mb - k0), ld = precond_ld(mb);
      float* Mb = A.M + A.poff[b];
      if (threadIdx.x < 2 * GJ_NB) pivot_block_invert(Mb, ld, k0, kn, sm);
      __syncthreads();
    }
    grid.sync();
    if (kb == 0) trace_mark(A, 4);
    // phase 2: row panel R <- P^-1 R (tiles of GJ_NB rows x GT columns)
    {
      int done = 0;
      for (int b = 0; b < A.nbodies; ++b) {
        const int mb = A.boff[b + 1] - A.boff[b];
        if (k0 >= mb) continue;
        const int kn = min(GJ_NB, mb - k0), ld = precond_ld(mb);
        float* Mb = A.M + A.poff[b];
        const int nt = (mb + GT - 1) / GT;
        for (int t = first_tile(done); t < nt; t += gridDim.x) {
          const int j0 = t * GT;
          tile_gemm(Mb, ld, Mb + (long long)k0 * ld + k0, ld, Mb + (long long)k0 * ld, ld, k0, j0, kn,
                    min(GT, mb - j0), kn, 1.0f, false, -1, -1, k0, k0 + kn, sm);
        }
        done += nt;
      }
    }
    grid.sync();
    if (kb == 0) trace_mark(A, 5);
    // phase 3a: S <- S - C R (rows and columns outside the pivot block)
    {
      int done = 0;
      for (int b = 0; b < A.nbodies; ++b) {
        const int mb = A.boff[b + 1] - A.boff[b];
        if (k0 >= mb) continue;
        const int kn = min(GJ_NB, mb - k0), ld = precond_ld(mb);
        float* Mb = A.M + A.poff[b];
        const int nt = (mb + GT - 1) / GT;
        for (int t = first_tile(done); t < nt * nt; t += gridDim.x) {
          const int i0 = (t / nt) * GT, j0 = (t % nt) * GT;
          tile_gemm(Mb, ld, Mb + (long long)i0 * ld + k0, ld, Mb + (long long)k0 * ld, ld, i0, j0,
                    min(GT, mb - i0), min(GT, mb - j0), kn, -1.0f, true, k0, k0 + kn, k0, k0 + kn, sm);
        }
        done += nt * nt;
      }
    }
    grid.sync();
    if (kb == 0) trace_mark(A, 6);
    // phase 3b: C <- -C P^-1 (rows outside, columns inside the pivot block)
    {
      int done = 0;
      for (int b = 0; b < A.nbodies; ++b) {
        const int mb = A.boff[b + 1] - A.boff[b];
        if (k0 >= mb) continue;
        const int kn = min(GJ_NB, mb - k0), ld = precond_ld(mb);
        float* Mb = A.M + A.poff[b];
        const int nt = (mb + GT - 1) / GT;
        for (int t = first_tile(done); t < nt; t += gridDim.x) {
          const int i0 = t * GT;
          tile_gemm(Mb, ld, Mb + (long long)i0 * ld + k0, ld, Mb + (long long)k0 * ld, ld, i0, k0,
                    min(GT, mb - i0), kn, kn, -1.0f, false, k0, k0 + kn, -1, -1, sm);
        }
        done += nt;
      }
    }
    grid.sync();
    if (kb == 0) trace_mark(A, 7);
  }
}

// Stages A-G of the separable preconditioner (sep.cuh) for all bodies and
// components, a grid barrier after each; the caller then reads each
// marker's z from the R0 rectangle (sep_marker_z).  With trace set (the
// set-up's first application) the end of each stage is time-stamped: slots
// 4-7 (unused by this preconditioner's rebuild) and 251-253 (after the
// iteration slots), from 250.
__device__ void sep_apply(const PcgArgs& A, cg::grid_group& grid, const SepIn& in, float* sm, bool trace) {
  const int marks[7] = {4, 5, 6, 7, 251, 252, 253};
  for (int st = 0; st < 7; ++st) {
    switch (st) {
      case 0: sep_gemm(A.sep, A.nbodies, 0, false, in, A.voff, sm); break;    // A  Y1 = X V
      case 1: sep_colpass(A.sep, A.nbodies, false, sm); break;                 // B  Y2 = H Y1
      case 2: sep_gemm(A.sep, A.nbodies, 2, true, in, A.voff, sm); break;     // C  T = Y2 V^T
      case 3: sep_schur(A.sep, A.nbodies, sm, A.smem_floats); break;          // D  u = S^-1 t
      case 4: sep_gemm(A.sep, A.nbodies, 1, false, in, A.voff, sm); break;    // E  W1 = U V
      case 5: sep_colpass(A.sep, A.nbodies, true, sm); break;                  // F  W2 = H W1
      default: sep_gemm(A.sep, A.nbodies, 3, true, in, A.voff, sm); break;    // G  Z = (Y2 - W2) V^T
    }
    grid.sync();
    if (trace) trace_mark(A, marks[st]);
  }
}

// Preconditioned CG on G w = B, three right-hand sides (velocity components)
// at once, two grid barriers per iteration, vectors and scalars in
// double-float.  A p is updated by the recurrence A p = G z + beta A p_old,
// so the SpMV reads z only and no direction is recomputed by its
// neighbours; r - alpha A p is formed in FP32 inside the preconditioner
// product.  SpMV rows go to warps in groups of four (8 lanes per row),
// preconditioner rows in pairs (2p, 2p + 1), pair p to block p mod gridDim.
__global__ void __launch_bounds__(PCG_THREADS, 1) k_pcg(PcgArgs A) {
  cg::grid_group grid = cg::this_grid();
  extern __shared__ __align__(16) float sm[];
  __shared__ double shd[3 * PCG_WARPS + 8];
  __shared__ df shdf[3 * PCG_WARPS + 8];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nthreads = gridDim.x * blockDim.x;
  const int m = A.m_total;
  const int row0 = blockIdx.x + gridDim.x * wib;       // this warp's first row (groups of 4 in the SpMV)
  const int rstep = gridDim.x * PCG_WARPS;

  // ---- optional preconditioner rebuild: M_b <- (G_b + sigma_b I)^-1 in FP32
  trace_mark(A, 0);
  // the separable factors are rebuilt by their own kernel on the host's
  // schedule only (sep_launch), so early requests apply to the dense path
  const bool rebuild = A.refresh || (!A.sep_on && A.info[1]);
  if (rebuild && !A.sep_on) {
    if (gtid == 0 && !A.refresh) A.info[3] += 1;   // early rebuilds (a slow previous solve)
    for (int b = 0; b < A.nbodies; ++b) {
      const int mb = A.boff[b + 1] - A.boff[b];
      const long long tot = (long long)mb * precond_ld(mb);
      for (long long e = gtid; e < tot; e += nthreads) A.M[A.poff[b] + e] = 0.f;
    }
    grid.sync();
    for (int l = gtid; l < m; l += nthreads) {
      const int b = A.body_of[l];
      const int o = A.boff[b], mb = A.boff[b + 1] - o, ld = precond_ld(mb);
      const double sigma = 1e-6 * __longlong_as_double((long long)A.rowsum_max[b]);
      float* Mb = A.M + A.poff[b];
      for (int j = 0; j < A.Gnnz[l]; ++j) {
        const int k = A.Gcol[(long long)l * G_MAXNNZ + j];
        if (A.body_of[k] != b) continue;   // block-Jacobi over bodies
        double v = df_to_double(A.Gv[(long long)l * G_MAXNNZ + j]);
        if (k == l) v += sigma;
        Mb[(long long)(l - o) * ld + (k - o)] = (float)v;
      }
    }
    grid.sync();
    gj_invert(A, grid, sm);
  }
  // the preconditioner is applied to row pairs (2p, 2p + 1), pair p owned by
  // block p mod gridDim, warp (p / gridDim) mod 32; this block's pairs
  // (jp-th: p = blockIdx.x + gridDim.x jp) stay in shared memory, rows 2jp
  // and 2jp + 1, for the whole solve when they fit
  const int npairs = (m + 1) >> 1;
  const int prow0 = blockIdx.x + gridDim.x * wib;
  float* mres = nullptr;
  if (A.row_slot > 0) {
    mres = sm + A.smem_floats;
    for (int jp = wib, pp = prow0; pp < npairs; jp += PCG_WARPS, pp += rstep)
      for (int h = 0; h < 2; ++h) {
        const int l = 2 * pp + h;
        if (l >= m) break;
        const int bd = A.body_of[l];
        const int o = A.boff[bd], ld = precond_ld(A.boff[bd + 1] - o);
        const float4* src = reinterpret_cast<const float4*>(A.M + A.poff[bd] + (long long)(l - o) * ld);
        float4* dst = reinterpret_cast<float4*>(mres + (long long)(2 * jp + h) * A.row_slot);
#pragma unroll 4
        for (int q = lane; q < (ld >> 2); q += 32) dst[q] = __ldcg(src + q);
      }
  }
  trace_mark(A, 1);

  // ---- set-up (double-float vectors): w0 = 0, the last solution,
  // 2 w_n-1 - w_n-2 once two exist, or 3 w_n-1 - 3 w_n-2 + w_n-3 once three
  // exist (the solution varies smoothly in time); r = B - G w0; FP32 copies;
  // p = A p = 0
  const df dzero = df_make(0.f, 0.f);
  if (A.warm >= 2) {
    for (int i = gtid; i < 3 * m; i += nthreads) {
      const df cur = A.wd[i], prev = A.wprevd[i];
      if (A.warm >= 3) {
        const df t = df_sub(cur, prev);
        A.wd[i] = df_add(df_add(df_add(A.wprev2d[i], t), t), t);
      } else {
        A.wd[i] = df_sub(df_make(2.f * cur.hi, 2.f * cur.lo), prev);
      }
      A.wprev2d[i] = prev;
      A.wprevd[i] = cur;
    }
    grid.sync();
  } else if (A.warm == 1) {
    for (int i = gtid; i < 3 * m; i += nthreads) {
      A.wprev2d[i] = A.wprevd[i];
      A.wprevd[i] = A.wd[i];
    }
  }
  for (int l = row0; l < m; l += rstep) {
    dfacc a0 = acc_zero(), a1 = acc_zero(), a2 = acc_zero();
    if (A.warm) {
      const int nnz = A.Gnnz[l];
      for (int j = lane; j < nnz; j += 32) {
        const int k = A.Gcol[(long long)l * G_MAXNNZ + j];
        const df v = A.Gv[(long long)l * G_MAXNNZ + j];
        acc_fma(a0, v, A.wd[3 * k]);
        acc_fma(a1, v, A.wd[3 * k + 1]);
        acc_fma(a2, v, A.wd[3 * k + 2]);
      }
    }
    const df g0 = df_warp_sum(acc_value(a0)), g1 = df_warp_sum(acc_value(a1)), g2 = df_warp_sum(acc_value(a2));
    if (lane < 3) {
      const int c = lane;
      const int vi = A.voff[A.body_of[l]] + 3 * (l - A.boff[A.body_of[l]]) + c;
      const df gx = c == 0 ? g0 : (c == 1 ? g1 : g2);
      const df b = df_from_double(A.B[3 * l + c]);
      const df r = df_sub(b, gx);
      A.rd[3 * l + c] = r;
      A.rf[vi] = r.hi;
      A.Bf[vi] = b.hi;
      A.pd[3 * l + c] = dzero;
      A.Apd[3 * l + c] = dzero;
      if (!A.warm) A.wd[3 * l + c] = dzero;
    }
  }
  grid.sync();
  // z = M r and the stopping scale B.(M B): lane c of each warp accumulates
  // component c; partials r.z (slots 3..5) and B.MB (0..2)
  const int gwarp = blockIdx.x * PCG_WARPS + wib, nwarp_all = gridDim.x * PCG_WARPS;
  if (A.sep_on) {
    df rz = dzero, bb = dzero;
    SepIn in;
    in.a = A.rf;
    in.b = nullptr;
    in.s[0] = in.s[1] = in.s[2] = 0.f;
    trace_mark(A, 250);
    sep_apply(A, grid, in, sm, true);
    for (int l = gwarp; l < m; l += nwarp_all) {
      const int bd = A.body_of[l];
      float z[3];
      sep_marker_z(A.sep[bd], l - A.boff[bd], z);
      if (lane < 3) {
        const float zc = lane == 0 ? z[0] : (lane == 1 ? z[1] : z[2]);
        A.zf[3 * l + lane] = zc;
        rz = df_add(rz, df_mul_f(A.rd[3 * l + lane], zc));
      }
    }
    grid.sync();   // every block has read its z before the next application writes R0
    in.a = A.Bf;
    sep_apply(A, grid, in, sm, false);
    for (int l = gwarp; l < m; l += nwarp_all) {
      const int bd = A.body_of[l];
      float z[3];
      sep_marker_z(A.sep[bd], l - A.boff[bd], z);
      if (lane < 3) {
        const float zc = lane == 0 ? z[0] : (lane == 1 ? z[1] : z[2]);
        bb = df_add(bb, df_mul_f(df_from_double(A.B[3 * l + lane]), zc));
      }
    }
    block_partial3(bb, shdf, A.red + blockIdx.x * 8);
    block_partial3(rz, shdf, A.red + blockIdx.x * 8 + 3);
  } else {
    df rz = dzero, bb = dzero;
    const float zero3[3] = {0.f, 0.f, 0.f};
    const float* xs = stage_x(A, A.rf, nullptr, zero3, sm);
    for (int jp = wib, pp = prow0; pp < npairs; jp += PCG_WARPS, pp += rstep) {
      float z6[2][3];
      precond_pair(A, pp, xs, A.rf, nullptr, zero3, z6[0], z6[1], lane, mres ? mres + (long long)(2 * jp) * A.row_slot : nullptr,
                   mres ? mres + (long long)(2 * jp + 1) * A.row_slot : nullptr);
      const int h = lane / 3, c = lane - 3 * (lane / 3), l = 2 * pp + h;
      if (lane < 6 && l < m) {
        const float zv = h == 0 ? z6[0][c] : z6[1][c];
        A.zf[3 * l + c] = zv;
        rz = df_add(rz, df_mul_f(A.rd[3 * l + c], zv));
      }
    }
    xs = stage_x(A, A.Bf, nullptr, zero3, sm);
    for (int jp = wib, pp = prow0; pp < npairs; jp += PCG_WARPS, pp += rstep) {
      float z6[2][3];
      precond_pair(A, pp, xs, A.Bf, nullptr, zero3, z6[0], z6[1], lane, mres ? mres + (long long)(2 * jp) * A.row_slot : nullptr,
                   mres ? mres + (long long)(2 * jp + 1) * A.row_slot : nullptr);
      const int h = lane / 3, c = lane - 3 * (lane / 3), l = 2 * pp + h;
      if (lane < 6 && l < m)
        bb = df_add(bb, df_mul_f(df_from_double(A.B[3 * l + c]), h == 0 ? z6[0][c] : z6[1][c]));
    }
    // lanes 3-5 hold the second row's components: fold them into lanes 0-2
    {
      const df r3 = df_make(__shfl_down_sync(0xffffffffu, rz.hi, 3), __shfl_down_sync(0xffffffffu, rz.lo, 3));
      const df b3 = df_make(__shfl_down_sync(0xffffffffu, bb.hi, 3), __shfl_down_sync(0xffffffffu, bb.lo, 3));
      if (lane < 3) {
        rz = df_add(rz, r3);
        bb = df_add(bb, b3);
      }
    }
    block_partial3(bb, shdf, A.red + blockIdx.x * 8);
    block_partial3(rz, shdf, A.red + blockIdx.x * 8 + 3);
  }
  grid.sync();
  trace_mark(A, 2);
  // Scalars of the recurrence live in shared memory: warp 0 of each block
  // forms them from the grid totals (every block gets bitwise the same values).
  __shared__ df s_rz[3], s_scale[3], s_beta[3], s_alpha[3];
  __shared__ float s_alphaf[3];
  __shared__ df s_stop[3];
  __shared__ int s_conv[3];
  if (wib < 3) {
    // warp c: totals of component c; the stopping threshold tol^2 (B.MB) once per solve
    const int c = wib;
    const df sc = grid_total_df(A.red, c);
    const df rz = grid_total_df(A.red, 3 + c);
    if (lane == 0) {
      s_scale[c] = sc;
      s_rz[c] = rz;
      s_beta[c] = dzero;
      s_stop[c] = df_from_double(A.tol * A.tol * df_to_double(sc));
      s_conv[c] = (c >= A.D || !df_greater(rz, s_stop[c])) ? 1 : 0;
    }
  }
  __syncthreads();
  const int s_done = s_conv[0] & s_conv[1] & s_conv[2];
  int it = 0;
  bool done = s_done != 0;
  // z of every marker (FP32) in shared memory for the SpMV when it fits
  const bool stage_z = 3 * m <= A.smem_floats;
  while (!done && it < PCG_MAX_ITERS) {
    // ---- P1: p = z + beta p;  A p = G z + beta A p;  partial p.Ap;  FP32 copies of r and A p
    // iterations 0..25 use slots 8..241; later ones are not traced (250-253 hold the set-up's marks)
    const int ts = it < 26 ? 8 + TRACE_PER_IT * it : TRACE_SLOTS;
    trace_mark(A, ts);
    {
      df pAp = dzero;
      const float* zs = A.zf;
      if (stage_z) {
        __syncthreads();
        const int n4 = (3 * m) >> 2;
        const float4* src = reinterpret_cast<const float4*>(A.zf);
        float4* dst = reinterpret_cast<float4*>(sm);
#pragma unroll 4
        for (int q = threadIdx.x; q < n4; q += blockDim.x) dst[q] = __ldcg(src + q);
        for (int q = 4 * n4 + threadIdx.x; q < 3 * m; q += blockDim.x) sm[q] = __ldcg(A.zf + q);
        __syncthreads();
        zs = sm;
      }
      trace_mark(A, ts + 1);
      // 8 lanes per row, 4 rows per warp
      const int sub = lane >> 3, sl = lane & 7;
      for (int l0 = row0 * 4; l0 < m; l0 += rstep * 4) {
        const int l = l0 + sub;
        // this lane's epilogue operands, fetched before the row product
        const int ce = sl < 3 ? sl : 0;
        const int le = l < m ? l : 0;
        const float z0 = A.zf[3 * le + ce];
        const df p0 = A.pd[3 * le + ce], ap0 = A.Apd[3 * le + ce], r0 = A.rd[3 * le + ce];
        dfacc a0 = acc_zero(), a1 = acc_zero(), a2 = acc_zero();
        if (l < m) {
          const int nnz = A.Gnnz[l];
          const int* gc = A.Gcol + (long long)l * G_MAXNNZ;
          const df* gv = A.Gv + (long long)l * G_MAXNNZ;
#pragma unroll 2
          for (int j = sl; j < nnz; j += 8) {
            const int k = gc[j];
            const df v = gv[j];
            acc_fma_f(a0, v, zs[3 * k]);
            acc_fma_f(a1, v, zs[3 * k + 1]);
            acc_fma_f(a2, v, zs[3 * k + 2]);
          }
        }
        const df gz0 = df_warp_sum(acc_value(a0), 8), gz1 = df_warp_sum(acc_value(a1), 8);
        const df gz2 = df_warp_sum(acc_value(a2), 8);
        df contrib = dzero;
        if (l < m && sl < 3) {
          const int c = sl;
          const int bd = A.body_of[l];
          const int vi = A.voff[bd] + 3 * (l - A.boff[bd]) + c;
          const df gz = c == 0 ? gz0 : (c == 1 ? gz1 : gz2);
          const df beta = s_beta[c];
          const df pl = df_add(df_from_float(z0), df_mul(beta, p0));
          const df ap = df_add(gz, df_mul(beta, ap0));
          A.pd[3 * l + c] = pl;
          A.Apd[3 * l + c] = ap;
          A.Apf[vi] = ap.hi;
          A.rf[vi] = r0.hi;
          contrib = df_mul(pl, ap);
        }
        // lane c < 3 gathers component c of the warp's four rows, in row order
        for (int r = 0; r < 4; ++r) {
          const int src = 8 * r + (lane & 7);
          const df v = df_make(__shfl_sync(0xffffffffu, contrib.hi, src), __shfl_sync(0xffffffffu, contrib.lo, src));
          if (lane < 3) pAp = df_add(pAp, v);
        }
      }
      trace_mark(A, ts + 2);
      block_partial3(pAp, shdf, A.red + blockIdx.x * 8);
      trace_mark(A, ts + 3);
    }
    grid.sync();
    trace_mark(A, ts + 4);
    // ---- P2: alpha;  z = M (r - alpha A p) in FP32;  w += alpha p;  r -= alpha A p;  partial r.z
    if (wib < 3) {
      // warp c: total p.Ap of component c and the step length
      const int c = wib;
      const df pAp = grid_total_df(A.red, c);
      if (lane == 0) {
        const df a = (pAp.hi > 0.f && s_rz[c].hi > 0.f) ? df_div(s_rz[c], pAp) : dzero;
        s_alpha[c] = a;
        s_alphaf[c] = a.hi;
      }
    }
    __syncthreads();
    trace_mark(A, ts + 5);
    const float alphaf[3] = {s_alphaf[0], s_alphaf[1], s_alphaf[2]};
    if (A.sep_on) {
      // z = M (r - alpha A p) through the separable factors; then, per
      // marker, w += alpha p, r -= alpha A p and the partial r.z
      df rz = dzero;
      SepIn in;
      in.a = A.rf;
      in.b = A.Apf;
      in.s[0] = alphaf[0];
      in.s[1] = alphaf[1];
      in.s[2] = alphaf[2];
      trace_mark(A, ts + 6);
      sep_apply(A, grid, in, sm, false);
      for (int l = gwarp; l < m; l += nwarp_all) {
        const int bd = A.body_of[l];
        float z[3];
        sep_marker_z(A.sep[bd], l - A.boff[bd], z);
        if (lane < 3) {
          const int c = lane;
          const float zl = c == 0 ? z[0] : (c == 1 ? z[1] : z[2]);
          const df alpha = s_alpha[c];
          const df w0 = A.wd[3 * l + c], p0 = A.pd[3 * l + c], r0 = A.rd[3 * l + c], ap0 = A.Apd[3 * l + c];
          A.wd[3 * l + c] = df_add(w0, df_mul(alpha, p0));
          const df rn = df_sub(r0, df_mul(alpha, ap0));
          A.rd[3 * l + c] = rn;
          A.zf[3 * l + c] = zl;
          rz = df_add(rz, df_mul_f(rn, zl));
        }
      }
      trace_mark(A, ts + 7);
      block_partial3(rz, shdf, A.red + blockIdx.x * 8 + 3);
    } else {
      df rz = dzero;
      const float* xs = stage_x(A, A.rf, A.Apf, alphaf, sm);
      trace_mark(A, ts + 6);
      for (int jp = wib, pp = prow0; pp < npairs; jp += PCG_WARPS, pp += rstep) {
        // lane h*3 + c (< 6) updates component c of row 2pp + h; its vector
        // entries are fetched before the product so that their latency overlaps it
        const int h = lane / 3, c = lane - 3 * (lane / 3);
        const int l = 2 * pp + (lane < 6 ? h : 0);
        const bool mine = lane < 6 && l < m;
        const int ls = mine ? l : 2 * pp, cs = mine ? c : 0;
        const df w0 = A.wd[3 * ls + cs], p0 = A.pd[3 * ls + cs], r0 = A.rd[3 * ls + cs], ap0 = A.Apd[3 * ls + cs];
        float z6[2][3];
        precond_pair(A, pp, xs, A.rf, A.Apf, alphaf, z6[0], z6[1], lane,
                     mres ? mres + (long long)(2 * jp) * A.row_slot : nullptr,
                     mres ? mres + (long long)(2 * jp + 1) * A.row_slot : nullptr);
        if (mine) {
          const float zl = h == 0 ? z6[0][c] : z6[1][c];
          const df alpha = s_alpha[c];
          A.wd[3 * l + c] = df_add(w0, df_mul(alpha, p0));
          const df rn = df_sub(r0, df_mul(alpha, ap0));
          A.rd[3 * l + c] = rn;
          A.zf[3 * l + c] = zl;
          rz = df_add(rz, df_mul_f(rn, zl));
        }
      }
      {
        const df r3 = df_make(__shfl_down_sync(0xffffffffu, rz.hi, 3), __shfl_down_sync(0xffffffffu, rz.lo, 3));
        if (lane < 3) rz = df_add(rz, r3);
      }
      trace_mark(A, ts + 7);
      block_partial3(rz, shdf, A.red + blockIdx.x * 8 + 3);
    }
    grid.sync();
    trace_mark(A, ts + 8);
    // warp c: total r.z of component c, beta for the next iteration, convergence test
    if (wib < 3) {
      const int c = wib;
      const df rzn = grid_total_df(A.red, 3 + c);
      if (lane == 0) {
        const df prev = s_rz[c];
        s_beta[c] = prev.hi > 0.f ? df_div(rzn, prev) : dzero;
        s_rz[c] = rzn;
        s_conv[c] = (c >= A.D || !df_greater(rzn, s_stop[c])) ? 1 : 0;
      }
    }
    __syncthreads();
    ++it;
    done = (s_conv[0] & s_conv[1] & s_conv[2]) != 0;
  }
  trace_mark(A, 3);
  // ---- FP64 copy of the solution for the spreading; body forces
  // F_w = -sum_l 2 rho_l w_l (Eq. 26 x ds, Sec. 3.7): block b reduces body b in
  // a fixed order (lane-strided FP64 sums, fixed shuffle tree, warp order)
  for (int i = gtid; i < 3 * m; i += nthreads) A.w[i] = df_to_double(A.wd[i]);
  // every block left the loop after the same barrier: the whole solution is
  // final, so the spreading runs here instead of in a kernel of its own
  {
    const long long tot = (long long)m * (A.geo.D == 3 ? 64 : 16);
    for (long long gi = gtid; gi < tot; gi += nthreads)
      spread_node(gi, m, A.base, A.wts, A.wd, A.tile_slot, A.geo, A.acc, A.status);
  }
  for (int b = blockIdx.x; b < A.nbodies; b += gridDim.x) {
    double v[3] = {0, 0, 0};
    for (int l = A.boff[b] + threadIdx.x; l < A.boff[b + 1]; l += blockDim.x)
      for (int c = 0; c < 3; ++c) {
        const double f = 2.0 * A.rho_l[l] * df_to_double(A.wd[3 * l + c]);   // force on the fluid
        A.mforce[3 * l + c] = f;
        v[c] += f;
      }
    for (int o = 16; o > 0; o >>= 1)
      for (int c = 0; c < 3; ++c) v[c] += __shfl_xor_sync(0xffffffffu, v[c], o);
    block_total3(v, shd);
    if (threadIdx.x == 0) {
      double* h = A.hist + ((long long)b * HIST_LEN + (A.step % HIST_LEN)) * 3;
      for (int c = 0; c < 3; ++c) h[c] = -v[c];   // force on the body
    }
  }
  if (gtid == 0) {
    double rel = 0.0;
    for (int c = 0; c < A.D; ++c)
      if (s_scale[c].hi > 0.f) rel = fmax(rel, sqrt(fmax(df_to_double(s_rz[c]), 0.0) / df_to_double(s_scale[c])));
    A.info[0] = it;
    if (rebuild) {
      A.info[4] = it;
      A.info[5] = 0;
    } else {
      A.info[5] = min(A.info[5] + max(it - max(A.info[4], REBUILD_ITERS_OK), 0), 1 << 30);
    }
    A.info[1] = (A.info[5] > A.rebuild_excess || !done) ? 1 : 0;
    A.info[2] = done ? 1 : 0;
    *A.res = rel;
    if (!done) atomicOr(A.status, ST_NOTCONV);
  }
}

// ------------------------------------------------------------------ forces
// Eulerian IB force density of the last step for every cell (band cells, zero elsewhere).
template <class R>
__global__ void k_force_field(long long N, int nx, int ny, TileGeom tg, const int* __restrict__ tile_slot,
                              const R* __restrict__ band_F, int D, double* __restrict__ out) {
  const long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= N) return;
  const int x = (int)(cell % nx);
  const long long yz = cell / nx;
  const int y = (int)(yz % ny), z = (int)(yz / ny);
  const int tile = ((z / tg.tz) * tg.nty + (y / tg.ty)) * tg.ntx + (x / tg.tx);
  const int s = tile_slot ? tile_slot[tile] : -1;
  const int local = ((z % tg.tz) * tg.ty + (y % tg.ty)) * tg.tx + (x % tg.tx);
  for (int a = 0; a < D; ++a)
    out[a * N + cell] = s >= 0 ? (double)band_F[(long long)s * 3 * TILE_CELLS + a * TILE_CELLS + local] : 0.0;
}

// ------------------------------------------------------------------ host orchestration
static Geo make_geo(ibl_ctx* c) {
  Geo g;
  g.D = c->D;
  g.n[0] = c->nx; g.n[1] = c->ny; g.n[2] = c->nz;
  for (int a = 0; a < 3; ++a) g.per[a] = (a < c->D) ? (c->bc[2 * a] == IBL_PERIODIC) : 1;
  g.tg = c->tg;
  return g;
}

static size_t real_size(ibl_ctx* c) { return c->prec == IBL_FP64 ? sizeof(double) : sizeof(float); }

#define IBL_CU(x)                       \
  do {                                  \
    cudaError_t e_ = (x);               \
    if (e_ != cudaSuccess) return e_;   \
  } while (0)

// The dense preconditioner is re-read by every iteration of every solve;
// while the bulk collide streams the populations through L2 on the other
// SMs it would be evicted each time.  Mark it persisting in L2 for the
// context's stream (the set-aside is a property of this process's context
// and ends with it).  Best effort: without support the solve only runs slower.
static void keep_in_l2(ibl_ctx* c, const void* ptr, size_t bytes) {
  int dev = 0, max_persist = 0, max_window = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, dev);
  cudaDeviceGetAttribute(&max_window, cudaDevAttrMaxAccessPolicyWindowSize, dev);
  if (max_persist <= 0 || max_window <= 0) return;
  // at most 64 MB: a larger set-aside starves the collide's streaming; a
  // matrix larger than that is left to stream from HBM (a partial window
  // saves the solve less than the smaller L2 costs the collide)
  const size_t cap = std::min<size_t>((size_t)max_persist, (size_t)64 << 20);
  if (bytes > cap) return;
  size_t cur = 0;
  cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize);
  const size_t want = bytes;
  if (cur < want && cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  cudaStreamAttrValue attr = {};
  attr.accessPolicyWindow.base_ptr = const_cast<void*>(ptr);
  attr.accessPolicyWindow.num_bytes = std::min<size_t>(bytes, (size_t)max_window);
  attr.accessPolicyWindow.hitRatio =
      (float)std::min(1.0, (double)want / (double)attr.accessPolicyWindow.num_bytes);
  attr.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
  attr.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
  if (cudaStreamSetAttribute(c->stream, cudaStreamAttributeAccessPolicyWindow, &attr) != cudaSuccess)
    cudaGetLastError();
}

cudaError_t ib_alloc(ibl_ctx* c) {
  ib_free(c);
  const int m = c->m_total;
  if (m == 0) return cudaSuccess;
  // band slots: a sheet of unit-spaced markers touches well under one tile per
  // marker; overflow is reported as IBL_EINVAL rather than silently dropped
  c->cap_slots = (int)std::min<long long>((long long)c->tg.n_tiles, (long long)m + 4096);
  const size_t rs = real_size(c);
  IBL_CU(cudaMalloc(&c->d_X0, sizeof(double) * 3 * m));
  IBL_CU(cudaMalloc(&c->d_ds, sizeof(double) * m));
  IBL_CU(cudaMalloc(&c->d_body, sizeof(int) * m));
  IBL_CU(cudaMalloc(&c->d_X, sizeof(double) * 3 * m));
  IBL_CU(cudaMalloc(&c->d_U, sizeof(double) * 3 * m));
  IBL_CU(cudaMalloc(&c->d_Xp, sizeof(double) * 3 * m));
  IBL_CU(cudaMalloc(&c->d_Up, sizeof(double) * 3 * m));
  IBL_CU(cudaMalloc(&c->d_tile_slot, sizeof(int) * c->tg.n_tiles));
  IBL_CU(cudaMemsetAsync(c->d_tile_slot, 0xff, sizeof(int) * c->tg.n_tiles, c->stream));
  IBL_CU(cudaMalloc(&c->d_slot_tile, sizeof(int) * c->cap_slots));
  IBL_CU(cudaMalloc(&c->d_band_count, sizeof(int)));
  IBL_CU(cudaMemsetAsync(c->d_band_count, 0, sizeof(int), c->stream));
  IBL_CU(cudaMalloc(&c->d_tile_mcount, sizeof(int) * c->cap_slots));
  IBL_CU(cudaMemsetAsync(c->d_tile_mcount, 0, sizeof(int) * c->cap_slots, c->stream));
  IBL_CU(cudaMalloc(&c->d_tile_markers, sizeof(int) * (size_t)c->cap_slots * TILE_MARKER_CAP));
  IBL_CU(cudaMalloc(&c->d_band_F, rs * 3 * TILE_CELLS * (size_t)c->cap_slots));
  IBL_CU(cudaMalloc(&c->d_acc, sizeof(unsigned long long) * 3 * TILE_CELLS * (size_t)c->cap_slots));
  IBL_CU(cudaMemsetAsync(c->d_acc, 0, sizeof(unsigned long long) * 3 * TILE_CELLS * (size_t)c->cap_slots, c->stream));
  IBL_CU(cudaMalloc(&c->d_slot_body, sizeof(int) * c->cap_slots));
  IBL_CU(cudaMemsetAsync(c->d_slot_body, 0xff, sizeof(int) * c->cap_slots, c->stream));
  IBL_CU(cudaMalloc(&c->d_mixed, 2 * sizeof(int)));   // [0] use tiles this step, [1] lists overflowed
  IBL_CU(cudaMalloc(&c->d_cand, sizeof(int) * (size_t)m * CAND_MAX));
  IBL_CU(cudaMalloc(&c->d_ncand, sizeof(int) * m));
  IBL_CU(cudaMalloc(&c->d_base, sizeof(int) * 3 * m));
  IBL_CU(cudaMalloc(&c->d_wts, sizeof(double) * 12 * m));
  IBL_CU(cudaMalloc(&c->d_rho_l, sizeof(double) * m));
  IBL_CU(cudaMalloc(&c->d_B, sizeof(double) * 3 * m));
  IBL_CU(cudaMalloc(&c->d_w, sizeof(double) * 3 * m));
  IBL_CU(cudaMalloc(&c->d_wprev, sizeof(double) * 3 * m));
  IBL_CU(cudaMalloc(&c->d_wprev2, sizeof(double) * 3 * m));
  IBL_CU(cudaMemsetAsync(c->d_w, 0, sizeof(double) * 3 * m, c->stream));
  IBL_CU(cudaMalloc(&c->d_r, sizeof(double) * 3 * m));
  IBL_CU(cudaMalloc(&c->d_p, sizeof(double) * 6 * m));
  IBL_CU(cudaMalloc(&c->d_Ap, sizeof(double) * 3 * m));
  IBL_CU(cudaMalloc(&c->d_z, sizeof(double) * 3 * m));
  // three padded FP32 vectors (r, A p, B); each body's slice starts at a
  // multiple of 12 floats and carries a zero tail up to a multiple of 4 markers
  size_t vf = 0;
  for (auto& b : c->bodies) vf += 3 * (size_t)((b.m + 3) & ~3) + 12;
  c->xf_floats = vf;
  IBL_CU(cudaMalloc(&c->d_xf, sizeof(float) * 3 * vf));
  IBL_CU(cudaMemsetAsync(c->d_xf, 0, sizeof(float) * 3 * vf, c->stream));
  IBL_CU(cudaMalloc(&c->d_trace, sizeof(unsigned long long) * 256));
  IBL_CU(cudaMemsetAsync(c->d_trace, 0, sizeof(unsigned long long) * 256, c->stream));
  IBL_CU(cudaMalloc(&c->d_Gcol, sizeof(int) * (size_t)m * G_MAXNNZ));
  IBL_CU(cudaMalloc(&c->d_Gval, sizeof(double) * (size_t)m * G_MAXNNZ));
  IBL_CU(cudaMalloc(&c->d_Gnnz, sizeof(int) * m));
  IBL_CU(cudaMalloc(&c->d_Gdiag_max, sizeof(double) * MAX_BODIES));
  // preconditioner: the separable factors when every body allows them and
  // they are asked for (or, automatically, for large bodies); else the dense
  // per-body inverses
  int max_m = 0;
  const bool separable = sep_all_separable(c, &max_m);
  if (c->precond_kind == 1 && !separable) return cudaErrorInvalidValue;
  const bool use_sep = c->precond_kind == 1 || (c->precond_kind < 0 && separable && max_m >= SEP_AUTO_MIN_MARKERS);
  size_t mf = 0;
  for (auto& b : c->bodies) {
    b.precond_offset = (int)mf;
    if (!use_sep) mf += (size_t)b.m * (size_t)((b.m + 3) & ~3);
  }
  c->M_floats = mf;
  if (use_sep) {
    IBL_CU(sep_alloc(c));
  } else {
    IBL_CU(cudaMalloc(&c->d_M, sizeof(float) * mf));
    keep_in_l2(c, c->d_M, sizeof(float) * mf);
  }
  IBL_CU(cudaMalloc(&c->d_red, sizeof(double) * 8 * 1024));
  IBL_CU(cudaMalloc(&c->d_cg_info, sizeof(int) * 8));
  IBL_CU(cudaMemsetAsync(c->d_cg_info, 0, sizeof(int) * 8, c->stream));
  IBL_CU(cudaMalloc(&c->d_cg_res, sizeof(double)));
  IBL_CU(cudaMemsetAsync(c->d_cg_res, 0, sizeof(double), c->stream));
  IBL_CU(cudaMalloc(&c->d_hist, sizeof(double) * 3 * (size_t)HIST_LEN * c->bodies.size()));
  IBL_CU(cudaMemsetAsync(c->d_hist, 0, sizeof(double) * 3 * (size_t)HIST_LEN * c->bodies.size(), c->stream));
  IBL_CU(cudaMalloc(&c->d_mforce, sizeof(double) * 3 * m));
  IBL_CU(cudaMemsetAsync(c->d_mforce, 0, sizeof(double) * 3 * m, c->stream));
  // body index per marker, body-frame coordinates and element sizes
  std::vector<int> body_of(m);
  for (size_t b = 0; b < c->bodies.size(); ++b)
    for (int l = 0; l < c->bodies[b].m; ++l) body_of[c->bodies[b].offset + l] = (int)b;
  IBL_CU(to_device(c, c->d_body, body_of.data(), sizeof(int) * m));
  std::vector<int> boff(c->bodies.size() + 1);
  for (size_t b = 0; b < c->bodies.size(); ++b) boff[b] = c->bodies[b].offset;
  boff[c->bodies.size()] = m;
  IBL_CU(cudaMalloc(&c->d_boff, sizeof(int) * boff.size()));
  IBL_CU(to_device(c, c->d_boff, boff.data(), sizeof(int) * boff.size()));
  c->cand_ready = false;
  c->precond_valid = false;
  c->warm = false;
  c->warm_steps = 0;
  c->ib_ready = true;
  return cudaSuccess;
}

void ib_free(ibl_ctx* c) {
  void* ptrs[] = {c->d_X0, c->d_ds, c->d_body, c->d_X, c->d_U, c->d_Xp, c->d_Up, c->d_tile_slot,
                  c->d_slot_tile, c->d_band_count, c->d_tile_mcount, c->d_tile_markers,
                  c->d_band_F, c->d_base, c->d_wts, c->d_rho_l, c->d_B, c->d_w, c->d_r, c->d_p,
                  c->d_Ap, c->d_z, c->d_Gcol, c->d_Gval, c->d_Gnnz, c->d_Gdiag_max, c->d_M, c->d_red,
                  c->d_cg_info, c->d_cg_res, c->d_hist, c->d_mforce, c->d_boff, c->d_xf, c->d_trace,
                  c->d_acc, c->d_slot_body, c->d_mixed, c->d_cand, c->d_ncand,
                  c->d_wprev, c->d_wprev2};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  c->d_X0 = c->d_ds = c->d_X = c->d_U = c->d_Xp = c->d_Up = nullptr;
  c->d_body = c->d_tile_slot = c->d_slot_tile = c->d_band_count = c->d_tile_mcount = nullptr;
  c->d_tile_markers = c->d_base = c->d_Gcol = c->d_Gnnz = c->d_cg_info = c->d_boff = nullptr;
  c->d_band_F = nullptr;
  c->d_wts = nullptr;
  c->d_rho_l = c->d_B = c->d_w = c->d_r = c->d_p = c->d_Ap = c->d_z = c->d_Gval = nullptr;
  c->d_Gdiag_max = c->d_red = c->d_cg_res = c->d_hist = c->d_mforce = nullptr;
  c->d_M = nullptr;
  c->d_xf = nullptr;
  c->d_trace = nullptr;
  c->d_acc = nullptr;
  c->d_slot_body = c->d_mixed = c->d_cand = c->d_ncand = nullptr;
  c->d_wprev = c->d_wprev2 = nullptr;
  sep_free(c);
  c->ib_ready = false;
}

template <int Q, class T>
static cudaError_t interpolate_q(ibl_ctx* c, const Geo& g) {
  using R = typename Store<T>::R;
  FluidParams<R> p;
  p.nx = c->nx; p.ny = c->ny; p.nz = c->nz; p.N = c->N;
  for (int i = 0; i < 6; ++i) p.bc[i] = c->bc[i];
  for (int a = 0; a < 3; ++a) { p.u_in[a] = (R)c->u_in[a]; p.G[a] = (R)c->G[a]; }
  p.rho_out = (R)c->rho_out;
  p.omega = (R)(1.0 / c->tau);
  p.pref = (R)(1.0 - 0.5 / c->tau);
  p.tg = c->tg;
  p.tile_slot = nullptr;
  p.band_acc = nullptr;
  p.band_F = nullptr;
  p.status = c->d_status;
  const T* src = (const T*)c->f[c->cur];
  const int m = c->m_total;
  const int wb = (m * 32 + 255) / 256;   // interpolation blocks (8 markers each)
  const int ab = (m + 7) / 8;            // assembly blocks (8 rows each)
  AssembleArgs aa;
  aa.tile_slot = c->d_tile_slot;
  aa.tile_mcount = c->d_tile_mcount;
  aa.tile_markers = c->d_tile_markers;
  aa.body_of = c->d_body;
  aa.Gcol = c->d_Gcol;
  aa.Gval = reinterpret_cast<df*>(c->d_Gval);
  aa.Gnnz = c->d_Gnnz;
  aa.rowsum_max = (unsigned long long*)c->d_Gdiag_max;
  aa.status = c->d_status;
  aa.cand = c->d_cand;
  aa.ncand = c->d_ncand;
  aa.use_tiles = c->d_mixed;
  aa.cand_bad = c->d_mixed + 1;
  const df* w = reinterpret_cast<const df*>(c->d_wts);
  if (c->poststream)
    k_interp_assemble<Q, T, false><<<wb + ab, 256, 0, c->stream>>>(wb, m, c->d_base, w, src, p, g, c->d_U, c->d_rho_l,
                                                                     c->d_B, aa);
  else
    k_interp_assemble<Q, T, true><<<wb + ab, 256, 0, c->stream>>>(wb, m, c->d_base, w, src, p, g, c->d_U, c->d_rho_l,
                                                                    c->d_B, aa);
  c->launches++;
  return cudaGetLastError();
}

static cudaError_t interpolate(ibl_ctx* c, const Geo& g) {
  if (c->Q == 9) {
    switch (c->prec) {
      case IBL_FP64: return interpolate_q<9, double>(c, g);
      case IBL_FP32: return interpolate_q<9, float>(c, g);
      case IBL_FP16DEV: return interpolate_q<9, __half>(c, g);
      default: return interpolate_q<9, __nv_bfloat16>(c, g);
    }
  }
  switch (c->prec) {
    case IBL_FP64: return interpolate_q<19, double>(c, g);
    case IBL_FP32: return interpolate_q<19, float>(c, g);
    case IBL_FP16DEV: return interpolate_q<19, __half>(c, g);
    default: return interpolate_q<19, __nv_bfloat16>(c, g);
  }
}

static int g_num_sms = 0;

int num_sms() {
  if (!g_num_sms) {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    g_num_sms = n > 0 ? n : 1;
  }
  return g_num_sms;
}

void phase_mark(ibl_ctx* c, int phase) {
  if (c->prof_level < 2) return;
  if (c->pev_used == c->pev_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    c->pev_pool.push_back(e);
  }
  cudaEvent_t e = c->pev_pool[c->pev_used++];
  cudaEventRecord(e, c->stream);
  c->pev_log.emplace_back(phase, e);
}

// Blocks of the cooperative solve: by default half the SMs (the other half
// runs the bulk collide concurrently when the step is split), all of them for
// marker sets too large to split for (the solve then dominates the step);
// fixed per context so that the solve's reduction order does not depend on
// the schedule.
int pcg_block_count(const ibl_ctx* c) {
  const bool half = c->overlap == 1 || c->m_total <= SPLIT_MAX_MARKERS;
  const int want = c->pcg_blocks > 0 ? c->pcg_blocks : (half ? num_sms() / 2 : num_sms());
  return std::max(1, std::min(std::min(std::min(want, num_sms()), MAX_PCG_BLOCKS), c->m_total));
}

// Wave value and rate at time t (Eqs. 20-23 and the reading of Eq. 23 as
// |sin|; TABLE: samples per step, central difference for the rate), in
// FP64 on the host: a handful of values per body and step, kept off the
// GPU's slow FP64 pipe.
static void wave_eval(const Wave& w, const std::vector<double>& table, double t, double f, double phi,
                      double& v, double& vd) {
  const double om = 2.0 * 3.14159265358979323846 * f;
  const double th = om * t + phi;
  switch (w.kind) {
    case IBL_WAVE_COS: v = w.offset + w.amp * std::cos(th); vd = -w.amp * om * std::sin(th); break;
    case IBL_WAVE_SIN: v = w.offset + w.amp * std::sin(th); vd = w.amp * om * std::cos(th); break;
    case IBL_WAVE_ABS_SIN: {
      const double sn = std::sin(th);
      const double sg = sn >= 0.0 ? 1.0 : -1.0;
      v = w.offset + w.amp * std::fabs(sn);
      vd = w.amp * om * std::cos(th) * sg;
      break;
    }
    case IBL_WAVE_TABLE: {
      const long long n = (long long)table.size();
      const long long k = std::llround(t);
      const long long i0 = ((k % n) + n) % n, ip = (((k + 1) % n) + n) % n, im = (((k - 1) % n) + n) % n;
      v = table[i0];
      vd = 0.5 * (table[ip] - table[im]);
      break;
    }
    default: v = w.offset; vd = 0.0; break;
  }
}

// Motion state of body b at time t shared by all of its markers: A, A',
// alpha', cos alpha, sin alpha, the stroke direction e_s (cos beta, sin beta), alpha.
static void body_state(const Body& B, double t, double st[8]) {
  double A, Ad, al, ald;
  wave_eval(B.A, B.hostA, t, B.f, B.phi, A, Ad);
  wave_eval(B.alpha, B.hostAlpha, t, B.f, B.phi, al, ald);
  st[0] = A;
  st[1] = Ad;
  st[2] = ald;
  st[3] = std::cos(al);
  st[4] = std::sin(al);
  st[5] = std::cos(B.beta);
  st[6] = std::sin(B.beta);
  st[7] = al;
}

// Kinematics and the band tiles of the step (the bulk collide may start
// once these are enqueued).
cudaError_t ib_step_front(ibl_ctx* c) {
  const int m = c->m_total;
  if (m == 0) return cudaSuccess;
  num_sms();
  Geo g = make_geo(c);
  if (!c->cand_ready) {
    IBL_CU(cudaMemsetAsync(c->d_mixed + 1, 0, sizeof(int), c->stream));
    k_build_candidates<<<(m * 32 + 255) / 256, 256, 0, c->stream>>>(m, c->d_X0, c->d_body, c->d_boff, c->D,
                                                                    c->d_cand, c->d_ncand, c->d_mixed + 1);
    c->launches++;
    c->cand_ready = true;
  }
  BodyTable bt;
  bt.n = (int)c->bodies.size();
  for (int b = 0; b < bt.n; ++b) {
    const Body& h = c->bodies[b];
    BodyDev& d = bt.b[b];
    d.offset = h.offset; d.m = h.m;
    for (int a = 0; a < 3; ++a) { d.hinge[a] = h.hinge[a]; d.axis[a] = h.axis[a]; d.origin[a] = h.origin[a]; }
    body_state(h, (double)c->step, d.st);
    d.prescribed = h.prescribed ? 1 : 0;
  }
  const int tb = 64;
  const int mb = (m + tb - 1) / tb;
  k_kinematics<<<(3 * m + 127) / 128, 128, 0, c->stream>>>(bt, m, c->d_body, c->d_X0, c->d_Xp, c->d_Up, c->d_X, c->d_U,
                                         c->d_base, reinterpret_cast<df*>(c->d_wts), (double)c->step, g,
                                         c->d_status);
  phase_mark(c, 0);
  // candidate-list assembly unless a body is driven by uploaded states this step
  bool any_prescribed = false;
  for (auto& b : c->bodies) any_prescribed |= b.prescribed;
  const int use_tiles_host = any_prescribed ? 1 : 0;
  IBL_CU(cudaMemsetAsync(c->d_mixed, use_tiles_host, sizeof(int), c->stream));
  IBL_CU(cudaMemsetAsync(c->d_band_count, 0, sizeof(int), c->stream));
  phase_mark(c, 1);
  k_mark_tiles<<<mb, tb, 0, c->stream>>>(m, c->d_base, g, c->d_tile_slot);
  phase_mark(c, 2);
  k_assign_slots<<<std::max(1, std::min((c->tg.n_tiles + 255) / 256, 2 * g_num_sms)), 256, 0, c->stream>>>(
      c->tg.n_tiles, c->d_tile_slot, c->d_slot_tile, c->d_band_count, c->cap_slots, c->d_tile_mcount,
      c->d_slot_body, c->d_status);
  phase_mark(c, 3);
  c->launches += 3;
  return cudaGetLastError();
}

// Marker lists, interpolation, assembly, the implicit solve and spreading.
cudaError_t ib_step_back(ibl_ctx* c) {
  const int m = c->m_total;
  if (m == 0) return cudaSuccess;
  Geo g = make_geo(c);
  const int tb = 64;
  const int mb = (m + tb - 1) / tb;
  k_append_markers<<<(8 * m + 255) / 256, 256, 0, c->stream>>>(m, c->d_base, g, c->d_tile_slot, c->d_tile_mcount,
                                             c->d_tile_markers, c->d_status, c->d_body, c->d_slot_body,
                                             c->d_mixed);
  phase_mark(c, 4);
  for (auto& b : c->bodies) b.prescribed = false;
  c->launches += 1;
  IBL_CU(cudaGetLastError());
  IBL_CU(cudaMemsetAsync(c->d_Gdiag_max, 0, sizeof(double) * MAX_BODIES, c->stream));
  IBL_CU(interpolate(c, g));   // interpolation and assembly, one launch
  phase_mark(c, 5);
  phase_mark(c, 6);
  // PCG (cooperative)
  PcgArgs A;
  A.m_total = m;
  A.D = c->D;
  A.nbodies = (int)c->bodies.size();
  for (int b = 0; b < A.nbodies; ++b) {
    A.boff[b] = c->bodies[b].offset;
    A.poff[b] = c->bodies[b].precond_offset;
  }
  A.boff[A.nbodies] = m;
  A.body_of = c->d_body;
  A.Gcol = c->d_Gcol; A.Gv = reinterpret_cast<const df*>(c->d_Gval); A.Gnnz = c->d_Gnnz;
  A.rowsum_max = (const unsigned long long*)c->d_Gdiag_max;
  A.B = c->d_B; A.w = c->d_w;
  // the double-float vectors reuse the FP64 work arrays (8 bytes per entry);
  // the search direction array holds two m x 3 vectors: p and the solution
  A.rd = reinterpret_cast<df*>(c->d_r);
  A.pd = reinterpret_cast<df*>(c->d_p);
  A.wd = reinterpret_cast<df*>(c->d_p) + 3 * (size_t)m;
  A.Apd = reinterpret_cast<df*>(c->d_Ap);
  A.zf = reinterpret_cast<float*>(c->d_z);
  A.wprevd = reinterpret_cast<df*>(c->d_wprev);
  A.wprev2d = reinterpret_cast<df*>(c->d_wprev2);
  A.rf = c->d_xf;
  A.Apf = c->d_xf + c->xf_floats;
  A.Bf = c->d_xf + 2 * c->xf_floats;
  {
    int vo = 0;
    for (int b = 0; b < A.nbodies; ++b) {
      A.voff[b] = vo;
      vo += 3 * ((c->bodies[b].m + 3) & ~3) + 12;
    }
    A.vtotal = vo;
  }
  // shared memory: a staging area (z for the SpMV, or the preconditioner
  // input, both FP32) and, when they fit, this block's preconditioner rows
  const int pcg_blocks = pcg_block_count(c);
  {
    // vectors larger than the shared memory are read from L2 instead of being staged
    size_t stage = std::max<size_t>((size_t)3 * m * sizeof(float), (size_t)A.vtotal * sizeof(float));
    stage = std::max(std::min((stage + 15) & ~(size_t)15, PCG_SMEM_MAX), GJ_SMEM);
    int slot = 0;
    for (int b = 0; b < A.nbodies; ++b) slot = std::max(slot, precond_ld(c->bodies[b].m));
    const size_t rows = 2 * (((size_t)(m + 1) / 2 + pcg_blocks - 1) / pcg_blocks);   // whole row pairs
    const size_t need = stage + rows * (size_t)slot * sizeof(float);
    if (c->sep_on) stage = std::max(stage, sep_smem_bytes(c));
    A.smem_floats = (int)(stage / sizeof(float));
    A.row_slot = (need <= PCG_SMEM_MAX && c->resident_rows != 0 && !c->sep_on) ? slot : 0;
    c->pcg_smem = A.row_slot ? need : stage;
  }
  A.tol = c->solver_tol > 0 ? c->solver_tol
                             : (c->prec == IBL_FP64 ? PCG_TOL : (c->prec == IBL_FP32 ? PCG_TOL_FP32 : PCG_TOL_HALF));
  A.M = c->d_M; A.red = reinterpret_cast<df*>(c->d_red); A.info = c->d_cg_info; A.res = c->d_cg_res;
  {
    double cube = 0, square = 0;
    for (int b = 0; b < A.nbodies; ++b) {
      const double mb = c->bodies[b].m;
      cube += 2 * mb * mb * mb;
      square += 6 * mb * mb;
    }
    A.rebuild_excess = (int)std::min(std::max(cube / std::max(square, 1.0), (double)REBUILD_MIN_EXCESS), 1e8);
  }
  A.warm = c->extrapolate < 0 ? 0
         : (c->extrapolate >= 2 && c->warm_steps >= 3 ? 3
            : (c->extrapolate >= 1 && c->warm_steps >= 2 ? 2 : (c->warm_steps >= 1 ? 1 : 0)));
  const bool sched = !c->precond_valid || (c->step - c->last_refresh_step) >= c->refresh_every;
  A.refresh = sched ? 1 : 0;
  if (sched) {
    c->last_refresh_step = c->step;
    c->refreshes++;
  }
  c->precond_valid = true;
  A.status = c->d_status;
  A.trace = c->d_trace;
  A.base = c->d_base;
  A.wts = reinterpret_cast<const df*>(c->d_wts);
  A.tile_slot = c->d_tile_slot;
  A.acc = c->d_acc;
  A.geo = g;
  A.rho_l = c->d_rho_l;
  A.mforce = c->d_mforce;
  A.hist = c->d_hist;
  A.step = c->step;
  A.sep = c->d_sep;
  A.sep_on = c->sep_on ? 1 : 0;
  if (c->sep_on && A.refresh) IBL_CU(sep_launch(c, g.n, g.per));
  static bool smem_set = false;
  if (!smem_set) {
    IBL_CU(cudaFuncSetAttribute((const void*)k_pcg, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PCG_SMEM_MAX));
    smem_set = true;
  }
  void* args[] = {&A};
  IBL_CU(cudaLaunchCooperativeKernel((void*)k_pcg, dim3(pcg_blocks), dim3(PCG_THREADS), args, c->pcg_smem,
                                     c->stream));
  phase_mark(c, 7);
  c->launches++;
  c->warm = true;
  c->warm_steps++;
  phase_mark(c, 8);   // the spreading runs at the end of the solve
  IBL_CU(cudaGetLastError());
  return cudaSuccess;
}

cudaError_t ib_step(ibl_ctx* c) {
  IBL_CU(ib_step_front(c));
  return ib_step_back(c);
}

cudaError_t launch_force_field(ibl_ctx* c, double* d_out) {
  const int bs = 256;
  const long long nb = (c->N + bs - 1) / bs;
  if (c->prec == IBL_FP64)
    k_force_field<double><<<(unsigned)nb, bs, 0, c->stream>>>(c->N, c->nx, c->ny, c->tg, c->m_total ? c->d_tile_slot : nullptr,
                                                              (const double*)c->d_band_F, c->D, d_out);
  else
    k_force_field<float><<<(unsigned)nb, bs, 0, c->stream>>>(c->N, c->nx, c->ny, c->tg, c->m_total ? c->d_tile_slot : nullptr,
                                                             (const float*)c->d_band_F, c->D, d_out);
  c->launches++;
  return cudaGetLastError();
}

}  // namespace ibl
