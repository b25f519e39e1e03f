// Immersed-boundary kernels: the implicit velocity-correction exchange of
// Sec. 2.2 (Wu and Shu's formulation) between the fluid and the markers.
//
// Per step, in the paper's order:
//   k_kinematics     marker positions X and wall velocities U_B (Eqs. 20-23,
//                    rotational velocity of Sec. 3.3), stencil base nodes and
//                    the 4-point cosine weights (Eq. 14) in FP64;
//   k_mark/assign/append
//                    grid tiles touched by a stencil get a band slot and a
//                    list of the markers that touch them;
//   k_band_moments   rho and u* = (sum c_i f_i + G/2)/rho on band tiles (Eq. 11);
//   k_interpolate    rho_l and u*_l (Eq. 17); B = U_B - u*_l (Eq. 19);
//   k_assemble       sparse G_lk = sum_x D(x-X_l) D(x-X_k) (Eq. 18 without
//                    ds_k: the solve is run on w = ds * du_B, G w = B);
//   k_pcg            preconditioned conjugate gradients for the three velocity
//                    components at once, FP64 vectors and SpMV, an FP32 dense
//                    per-body approximate inverse as preconditioner, rebuilt
//                    in-kernel (blocked Gauss-Jordan) every few steps;
//   k_spread         du(x) = sum_l w_l D(x - X_l) (Eq. 15) as a per-tile gather
//                    over the tile's markers in marker-index order (no float
//                    atomics), F = 2 rho du (Eq. 26) into the band force;
//   k_force_reduce   F_w = -sum_l 2 rho_l w_l per body in FP64, fixed order.
#include <cooperative_groups.h>

#include "ibl_internal.cuh"

namespace cg = cooperative_groups;

namespace ibl {

constexpr int MAX_BODIES = 16;
constexpr int GJ_NB = 32;          // Gauss-Jordan pivot block
constexpr int PCG_MAX_ITERS = 200;
constexpr double PCG_TOL = 1e-10;  // relative preconditioned residual (field A-norm)
constexpr int REFRESH_EVERY = 64;  // steps between preconditioner rebuilds
constexpr int REFRESH_ITERS = 40;  // rebuild early if a solve needed more

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
  v %= n;
  return v < 0 ? v + n : v;
}

__device__ __forceinline__ double phi_cos(double r) {
  // Eq. 14: (1 + cos(pi |r| / 2)) / 4 for |r| <= 2
  const double a = fabs(r);
  return a <= 2.0 ? 0.25 * (1.0 + cospi(0.5 * a)) : 0.0;
}

__device__ void wave_eval(const Wave& w, double t, double f, double phi, double& v, double& vd) {
  const double om = 2.0 * 3.14159265358979323846 * f;
  const double th = om * t + phi;
  switch (w.kind) {
    case IBL_WAVE_COS: v = w.offset + w.amp * cos(th); vd = -w.amp * om * sin(th); break;
    case IBL_WAVE_SIN: v = w.offset + w.amp * sin(th); vd = w.amp * om * cos(th); break;
    case IBL_WAVE_ABS_SIN: {
      const double s = sin(th);
      const double sg = s >= 0.0 ? 1.0 : -1.0;
      v = w.offset + w.amp * fabs(s);
      vd = w.amp * om * cos(th) * sg;
      break;
    }
    case IBL_WAVE_TABLE: {
      const long long n = w.n_table;
      long long k = llround(t);
      const long long i0 = ((k % n) + n) % n, ip = (((k + 1) % n) + n) % n, im = (((k - 1) % n) + n) % n;
      v = w.table[i0];
      vd = 0.5 * (w.table[ip] - w.table[im]);
      break;
    }
    default: v = w.offset; vd = 0.0; break;
  }
}

// ------------------------------------------------------------------ kinematics + stencil
__global__ void k_kinematics(BodyTable bt, int m_total, const int* __restrict__ body_of,
                             const double* __restrict__ X0, const double* __restrict__ Xp,
                             const double* __restrict__ Up, double* __restrict__ X,
                             double* __restrict__ U, int* __restrict__ base,
                             double* __restrict__ wts, double t, Geo geo, int* status) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= m_total) return;
  const BodyDev& B = bt.b[body_of[l]];
  double x[3], u[3];
  if (B.prescribed) {
    for (int a = 0; a < 3; ++a) { x[a] = Xp[3 * l + a]; u[a] = Up[3 * l + a]; }
  } else {
    double A, Ad, al, ald;
    wave_eval(B.A, t, B.f, B.phi, A, Ad);
    wave_eval(B.alpha, t, B.f, B.phi, al, ald);
    const double es[3] = {cos(B.beta), sin(B.beta), 0.0};
    const double* e = B.axis;
    double d[3];
    for (int a = 0; a < 3; ++a) d[a] = X0[3 * l + a] - B.hinge[a];
    // Rodrigues: r = d cos + (e x d) sin + e (e.d)(1 - cos)
    const double c = cos(al), s = sin(al);
    const double ed = e[0] * d[0] + e[1] * d[1] + e[2] * d[2];
    const double exd[3] = {e[1] * d[2] - e[2] * d[1], e[2] * d[0] - e[0] * d[2],
                           e[0] * d[1] - e[1] * d[0]};
    double r[3];
    for (int a = 0; a < 3; ++a) r[a] = d[a] * c + exd[a] * s + e[a] * ed * (1.0 - c);
    const double exr[3] = {e[1] * r[2] - e[2] * r[1], e[2] * r[0] - e[0] * r[2],
                           e[0] * r[1] - e[1] * r[0]};
    for (int a = 0; a < 3; ++a) {
      x[a] = B.origin[a] + B.hinge[a] + r[a] + A * es[a];
      u[a] = Ad * es[a] + ald * exr[a];
    }
  }
  if (geo.D == 2) { x[2] = 0.0; u[2] = 0.0; }
  for (int a = 0; a < 3; ++a) { X[3 * l + a] = x[a]; U[3 * l + a] = u[a]; }
  for (int a = 0; a < 3; ++a) {
    if (a >= geo.D) {
      base[3 * l + a] = 0;
      wts[12 * l + 4 * a + 0] = 1.0;
      wts[12 * l + 4 * a + 1] = 0.0;
      wts[12 * l + 4 * a + 2] = 0.0;
      wts[12 * l + 4 * a + 3] = 0.0;
      continue;
    }
    const int b0 = (int)floor(x[a]) - 1;
    if (!geo.per[a] && (b0 < 0 || b0 + 3 >= geo.n[a])) atomicOr(status, ST_OVERFLOW);
    base[3 * l + a] = b0;
    for (int k = 0; k < 4; ++k) wts[12 * l + 4 * a + k] = phi_cos((double)(b0 + k) - x[a]);
  }
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

__global__ void k_clear_tiles(int* __restrict__ tile_slot, const int* __restrict__ slot_tile,
                              const int* __restrict__ band_count, int* __restrict__ tile_mcount,
                              int cap) {
  const int n = min(*band_count, cap);
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    tile_slot[slot_tile[s]] = -1;
    tile_mcount[s] = 0;
  }
}

__global__ void k_mark_tiles(int m_total, const int* __restrict__ base, Geo g,
                             int* __restrict__ tile_slot) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= m_total) return;
  int t[8];
  const int n = touched_tiles(g, base + 3 * l, t);
  for (int i = 0; i < n; ++i) tile_slot[t[i]] = -2;
}

__global__ void k_assign_slots(int n_tiles, int* __restrict__ tile_slot, int* __restrict__ slot_tile,
                               int* __restrict__ band_count, int cap, int* status) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n_tiles; t += gridDim.x * blockDim.x) {
    if (tile_slot[t] == -2) {
      const int s = atomicAdd(band_count, 1);
      if (s < cap) {
        tile_slot[t] = s;
        slot_tile[s] = t;
      } else {
        tile_slot[t] = -1;
        atomicOr(status, ST_OVERFLOW);
      }
    }
  }
}

__global__ void k_append_markers(int m_total, const int* __restrict__ base, Geo g,
                                 const int* __restrict__ tile_slot, int* __restrict__ tile_mcount,
                                 int* __restrict__ tile_markers, int* status) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= m_total) return;
  int t[8];
  const int n = touched_tiles(g, base + 3 * l, t);
  for (int i = 0; i < n; ++i) {
    const int s = tile_slot[t[i]];
    if (s < 0) continue;
    const int pos = atomicAdd(&tile_mcount[s], 1);
    if (pos < TILE_MARKER_CAP) tile_markers[s * TILE_MARKER_CAP + pos] = l;
    else atomicOr(status, ST_OVERFLOW);
  }
}

}  // namespace ibl

// The gather/Zou-He code of the fluid kernels is reused for the band moments
// so that rho and u* on the band are bitwise the values the collision
// recomputes.
#include "lbm_gather.cuh"

namespace ibl {

template <int Q, class T, bool PULL>
__global__ void k_band_moments(const T* __restrict__ src, FluidParams<typename Store<T>::R> p,
                               const int* __restrict__ slot_tile, const int* __restrict__ band_count,
                               int cap, typename Store<T>::R* __restrict__ band_mom) {
  using R = typename Store<T>::R;
  const int n = min(*band_count, cap);
  const TileGeom& tg = p.tg;
  for (int s = blockIdx.x; s < n; s += gridDim.x) {
    const int tile = slot_tile[s];
    const int tx0 = (tile % tg.ntx) * tg.tx;
    const int ty0 = ((tile / tg.ntx) % tg.nty) * tg.ty;
    const int tz0 = (tile / (tg.ntx * tg.nty)) * tg.tz;
    const int local = threadIdx.x;
    const int lx = local % tg.tx, ly = (local / tg.tx) % tg.ty, lz = local / (tg.tx * tg.ty);
    const int x = tx0 + lx, y = ty0 + ly, z = tz0 + lz;
    R rho = R(1), u0 = R(0), u1 = R(0), u2 = R(0);
    if (x < p.nx && y < p.ny && z < p.nz) {
      const long long cell = ((long long)z * p.ny + y) * p.nx + x;
      R g[Q];
      gather_q<Q, T, PULL, R>(src, x, y, z, cell, p, g);
      R drho = R(0), m0 = R(0), m1 = R(0), m2 = R(0);
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        drho += g[i];
        if (Lat<Q>::cx(i)) m0 += R(Lat<Q>::cx(i)) * g[i];
        if (Lat<Q>::cy(i)) m1 += R(Lat<Q>::cy(i)) * g[i];
        if (Lat<Q>::cz(i)) m2 += R(Lat<Q>::cz(i)) * g[i];
      }
      rho = R(1) + drho;
      const R inv = R(1) / rho;
      u0 = (m0 + R(0.5) * p.G[0]) * inv;    // Eq. 11 with the uniform body force
      u1 = (m1 + R(0.5) * p.G[1]) * inv;
      u2 = (m2 + R(0.5) * p.G[2]) * inv;
    }
    R* o = band_mom + (long long)s * 4 * TILE_CELLS + local;
    o[0] = rho;
    o[TILE_CELLS] = u0;
    o[2 * TILE_CELLS] = u1;
    o[3 * TILE_CELLS] = u2;
  }
}

// ------------------------------------------------------------------ interpolation
template <class R>
__global__ void k_interpolate(int m_total, const int* __restrict__ base, const double* __restrict__ wts,
                              const R* __restrict__ band_mom, const int* __restrict__ tile_slot, Geo g,
                              const double* __restrict__ U, double* __restrict__ rho_l,
                              double* __restrict__ B) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= m_total) return;
  const int l = warp;
  const int* b = base + 3 * l;
  const double* w = wts + 12 * l;
  const int nnodes = g.D == 3 ? 64 : 16;
  double acc[4] = {0, 0, 0, 0};
  for (int k = lane; k < nnodes; k += 32) {
    const int i = k & 3, j = (k >> 2) & 3, q = k >> 4;
    int node[3] = {b[0] + i, b[1] + j, g.D == 3 ? b[2] + q : 0};
    for (int a = 0; a < g.D; ++a)
      if (g.per[a]) node[a] = wrap(node[a], g.n[a]);
    const double wt = w[i] * w[4 + j] * w[8 + (g.D == 3 ? q : 0)];
    const int tile = tile_of(g, node[0], node[1], node[2]);
    const int s = tile_slot[tile];
    if (s < 0) continue;   // cannot happen: every stencil tile has a slot
    const int local = ((node[2] % g.tg.tz) * g.tg.ty + (node[1] % g.tg.ty)) * g.tg.tx + (node[0] % g.tg.tx);
    const R* mo = band_mom + (long long)s * 4 * TILE_CELLS + local;
    acc[0] += wt * (double)mo[0];
    acc[1] += wt * (double)mo[TILE_CELLS];
    acc[2] += wt * (double)mo[2 * TILE_CELLS];
    acc[3] += wt * (double)mo[3 * TILE_CELLS];
  }
  for (int o = 16; o > 0; o >>= 1)
    for (int c = 0; c < 4; ++c) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
  if (lane == 0) {
    rho_l[l] = acc[0];
    for (int a = 0; a < 3; ++a) B[3 * l + a] = (a < g.D) ? U[3 * l + a] - acc[1 + a] : 0.0;
  }
}

// ------------------------------------------------------------------ system assembly
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
__global__ void k_assemble(int m_total, const int* __restrict__ base, const double* __restrict__ wts,
                           const int* __restrict__ tile_slot, const int* __restrict__ tile_mcount,
                           const int* __restrict__ tile_markers, Geo g, const int* __restrict__ body_of,
                           int* __restrict__ Gcol, double* __restrict__ Gval, int* __restrict__ Gnnz,
                           unsigned long long* __restrict__ rowsum_max, int* status) {
  __shared__ int s_col[8][G_MAXNNZ];
  __shared__ double s_val[8][G_MAXNNZ];
  const int wib = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int l = blockIdx.x * 8 + wib;
  if (l >= m_total) return;
  const int* bl = base + 3 * l;
  const double* wl = wts + 12 * l;
  int tiles[8];
  const int nt = touched_tiles(g, bl, tiles);
  int count = 0;
  double rowsum = 0.0;
  for (int ti = 0; ti < nt; ++ti) {
    const int t = tiles[ti];
    const int s = tile_slot[t];
    if (s < 0) continue;
    const int cnt = min(tile_mcount[s], TILE_MARKER_CAP);
    for (int j0 = 0; j0 < cnt; j0 += 32) {
      const int j = j0 + lane;
      bool take = false;
      double val = 0.0;
      int k = -1;
      if (j < cnt) {
        k = tile_markers[s * TILE_MARKER_CAP + j];
        const int* bk = base + 3 * k;
        const double* wk = wts + 12 * k;
        take = true;
        int lo[3];
        double prod = 1.0;
        for (int a = 0; a < 3 && take; ++a) {
          if (a >= g.D) { lo[a] = 0; continue; }
          const int d = base_diff(bk[a], bl[a], g.n[a], g.per[a]);   // base_k - base_l
          if (d < -3 || d > 3) { take = false; break; }
          // overlap nodes in l's frame: o in [max(0,d), min(3,3+d)]
          const int o0 = d > 0 ? d : 0, o1 = d < 0 ? 3 + d : 3;
          double s1 = 0.0;
          for (int o = o0; o <= o1; ++o) s1 += wl[4 * a + o] * wk[4 * a + (o - d)];
          prod *= s1;
          int node = bl[a] + o0;
          lo[a] = g.per[a] ? wrap(node, g.n[a]) : node;
        }
        if (take) {
          if (tile_of(g, lo[0], lo[1], g.D == 3 ? lo[2] : 0) != t) take = false;
          val = prod;
        }
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
        rowsum += fabs(val);
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
    atomicMax(&rowsum_max[body_of[l]], (unsigned long long)__double_as_longlong(rowsum));
  }
}

// ------------------------------------------------------------------ PCG with in-kernel preconditioner rebuild
struct PcgArgs {
  int m_total;
  int D;
  int nbodies;
  int boff[MAX_BODIES + 1];     // marker offsets
  long long poff[MAX_BODIES];   // preconditioner offsets (floats)
  const int* body_of;
  const int* Gcol;
  const double* Gval;
  const int* Gnnz;
  const unsigned long long* rowsum_max;
  const double* B;
  double* w;
  double* r;
  double* p;
  double* Ap;
  double* z;
  float* M;
  double* red;      // [gridDim][8] partials
  int* info;        // [0] iterations, [1] refresh request, [2] converged flag
  double* res;      // final relative residual
  int warm;
  int refresh;      // host-scheduled rebuild
  int* status;
};

// Deterministic block reduction of nv doubles; result valid in thread 0.
template <int NV>
__device__ void block_sum(double v[NV], double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int o = 16; o > 0; o >>= 1)
    for (int c = 0; c < NV; ++c) v[c] += __shfl_xor_sync(0xffffffffu, v[c], o);
  __syncthreads();
  if (lane == 0)
    for (int c = 0; c < NV; ++c) sh[wid * NV + c] = v[c];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int c = 0; c < NV; ++c) {
      double s = 0;
      for (int w = 0; w < nw; ++w) s += sh[w * NV + c];
      v[c] = s;
    }
  }
  __syncthreads();
}

// Sum of the per-block partials in block order (every block gets the same bits).
template <int NV>
__device__ void grid_total(const double* red, int slot, double out[NV]) {
  for (int c = 0; c < NV; ++c) out[c] = 0.0;
  for (int b = 0; b < (int)gridDim.x; ++b)
    for (int c = 0; c < NV; ++c) out[c] += red[b * 8 + slot + c];
}

// y = G x for the rows of this warp (strided over all warps).
__device__ void spmv_rows(const PcgArgs& A, const double* __restrict__ x, double* __restrict__ y,
                          int gwarp, int nwarps, int lane) {
  for (int l = gwarp; l < A.m_total; l += nwarps) {
    const int nnz = A.Gnnz[l];
    double s0 = 0, s1 = 0, s2 = 0;
    for (int j = lane; j < nnz; j += 32) {
      const int k = A.Gcol[(long long)l * G_MAXNNZ + j];
      const double v = A.Gval[(long long)l * G_MAXNNZ + j];
      s0 += v * x[3 * k];
      s1 += v * x[3 * k + 1];
      s2 += v * x[3 * k + 2];
    }
    for (int o = 16; o > 0; o >>= 1) {
      s0 += __shfl_xor_sync(0xffffffffu, s0, o);
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
      s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if (lane == 0) { y[3 * l] = s0; y[3 * l + 1] = s1; y[3 * l + 2] = s2; }
  }
}

// y = M_b x (FP32 dense preconditioner of the row's body, FP64 accumulation per lane).
__device__ void precond_rows(const PcgArgs& A, const double* __restrict__ x, double* __restrict__ y,
                             int gwarp, int nwarps, int lane) {
  for (int l = gwarp; l < A.m_total; l += nwarps) {
    const int b = A.body_of[l];
    const int o = A.boff[b], mb = A.boff[b + 1] - o;
    const float* row = A.M + A.poff[b] + (long long)(l - o) * mb;
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
    for (int j = lane; j < mb; j += 32) {
      const float v = row[j];
      const int k = o + j;
      s0 = fmaf(v, (float)x[3 * k], s0);
      s1 = fmaf(v, (float)x[3 * k + 1], s1);
      s2 = fmaf(v, (float)x[3 * k + 2], s2);
    }
    for (int off = 16; off > 0; off >>= 1) {
      s0 += __shfl_xor_sync(0xffffffffu, s0, off);
      s1 += __shfl_xor_sync(0xffffffffu, s1, off);
      s2 += __shfl_xor_sync(0xffffffffu, s2, off);
    }
    if (lane == 0) { y[3 * l] = s0; y[3 * l + 1] = s1; y[3 * l + 2] = s2; }
  }
}

// In-place blocked Gauss-Jordan inverse of every body's dense SPD matrix
// (no pivoting; the matrix is G_b + sigma I).  For the pivot block P:
//   P <- P^-1;  row panel R <- P^-1 R;  rest S <- S - C R;  column panel C <- -C P^-1.
__device__ void gj_invert(const PcgArgs& A, cg::grid_group& grid, float* sh) {
  int maxnb = 0;
  for (int b = 0; b < A.nbodies; ++b) {
    const int mb = A.boff[b + 1] - A.boff[b];
    maxnb = max(maxnb, (mb + GJ_NB - 1) / GJ_NB);
  }
  const int nthreads = gridDim.x * blockDim.x;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  float* piv = sh;                          // GJ_NB x GJ_NB
  for (int kb = 0; kb < maxnb; ++kb) {
    // phase 1: invert the pivot blocks (block b of the grid handles body b)
    for (int b = blockIdx.x; b < A.nbodies; b += gridDim.x) {
      const int mb = A.boff[b + 1] - A.boff[b];
      const int k0 = kb * GJ_NB;
      if (k0 >= mb) continue;
      const int kn = min(GJ_NB, mb - k0);
      float* Mb = A.M + A.poff[b];
      for (int e = threadIdx.x; e < kn * kn; e += blockDim.x)
        piv[e] = Mb[(long long)(k0 + e / kn) * mb + k0 + e % kn];
      __syncthreads();
      for (int k = 0; k < kn; ++k) {
        const float pk = 1.0f / piv[k * kn + k];
        __syncthreads();
        // row k scaled, other rows eliminated (unblocked Gauss-Jordan)
        for (int e = threadIdx.x; e < kn * kn; e += blockDim.x) {
          const int i = e / kn, j = e % kn;
          float v;
          if (i == k && j == k) v = pk;
          else if (i == k) v = piv[k * kn + j] * pk;
          else if (j == k) v = -piv[i * kn + k] * pk;
          else v = piv[i * kn + j] - piv[i * kn + k] * piv[k * kn + j] * pk;
          sh[GJ_NB * GJ_NB + e] = v;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < kn * kn; e += blockDim.x) piv[e] = sh[GJ_NB * GJ_NB + e];
        __syncthreads();
      }
      for (int e = threadIdx.x; e < kn * kn; e += blockDim.x)
        Mb[(long long)(k0 + e / kn) * mb + k0 + e % kn] = piv[e];
      __syncthreads();
    }
    grid.sync();
    // phase 2: row panel R <- P^-1 R (one thread per column outside the pivot block)
    for (int b = 0; b < A.nbodies; ++b) {
      const int mb = A.boff[b + 1] - A.boff[b];
      const int k0 = kb * GJ_NB;
      if (k0 >= mb) continue;
      const int kn = min(GJ_NB, mb - k0);
      float* Mb = A.M + A.poff[b];
      for (int j = gtid; j < mb; j += nthreads) {
        if (j >= k0 && j < k0 + kn) continue;
        float col[GJ_NB];
        for (int i = 0; i < kn; ++i) col[i] = Mb[(long long)(k0 + i) * mb + j];
        for (int i = 0; i < kn; ++i) {
          float s = 0.f;
          for (int q = 0; q < kn; ++q) s = fmaf(Mb[(long long)(k0 + i) * mb + k0 + q], col[q], s);
          Mb[(long long)(k0 + i) * mb + j] = s;
        }
      }
    }
    grid.sync();
    // phase 3a: S <- S - C R (rows and columns outside the pivot block)
    for (int b = 0; b < A.nbodies; ++b) {
      const int mb = A.boff[b + 1] - A.boff[b];
      const int k0 = kb * GJ_NB;
      if (k0 >= mb) continue;
      const int kn = min(GJ_NB, mb - k0);
      float* Mb = A.M + A.poff[b];
      const long long total = (long long)mb * mb;
      for (long long e = gtid; e < total; e += nthreads) {
        const int i = (int)(e / mb), j = (int)(e % mb);
        if ((i >= k0 && i < k0 + kn) || (j >= k0 && j < k0 + kn)) continue;
        float s = Mb[e];
        const float* ci = Mb + (long long)i * mb + k0;
        for (int q = 0; q < kn; ++q) s = fmaf(-ci[q], Mb[(long long)(k0 + q) * mb + j], s);
        Mb[e] = s;
      }
    }
    grid.sync();
    // phase 3b: C <- -C P^-1 (rows outside, columns inside the pivot block)
    for (int b = 0; b < A.nbodies; ++b) {
      const int mb = A.boff[b + 1] - A.boff[b];
      const int k0 = kb * GJ_NB;
      if (k0 >= mb) continue;
      const int kn = min(GJ_NB, mb - k0);
      float* Mb = A.M + A.poff[b];
      for (int i = gtid; i < mb; i += nthreads) {
        if (i >= k0 && i < k0 + kn) continue;
        float row[GJ_NB];
        for (int q = 0; q < kn; ++q) row[q] = Mb[(long long)i * mb + k0 + q];
        for (int j = 0; j < kn; ++j) {
          float s = 0.f;
          for (int q = 0; q < kn; ++q) s = fmaf(row[q], Mb[(long long)(k0 + q) * mb + k0 + j], s);
          Mb[(long long)i * mb + k0 + j] = -s;
        }
      }
    }
    grid.sync();
  }
}

__global__ void __launch_bounds__(256) k_pcg(PcgArgs A) {
  cg::grid_group grid = cg::this_grid();
  __shared__ float sh[2 * GJ_NB * GJ_NB];
  __shared__ double shd[8 * 8];
  const int lane = threadIdx.x & 31;
  const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nthreads = gridDim.x * blockDim.x;
  const int m3 = 3 * A.m_total;

  // ---- optional preconditioner rebuild: M_b <- (G_b + sigma_b I)^-1 in FP32
  const bool rebuild = A.refresh || A.info[1];
  if (rebuild) {
    for (int b = 0; b < A.nbodies; ++b) {
      const int mb = A.boff[b + 1] - A.boff[b];
      const long long tot = (long long)mb * mb;
      for (long long e = gtid; e < tot; e += nthreads) A.M[A.poff[b] + e] = 0.f;
    }
    grid.sync();
    for (int l = gtid; l < A.m_total; l += nthreads) {
      const int b = A.body_of[l];
      const int o = A.boff[b], mb = A.boff[b + 1] - o;
      const double sigma = 1e-6 * __longlong_as_double((long long)A.rowsum_max[b]);
      float* Mb = A.M + A.poff[b];
      for (int j = 0; j < A.Gnnz[l]; ++j) {
        const int k = A.Gcol[(long long)l * G_MAXNNZ + j];
        if (A.body_of[k] != b) continue;   // block-Jacobi over bodies
        double v = A.Gval[(long long)l * G_MAXNNZ + j];
        if (k == l) v += sigma;
        Mb[(long long)(l - o) * mb + (k - o)] = (float)v;
      }
    }
    grid.sync();
    gj_invert(A, grid, sh);
  }

  // ---- setup: x0 = warm ? w : 0;  r = B - G x0;  z = M r;  p = z
  if (!A.warm)
    for (int i = gtid; i < m3; i += nthreads) A.w[i] = 0.0;
  grid.sync();
  spmv_rows(A, A.w, A.Ap, gwarp, nwarps, lane);
  grid.sync();
  for (int i = gtid; i < m3; i += nthreads) A.r[i] = A.B[i] - A.Ap[i];
  grid.sync();
  precond_rows(A, A.r, A.z, gwarp, nwarps, lane);
  precond_rows(A, A.B, A.Ap, gwarp, nwarps, lane);   // M B for the stopping scale
  grid.sync();
  {
    double v[6] = {0, 0, 0, 0, 0, 0};
    for (int i = gtid; i < m3; i += nthreads) {
      const int c = i % 3;
      v[c] += A.r[i] * A.z[i];
      v[3 + c] += A.B[i] * A.Ap[i];
    }
    block_sum<6>(v, shd);
    if (threadIdx.x == 0)
      for (int c = 0; c < 6; ++c) A.red[blockIdx.x * 8 + c] = v[c];
  }
  for (int i = gtid; i < m3; i += nthreads) A.p[i] = A.z[i];
  grid.sync();
  double tot[6];
  grid_total<6>(A.red, 0, tot);
  double rz[3] = {tot[0], tot[1], tot[2]};
  double scale[3] = {tot[3], tot[4], tot[5]};
  grid.sync();   // everyone has read the partials before they are overwritten

  int it = 0;
  bool done = true;
  for (int c = 0; c < A.D; ++c) done &= !(rz[c] > PCG_TOL * PCG_TOL * scale[c]);
  while (!done && it < PCG_MAX_ITERS) {
    // Ap = G p;  partial p.Ap
    spmv_rows(A, A.p, A.Ap, gwarp, nwarps, lane);
    grid.sync();
    {
      double v[3] = {0, 0, 0};
      for (int i = gtid; i < m3; i += nthreads) v[i % 3] += A.p[i] * A.Ap[i];
      block_sum<3>(v, shd);
      if (threadIdx.x == 0)
        for (int c = 0; c < 3; ++c) A.red[blockIdx.x * 8 + c] = v[c];
    }
    grid.sync();
    double pAp[3];
    grid_total<3>(A.red, 0, pAp);
    double alpha[3];
    for (int c = 0; c < 3; ++c) alpha[c] = (pAp[c] > 0.0 && rz[c] > 0.0) ? rz[c] / pAp[c] : 0.0;
    for (int i = gtid; i < m3; i += nthreads) {
      const int c = i % 3;
      A.w[i] += alpha[c] * A.p[i];
      A.r[i] -= alpha[c] * A.Ap[i];
    }
    grid.sync();
    // z = M r;  partial r.z
    precond_rows(A, A.r, A.z, gwarp, nwarps, lane);
    grid.sync();
    {
      double v[3] = {0, 0, 0};
      for (int i = gtid; i < m3; i += nthreads) v[i % 3] += A.r[i] * A.z[i];
      block_sum<3>(v, shd);
      if (threadIdx.x == 0)
        for (int c = 0; c < 3; ++c) A.red[blockIdx.x * 8 + 3 + c] = v[c];
    }
    grid.sync();
    double rzn[3];
    grid_total<3>(A.red, 3, rzn);
    double beta[3];
    for (int c = 0; c < 3; ++c) beta[c] = rz[c] > 0.0 ? rzn[c] / rz[c] : 0.0;
    for (int i = gtid; i < m3; i += nthreads) A.p[i] = A.z[i] + beta[i % 3] * A.p[i];
    for (int c = 0; c < 3; ++c) rz[c] = rzn[c];
    ++it;
    done = true;
    for (int c = 0; c < A.D; ++c) done &= !(rz[c] > PCG_TOL * PCG_TOL * scale[c]);
    grid.sync();
  }
  if (gtid == 0) {
    double rel = 0.0;
    for (int c = 0; c < A.D; ++c)
      if (scale[c] > 0.0) rel = fmax(rel, sqrt(fmax(rz[c], 0.0) / scale[c]));
    A.info[0] = it;
    A.info[1] = (it > REFRESH_ITERS || !done) ? 1 : 0;
    A.info[2] = done ? 1 : 0;
    *A.res = rel;
    if (!done) atomicOr(A.status, ST_NOTCONV);
  }
}

// ------------------------------------------------------------------ spreading and force density
template <class R>
__global__ void k_spread(const int* __restrict__ slot_tile, const int* __restrict__ band_count, int cap,
                         const int* __restrict__ tile_mcount, const int* __restrict__ tile_markers,
                         const int* __restrict__ base, const double* __restrict__ wts,
                         const double* __restrict__ wsol, const R* __restrict__ band_mom,
                         R* __restrict__ band_F, Geo g) {
  __shared__ int s_list[TILE_MARKER_CAP];
  __shared__ int s_sorted[TILE_MARKER_CAP];
  const int n = min(*band_count, cap);
  for (int s = blockIdx.x; s < n; s += gridDim.x) {
    const int cnt = min(tile_mcount[s], TILE_MARKER_CAP);
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) s_list[i] = tile_markers[s * TILE_MARKER_CAP + i];
    __syncthreads();
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
      const int key = s_list[i];
      int rank = 0;
      for (int j = 0; j < cnt; ++j) rank += s_list[j] < key;
      s_sorted[rank] = key;
    }
    __syncthreads();
    const int tile = slot_tile[s];
    const int local = threadIdx.x;
    const int x = (tile % g.tg.ntx) * g.tg.tx + local % g.tg.tx;
    const int y = ((tile / g.tg.ntx) % g.tg.nty) * g.tg.ty + (local / g.tg.tx) % g.tg.ty;
    const int z = (tile / (g.tg.ntx * g.tg.nty)) * g.tg.tz + local / (g.tg.tx * g.tg.ty);
    const int node[3] = {x, y, z};
    double du[3] = {0, 0, 0};
    for (int j = 0; j < cnt; ++j) {
      const int k = s_sorted[j];
      const int* bk = base + 3 * k;
      double wt = 1.0;
      bool in = true;
      for (int a = 0; a < g.D; ++a) {
        int o = node[a] - bk[a];
        if (g.per[a]) o = wrap(o, g.n[a]);
        if (o < 0 || o > 3) { in = false; break; }
        wt *= wts[12 * k + 4 * a + o];
      }
      if (!in) continue;
      du[0] += wt * wsol[3 * k];
      du[1] += wt * wsol[3 * k + 1];
      du[2] += wt * wsol[3 * k + 2];
    }
    const R* mo = band_mom + (long long)s * 4 * TILE_CELLS + local;
    const double rho = (double)mo[0];
    R* f = band_F + (long long)s * 3 * TILE_CELLS + local;
    f[0] = (R)(2.0 * rho * du[0]);      // Eq. 26: F = 2 rho du / dt
    f[TILE_CELLS] = (R)(2.0 * rho * du[1]);
    f[2 * TILE_CELLS] = (R)(g.D == 3 ? 2.0 * rho * du[2] : 0.0);
    __syncthreads();
  }
}

// ------------------------------------------------------------------ forces
__global__ void k_force_reduce(int nbodies, const int* __restrict__ boff, const double* __restrict__ rho_l,
                               const double* __restrict__ wsol, double* __restrict__ mforce,
                               double* __restrict__ hist, long long step) {
  __shared__ double sh[8 * 3];
  const int b = blockIdx.x;
  if (b >= nbodies) return;
  const int o = boff[b], e = boff[b + 1];
  double v[3] = {0, 0, 0};
  for (int l = o + threadIdx.x; l < e; l += blockDim.x) {
    for (int a = 0; a < 3; ++a) {
      const double f = 2.0 * rho_l[l] * wsol[3 * l + a];   // force on the fluid (Eq. 26 x ds)
      mforce[3 * l + a] = f;
      v[a] += f;
    }
  }
  block_sum<3>(v, sh);
  if (threadIdx.x == 0) {
    double* h = hist + ((long long)b * HIST_LEN + (step % HIST_LEN)) * 3;
    for (int a = 0; a < 3; ++a) h[a] = -v[a];   // force on the body
  }
}

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

cudaError_t ib_alloc(ibl_ctx* c) {
  ib_free(c);
  const int m = c->m_total;
  if (m == 0) return cudaSuccess;
  c->cap_slots = (int)std::min<long long>((long long)c->tg.n_tiles, 8LL * m + 64);
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
  IBL_CU(cudaMalloc(&c->d_band_mom, rs * 4 * TILE_CELLS * (size_t)c->cap_slots));
  IBL_CU(cudaMalloc(&c->d_band_F, rs * 3 * TILE_CELLS * (size_t)c->cap_slots));
  IBL_CU(cudaMalloc(&c->d_base, sizeof(int) * 3 * m));
  IBL_CU(cudaMalloc(&c->d_wts, sizeof(double) * 12 * m));
  IBL_CU(cudaMalloc(&c->d_rho_l, sizeof(double) * m));
  IBL_CU(cudaMalloc(&c->d_B, sizeof(double) * 3 * m));
  IBL_CU(cudaMalloc(&c->d_w, sizeof(double) * 3 * m));
  IBL_CU(cudaMemsetAsync(c->d_w, 0, sizeof(double) * 3 * m, c->stream));
  IBL_CU(cudaMalloc(&c->d_r, sizeof(double) * 3 * m));
  IBL_CU(cudaMalloc(&c->d_p, sizeof(double) * 6 * m));
  IBL_CU(cudaMalloc(&c->d_Ap, sizeof(double) * 3 * m));
  IBL_CU(cudaMalloc(&c->d_z, sizeof(double) * 3 * m));
  IBL_CU(cudaMalloc(&c->d_Gcol, sizeof(int) * (size_t)m * G_MAXNNZ));
  IBL_CU(cudaMalloc(&c->d_Gval, sizeof(double) * (size_t)m * G_MAXNNZ));
  IBL_CU(cudaMalloc(&c->d_Gnnz, sizeof(int) * m));
  IBL_CU(cudaMalloc(&c->d_Gdiag_max, sizeof(double) * MAX_BODIES));
  size_t mf = 0;
  for (auto& b : c->bodies) {
    b.precond_offset = (int)mf;
    mf += (size_t)b.m * b.m;
  }
  c->M_floats = mf;
  IBL_CU(cudaMalloc(&c->d_M, sizeof(float) * mf));
  IBL_CU(cudaMalloc(&c->d_red, sizeof(double) * 8 * 1024));
  IBL_CU(cudaMalloc(&c->d_cg_info, sizeof(int) * 4));
  IBL_CU(cudaMemsetAsync(c->d_cg_info, 0, sizeof(int) * 4, c->stream));
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
  IBL_CU(cudaMemcpy(c->d_body, body_of.data(), sizeof(int) * m, cudaMemcpyHostToDevice));
  std::vector<int> boff(c->bodies.size() + 1);
  for (size_t b = 0; b < c->bodies.size(); ++b) boff[b] = c->bodies[b].offset;
  boff[c->bodies.size()] = m;
  IBL_CU(cudaMalloc(&c->d_boff, sizeof(int) * boff.size()));
  IBL_CU(cudaMemcpy(c->d_boff, boff.data(), sizeof(int) * boff.size(), cudaMemcpyHostToDevice));
  c->precond_valid = false;
  c->warm = false;
  c->ib_ready = true;
  return cudaSuccess;
}

void ib_free(ibl_ctx* c) {
  void* ptrs[] = {c->d_X0, c->d_ds, c->d_body, c->d_X, c->d_U, c->d_Xp, c->d_Up, c->d_tile_slot,
                  c->d_slot_tile, c->d_band_count, c->d_tile_mcount, c->d_tile_markers, c->d_band_mom,
                  c->d_band_F, c->d_base, c->d_wts, c->d_rho_l, c->d_B, c->d_w, c->d_r, c->d_p,
                  c->d_Ap, c->d_z, c->d_Gcol, c->d_Gval, c->d_Gnnz, c->d_Gdiag_max, c->d_M, c->d_red,
                  c->d_cg_info, c->d_cg_res, c->d_hist, c->d_mforce, c->d_boff};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  c->d_X0 = c->d_ds = c->d_X = c->d_U = c->d_Xp = c->d_Up = nullptr;
  c->d_body = c->d_tile_slot = c->d_slot_tile = c->d_band_count = c->d_tile_mcount = nullptr;
  c->d_tile_markers = c->d_base = c->d_Gcol = c->d_Gnnz = c->d_cg_info = c->d_boff = nullptr;
  c->d_band_mom = c->d_band_F = nullptr;
  c->d_wts = nullptr;
  c->d_rho_l = c->d_B = c->d_w = c->d_r = c->d_p = c->d_Ap = c->d_z = c->d_Gval = nullptr;
  c->d_Gdiag_max = c->d_red = c->d_cg_res = c->d_hist = c->d_mforce = nullptr;
  c->d_M = nullptr;
  c->ib_ready = false;
}

template <int Q, class T>
static cudaError_t band_moments_q(ibl_ctx* c, int grid) {
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
  p.band_F = nullptr;
  p.status = c->d_status;
  const T* src = (const T*)c->f[c->cur];
  if (c->poststream)
    k_band_moments<Q, T, false><<<grid, TILE_CELLS, 0, c->stream>>>(src, p, c->d_slot_tile, c->d_band_count,
                                                                  c->cap_slots, (R*)c->d_band_mom);
  else
    k_band_moments<Q, T, true><<<grid, TILE_CELLS, 0, c->stream>>>(src, p, c->d_slot_tile, c->d_band_count,
                                                                 c->cap_slots, (R*)c->d_band_mom);
  c->launches++;
  return cudaGetLastError();
}

static cudaError_t band_moments(ibl_ctx* c, int grid) {
  if (c->Q == 9) {
    switch (c->prec) {
      case IBL_FP64: return band_moments_q<9, double>(c, grid);
      case IBL_FP32: return band_moments_q<9, float>(c, grid);
      case IBL_FP16DEV: return band_moments_q<9, __half>(c, grid);
      default: return band_moments_q<9, __nv_bfloat16>(c, grid);
    }
  }
  switch (c->prec) {
    case IBL_FP64: return band_moments_q<19, double>(c, grid);
    case IBL_FP32: return band_moments_q<19, float>(c, grid);
    case IBL_FP16DEV: return band_moments_q<19, __half>(c, grid);
    default: return band_moments_q<19, __nv_bfloat16>(c, grid);
  }
}

static int g_num_sms = 0;

cudaError_t ib_step(ibl_ctx* c) {
  const int m = c->m_total;
  if (m == 0) return cudaSuccess;
  if (!g_num_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 1;
  }
  Geo g = make_geo(c);
  BodyTable bt;
  bt.n = (int)c->bodies.size();
  for (int b = 0; b < bt.n; ++b) {
    const Body& h = c->bodies[b];
    BodyDev& d = bt.b[b];
    d.offset = h.offset; d.m = h.m;
    for (int a = 0; a < 3; ++a) { d.hinge[a] = h.hinge[a]; d.axis[a] = h.axis[a]; d.origin[a] = h.origin[a]; }
    d.beta = h.beta; d.phi = h.phi; d.f = h.f;
    d.A = h.A; d.alpha = h.alpha;
    d.A.table = h.tableA; d.alpha.table = h.tableAlpha;
    d.prescribed = h.prescribed ? 1 : 0;
  }
  const int tb = 128;
  const int mb = (m + tb - 1) / tb;
  k_kinematics<<<mb, tb, 0, c->stream>>>(bt, m, c->d_body, c->d_X0, c->d_Xp, c->d_Up, c->d_X, c->d_U,
                                         c->d_base, c->d_wts, (double)c->step, g, c->d_status);
  for (auto& b : c->bodies) b.prescribed = false;
  const int cg_grid = std::min(c->cap_slots, 4 * g_num_sms);
  k_clear_tiles<<<std::max(1, std::min(c->cap_slots / 256 + 1, g_num_sms)), 256, 0, c->stream>>>(
      c->d_tile_slot, c->d_slot_tile, c->d_band_count, c->d_tile_mcount, c->cap_slots);
  IBL_CU(cudaMemsetAsync(c->d_band_count, 0, sizeof(int), c->stream));
  k_mark_tiles<<<mb, tb, 0, c->stream>>>(m, c->d_base, g, c->d_tile_slot);
  k_assign_slots<<<std::max(1, std::min((c->tg.n_tiles + 255) / 256, 2 * g_num_sms)), 256, 0, c->stream>>>(
      c->tg.n_tiles, c->d_tile_slot, c->d_slot_tile, c->d_band_count, c->cap_slots, c->d_status);
  k_append_markers<<<mb, tb, 0, c->stream>>>(m, c->d_base, g, c->d_tile_slot, c->d_tile_mcount,
                                             c->d_tile_markers, c->d_status);
  c->launches += 6;
  IBL_CU(cudaGetLastError());
  IBL_CU(band_moments(c, cg_grid));
  const int wb = (m * 32 + 255) / 256;
  if (c->prec == IBL_FP64)
    k_interpolate<double><<<wb, 256, 0, c->stream>>>(m, c->d_base, c->d_wts, (const double*)c->d_band_mom,
                                                     c->d_tile_slot, g, c->d_U, c->d_rho_l, c->d_B);
  else
    k_interpolate<float><<<wb, 256, 0, c->stream>>>(m, c->d_base, c->d_wts, (const float*)c->d_band_mom,
                                                    c->d_tile_slot, g, c->d_U, c->d_rho_l, c->d_B);
  IBL_CU(cudaMemsetAsync(c->d_Gdiag_max, 0, sizeof(double) * MAX_BODIES, c->stream));
  k_assemble<<<(m + 7) / 8, 256, 0, c->stream>>>(m, c->d_base, c->d_wts, c->d_tile_slot,
                                                 c->d_tile_mcount, c->d_tile_markers, g, c->d_body, c->d_Gcol,
                                                 c->d_Gval, c->d_Gnnz, (unsigned long long*)c->d_Gdiag_max,
                                                 c->d_status);
  c->launches += 2;
  IBL_CU(cudaGetLastError());
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
  A.Gcol = c->d_Gcol; A.Gval = c->d_Gval; A.Gnnz = c->d_Gnnz;
  A.rowsum_max = (const unsigned long long*)c->d_Gdiag_max;
  A.B = c->d_B; A.w = c->d_w; A.r = c->d_r; A.p = c->d_p; A.Ap = c->d_Ap; A.z = c->d_z;
  A.M = c->d_M; A.red = c->d_red; A.info = c->d_cg_info; A.res = c->d_cg_res;
  A.warm = c->warm ? 1 : 0;
  const bool sched = !c->precond_valid || (c->step - c->last_refresh_step) >= REFRESH_EVERY;
  A.refresh = sched ? 1 : 0;
  if (sched) {
    c->last_refresh_step = c->step;
    c->refreshes++;
  }
  c->precond_valid = true;
  A.status = c->d_status;
  static int max_blocks_per_sm = 0;
  if (!max_blocks_per_sm) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&max_blocks_per_sm, k_pcg, 256, 0);
    if (max_blocks_per_sm <= 0) max_blocks_per_sm = 1;
  }
  int pcg_blocks = std::min(g_num_sms * std::min(max_blocks_per_sm, 1), std::max(1, (m + 15) / 16));
  pcg_blocks = std::min(pcg_blocks, 1024);
  void* args[] = {&A};
  IBL_CU(cudaLaunchCooperativeKernel((void*)k_pcg, dim3(pcg_blocks), dim3(256), args, 0, c->stream));
  c->launches++;
  c->warm = true;
  // spreading
  if (c->prec == IBL_FP64)
    k_spread<double><<<cg_grid, TILE_CELLS, 0, c->stream>>>(c->d_slot_tile, c->d_band_count, c->cap_slots,
                                                            c->d_tile_mcount, c->d_tile_markers, c->d_base,
                                                            c->d_wts, c->d_w, (const double*)c->d_band_mom,
                                                            (double*)c->d_band_F, g);
  else
    k_spread<float><<<cg_grid, TILE_CELLS, 0, c->stream>>>(c->d_slot_tile, c->d_band_count, c->cap_slots,
                                                           c->d_tile_mcount, c->d_tile_markers, c->d_base,
                                                           c->d_wts, c->d_w, (const float*)c->d_band_mom,
                                                           (float*)c->d_band_F, g);
  c->launches++;
  IBL_CU(cudaGetLastError());
  return cudaSuccess;
}

cudaError_t ib_after_collide(ibl_ctx* c) {
  if (c->m_total == 0) return cudaSuccess;
  const int nb = (int)c->bodies.size();
  k_force_reduce<<<nb, 256, 0, c->stream>>>(nb, c->d_boff, c->d_rho_l, c->d_w, c->d_mforce, c->d_hist, c->step);
  c->launches++;
  return cudaGetLastError();
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
