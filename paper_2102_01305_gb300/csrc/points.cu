// Stand-alone immersed-boundary transfers on an arbitrary point cloud: the
// interpolation of Eq. 17 and the spreading of Eq. 15 on device arrays,
// without the implicit solve.  They run the same per-node arithmetic as the
// IB step (stencil_axis, node_moments, double-float weights and sums), one
// warp per point, after a pre-pass that evaluates every point's stencil.
#include <algorithm>

#include "ib_stencil.cuh"

namespace ibl {
namespace {

constexpr double PT_FIX_SCALE = 70368744177664.0;   // 2^46
constexpr double PT_FIX_LIMIT = 9.0e18 / PT_FIX_SCALE;
constexpr int PT_BAD_STENCIL = 1;
constexpr int PT_BAD_RANGE = 2;

struct PtGeo {
  int D;
  int n[3];
  int per[3];
};

__device__ __forceinline__ int wrap_once(int v, int n) { return v >= n ? v - n : v; }

__device__ __forceinline__ long long stencil_node(const PtGeo& g, const int b[3], int k, int node[3]) {
  const int i = k & 3, j = (k >> 2) & 3, q = k >> 4;
  node[0] = b[0] + i;
  node[1] = b[1] + j;
  node[2] = g.D == 3 ? b[2] + q : 0;
  for (int a = 0; a < g.D; ++a)
    if (g.per[a]) node[a] = wrap_once(node[a], g.n[a]);
  return ((long long)node[2] * g.n[1] + node[1]) * g.n[0] + node[0];
}

// The stencils of all points, computed before the transfers with one
// thread per (point, axis): the FP64 evaluation of Eq. 14 then fills every
// lane of the FP64 pipe, where inside the transfers (one warp per point)
// only D lanes of a warp would use it.  base[3 l + a] is the first node on
// axis a (-1 if the stencil leaves a bounded axis or x is not finite),
// wts[4 (3 l + a) + k] the double-float weights; axes a >= D get base 0
// and weights (1, 0, 0, 0).
__global__ void k_pt_stencils(int m, const double* __restrict__ X, PtGeo g, int* __restrict__ base,
                              df* __restrict__ wts, int* flag) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3LL * m) return;
  const int l = (int)(t / 3), a = (int)(t % 3);
  int mb = 0;
  df mw[4] = {df_make(1.f, 0.f), df_make(0.f, 0.f), df_make(0.f, 0.f), df_make(0.f, 0.f)};
  bool ok = true;
  if (a < g.D) {
    double wd[4];
    ok = stencil_axis(X[3 * l + a], g.n[a], g.per[a] != 0, mb, wd);
    for (int k = 0; k < 4; ++k) mw[k] = df_from_double(wd[k]);
  }
  base[t] = ok ? mb : -1;
  for (int k = 0; k < 4; ++k) wts[4 * t + k] = mw[k];
  if (!ok) atomicOr(flag, PT_BAD_STENCIL);
}

// Point l's stencil from the pre-pass; false if an axis failed (the caller
// then touches no memory).
__device__ __forceinline__ bool load_stencil(const int* __restrict__ base, const df* __restrict__ wts, int l,
                                             int b[3], df w[3][4]) {
  bool ok = true;
  for (int a = 0; a < 3; ++a) {
    b[a] = base[3 * l + a];
    ok = ok && b[a] >= 0;
    for (int k = 0; k < 4; ++k) w[a][k] = wts[4 * (3 * l + a) + k];
  }
  return ok;
}

template <int Q, class T, bool PULL>
__global__ void k_points_interpolate(int m, const int* __restrict__ sbase, const df* __restrict__ swts,
                                     const T* __restrict__ src, FluidParams<typename Store<T>::R> p, PtGeo g,
                                     double* __restrict__ U, double* __restrict__ rho_out,
                                     const int* __restrict__ perm) {
  const int wl = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (wl >= m) return;
  const int l = perm ? perm[wl] : wl;
  int b[3];
  df w[3][4];
  if (!load_stencil(sbase, swts, l, b, w)) return;
  using R = typename Store<T>::R;
  const int nn = g.D == 3 ? 64 : 16;
  dfacc acc[4] = {acc_zero(), acc_zero(), acc_zero(), acc_zero()};
  for (int k = lane; k < nn; k += 32) {
    int node[3];
    const long long cell = stencil_node(g, b, k, node);
    df wt = df_mul(w[0][k & 3], w[1][(k >> 2) & 3]);
    if (g.D == 3) wt = df_mul(wt, w[2][k >> 4]);
    R drho, u[3];
    node_moments<Q, T, PULL>(src, node[0], node[1], node[2], cell, p, drho, u);
    acc_fma(acc[0], wt, df_from_float(1.f));
    acc_fma(acc[0], wt, to_df(drho));
    for (int c = 0; c < 3; ++c) acc_fma(acc[1 + c], wt, to_df(u[c]));
  }
  df v[4];
  for (int c = 0; c < 4; ++c) v[c] = df_warp_sum(acc_value(acc[c]));
  if (lane == 0) {
    if (rho_out) rho_out[l] = df_to_double(v[0]);
    for (int a = 0; a < g.D; ++a) U[(long long)g.D * l + a] = df_to_double(v[1 + a]);
  }
}

// Large point clouds cover most cells several times over, so the pulls of
// k_points_interpolate repeat: the moments of every cell are formed once
// (k_cell_moments, the same node_moments) into a context scratch array of
// 4 N values (drho, u*), and the interpolation reads four values per node
// (k_points_interpolate_cached, the same weights and accumulation order).
// Both paths give bitwise the same results.
template <int Q, class T, bool PULL>
__global__ void k_cell_moments(const T* __restrict__ src, FluidParams<typename Store<T>::R> p,
                               typename Store<T>::R* __restrict__ mom) {
  using R = typename Store<T>::R;
  const long long N = p.N;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x; cell < N; cell += stride) {
    const int x = (int)(cell % p.nx);
    const long long yz = cell / p.nx;
    const int y = (int)(yz % p.ny), z = (int)(yz / p.ny);
    R drho, u[3];
    node_moments<Q, T, PULL>(src, x, y, z, cell, p, drho, u);
    mom[cell] = drho;
    mom[N + cell] = u[0];
    mom[2 * N + cell] = u[1];
    mom[3 * N + cell] = u[2];
  }
}

template <class R>
__global__ void k_points_interpolate_cached(int m, const int* __restrict__ sbase, const df* __restrict__ swts,
                                            const R* __restrict__ mom, long long N, PtGeo g,
                                            double* __restrict__ U, double* __restrict__ rho_out,
                                            const int* __restrict__ perm) {
  const int wl = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (wl >= m) return;
  const int l = perm ? perm[wl] : wl;
  int b[3];
  df w[3][4];
  if (!load_stencil(sbase, swts, l, b, w)) return;
  const int nn = g.D == 3 ? 64 : 16;
  dfacc acc[4] = {acc_zero(), acc_zero(), acc_zero(), acc_zero()};
  for (int k = lane; k < nn; k += 32) {
    int node[3];
    const long long cell = stencil_node(g, b, k, node);
    df wt = df_mul(w[0][k & 3], w[1][(k >> 2) & 3]);
    if (g.D == 3) wt = df_mul(wt, w[2][k >> 4]);
    const R drho = mom[cell];
    const R u[3] = {mom[N + cell], mom[2 * N + cell], mom[3 * N + cell]};
    acc_fma(acc[0], wt, df_from_float(1.f));
    acc_fma(acc[0], wt, to_df(drho));
    for (int c = 0; c < 3; ++c) acc_fma(acc[1 + c], wt, to_df(u[c]));
  }
  df v[4];
  for (int c = 0; c < 4; ++c) v[c] = df_warp_sum(acc_value(acc[c]));
  if (lane == 0) {
    if (rho_out) rho_out[l] = df_to_double(v[0]);
    for (int a = 0; a < g.D; ++a) U[(long long)g.D * l + a] = df_to_double(v[1 + a]);
  }
}

// Fixed-point scatter into the caller's output array reinterpreted as int64
// (the same 8 bytes per entry): integer sums do not depend on atomic order.
__global__ void k_points_spread(int m, const int* __restrict__ sbase, const df* __restrict__ swts,
                                const double* __restrict__ V, const double* __restrict__ ds, PtGeo g, long long N,
                                unsigned long long* __restrict__ acc, int* flag, const int* __restrict__ perm) {
  const int wl = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (wl >= m) return;
  const int l = perm ? perm[wl] : wl;
  int b[3];
  df w[3][4];
  if (!load_stencil(sbase, swts, l, b, w)) return;
  // V_l ds_l per component, formed by lane c and broadcast
  df vc = df_make(0.f, 0.f);
  if (lane < g.D) vc = df_from_double(V[(long long)g.D * l + lane] * ds[l]);
  df v[3];
  for (int c = 0; c < 3; ++c) v[c] = df_make(__shfl_sync(0xffffffffu, vc.hi, c), __shfl_sync(0xffffffffu, vc.lo, c));
  const int nn = g.D == 3 ? 64 : 16;
  for (int k = lane; k < nn; k += 32) {
    int node[3];
    const long long cell = stencil_node(g, b, k, node);
    df wt = df_mul(w[0][k & 3], w[1][(k >> 2) & 3]);
    if (g.D == 3) wt = df_mul(wt, w[2][k >> 4]);
    for (int c = 0; c < g.D; ++c) {
      // the double-float product in fixed point, part by part (error <= 1 unit of 2^-46)
      const df val = df_mul(wt, v[c]);
      if (!(fabsf(val.hi) < (float)PT_FIX_LIMIT)) {
        atomicOr(flag, PT_BAD_RANGE);
        continue;
      }
      const long long fx = __float2ll_rn(val.hi * (float)PT_FIX_SCALE) + __float2ll_rn(val.lo * (float)PT_FIX_SCALE);
      atomicAdd(acc + c * N + cell, (unsigned long long)fx);
    }
  }
}

__global__ void k_fixed_to_double(unsigned long long* a, long long n) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    reinterpret_cast<double*>(a)[i] = (double)(long long)a[i] * (1.0 / PT_FIX_SCALE);
}

// ---- spatial order of the points: a counting sort by the 16 x 4 x 4 (2D:
// 16 x 16) tile holding each point's cell, so that neighbouring warps touch
// neighbouring cells (cache and atomic locality); the results do not depend
// on the order (interpolation is per point, spreading sums in fixed point).
__device__ __forceinline__ int point_bin(const double* X, int l, const PtGeo& g, const TileGeom& t) {
  int c[3] = {0, 0, 0};
  for (int a = 0; a < g.D; ++a) {
    const double x = X[3 * l + a];
    double f = isfinite(x) ? floor(x) : 0.0;
    if (g.per[a]) {
      f = fmod(f, (double)g.n[a]);
      if (f < 0.0) f += (double)g.n[a];
    }
    c[a] = (int)fmin(fmax(f, 0.0), (double)(g.n[a] - 1));
  }
  return ((c[2] / t.tz) * t.nty + (c[1] / t.ty)) * t.ntx + (c[0] / t.tx);
}

__global__ void k_pt_count(int m, const double* __restrict__ X, PtGeo g, TileGeom t, int* __restrict__ cnt) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l < m) atomicAdd(&cnt[point_bin(X, l, g, t)], 1);
}

// Exclusive scan of n counters in place, one block of 1024 threads.
__global__ void __launch_bounds__(1024) k_pt_scan(int n, int* __restrict__ cnt) {
  __shared__ int wsum[32];
  const int per = (n + blockDim.x - 1) / blockDim.x;
  const int b0 = threadIdx.x * per, b1 = min(n, b0 + per);
  int s = 0;
  for (int i = b0; i < b1; ++i) s += cnt[i];
  // inclusive scan of the per-thread sums across the block
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int v = s;
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  if (lane == 31) wsum[w] = v;
  __syncthreads();
  if (w == 0) {
    int x = wsum[lane];
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += t;
    }
    wsum[lane] = x;
  }
  __syncthreads();
  int run = v - s + (w > 0 ? wsum[w - 1] : 0);   // exclusive prefix of this thread's chunk
  for (int i = b0; i < b1; ++i) {
    const int c = cnt[i];
    cnt[i] = run;
    run += c;
  }
}

__global__ void k_pt_scatter(int m, const double* __restrict__ X, PtGeo g, TileGeom t, int* __restrict__ off,
                             int* __restrict__ perm) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l < m) perm[atomicAdd(&off[point_bin(X, l, g, t)], 1)] = l;
}

PtGeo pt_geo(const ibl_ctx* c) {
  PtGeo g;
  g.D = c->D;
  g.n[0] = c->nx;
  g.n[1] = c->ny;
  g.n[2] = c->nz;
  for (int a = 0; a < 3; ++a) g.per[a] = c->bc[2 * a] == IBL_PERIODIC;
  return g;
}

// Sorted point order in the context's scratch (grown on demand); nullptr
// (identity order) for small clouds, where the sort costs more than it saves.
constexpr int SORT_MIN_POINTS = 4096;
const int* point_order(ibl_ctx* c, int m, const double* X, cudaError_t& e) {
  e = cudaSuccess;
  if (m < SORT_MIN_POINTS) return nullptr;
  const int nb = c->tg.n_tiles;
  if (c->pt_cap < (size_t)m || !c->d_pt_bins) {
    if (c->d_pt_perm) cudaFree(c->d_pt_perm);
    if (c->d_pt_bins) cudaFree(c->d_pt_bins);
    c->d_pt_perm = nullptr;
    c->d_pt_bins = nullptr;
    c->pt_cap = 0;
    e = cudaMalloc(&c->d_pt_perm, sizeof(int) * (size_t)m);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_pt_bins, sizeof(int) * (size_t)nb);
    if (e != cudaSuccess) return nullptr;
    c->pt_cap = (size_t)m;
  }
  const PtGeo g = pt_geo(c);
  e = cudaMemsetAsync(c->d_pt_bins, 0, sizeof(int) * (size_t)nb, c->stream);
  if (e != cudaSuccess) return nullptr;
  const unsigned b = (unsigned)((m + 255) / 256);
  k_pt_count<<<b, 256, 0, c->stream>>>(m, X, g, c->tg, c->d_pt_bins);
  k_pt_scan<<<1, 1024, 0, c->stream>>>(nb, c->d_pt_bins);
  k_pt_scatter<<<b, 256, 0, c->stream>>>(m, X, g, c->tg, c->d_pt_bins, c->d_pt_perm);
  c->launches += 3;
  e = cudaGetLastError();
  return e == cudaSuccess ? c->d_pt_perm : nullptr;
}

// Stencils of the m points in the context's scratch (grown on demand).
bool point_stencils(ibl_ctx* c, int m, const double* X, const int*& base, const df*& wts, cudaError_t& e) {
  e = cudaSuccess;
  if (c->pt_st_cap < (size_t)m) {
    if (c->d_pt_sbase) cudaFree(c->d_pt_sbase);
    if (c->d_pt_swts) cudaFree(c->d_pt_swts);
    c->d_pt_sbase = nullptr;
    c->d_pt_swts = nullptr;
    c->pt_st_cap = 0;
    e = cudaMalloc(&c->d_pt_sbase, sizeof(int) * 3 * (size_t)m);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_pt_swts, sizeof(df) * 12 * (size_t)m);
    if (e != cudaSuccess) return false;
    c->pt_st_cap = (size_t)m;
  }
  int* b = static_cast<int*>(c->d_pt_sbase);
  df* w = static_cast<df*>(c->d_pt_swts);
  k_pt_stencils<<<(unsigned)((3LL * m + 255) / 256), 256, 0, c->stream>>>(m, X, pt_geo(c), b, w, c->d_status + 1);
  c->launches++;
  e = cudaGetLastError();
  base = b;
  wts = w;
  return e == cudaSuccess;
}

unsigned point_blocks(int m) { return (unsigned)(((long long)m * 32 + 255) / 256); }

template <int Q, class T>
void launch_interpolate(ibl_ctx* c, int m, const int* sbase, const df* swts, double* U, double* rho,
                        const int* perm) {
  using R = typename Store<T>::R;
  FluidParams<R> p{};
  p.nx = c->nx;
  p.ny = c->ny;
  p.nz = c->nz;
  p.N = c->N;
  for (int i = 0; i < 6; ++i) p.bc[i] = c->bc[i];
  for (int a = 0; a < 3; ++a) {
    p.u_in[a] = (R)c->u_in[a];
    p.G[a] = (R)c->G[a];
  }
  p.rho_out = (R)c->rho_out;
  p.tg = c->tg;
  p.status = c->d_status;
  const T* src = (const T*)c->f[c->cur];
  const PtGeo g = pt_geo(c);
  const long long nn = c->D == 3 ? 64 : 16;
  if ((long long)m * nn >= c->N) {
    // as many stencil nodes as cells or more: moments once per cell first
    const size_t bytes = 4 * sizeof(R) * (size_t)c->N;
    if (c->pt_mom_bytes < bytes) {
      if (c->d_pt_mom) cudaFree(c->d_pt_mom);
      c->d_pt_mom = nullptr;
      c->pt_mom_bytes = 0;
      if (cudaMalloc(&c->d_pt_mom, bytes) != cudaSuccess) return;   // reported by the caller's error check
      c->pt_mom_bytes = bytes;
    }
    R* mom = static_cast<R*>(c->d_pt_mom);
    const unsigned cb = (unsigned)std::min<long long>((c->N + 255) / 256, 152LL * 16);
    if (c->poststream) k_cell_moments<Q, T, false><<<cb, 256, 0, c->stream>>>(src, p, mom);
    else k_cell_moments<Q, T, true><<<cb, 256, 0, c->stream>>>(src, p, mom);
    k_points_interpolate_cached<R><<<point_blocks(m), 256, 0, c->stream>>>(m, sbase, swts, mom, c->N, g, U, rho,
                                                                           perm);
    c->launches++;
    return;
  }
  if (c->poststream)
    k_points_interpolate<Q, T, false><<<point_blocks(m), 256, 0, c->stream>>>(m, sbase, swts, src, p, g, U, rho,
                                                                               perm);
  else
    k_points_interpolate<Q, T, true><<<point_blocks(m), 256, 0, c->stream>>>(m, sbase, swts, src, p, g, U, rho,
                                                                              perm);
}

template <int Q>
void launch_interpolate_q(ibl_ctx* c, int m, const int* sbase, const df* swts, double* U, double* rho,
                          const int* perm) {
  switch (c->prec) {
    case IBL_FP64: launch_interpolate<Q, double>(c, m, sbase, swts, U, rho, perm); break;
    case IBL_FP32: launch_interpolate<Q, float>(c, m, sbase, swts, U, rho, perm); break;
    case IBL_FP16DEV: launch_interpolate<Q, __half>(c, m, sbase, swts, U, rho, perm); break;
    default: launch_interpolate<Q, __nv_bfloat16>(c, m, sbase, swts, U, rho, perm); break;
  }
}

bool axes_ok(const ibl_ctx* c) {
  const int n[3] = {c->nx, c->ny, c->nz};
  for (int a = 0; a < c->D; ++a)
    if (n[a] < 8) return false;
  return true;
}

// Reads and clears the point-operator flag after the stream drains.
ibl_status finish(ibl_ctx* c, cudaError_t e, const char* what) {
  int flag = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, c->d_status + 1, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_status + 1, 0, sizeof(int), c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_check(c, e, what);
  if (flag & PT_BAD_STENCIL) return fail(c, IBL_EINVAL, "a point's stencil leaves a bounded axis (or is not finite)");
  if (flag & PT_BAD_RANGE) return fail(c, IBL_EINVAL, "|V ds| exceeds the fixed-point range of the spreading");
  return IBL_OK;
}

}  // namespace
}  // namespace ibl

using namespace ibl;

extern "C" {

ibl_status ibl_interpolate_points(ibl_ctx* c, int32_t m, const double* d_X, double* d_U, double* d_rho) {
  if (!c) return IBL_EINVAL;
  if (m < 0 || (m > 0 && (!d_X || !d_U))) return fail(c, IBL_EINVAL, "ibl_interpolate_points: bad arguments");
  if (!axes_ok(c)) return fail(c, IBL_EINVAL, "axes carrying points need at least 8 nodes");
  if (!c->initialised) return fail(c, IBL_ESTATE, "fluid not initialised");
  const ibl_status s = sync_and_collect(c);
  if (s != IBL_OK && s != IBL_ENOTCONV) return s;
  if (m == 0) return s;
  cudaError_t pe;
  const int* perm = point_order(c, m, d_X, pe);
  if (pe != cudaSuccess) return cuda_check(c, pe, "ibl_interpolate_points: point order");
  const int* sbase = nullptr;
  const df* swts = nullptr;
  if (!point_stencils(c, m, d_X, sbase, swts, pe)) return cuda_check(c, pe, "ibl_interpolate_points: stencils");
  if (c->Q == 9) launch_interpolate_q<9>(c, m, sbase, swts, d_U, d_rho, perm);
  else launch_interpolate_q<19>(c, m, sbase, swts, d_U, d_rho, perm);
  c->launches++;
  const ibl_status r = finish(c, cudaGetLastError(), "ibl_interpolate_points");
  return r != IBL_OK ? r : s;
}

ibl_status ibl_spread_points(ibl_ctx* c, int32_t m, const double* d_X, const double* d_V, const double* d_ds,
                             double* d_out) {
  if (!c) return IBL_EINVAL;
  if (m < 0 || !d_out || (m > 0 && (!d_X || !d_V || !d_ds)))
    return fail(c, IBL_EINVAL, "ibl_spread_points: bad arguments");
  if (!axes_ok(c)) return fail(c, IBL_EINVAL, "axes carrying points need at least 8 nodes");
  const ibl_status s = sync_and_collect(c);
  if (s != IBL_OK && s != IBL_ENOTCONV) return s;
  const long long tot = (long long)c->D * c->N;
  unsigned long long* acc = reinterpret_cast<unsigned long long*>(d_out);
  cudaError_t e = cudaMemsetAsync(d_out, 0, sizeof(double) * tot, c->stream);
  const int* perm = nullptr;
  const int* sbase = nullptr;
  const df* swts = nullptr;
  if (e == cudaSuccess && m > 0) perm = point_order(c, m, d_X, e);
  if (e == cudaSuccess && m > 0) point_stencils(c, m, d_X, sbase, swts, e);
  if (e == cudaSuccess && m > 0) {
    k_points_spread<<<point_blocks(m), 256, 0, c->stream>>>(m, sbase, swts, d_V, d_ds, pt_geo(c), c->N, acc,
                                                            c->d_status + 1, perm);
    c->launches++;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    k_fixed_to_double<<<152 * 8, 256, 0, c->stream>>>(acc, tot);
    c->launches++;
    e = cudaGetLastError();
  }
  const ibl_status r = finish(c, e, "ibl_spread_points");
  return r != IBL_OK ? r : s;
}

}  // extern "C"
