// Stand-alone immersed-boundary transfers on an arbitrary point cloud: the
// interpolation of Eq. 17 and the spreading of Eq. 15 on device arrays,
// without the implicit solve.  They run the same per-node arithmetic as the
// IB step (stencil_axis, node_rho_u), one warp per point.
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

// Stencil of point l: bases and per-axis weights; false (flag set) if it
// leaves a bounded axis, in which case the caller touches no memory.
__device__ __forceinline__ bool point_stencil(const PtGeo& g, const double* X, int l, int b[3],
                                              double w[3][4], int* flag) {
  bool ok = true;
  for (int a = 0; a < 3; ++a) {
    if (a < g.D) {
      ok &= stencil_axis(X[3 * l + a], g.n[a], g.per[a] != 0, b[a], w[a]);
    } else {
      b[a] = 0;
      w[a][0] = 1.0;
      w[a][1] = w[a][2] = w[a][3] = 0.0;
    }
  }
  if (!ok) atomicOr(flag, PT_BAD_STENCIL);
  return ok;
}

__device__ __forceinline__ long long stencil_node(const PtGeo& g, const int b[3], int k, int node[3]) {
  const int i = k & 3, j = (k >> 2) & 3, q = k >> 4;
  node[0] = b[0] + i;
  node[1] = b[1] + j;
  node[2] = g.D == 3 ? b[2] + q : 0;
  for (int a = 0; a < g.D; ++a)
    if (g.per[a]) node[a] = wrap_once(node[a], g.n[a]);
  return ((long long)node[2] * g.n[1] + node[1]) * g.n[0] + node[0];
}

template <int Q, class T, bool PULL>
__global__ void k_points_interpolate(int m, const double* __restrict__ X, const T* __restrict__ src,
                                     FluidParams<typename Store<T>::R> p, PtGeo g, double* __restrict__ U,
                                     double* __restrict__ rho_out, int* flag) {
  const int l = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (l >= m) return;
  int b[3];
  double w[3][4];
  if (!point_stencil(g, X, l, b, w, flag)) return;
  const int nn = g.D == 3 ? 64 : 16;
  double acc[4] = {0, 0, 0, 0};
  for (int k = lane; k < nn; k += 32) {
    int node[3];
    const long long cell = stencil_node(g, b, k, node);
    const double wt = w[0][k & 3] * w[1][(k >> 2) & 3] * w[2][g.D == 3 ? k >> 4 : 0];
    double rho, u[3];
    node_rho_u<Q, T, PULL>(src, node[0], node[1], node[2], cell, p, rho, u);
    acc[0] += wt * rho;
    acc[1] += wt * u[0];
    acc[2] += wt * u[1];
    acc[3] += wt * u[2];
  }
  for (int o = 16; o > 0; o >>= 1)
    for (int c = 0; c < 4; ++c) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
  if (lane == 0) {
    if (rho_out) rho_out[l] = acc[0];
    for (int a = 0; a < g.D; ++a) U[(long long)g.D * l + a] = acc[1 + a];
  }
}

// Fixed-point scatter into the caller's output array reinterpreted as int64
// (the same 8 bytes per entry): integer sums do not depend on atomic order.
__global__ void k_points_spread(int m, const double* __restrict__ X, const double* __restrict__ V,
                                const double* __restrict__ ds, PtGeo g, long long N,
                                unsigned long long* __restrict__ acc, int* flag) {
  const int l = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (l >= m) return;
  int b[3];
  double w[3][4];
  if (!point_stencil(g, X, l, b, w, flag)) return;
  double v[3] = {0, 0, 0};
  for (int a = 0; a < g.D; ++a) v[a] = V[(long long)g.D * l + a] * ds[l];
  const int nn = g.D == 3 ? 64 : 16;
  for (int k = lane; k < nn; k += 32) {
    int node[3];
    const long long cell = stencil_node(g, b, k, node);
    const double wt = w[0][k & 3] * w[1][(k >> 2) & 3] * w[2][g.D == 3 ? k >> 4 : 0];
    for (int c = 0; c < g.D; ++c) {
      const double val = wt * v[c];
      if (!(fabs(val) < PT_FIX_LIMIT)) {
        atomicOr(flag, PT_BAD_RANGE);
        continue;
      }
      atomicAdd(acc + c * N + cell, (unsigned long long)__double2ll_rn(val * PT_FIX_SCALE));
    }
  }
}

__global__ void k_fixed_to_double(unsigned long long* a, long long n) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    reinterpret_cast<double*>(a)[i] = (double)(long long)a[i] * (1.0 / PT_FIX_SCALE);
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

unsigned point_blocks(int m) { return (unsigned)(((long long)m * 32 + 255) / 256); }

template <int Q, class T>
void launch_interpolate(ibl_ctx* c, int m, const double* X, double* U, double* rho, int* flag) {
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
  if (c->poststream)
    k_points_interpolate<Q, T, false><<<point_blocks(m), 256, 0, c->stream>>>(m, X, src, p, g, U, rho, flag);
  else
    k_points_interpolate<Q, T, true><<<point_blocks(m), 256, 0, c->stream>>>(m, X, src, p, g, U, rho, flag);
}

template <int Q>
void launch_interpolate_q(ibl_ctx* c, int m, const double* X, double* U, double* rho, int* flag) {
  switch (c->prec) {
    case IBL_FP64: launch_interpolate<Q, double>(c, m, X, U, rho, flag); break;
    case IBL_FP32: launch_interpolate<Q, float>(c, m, X, U, rho, flag); break;
    case IBL_FP16DEV: launch_interpolate<Q, __half>(c, m, X, U, rho, flag); break;
    default: launch_interpolate<Q, __nv_bfloat16>(c, m, X, U, rho, flag); break;
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
  if (c->Q == 9) launch_interpolate_q<9>(c, m, d_X, d_U, d_rho, c->d_status + 1);
  else launch_interpolate_q<19>(c, m, d_X, d_U, d_rho, c->d_status + 1);
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
  if (e == cudaSuccess && m > 0) {
    k_points_spread<<<point_blocks(m), 256, 0, c->stream>>>(m, d_X, d_V, d_ds, pt_geo(c), c->N, acc,
                                                            c->d_status + 1);
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
