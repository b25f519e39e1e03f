// Per-marker pieces of the IB transfers shared by the step's kernels and the
// stand-alone point operators: the stencil of Eq. 14 along one axis and the
// moments (Eq. 11) of one node's post-streaming populations.
#pragma once

#include "df.cuh"
#include "lbm_gather.cuh"

namespace ibl {

// Eq. 14 at the four nodes base..base+3 of one axis for a point at x.  With
// s = x - floor(x) the nodes sit at |r| = 1+s, s, 1-s, 2-s, whose
// cos(pi |r| / 2) are -sin, cos, sin, -cos of (pi s / 2).  A periodic axis
// reduces the base into [0, n) so that node offsets wrap once at most.  On a
// bounded axis a stencil that leaves [0, n), or a non-finite x, returns false
// and the base is clamped into [0, n - 4], so that no later access leaves the
// arrays (n >= 8 on every axis that carries points).
__device__ __forceinline__ bool stencil_axis(double x, int n, bool per, int& base, double w[4]) {
  const bool finite = isfinite(x);
  const double xx = finite ? x : 0.0;
  const double fl = floor(xx);
  double sn, cs;
  sincospi(0.5 * (xx - fl), &sn, &cs);
  w[0] = 0.25 * (1.0 - sn);
  w[1] = 0.25 * (1.0 + cs);
  w[2] = 0.25 * (1.0 + sn);
  w[3] = 0.25 * (1.0 - cs);
  if (per) {
    double r = fmod(fl - 1.0, (double)n);
    if (r < 0.0) r += (double)n;
    base = (int)r;
    return finite;
  }
  base = (int)fmin(fmax(fl - 1.0, 0.0), (double)(n - 4));
  return finite && fl - 1.0 >= 0.0 && fl + 2.0 < (double)n;
}

// Fused multiply-add rounded once, with no room for the compiler to round
// differently in different kernels (the point operators compute a node's
// moments either inside the interpolation or once per cell beforehand, and
// both must give the same bits).
__device__ __forceinline__ float rn_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double rn_fma(double a, double b, double c) { return __fma_rn(a, b, c); }

// drho and u* of one node from its post-streaming deviations, in the
// storage's compute precision (Eq. 11 with the uniform body force G:
// u* = (m + G/2) / rho, formed as m - m drho / rho).
template <int Q, class T, bool PULL>
__device__ __forceinline__ void node_moments(const T* __restrict__ src, int x, int y, int z, long long cell,
                                             const FluidParams<typename Store<T>::R>& p,
                                             typename Store<T>::R& drho_out, typename Store<T>::R u[3]) {
  using R = typename Store<T>::R;
  R gg[Q];
  gather_q<Q, T, PULL, R>(src, x, y, z, cell, p, gg);
  R drho = gg[0], m0 = R(0), m1 = R(0), m2 = R(0);
#pragma unroll
  for (int e = 1; e < Q; e += 2) {
    drho += gg[e] + gg[e + 1];
    const R d = gg[e] - gg[e + 1];
    if (Lat<Q>::cx(e)) m0 += R(Lat<Q>::cx(e)) * d;
    if (Lat<Q>::cy(e)) m1 += R(Lat<Q>::cy(e)) * d;
    if (Lat<Q>::cz(e)) m2 += R(Lat<Q>::cz(e)) * d;
  }
  const R qd = drho / (R(1) + drho);
  R u0 = rn_fma(R(0.5), p.G[0], m0), u1 = rn_fma(R(0.5), p.G[1], m1), u2 = rn_fma(R(0.5), p.G[2], m2);
  u0 = rn_fma(-u0, qd, u0);
  u1 = rn_fma(-u1, qd, u1);
  u2 = rn_fma(-u2, qd, u2);
  drho_out = drho;
  u[0] = u0;
  u[1] = u1;
  u[2] = u2;
}

// The same moments as FP64 rho and u*.
template <int Q, class T, bool PULL>
__device__ __forceinline__ void node_rho_u(const T* __restrict__ src, int x, int y, int z, long long cell,
                                           const FluidParams<typename Store<T>::R>& p, double& rho,
                                           double u[3]) {
  typename Store<T>::R drho, uu[3];
  node_moments<Q, T, PULL>(src, x, y, z, cell, p, drho, uu);
  rho = 1.0 + (double)drho;
  u[0] = (double)uu[0];
  u[1] = (double)uu[1];
  u[2] = (double)uu[2];
}

// A storage-precision value as a double-float (exact).
__device__ __forceinline__ df to_df(float v) { return df_from_float(v); }
__device__ __forceinline__ df to_df(double v) { return df_from_double(v); }

}  // namespace ibl
