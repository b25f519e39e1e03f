// Set-up and rebuild of the separable preconditioner (sep.cuh holds the
// derivation and the application used by the solve kernel).
//
//   sep_detect        host: does a body's marker set factor into chord x
//                     span positions with the rotation axis along z?  Index
//                     maps of the bounding rectangle (set-up bookkeeping).
//   k_sep_span_eigen  once per context: the span factor Z (Eq. 18's overlap
//                     sum along z, fixed while the body turns about z) and
//                     its eigen-decomposition by cyclic Jacobi rotations in
//                     FP64, one block per body.
//   k_sep_rebuild     at every scheduled rebuild: the chord factor C
//                     (overlap sums in the plane of rotation), the per-mode
//                     blocks H_j = (lambda_j C + sigma I)^-1, the Schur block
//                     S = (K^-1)_cc and its inverse by blocked Gauss-Jordan,
//                     all in FP64 (S has condition numbers of ~5e5 at 2 x 6292
//                     markers; FP32 elimination loses it); V and H_j are
//                     stored in FP32, S^-1 as double-float pairs.
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <utility>
#include <vector>

#include "ibl_internal.cuh"
#include "sep.cuh"

namespace cg = cooperative_groups;

namespace ibl {

constexpr int SEP_THREADS = 256;
constexpr int GJ64_NB = 32;              // pivot block and tile edge of the FP64 elimination
constexpr int GJ64_LD = GJ64_NB + 1;     // padded shared-memory row
constexpr int JACOBI_MAX_SWEEPS = 40;
// Relative shift of the separable preconditioner (see the rebuild).  Emulated
// on the 2 x 6292-marker wings (zero initial guess, tolerance 1e-7): 1e-6
// takes 31-57 iterations, 2e-7 16-28; at 1e-7 the preconditioned residual
// no longer tracks the error (the stopping test stops firing first).
constexpr double SEP_SHIFT = 2e-7;

// Overlap sum of two markers' stencils along axis a in FP64 (the 1D factor of
// an Eq. 18 entry): sum_o w_l[o] w_k[o - d], d the minimal-image difference
// of the stencil bases; 0 when the stencils do not meet.
__device__ double axis_overlap(const int* __restrict__ base, const df* __restrict__ wts, int l, int k, int a,
                               int n, int per) {
  int d = base[3 * k + a] - base[3 * l + a];
  if (per) {
    if (d < 0) d += n;
    else if (d >= n) d -= n;
    if (d > n / 2) d -= n;
  }
  if (d < -3 || d > 3) return 0.0;
  const int o0 = d > 0 ? d : 0, o1 = d < 0 ? 3 + d : 3;
  double s = 0.0;
  for (int o = o0; o <= o1; ++o)
    s += df_to_double(wts[12 * l + 4 * a + o]) * df_to_double(wts[12 * k + 4 * a + (o - d)]);
  return s;
}

// --------------------------------------------------------------- span factor
// Z[k][k2] = overlap along z of the span positions' stencils, then Z = V
// diag(lambda) V^T by cyclic Jacobi rotations: each round applies n/2
// disjoint rotations (round-robin pairing), rows first, then columns and V.
__global__ void __launch_bounds__(1024) k_sep_span_eigen(SepBody* sb, const int* __restrict__ boff,
                                                         const int* __restrict__ base, const df* __restrict__ wts,
                                                         int nz, int perz) {
  SepBody& B = sb[blockIdx.x];
  const int n = B.nk, o = boff[blockIdx.x];
  double* A = B.Z64;
  double* V = B.V64;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int k = e / n, k2 = e - k * n;
    A[e] = axis_overlap(base, wts, o + B.rep_k[k], o + B.rep_k[k2], 2, nz, perz);
    V[e] = k == k2 ? 1.0 : 0.0;
  }
  __shared__ int pp[SEP_NK_MAX / 2 + 1], qq[SEP_NK_MAX / 2 + 1];
  __shared__ double cs[SEP_NK_MAX / 2 + 1], sn[SEP_NK_MAX / 2 + 1];
  __shared__ double red[32];
  __shared__ int s_more;
  const int N = (n + 1) & ~1;   // even count; index n (when n is odd) is a dummy
  const int npair = N / 2;
  __syncthreads();
  for (int sweep = 0; sweep < JACOBI_MAX_SWEEPS; ++sweep) {
    for (int r = 0; r < N - 1; ++r) {
      // round r of the round-robin: position 0 fixed, the others rotated
      for (int t = threadIdx.x; t < npair; t += blockDim.x) {
        auto at = [&](int pos) { return pos == 0 ? 0 : 1 + (pos - 1 + r) % (N - 1); };
        int p = at(t), q = at(N - 1 - t);
        if (p > q) { const int w = p; p = q; q = w; }
        double c = 1.0, s = 0.0;
        if (q < n) {
          const double apq = A[p * n + q];
          if (apq != 0.0) {
            const double th = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
            const double tt = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
            c = 1.0 / sqrt(tt * tt + 1.0);
            s = tt * c;
          }
        }
        pp[t] = p;
        qq[t] = q < n ? q : p;
        cs[t] = c;
        sn[t] = q < n ? s : 0.0;
      }
      __syncthreads();
      // rows: A <- P^T A
      for (int e = threadIdx.x; e < npair * n; e += blockDim.x) {
        const int t = e / n, j = e - t * n;
        const int p = pp[t], q = qq[t];
        if (p == q) continue;
        const double c = cs[t], s = sn[t];
        const double ap = A[p * n + j], aq = A[q * n + j];
        A[p * n + j] = c * ap - s * aq;
        A[q * n + j] = s * ap + c * aq;
      }
      __syncthreads();
      // columns: A <- A P and V <- V P
      for (int e = threadIdx.x; e < npair * n; e += blockDim.x) {
        const int t = e / n, i = e - t * n;
        const int p = pp[t], q = qq[t];
        if (p == q) continue;
        const double c = cs[t], s = sn[t];
        const double ap = A[i * n + p], aq = A[i * n + q];
        A[i * n + p] = c * ap - s * aq;
        A[i * n + q] = s * ap + c * aq;
        const double vp = V[i * n + p], vq = V[i * n + q];
        V[i * n + p] = c * vp - s * vq;
        V[i * n + q] = s * vp + c * vq;
      }
      __syncthreads();
    }
    // convergence: off-diagonal against the whole Frobenius norm
    double off = 0.0, all = 0.0;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      const double v = A[e] * A[e];
      all += v;
      if (e / n != e % n) off += v;
    }
    for (int w = 16; w > 0; w >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, w);
      all += __shfl_xor_sync(0xffffffffu, all, w);
    }
    if ((threadIdx.x & 31) == 0) {
      red[threadIdx.x >> 5] = off;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double o2 = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) o2 += red[w];
      red[31] = o2;
    }
    __syncthreads();
    const double off_tot = red[31];
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = all;
    __syncthreads();
    if (threadIdx.x == 0) {
      double a2 = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a2 += red[w];
      s_more = off_tot > 1e-26 * a2 ? 1 : 0;
    }
    __syncthreads();
    if (!s_more) break;
  }
  for (int k = threadIdx.x; k < n; k += blockDim.x) B.lam[k] = A[k * n + k];
  const int ldv = sep_ldv(n);
  for (int e = threadIdx.x; e < n * ldv; e += blockDim.x) {
    const int k = e / ldv, j = e % ldv;
    B.V[e] = j < n ? (float)V[k * n + j] : 0.f;
  }
}

// --------------------------------------------------------------- rebuild
struct SepRebuildArgs {
  SepBody* sb;
  int nb;
  const int* boff;
  const int* base;
  const df* wts;
  int n[3], per[3];
  const unsigned long long* rowsum_max;   // per body, FP64 bits: the shift's scale
};

// In-place Gauss-Jordan inverse of a kn x kn block in shared memory (row
// stride ld), no pivoting (the matrices are symmetric positive definite).
__device__ void gj_small_inplace(double* M, int kn, int ld) {
  for (int k = 0; k < kn; ++k) {
    __syncthreads();
    const double pk = 1.0 / M[k * ld + k];
    __syncthreads();
    for (int e = threadIdx.x; e < kn * kn; e += blockDim.x) {
      const int i = e / kn, j = e - i * kn;
      if (i == k || j == k) continue;
      M[i * ld + j] -= M[i * ld + k] * M[k * ld + j] * pk;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < kn; j += blockDim.x) {
      if (j == k) continue;
      M[k * ld + j] *= pk;    // row k
    }
    for (int i = threadIdx.x; i < kn; i += blockDim.x) {
      if (i == k) continue;
      M[i * ld + k] *= -pk;   // column k
    }
    __syncthreads();
    if (threadIdx.x == 0) M[k * ld + k] = pk;
  }
  __syncthreads();
}

// out (32 x 32 tile, row stride ldo) = alpha * A (32 x K) * B (K x 32) [+ out],
// A and B staged in shared memory with row stride GJ64_LD.
__device__ __forceinline__ void tile64_mma(const double* As, const double* Bs, int K, double acc[4]) {
  const int r = threadIdx.x >> 3, c0 = (threadIdx.x & 7) << 2;
  for (int e = 0; e < 4; ++e) acc[e] = 0.0;
  for (int q = 0; q < K; ++q) {
    const double a = As[r * GJ64_LD + q];
#pragma unroll
    for (int e = 0; e < 4; ++e) acc[e] = fma(a, Bs[q * GJ64_LD + c0 + e], acc[e]);
  }
}

__device__ void load_tile64(double* dst, const double* S, int ld, int r0, int c0, int nr, int nc) {
  for (int e = threadIdx.x; e < GJ64_NB * GJ64_NB; e += blockDim.x) {
    const int r = e >> 5, c = e & 31;
    dst[r * GJ64_LD + c] = (r < nr && c < nc) ? __ldcg(S + (long long)(r0 + r) * ld + c0 + c) : 0.0;
  }
}

// Blocked Gauss-Jordan inverse, in place, of every body's S64 (n_c x n_c,
// row stride n_c), all bodies at once; four grid-wide phases per pivot block.
__device__ void gj64_all(const SepRebuildArgs& R, cg::grid_group& grid, double* sm) {
  double* T0 = sm;
  double* T1 = sm + GJ64_NB * GJ64_LD;
  double* T2 = sm + 2 * GJ64_NB * GJ64_LD;
  int maxt = 0;
  for (int b = 0; b < R.nb; ++b) maxt = max(maxt, (R.sb[b].nc + GJ64_NB - 1) / GJ64_NB);
  const int r = threadIdx.x >> 3, c0 = (threadIdx.x & 7) << 2;
  for (int kb = 0; kb < maxt; ++kb) {
    const int k0 = kb * GJ64_NB;
    // P1: pivot block inverse (body b by block b)
    for (int b = blockIdx.x; b < R.nb; b += gridDim.x) {
      const SepBody& B = R.sb[b];
      if (k0 >= B.nc) continue;
      const int kn = min(GJ64_NB, B.nc - k0);
      load_tile64(T0, B.S64, B.nc, k0, k0, kn, kn);
      __syncthreads();
      gj_small_inplace(T0, kn, GJ64_LD);
      for (int e = threadIdx.x; e < kn * kn; e += blockDim.x) {
        const int i = e / kn, j = e - i * kn;
        B.S64[(long long)(k0 + i) * B.nc + k0 + j] = T0[i * GJ64_LD + j];
      }
      __syncthreads();
    }
    grid.sync();
    // P2: row panel R <- P^-1 R (tiles of 32 columns outside the pivot block)
    {
      long long item = blockIdx.x;
      for (int b = 0; b < R.nb; ++b) {
        const SepBody& B = R.sb[b];
        const int nt = (B.nc + GJ64_NB - 1) / GJ64_NB;
        if (k0 >= B.nc) { continue; }
        const int kn = min(GJ64_NB, B.nc - k0);
        for (; item < nt; item += gridDim.x) {
          const int jt = (int)item;
          if (jt == kb) continue;
          const int j0 = jt * GJ64_NB, nj = min(GJ64_NB, B.nc - j0);
          __syncthreads();
          load_tile64(T0, B.S64, B.nc, k0, k0, kn, kn);
          load_tile64(T1, B.S64, B.nc, k0, j0, kn, nj);
          __syncthreads();
          double acc[4];
          tile64_mma(T0, T1, kn, acc);
          __syncthreads();
          for (int e = 0; e < 4; ++e)
            if (r < kn && c0 + e < nj) B.S64[(long long)(k0 + r) * B.nc + j0 + c0 + e] = acc[e];
        }
        item -= nt;
      }
    }
    grid.sync();
    // P3: trailing update S <- S - C R (tiles outside the pivot rows and columns)
    {
      long long item = blockIdx.x;
      for (int b = 0; b < R.nb; ++b) {
        const SepBody& B = R.sb[b];
        const int nt = (B.nc + GJ64_NB - 1) / GJ64_NB;
        if (k0 >= B.nc) { continue; }
        const int kn = min(GJ64_NB, B.nc - k0);
        const long long cnt = (long long)nt * nt;
        for (; item < cnt; item += gridDim.x) {
          const int it = (int)(item / nt), jt = (int)(item % nt);
          if (it == kb || jt == kb) continue;
          const int i0 = it * GJ64_NB, ni = min(GJ64_NB, B.nc - i0);
          const int j0 = jt * GJ64_NB, nj = min(GJ64_NB, B.nc - j0);
          __syncthreads();
          load_tile64(T0, B.S64, B.nc, i0, k0, ni, kn);   // C
          load_tile64(T1, B.S64, B.nc, k0, j0, kn, nj);   // R (updated)
          load_tile64(T2, B.S64, B.nc, i0, j0, ni, nj);
          __syncthreads();
          double acc[4];
          tile64_mma(T0, T1, kn, acc);
          for (int e = 0; e < 4; ++e)
            if (r < ni && c0 + e < nj)
              B.S64[(long long)(i0 + r) * B.nc + j0 + c0 + e] = T2[r * GJ64_LD + c0 + e] - acc[e];
        }
        item -= cnt;
      }
    }
    grid.sync();
    // P4: column panel C <- -C P^-1
    {
      long long item = blockIdx.x;
      for (int b = 0; b < R.nb; ++b) {
        const SepBody& B = R.sb[b];
        const int nt = (B.nc + GJ64_NB - 1) / GJ64_NB;
        if (k0 >= B.nc) { continue; }
        const int kn = min(GJ64_NB, B.nc - k0);
        for (; item < nt; item += gridDim.x) {
          const int it = (int)item;
          if (it == kb) continue;
          const int i0 = it * GJ64_NB, ni = min(GJ64_NB, B.nc - i0);
          __syncthreads();
          load_tile64(T0, B.S64, B.nc, i0, k0, ni, kn);
          load_tile64(T1, B.S64, B.nc, k0, k0, kn, kn);
          __syncthreads();
          double acc[4];
          tile64_mma(T0, T1, kn, acc);
          __syncthreads();
          for (int e = 0; e < 4; ++e)
            if (r < ni && c0 + e < kn) B.S64[(long long)(i0 + r) * B.nc + k0 + c0 + e] = -acc[e];
        }
        item -= nt;
      }
    }
    grid.sync();
  }
}

__global__ void __launch_bounds__(SEP_THREADS) k_sep_rebuild(SepRebuildArgs R) {
  cg::grid_group grid = cg::this_grid();
  extern __shared__ __align__(16) double smd[];
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nthreads = gridDim.x * blockDim.x;
  // chord factor C (FP64): overlaps in the plane of rotation (axes x, y)
  {
    long long tot = 0;
    for (int b = 0; b < R.nb; ++b) tot += (long long)R.sb[b].ni * R.sb[b].ni;
    for (long long e = gtid; e < tot; e += nthreads) {
      long long li = e;
      int b = 0;
      while (li >= (long long)R.sb[b].ni * R.sb[b].ni) { li -= (long long)R.sb[b].ni * R.sb[b].ni; ++b; }
      const SepBody& B = R.sb[b];
      const int i = (int)(li / B.ni), i2 = (int)(li % B.ni);
      const int l = R.boff[b] + B.rep_i[i], k = R.boff[b] + B.rep_i[i2];
      B.C64[li] = axis_overlap(R.base, R.wts, l, k, 0, R.n[0], R.per[0]) *
                  axis_overlap(R.base, R.wts, l, k, 1, R.n[1], R.per[1]);
    }
  }
  grid.sync();
  // per span mode j: H_j = (lambda_j C + sigma I)^-1, sigma = SEP_SHIFT times
  // the largest absolute row sum of the system (the dense path's FP32
  // inverse needs 1e-6; with the Schur block in double-float a smaller shift
  // is safe here and cuts the iterations by about 40 %)
  {
    long long tot = 0;
    for (int b = 0; b < R.nb; ++b) tot += R.sb[b].nk;
    for (long long e = blockIdx.x; e < tot; e += gridDim.x) {
      long long j = e;
      int b = 0;
      while (j >= R.sb[b].nk) { j -= R.sb[b].nk; ++b; }
      const SepBody& B = R.sb[b];
      const int ni = B.ni, ld = SEP_NI_MAX + 1;
      const double sigma = SEP_SHIFT * __longlong_as_double((long long)R.rowsum_max[b]);
      const double lj = B.lam[j];
      __syncthreads();
      for (int q = threadIdx.x; q < ni * ni; q += blockDim.x) {
        const int i = q / ni, i2 = q - i * ni;
        smd[i * ld + i2] = lj * B.C64[q] + (i == i2 ? sigma : 0.0);
      }
      __syncthreads();
      gj_small_inplace(smd, ni, ld);
      for (int q = threadIdx.x; q < ni * ni; q += blockDim.x) {
        const int i = q / ni, i2 = q - i * ni;
        const double h = smd[i * ld + i2];
        B.H64[(long long)j * ni * ni + q] = h;
        B.Ht[((long long)j * ni + i2) * ni + i] = (float)h;
      }
    }
  }
  grid.sync();
  // Schur block S[p][q] = sum_j V[k_p][j] V[k_q][j] H_j[i_p][i_q] (FP64)
  {
    long long tot = 0;
    for (int b = 0; b < R.nb; ++b) tot += (long long)R.sb[b].nc * R.sb[b].nc;
    for (long long e = gtid; e < tot; e += nthreads) {
      long long li = e;
      int b = 0;
      while (li >= (long long)R.sb[b].nc * R.sb[b].nc) { li -= (long long)R.sb[b].nc * R.sb[b].nc; ++b; }
      const SepBody& B = R.sb[b];
      const int p = (int)(li / B.nc), q = (int)(li % B.nc);
      const int rp = B.crect[p], rq = B.crect[q];
      const int ip = rp / B.nk, kp = rp - ip * B.nk, iq = rq / B.nk, kq = rq - iq * B.nk;
      const double* vp = B.V64 + (long long)kp * B.nk;
      const double* vq = B.V64 + (long long)kq * B.nk;
      const double* h = B.H64 + (long long)ip * B.ni + iq;
      double s = 0.0;
      for (int j = 0; j < B.nk; ++j) s = fma(vp[j] * vq[j], h[(long long)j * B.ni * B.ni], s);
      B.S64[li] = s;
    }
  }
  grid.sync();
  gj64_all(R, grid, smd);
  // double-float copy (hi, lo pairs) with zero padding up to the row stride
  {
    long long tot = 0;
    for (int b = 0; b < R.nb; ++b) tot += (long long)R.sb[b].nc * R.sb[b].ldc;
    for (long long e = gtid; e < tot; e += nthreads) {
      long long li = e;
      int b = 0;
      while (li >= (long long)R.sb[b].nc * R.sb[b].ldc) { li -= (long long)R.sb[b].nc * R.sb[b].ldc; ++b; }
      const SepBody& B = R.sb[b];
      const int p = (int)(li / B.ldc), q = (int)(li % B.ldc);
      const df v = q < B.nc ? df_from_double(__ldcg(B.S64 + (long long)p * B.nc + q)) : df_make(0.f, 0.f);
      B.Sinv[2 * li] = v.hi;
      B.Sinv[2 * li + 1] = v.lo;
    }
  }
}

// --------------------------------------------------------------- host side
// A body's marker set is separable when the rotation axis is the grid's z
// axis, every marker's body-frame (x, y) takes one of n_i values and z one of
// n_k values, and no (x, y, z) repeats.  Exact comparisons: the mesh
// generator places the markers at exact multiples of the spacing.
struct SepHost {
  int ni = 0, nk = 0, nc = 0, m = 0;
  std::vector<int> rect, mrect, crect, rep_i, rep_k;
};

static bool sep_detect(const ibl_ctx* c, const Body& b, SepHost& h) {
  if (c->D != 3 || b.axis[0] != 0.0 || b.axis[1] != 0.0) return false;
  const double* X0 = c->h_X0.data() + 3 * (size_t)b.offset;
  std::map<std::pair<double, double>, int> ci;
  std::map<double, int> ck;
  for (int l = 0; l < b.m; ++l) {
    ci.emplace(std::make_pair(X0[3 * l], X0[3 * l + 1]), 0);
    ck.emplace(X0[3 * l + 2], 0);
  }
  if ((int)ci.size() > SEP_NI_MAX || (int)ck.size() > SEP_NK_MAX) return false;
  int t = 0;
  for (auto& kv : ci) kv.second = t++;
  t = 0;
  for (auto& kv : ck) kv.second = t++;
  h.ni = (int)ci.size();
  h.nk = (int)ck.size();
  h.m = b.m;
  h.rect.assign((size_t)h.ni * h.nk, INT32_MIN);
  h.mrect.resize(b.m);
  h.rep_i.assign(h.ni, -1);
  h.rep_k.assign(h.nk, -1);
  for (int l = 0; l < b.m; ++l) {
    const int i = ci[std::make_pair(X0[3 * l], X0[3 * l + 1])], k = ck[X0[3 * l + 2]];
    const int r = i * h.nk + k;
    if (h.rect[r] != INT32_MIN) return false;   // two markers at one mesh point
    h.rect[r] = l;
    h.mrect[l] = r;
    if (h.rep_i[i] < 0) h.rep_i[i] = l;
    if (h.rep_k[k] < 0) h.rep_k[k] = l;
  }
  h.crect.clear();
  for (int r = 0; r < h.ni * h.nk; ++r)
    if (h.rect[r] == INT32_MIN) {
      h.rect[r] = -(int)h.crect.size() - 1;
      h.crect.push_back(r);
    }
  h.nc = (int)h.crect.size();
  return true;
}

bool sep_all_separable(const ibl_ctx* c, int* max_markers) {
  int mx = 0;
  for (const auto& b : c->bodies) {
    SepHost h;
    if (!sep_detect(c, b, h)) return false;
    mx = std::max(mx, b.m);
  }
  if (max_markers) *max_markers = mx;
  return !c->bodies.empty();
}

#define SEP_CU(x)                       \
  do {                                  \
    cudaError_t e_ = (x);               \
    if (e_ != cudaSuccess) return e_;   \
  } while (0)

template <class T>
static cudaError_t sep_upload(ibl_ctx* c, T** dst, const T* src, size_t n) {
  void* p = nullptr;
  SEP_CU(cudaMalloc(&p, sizeof(T) * std::max<size_t>(n, 1)));
  c->sep_allocs.push_back(p);
  *dst = static_cast<T*>(p);
  if (src && n) SEP_CU(to_device(c, p, src, sizeof(T) * n));
  return cudaSuccess;
}

cudaError_t sep_alloc(ibl_ctx* c) {
  sep_free(c);
  std::vector<SepBody> tab;
  for (const auto& b : c->bodies) {
    SepHost h;
    if (!sep_detect(c, b, h)) return cudaErrorInvalidValue;
    SepBody s{};
    s.ni = h.ni; s.nk = h.nk; s.nc = h.nc; s.m = h.m;
    s.ldc = std::max(4, (h.nc + 3) & ~3);
    const size_t rect = (size_t)h.ni * h.nk;
    int* ip = nullptr;
    SEP_CU(sep_upload(c, &ip, h.rect.data(), rect)); s.rect = ip;
    SEP_CU(sep_upload(c, &ip, h.mrect.data(), h.mrect.size())); s.mrect = ip;
    SEP_CU(sep_upload(c, &ip, h.crect.data(), h.crect.size())); s.crect = ip;
    SEP_CU(sep_upload(c, &ip, h.rep_i.data(), h.rep_i.size())); s.rep_i = ip;
    SEP_CU(sep_upload(c, &ip, h.rep_k.data(), h.rep_k.size())); s.rep_k = ip;
    SEP_CU(sep_upload<float>(c, &s.V, nullptr, (size_t)h.nk * sep_ldv(h.nk)));
    SEP_CU(sep_upload<float>(c, &s.Ht, nullptr, (size_t)h.nk * h.ni * h.ni));
    SEP_CU(sep_upload<float>(c, &s.Sinv, nullptr, 2 * (size_t)h.nc * s.ldc));
    SEP_CU(sep_upload<float>(c, &s.R0, nullptr, 3 * rect));
    SEP_CU(sep_upload<float>(c, &s.R1, nullptr, 3 * rect));
    SEP_CU(sep_upload<float>(c, &s.R2, nullptr, 3 * rect));
    SEP_CU(sep_upload<float>(c, &s.Tc, nullptr, 3 * (size_t)std::max(h.nc, 1)));
    SEP_CU(sep_upload<float>(c, &s.U, nullptr, 3 * (size_t)std::max(h.nc, 1)));
    SEP_CU(sep_upload<double>(c, &s.lam, nullptr, h.nk));
    SEP_CU(sep_upload<double>(c, &s.V64, nullptr, (size_t)h.nk * h.nk));
    SEP_CU(sep_upload<double>(c, &s.Z64, nullptr, (size_t)h.nk * h.nk));
    SEP_CU(sep_upload<double>(c, &s.C64, nullptr, (size_t)h.ni * h.ni));
    SEP_CU(sep_upload<double>(c, &s.H64, nullptr, (size_t)h.nk * h.ni * h.ni));
    SEP_CU(sep_upload<double>(c, &s.S64, nullptr, (size_t)h.nc * h.nc));
    // Sinv rows start 16-byte aligned (ldc is a multiple of 4 entries of 8
    // bytes, cudaMalloc aligns to 256 B): the Schur product reads float4s
    SEP_CU(fill_zero(c, s.Sinv, sizeof(float) * 2 * (size_t)h.nc * s.ldc));
    SEP_CU(fill_zero(c, s.U, sizeof(float) * 3 * std::max(h.nc, 1)));
    tab.push_back(s);
  }
  // shared memory of the solve's separable stages: the staged tiles, and t
  // of the Schur product (3 n_c floats) when it fits
  int ncmax = 0;
  for (const auto& t : tab) ncmax = std::max(ncmax, t.nc);
  const size_t tiles = sizeof(float) * (size_t)std::max(SEP_GEMM_FLOATS, SEP_COL_FLOATS);
  c->sep_smem = std::max(tiles, std::min(sizeof(float) * 3 * (size_t)ncmax, (size_t)200 << 10));
  SepBody* d = nullptr;
  SEP_CU(sep_upload(c, &d, tab.data(), tab.size()));
  c->d_sep = d;
  c->sep_on = true;
  c->sep_eigen_ready = false;
  return cudaSuccess;
}

void sep_free(ibl_ctx* c) {
  for (void* p : c->sep_allocs)
    if (p) cudaFree(p);
  c->sep_allocs.clear();
  c->d_sep = nullptr;
  c->sep_on = false;
  c->sep_eigen_ready = false;
}

size_t sep_smem_bytes(const ibl_ctx* c) { return c->sep_smem; }

// Span eigen-decomposition (first use) and the rebuild of the factors, on
// the steps the host schedules a rebuild.  Early rebuilds, which the dense
// path takes when the iteration counts grow, are not needed here: the FP32
// application bounds the iteration count more than the factors' age does.
cudaError_t sep_launch(ibl_ctx* c, const int geo_n[3], const int geo_per[3]) {
  const int nb = (int)c->bodies.size();
  std::vector<int> boff(nb + 1);
  for (int b = 0; b < nb; ++b) boff[b] = c->bodies[b].offset;
  boff[nb] = c->m_total;
  if (!c->sep_eigen_ready) {
    k_sep_span_eigen<<<nb, 1024, 0, c->stream>>>(c->d_sep, c->d_boff, c->d_base,
                                                  reinterpret_cast<const df*>(c->d_wts), geo_n[2], geo_per[2]);
    c->launches++;
    SEP_CU(cudaGetLastError());
    c->sep_eigen_ready = true;
  }
  SepRebuildArgs R;
  R.sb = c->d_sep;
  R.nb = nb;
  R.boff = c->d_boff;
  R.base = c->d_base;
  R.wts = reinterpret_cast<const df*>(c->d_wts);
  for (int a = 0; a < 3; ++a) { R.n[a] = geo_n[a]; R.per[a] = geo_per[a]; }
  R.rowsum_max = (const unsigned long long*)c->d_Gdiag_max;
  const size_t smem = std::max(sizeof(double) * 3 * GJ64_NB * GJ64_LD,
                               sizeof(double) * SEP_NI_MAX * (SEP_NI_MAX + 1));
  if (!c->sep_blocks) {
    SEP_CU(cudaFuncSetAttribute((const void*)k_sep_rebuild, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    SEP_CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sep_rebuild, SEP_THREADS, smem));
    c->sep_blocks = std::max(1, std::min(per_sm, 4)) * num_sms();
  }
  void* args[] = {&R};
  SEP_CU(cudaLaunchCooperativeKernel((void*)k_sep_rebuild, dim3(c->sep_blocks), dim3(SEP_THREADS), args, smem,
                                     c->stream));
  c->launches++;
  return cudaGetLastError();
}

}  // namespace ibl
