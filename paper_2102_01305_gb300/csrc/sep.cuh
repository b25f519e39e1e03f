// Separable preconditioner of the implicit IB system (Eqs. 18-19) for rigid
// bodies whose markers lie on a product mesh: a chord index i (a position in
// the plane normal to the body's rotation axis) times a span index k (a
// position along that axis), with the rotation axis along the grid's z axis.
// The wing planforms are such meshes (a unit-spaced chord x span grid
// clipped to an ellipse, hinged about a spanwise axis).
//
// For such a body the 3D delta of Eq. 13 factors, D(x - X_ik) =
// [phi(x - X_i) phi(y - Y_i)] phi(z - Z_k), so the system matrix of Eq. 18
// is a principal submatrix of a Kronecker product:
//     G_(ik),(i'k') = C_ii' Z_kk',   C: chord-plane overlaps (change as the
//     body turns), Z: span overlaps (fixed: rotation about z keeps every z).
// With Omega the markers and R the bounding rectangle of the mesh (n_i x n_k,
// complement c = R \ Omega), and K = C (x) Z + sigma I, the inverse of
// G + sigma I = K_OmegaOmega is, by the block-inverse identity,
//     (G + sigma I)^-1 = (K^-1)_OmegaOmega - (K^-1)_Omega,c S^-1 (K^-1)_c,Omega,
//     S = (K^-1)_cc  (n_c x n_c).
// K^-1 is applied through the eigenvectors of Z (Z = V diag(lambda) V^T,
// computed once): K^-1 = (I (x) V) blockdiag_j H_j (I (x) V^T) with
// H_j = (lambda_j C + sigma I)^-1 (n_i x n_i per span mode j).  So
//     M r = [ K^-1 (P_Omega^T r - P_c^T u) ]_Omega,   u = S^-1 (K^-1 P_Omega^T r)_c,
// which is exactly the preconditioner the dense path stores (the shifted
// inverse of the same matrix), held in O(n_k^2 + n_k n_i^2 + n_c^2) numbers
// instead of O(m^2): at 2 x 6292 markers 2 x 25 MB instead of 2 x 158 MB.
//
// Application, for the three right-hand sides (velocity components) at once,
// in seven stages separated by grid barriers; rectangles are n_i x n_k FP32
// arrays:
//   A  Y1 = X V           X: the input on the markers, 0 on c (rows i)
//   B  Y2[:,j] = H_j Y1[:,j]                                  (columns j)
//   C  T = Y2 V^T         (t = T on c)
//   D  u = S^-1 t         (S^-1 stored as double-float pairs, products
//                          accumulated in double-float: the only stage whose
//                          FP32 rounding the Schur subtraction does not
//                          tolerate - at 2 x 6292 markers with the wings
//                          aligned to the grid (alpha = 0, every clap) an
//                          FP32 S^-1 makes the preconditioner indefinite)
//   E  W1 = U V           U: u on c, 0 on the markers
//   F  W2[:,j] = H_j W1[:,j]
//   G  Z = (Y2 - W2) V^T  (z = Z on the markers, read by the caller after
//                          a grid barrier)
#pragma once

#include "df.cuh"

namespace ibl {

constexpr int SEP_NK_MAX = 256;    // span positions per body
constexpr int SEP_NI_MAX = 64;     // chord positions per body
// Rectangle products (stages A, C, E, G): a block computes SEP_GR chord rows
// x SEP_GC columns of all three components, its 1024 threads splitting the
// reduction into SEP_GK groups.
constexpr int SEP_GR = 8;
constexpr int SEP_GC = 32;
constexpr int SEP_GK = 4;
// Column passes: a block applies SEP_JG consecutive span modes' H_j.
constexpr int SEP_JG = 2;
__host__ __device__ constexpr int sep_ldv(int nk) { return (nk + 3) & ~3; }   // V row stride (16-byte rows)

struct SepBody {
  int ni, nk, nc, m;      // chord positions, span positions, complement entries, markers
  int ldc;                // row stride of Sinv (n_c rounded up to 4)
  const int* rect;        // n_i n_k: local marker index (>= 0) or -(p + 1) for complement entry p
  const int* mrect;       // m: rectangle index i n_k + k of each marker
  const int* crect;       // n_c: rectangle index of each complement entry
  const int* rep_i;       // n_i: a marker (local index) at each chord position
  const int* rep_k;       // n_k: a marker (local index) at each span position
  float* V;               // n_k x ldv eigenvectors of Z, V[k ldv + j], ldv = sep_ldv(n_k), zero padded
  float* Ht;              // n_k x n_i x n_i: Ht[(j n_i + i2) n_i + i] = H_j[i][i2]
  float* Sinv;            // n_c x ldc double-float pairs (hi, lo), 2 ldc floats per row
  float* R0;              // 3 x n_i x n_k scratch (Y1, then W1)
  float* R1;              // 3 x n_i x n_k (Y2)
  float* R2;              // 3 x n_i x n_k (W2)
  float* Tc;              // 3 x n_c (t)
  float* U;               // 3 x n_c (u)
  // FP64 data of the rebuild
  double* lam;            // n_k eigenvalues of Z
  double* V64;            // n_k x n_k
  double* Z64;            // n_k x n_k (work of the eigensolver)
  double* C64;            // n_i x n_i
  double* H64;            // n_k x n_i x n_i
  double* S64;            // n_c x n_c, inverted in place
};

// Input of one application: x = a - s_c b at each marker's slot of the padded
// FP32 vectors (b may be null).
struct SepIn {
  const float* a;
  const float* b;
  float s[3];
};

// Items of a stage are dealt over all bodies in order; item -> (body, local item).
//   kind 0: rectangle-product tiles, one per block
//   kind 1: column-pass groups of SEP_JG modes, one per block
//   kind 2: groups of 32 Schur rows, one per block;  kind 3: markers
__device__ __forceinline__ long long sep_count(const SepBody& B, int kind) {
  switch (kind) {
    case 0: return (long long)((B.ni + SEP_GR - 1) / SEP_GR) * ((B.nk + SEP_GC - 1) / SEP_GC);
    case 1: return (B.nk + SEP_JG - 1) / SEP_JG;
    case 2: return (B.nc + 31) / 32;
    default: return B.m;
  }
}

__device__ __forceinline__ int sep_item_body(const SepBody* sb, int nb, int kind, long long& item) {
  for (int b = 0; b < nb; ++b) {
    const long long cnt = sep_count(sb[b], kind);
    if (item < cnt) return b;
    item -= cnt;
  }
  return -1;
}

__device__ __forceinline__ long long sep_items(const SepBody* sb, int nb, int kind) {
  long long t = 0;
  for (int b = 0; b < nb; ++b) t += sep_count(sb[b], kind);
  return t;
}

// dst[e] = f(e) for e < n by the whole block, U elements per thread per pass:
// the U loads (or load chains) of a thread are issued before the first store,
// so a pass costs one round trip instead of U.
template <int U, class F>
__device__ __forceinline__ void sep_stage(float* dst, int n, F f) {
  for (int base = 0; base < n; base += U * (int)blockDim.x) {
    float v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = base + u * (int)blockDim.x + (int)threadIdx.x;
      v[u] = e < n ? f(e) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = base + u * (int)blockDim.x + (int)threadIdx.x;
      if (e < n) dst[e] = v[u];
    }
  }
}

// Shared memory of the rectangle products and column passes, in floats (the
// Schur product adds 3 n_c, see sep_smem_bytes).
constexpr int SEP_GEMM_FLOATS = 3 * SEP_GR * SEP_NK_MAX + SEP_NK_MAX * SEP_GC + SEP_GK * 3 * SEP_GR * SEP_GC;
constexpr int SEP_COL_FLOATS = SEP_JG * (SEP_NI_MAX * SEP_NI_MAX + 3 * SEP_NI_MAX);

// Rectangle product (stages A, C, E, G), all three components:
//   trans = false:  R0[c][i][j] = sum_k in[c][i][k] V[k][j]        (to the span modes)
//   trans = true:   R0[c][i][k] = sum_j in[c][i][j] V[k][j]        (back to the span positions)
// with in = mode 0: x on the markers (x = a - s b, 0 on the complement),
// 1: u on the complement (0 on the markers), 2: R1, 3: R1 - R2.  A tile's
// input rows and its V tile are staged in shared memory; thread (g, r, jj)
// sums the g-th quarter of the reduction, and the quarters are added in a
// fixed order.  Needs blockDim.x == SEP_GK * SEP_GR * SEP_GC.
static __device__ void sep_gemm(const SepBody* sb, int nb, int mode, bool trans, const SepIn& in,
                                const int* voff, float* sm) {
  const long long total = sep_items(sb, nb, 0);
  for (long long it = blockIdx.x; it < total; it += gridDim.x) {
    long long li = it;
    const int b = sep_item_body(sb, nb, 0, li);
    const SepBody& B = sb[b];
    const int nk = B.nk, ldv = sep_ldv(nk);
    const int nct = (nk + SEP_GC - 1) / SEP_GC;
    const int i0 = (int)(li / nct) * SEP_GR, j0 = (int)(li % nct) * SEP_GC;
    const long long plane = (long long)B.ni * nk;
    float* xs = sm;                                  // [3][SEP_GR][nk]
    float* ws = xs + 3 * SEP_GR * nk;                // [nk][SEP_GC]
    float* red = ws + nk * SEP_GC;                   // [SEP_GK][3][SEP_GR][SEP_GC]
    __syncthreads();
    const int ni = B.ni, nc = B.nc;
    const int* rect = B.rect;
    const float *R1 = B.R1, *R2 = B.R2, *Uc = B.U, *V = B.V;
    const float *ina = in.a, *inb = in.b;
    const int vo = voff[b];
    sep_stage<8>(xs, 3 * SEP_GR * nk, [&](int e) {
      const int c = e / (SEP_GR * nk), r = (e / nk) % SEP_GR, k = e % nk;
      const int i = i0 + r;
      float v = 0.f;
      if (i < ni) {
        if (mode >= 2) {
          const long long o = c * plane + (long long)i * nk + k;
          v = __ldcg(R1 + o);
          if (mode == 3) v -= __ldcg(R2 + o);
        } else {
          const int slot = rect[i * nk + k];
          if (mode == 0) {
            if (slot >= 0) {
              const int vi = vo + 3 * slot + c;
              v = __ldcg(ina + vi);
              if (inb) v = fmaf(-in.s[c], __ldcg(inb + vi), v);
            }
          } else if (slot < 0) {
            v = __ldcg(Uc + c * nc + (-slot - 1));
          }
        }
      }
      return v;
    });
    if (!trans) {
      // ws[k][jj] = V[k][j0 + jj] (rows are zero padded to ldv)
      sep_stage<8>(ws, nk * SEP_GC, [&](int e) {
        const int k = e / SEP_GC, j = j0 + e % SEP_GC;
        return j < ldv ? __ldg(V + (long long)k * ldv + j) : 0.f;
      });
    } else {
      // ws[j][kk] = V[j0 + kk][j]: rows j0 .. j0 + SEP_GC of V, transposed
      sep_stage<8>(ws, SEP_GC * nk, [&](int e) {
        const int j = e / SEP_GC, kk = e % SEP_GC, k = j0 + kk;
        return k < nk ? __ldg(V + (long long)k * ldv + j) : 0.f;
      });
    }
    __syncthreads();
    const int g = threadIdx.x / (SEP_GR * SEP_GC), r = (threadIdx.x / SEP_GC) % SEP_GR, jj = threadIdx.x % SEP_GC;
    const int kq = (nk + SEP_GK - 1) / SEP_GK, k0 = g * kq, k1 = min(nk, k0 + kq);
    const float* x0 = xs + r * nk;
    const float* x1 = x0 + SEP_GR * nk;
    const float* x2 = x1 + SEP_GR * nk;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll 4
    for (int k = k0; k < k1; ++k) {
      const float v = ws[k * SEP_GC + jj];
      a0 = fmaf(x0[k], v, a0);
      a1 = fmaf(x1[k], v, a1);
      a2 = fmaf(x2[k], v, a2);
    }
    float* rd = red + (g * 3 * SEP_GR + r) * SEP_GC + jj;
    rd[0] = a0;
    rd[SEP_GR * SEP_GC] = a1;
    rd[2 * SEP_GR * SEP_GC] = a2;
    __syncthreads();
    if (g == 0) {
      const int i = i0 + r, j = j0 + jj;
      if (i < B.ni && j < nk) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          float t = 0.f;
#pragma unroll
          for (int q = 0; q < SEP_GK; ++q) t += red[((q * 3 + c) * SEP_GR + r) * SEP_GC + jj];
          B.R0[c * plane + (long long)i * nk + j] = t;
        }
      }
    }
  }
}

// Column pass (stages B and F): dst[c][i][j] = sum_i2 H_j[i][i2] src[c][i2][j]
// with src = R0.  One block per group of SEP_JG modes: their H_j and the
// source columns are staged in shared memory, then one thread per
// (mode, component, row) output.
static __device__ void sep_colpass(const SepBody* sb, int nb, bool second, float* sm) {
  const long long total = sep_items(sb, nb, 1);
  for (long long it = blockIdx.x; it < total; it += gridDim.x) {
    long long li = it;
    const int b = sep_item_body(sb, nb, 1, li);
    const SepBody& B = sb[b];
    const int ni = B.ni, nk = B.nk;
    const int j0 = (int)li * SEP_JG, nj = min(SEP_JG, nk - j0);
    const long long plane = (long long)ni * nk;
    float* hs = sm;                                   // [SEP_JG][ni][ni] in the Ht layout
    float* ys = sm + SEP_JG * ni * ni;                // [SEP_JG][3][ni]
    __syncthreads();
    const float* hsrc = B.Ht + (long long)j0 * ni * ni;
    const float* R0 = B.R0;
    sep_stage<8>(hs, nj * ni * ni, [&](int e) { return __ldg(hsrc + e); });
    sep_stage<1>(ys, nj * 3 * ni, [&](int e) {
      const int jj = e / (3 * ni), c = (e / ni) % 3, i2 = e % ni;
      return __ldcg(R0 + c * plane + (long long)i2 * nk + j0 + jj);
    });
    __syncthreads();
    for (int e = threadIdx.x; e < nj * 3 * ni; e += blockDim.x) {
      const int jj = e / (3 * ni), c = (e / ni) % 3, i = e % ni;
      const float* h = hs + jj * ni * ni + i;
      const float* y = ys + (jj * 3 + c) * ni;
      float acc = 0.f;
#pragma unroll 4
      for (int i2 = 0; i2 < ni; ++i2) acc = fmaf(h[i2 * ni], y[i2], acc);
      (second ? B.R2 : B.R1)[c * plane + (long long)i * nk + j0 + jj] = acc;
    }
  }
}

// Stage D: u = S^-1 t.  The complement rows of all bodies are split into
// equal contiguous ranges, one per block, so that every SM takes part; per
// body in its range a block stages t (the complement entries of R0, three
// components) in shared memory when it fits, then one warp per row; each
// double-float entry of S^-1 times an FP32 t enters a double-float
// accumulator (the product's rounding error included).  A row's sum does not
// depend on the block that forms it.
#ifndef IBL_SCHUR_BATCH
#define IBL_SCHUR_BATCH 2
#endif
constexpr int SCHUR_BATCH = IBL_SCHUR_BATCH;   // 128-bit loads per lane in flight in stage D
static __device__ void sep_schur(const SepBody* sb, int nb, float* sm, int smem_floats) {
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int warps = blockDim.x >> 5;
  // the complement rows of all bodies, split into equal contiguous ranges,
  // one per block (every SM takes part), one warp per row
  long long rows = 0;
  for (int b = 0; b < nb; ++b) rows += sb[b].nc;
  const long long r0 = (long long)blockIdx.x * rows / gridDim.x;
  const long long r1 = (long long)(blockIdx.x + 1) * rows / gridDim.x;
  long long base = 0;
  for (int b = 0; b < nb; ++b) {
    const SepBody& B = sb[b];
    const int nc = B.nc;
    const long long lo = r0 > base ? r0 : base, hi = r1 < base + nc ? r1 : base + nc;
    base += nc;
    if (lo >= hi) continue;
    const long long plane = (long long)B.ni * B.nk;
    const bool stage_t = 3 * nc <= smem_floats;
    __syncthreads();
    if (stage_t) {
      const float* R0 = B.R0;
      const int* crect = B.crect;
      sep_stage<8>(sm, 3 * nc, [&](int e) {
        const int c = e / nc, q = e % nc;
        return __ldcg(R0 + c * plane + crect[q]);
      });
    }
    __syncthreads();
    for (long long pr = lo + wib; pr < hi; pr += warps) {
      const int p = (int)(pr - (base - nc));
      // two (hi, lo) entries per 128-bit load
      const float4* row = reinterpret_cast<const float4*>(B.Sinv + 2LL * p * B.ldc);
      dfacc a0 = acc_zero(), a1 = acc_zero(), a2 = acc_zero();
      const int nq = B.ldc >> 1;
      // SCHUR_BATCH loads of a lane are issued before their products (2:
      // 26 us for the stage at 2 x 1708 complement rows, 29 us with one at a
      // time, 34 us with 8, which spills); the accumulation order is unchanged
      for (int q0 = lane; q0 < nq; q0 += 32 * SCHUR_BATCH) {
        float4 s4b[SCHUR_BATCH];
#pragma unroll
        for (int u = 0; u < SCHUR_BATCH; ++u)
          s4b[u] = q0 + 32 * u < nq ? __ldg(row + q0 + 32 * u) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int u = 0; u < SCHUR_BATCH; ++u) {
        const int q = q0 + 32 * u;
        const float4 s4 = s4b[u];
        const df sv[2] = {df_make(s4.x, s4.y), df_make(s4.z, s4.w)};
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int col = 2 * q + e;
          if (q < nq && col < nc) {
            float t0, t1, t2;
            if (stage_t) {
              t0 = sm[col];
              t1 = sm[nc + col];
              t2 = sm[2 * nc + col];
            } else {
              const int r = B.crect[col];
              t0 = __ldcg(B.R0 + r);
              t1 = __ldcg(B.R0 + plane + r);
              t2 = __ldcg(B.R0 + 2 * plane + r);
            }
            acc_fma_f(a0, sv[e], t0);
            acc_fma_f(a1, sv[e], t1);
            acc_fma_f(a2, sv[e], t2);
          }
        }
        }
      }
      const df u0 = df_warp_sum(acc_value(a0)), u1 = df_warp_sum(acc_value(a1)), u2 = df_warp_sum(acc_value(a2));
      if (lane == 0) {
        B.U[p] = u0.hi + u0.lo;
        B.U[nc + p] = u1.hi + u1.lo;
        B.U[2 * nc + p] = u2.hi + u2.lo;
      }
    }
  }
}

// z of one marker (local index l of body B) after stage G: its entry of
// the R0 rectangle, three components.
__device__ __forceinline__ void sep_marker_z(const SepBody& B, int l, float z[3]) {
  const long long plane = (long long)B.ni * B.nk;
  const int r = B.mrect[l];
  z[0] = __ldcg(B.R0 + r);
  z[1] = __ldcg(B.R0 + plane + r);
  z[2] = __ldcg(B.R0 + 2 * plane + r);
}

}  // namespace ibl
