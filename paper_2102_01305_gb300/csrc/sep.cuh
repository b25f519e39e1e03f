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
// Application, per right-hand side (velocity component), in seven stages
// separated by grid barriers; rectangles are n_i x n_k FP32 arrays:
//   A  Y1 = X V           X: the input on the markers, 0 on c (rows i)
//   B  Y2[:,j] = H_j Y1[:,j]                                  (columns j)
//   C  t_p = (Y2 V^T)[p] for p in c
//   D  u = S^-1 t         (S^-1 stored as double-float pairs, products
//                          accumulated in double-float: the only stage whose
//                          FP32 rounding the Schur subtraction does not
//                          tolerate - at 2 x 6292 markers with the wings
//                          aligned to the grid (alpha = 0, every clap) an
//                          FP32 S^-1 makes the preconditioner indefinite)
//   E  W1 = U V           U: u on c, 0 on the markers
//   F  W2[:,j] = H_j W1[:,j]
//   G  z_l = ((Y2 - W2) V^T)[l] for the markers l  (done by the caller)
#pragma once

#include "df.cuh"

namespace ibl {

constexpr int SEP_RG = 4;          // chord rows per warp item of a row pass
constexpr int SEP_NK_MAX = 256;    // span positions per body (shared-memory rows)
constexpr int SEP_NI_MAX = 64;     // chord positions per body

struct SepBody {
  int ni, nk, nc, m;      // chord positions, span positions, complement entries, markers
  int ldc;                // row stride of Sinv (n_c rounded up to 4)
  const int* rect;        // n_i n_k: local marker index (>= 0) or -(p + 1) for complement entry p
  const int* mrect;       // m: rectangle index i n_k + k of each marker
  const int* crect;       // n_c: rectangle index of each complement entry
  const int* rep_i;       // n_i: a marker (local index) at each chord position
  const int* rep_k;       // n_k: a marker (local index) at each span position
  float* V;               // n_k x n_k eigenvectors of Z, V[k n_k + j]
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

// Warp items of a stage are dealt over all bodies in order; item -> (body, local item).
__device__ __forceinline__ int sep_item_body(const SepBody* sb, int nb, int per_body_kind, long long& item) {
  for (int b = 0; b < nb; ++b) {
    const SepBody& B = sb[b];
    long long cnt;
    switch (per_body_kind) {
      case 0: cnt = 3LL * ((B.ni + SEP_RG - 1) / SEP_RG) * ((B.nk + 31) / 32); break;   // row pass
      case 1: cnt = 3LL * B.nk * ((B.ni + 31) / 32); break;                              // column pass
      case 2: cnt = B.nc; break;                                                          // per complement entry
      default: cnt = B.m; break;                                                          // per marker
    }
    if (item < cnt) return b;
    item -= cnt;
  }
  return -1;
}

__device__ __forceinline__ long long sep_items(const SepBody* sb, int nb, int kind) {
  long long t = 0;
  for (int b = 0; b < nb; ++b) {
    const SepBody& B = sb[b];
    switch (kind) {
      case 0: t += 3LL * ((B.ni + SEP_RG - 1) / SEP_RG) * ((B.nk + 31) / 32); break;
      case 1: t += 3LL * B.nk * ((B.ni + 31) / 32); break;
      case 2: t += B.nc; break;
      default: t += B.m; break;
    }
  }
  return t;
}

// Row pass (stages A and E): out[c][i][j] = sum_k in[c][i][k] V[k][j].
// mode 0: in = x on the markers (0 on c); mode 1: in = u on c (0 on the
// markers).  One warp per (body, component, group of SEP_RG rows, 32
// columns); the rows are gathered into the warp's shared-memory slice.
static __device__ void sep_rowpass(const SepBody* sb, int nb, int mode, const SepIn& in, const int* voff,
                            float* sm) {
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  float* xs = sm + wib * SEP_RG * SEP_NK_MAX;
  const long long total = sep_items(sb, nb, 0);
  for (long long it = (long long)blockIdx.x * nwarps + wib; it < total; it += (long long)gridDim.x * nwarps) {
    long long li = it;
    const int b = sep_item_body(sb, nb, 0, li);
    const SepBody& B = sb[b];
    const int njc = (B.nk + 31) / 32, nig = (B.ni + SEP_RG - 1) / SEP_RG;
    const int jc = (int)(li % njc);
    const int ig = (int)((li / njc) % nig);
    const int c = (int)(li / ((long long)njc * nig));
    const int i0 = ig * SEP_RG;
    __syncwarp();
    for (int r = 0; r < SEP_RG; ++r) {
      const int i = i0 + r;
      for (int k = lane; k < B.nk; k += 32) {
        float v = 0.f;
        if (i < B.ni) {
          const int slot = B.rect[i * B.nk + k];
          if (mode == 0) {
            if (slot >= 0) {
              const int vi = voff[b] + 3 * slot + c;
              v = __ldcg(in.a + vi);
              if (in.b) v = fmaf(-in.s[c], __ldcg(in.b + vi), v);
            }
          } else if (slot < 0) {
            v = __ldcg(B.U + c * B.nc + (-slot - 1));
          }
        }
        xs[r * SEP_NK_MAX + k] = v;
      }
    }
    __syncwarp();
    const int j = jc * 32 + lane;
    if (j < B.nk) {
      float acc[SEP_RG];
#pragma unroll
      for (int r = 0; r < SEP_RG; ++r) acc[r] = 0.f;
      const float* Vj = B.V + j;
#pragma unroll 4
      for (int k = 0; k < B.nk; ++k) {
        const float v = __ldg(Vj + (long long)k * B.nk);
#pragma unroll
        for (int r = 0; r < SEP_RG; ++r) acc[r] = fmaf(xs[r * SEP_NK_MAX + k], v, acc[r]);
      }
      float* out = B.R0 + (long long)c * B.ni * B.nk;
#pragma unroll
      for (int r = 0; r < SEP_RG; ++r)
        if (i0 + r < B.ni) out[(long long)(i0 + r) * B.nk + j] = acc[r];
    }
  }
}

// Column pass (stages B and F): dst[c][i][j] = sum_i2 H_j[i][i2] src[c][i2][j].
// One warp per (body, component, span mode j, 32 chord rows).
static __device__ void sep_colpass(const SepBody* sb, int nb, bool second) {
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  const long long total = sep_items(sb, nb, 1);
  for (long long it = (long long)blockIdx.x * nwarps + wib; it < total; it += (long long)gridDim.x * nwarps) {
    long long li = it;
    const int b = sep_item_body(sb, nb, 1, li);
    const SepBody& B = sb[b];
    const int nic = (B.ni + 31) / 32;
    const int ic = (int)(li % nic);
    const int j = (int)((li / nic) % B.nk);
    const int c = (int)(li / ((long long)nic * B.nk));
    const int i = ic * 32 + lane;
    const float* src = B.R0 + (long long)c * B.ni * B.nk + j;
    float* dst = (second ? B.R2 : B.R1) + (long long)c * B.ni * B.nk + j;
    const float* h = B.Ht + (long long)j * B.ni * B.ni + i;
    float acc = 0.f;
    if (i < B.ni) {
#pragma unroll 4
      for (int i2 = 0; i2 < B.ni; ++i2) acc = fmaf(__ldg(h + (long long)i2 * B.ni), __ldcg(src + (long long)i2 * B.nk), acc);
      dst[(long long)i * B.nk] = acc;
    }
  }
}

// Stage C: t_p = sum_j Y2[i_p][j] V[k_p][j] for every complement entry p,
// three components; one warp per entry.
static __device__ void sep_complement_values(const SepBody* sb, int nb) {
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  const long long total = sep_items(sb, nb, 2);
  for (long long it = (long long)blockIdx.x * nwarps + wib; it < total; it += (long long)gridDim.x * nwarps) {
    long long p = it;
    const int b = sep_item_body(sb, nb, 2, p);
    const SepBody& B = sb[b];
    const int r = B.crect[p];
    const int i = r / B.nk, k = r - i * B.nk;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f;
    const long long plane = (long long)B.ni * B.nk;
    const float* y = B.R1 + (long long)i * B.nk;
    const float* v = B.V + (long long)k * B.nk;
    for (int j = lane; j < B.nk; j += 32) {
      const float vj = __ldg(v + j);
      a0 = fmaf(__ldcg(y + j), vj, a0);
      a1 = fmaf(__ldcg(y + plane + j), vj, a1);
      a2 = fmaf(__ldcg(y + 2 * plane + j), vj, a2);
    }
    for (int o = 16; o > 0; o >>= 1) {
      a0 += __shfl_xor_sync(0xffffffffu, a0, o);
      a1 += __shfl_xor_sync(0xffffffffu, a1, o);
      a2 += __shfl_xor_sync(0xffffffffu, a2, o);
    }
    if (lane == 0) {
      B.Tc[p] = a0;
      B.Tc[B.nc + p] = a1;
      B.Tc[2 * B.nc + p] = a2;
    }
  }
}

// Stage D: u = S^-1 t, one warp per row p, three components; each
// double-float entry of S^-1 times an FP32 t enters a double-float
// accumulator (the product's rounding error included).
static __device__ void sep_schur(const SepBody* sb, int nb) {
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  const long long total = sep_items(sb, nb, 2);
  for (long long it = (long long)blockIdx.x * nwarps + wib; it < total; it += (long long)gridDim.x * nwarps) {
    long long p = it;
    const int b = sep_item_body(sb, nb, 2, p);
    const SepBody& B = sb[b];
    // two (hi, lo) entries per 128-bit load
    const float4* row = reinterpret_cast<const float4*>(B.Sinv + 2LL * p * B.ldc);
    dfacc a0 = acc_zero(), a1 = acc_zero(), a2 = acc_zero();
    const int nq = B.ldc >> 1;
    for (int q = lane; q < nq; q += 32) {
      const float4 s = __ldg(row + q);
      const df sv[2] = {df_make(s.x, s.y), df_make(s.z, s.w)};
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int col = 2 * q + e;
        if (col < B.nc) {
          acc_fma_f(a0, sv[e], __ldcg(B.Tc + col));
          acc_fma_f(a1, sv[e], __ldcg(B.Tc + B.nc + col));
          acc_fma_f(a2, sv[e], __ldcg(B.Tc + 2 * B.nc + col));
        }
      }
    }
    const df u0 = df_warp_sum(acc_value(a0)), u1 = df_warp_sum(acc_value(a1)), u2 = df_warp_sum(acc_value(a2));
    if (lane == 0) {
      B.U[p] = u0.hi + u0.lo;
      B.U[B.nc + p] = u1.hi + u1.lo;
      B.U[2 * B.nc + p] = u2.hi + u2.lo;
    }
  }
}

// Stage G for one marker (local index l of body B), in every lane of the
// calling warp: z[c] = sum_j (Y2 - W2)[c][i_l][j] V[k_l][j].
__device__ __forceinline__ void sep_marker_z(const SepBody& B, int l, float z[3]) {
  const int lane = threadIdx.x & 31;
  const int r = B.mrect[l];
  const int i = r / B.nk, k = r - i * B.nk;
  const long long plane = (long long)B.ni * B.nk;
  const float* y = B.R1 + (long long)i * B.nk;
  const float* w = B.R2 + (long long)i * B.nk;
  const float* v = B.V + (long long)k * B.nk;
  float a0 = 0.f, a1 = 0.f, a2 = 0.f;
  for (int j = lane; j < B.nk; j += 32) {
    const float vj = __ldg(v + j);
    a0 = fmaf(__ldcg(y + j) - __ldcg(w + j), vj, a0);
    a1 = fmaf(__ldcg(y + plane + j) - __ldcg(w + plane + j), vj, a1);
    a2 = fmaf(__ldcg(y + 2 * plane + j) - __ldcg(w + 2 * plane + j), vj, a2);
  }
  for (int o = 16; o > 0; o >>= 1) {
    a0 += __shfl_xor_sync(0xffffffffu, a0, o);
    a1 += __shfl_xor_sync(0xffffffffu, a1, o);
    a2 += __shfl_xor_sync(0xffffffffu, a2, o);
  }
  z[0] = a0;
  z[1] = a1;
  z[2] = a2;
}

}  // namespace ibl
