// Streaming (pull) + face conditions of one cell, shared by the fluid kernels
// and the IB band-moment kernel so that both see bitwise the same
// post-streaming populations.
#pragma once

#include "ibl_internal.cuh"

namespace ibl {

template <int Q>
__device__ __forceinline__ int comp(int i, int a) {
  return a == 0 ? Lat<Q>::cx(i) : (a == 1 ? Lat<Q>::cy(i) : Lat<Q>::cz(i));
}

// Zou-He reconstruction of the populations entering through `face`, in
// deviation form g = f - w (non-equilibrium bounce-back with the transverse
// momentum correction; valid for D2Q9 and D3Q19).
template <int Q, class R>
__device__ __forceinline__ void zou_he(R g[Q], int face, const FluidParams<R>& p) {
  const int a = face >> 1;
  const int s = (face & 1) ? -1 : 1;     // inward normal = s * e_a
  R S0 = R(0), Sm = R(0);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int cn = comp<Q>(i, a) * s;
    if (cn == 0) S0 += g[i];
    else if (cn == -1) Sm += g[i];
  }
  R u[3];
  R rho;
  if (p.bc[face] == IBL_VEL_INLET) {
    u[0] = p.u_in[0]; u[1] = p.u_in[1]; u[2] = p.u_in[2];
    const R un = u[a] * R(s);
    rho = (R(1) + S0 + R(2) * Sm) / (R(1) - un);
  } else {
    rho = p.rho_out;
    const R un = R(1) - (R(1) + S0 + R(2) * Sm) / rho;
    u[0] = u[1] = u[2] = R(0);
    u[a] = un * R(s);
  }
  R Nt[3] = {R(0), R(0), R(0)};
#pragma unroll
  for (int t = 0; t < Lat<Q>::D; ++t) {
    if (t == a) continue;
    R acc = R(0);
#pragma unroll
    for (int i = 0; i < Q; ++i)
      if (comp<Q>(i, a) == 0 && comp<Q>(i, t) != 0) acc += R(comp<Q>(i, t)) * g[i];
    Nt[t] = R(0.5) * acc - rho * u[t] / R(3);
  }
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    if (comp<Q>(i, a) * s != 1) continue;
    R cu = R(0);
#pragma unroll
    for (int b = 0; b < Lat<Q>::D; ++b) cu += R(comp<Q>(i, b)) * u[b];
    R v = g[opp(i)] + R(6.0 * Lat<Q>::w(i)) * rho * cu;
#pragma unroll
    for (int t = 0; t < Lat<Q>::D; ++t)
      if (t != a && comp<Q>(i, t) != 0) v -= R(comp<Q>(i, t)) * Nt[t];
    g[i] = v;
  }
}

// Post-streaming populations of one cell.  PULL=false: the buffer already
// holds post-streaming values (first step after initialisation).
template <int Q, class T, bool PULL, class R>
__device__ __forceinline__ void gather_q(const T* __restrict__ src, int x, int y, int z,
                                       long long cell, const FluidParams<R>& p, R g[Q]) {
  const long long N = p.N;
  if (!PULL) {
#pragma unroll
    for (int i = 0; i < Q; ++i) g[i] = Store<T>::ld(src[i * N + cell]);
    return;
  }
  int zh_face = -1;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    int xs = x - Lat<Q>::cx(i), ys = y - Lat<Q>::cy(i), zs = z - Lat<Q>::cz(i);
    int refl = 0, unk = -1;
    if (Lat<Q>::cx(i) != 0) {
      if (xs < 0) {
        const int b = p.bc[0];
        if (b == IBL_PERIODIC) xs += p.nx; else if (b == IBL_BOUNCEBACK) refl = 1; else unk = 0;
      } else if (xs >= p.nx) {
        const int b = p.bc[1];
        if (b == IBL_PERIODIC) xs -= p.nx; else if (b == IBL_BOUNCEBACK) refl = 1; else unk = 1;
      }
    }
    if (Lat<Q>::cy(i) != 0) {
      if (ys < 0) {
        const int b = p.bc[2];
        if (b == IBL_PERIODIC) ys += p.ny; else if (b == IBL_BOUNCEBACK) refl = 1; else unk = 2;
      } else if (ys >= p.ny) {
        const int b = p.bc[3];
        if (b == IBL_PERIODIC) ys -= p.ny; else if (b == IBL_BOUNCEBACK) refl = 1; else unk = 3;
      }
    }
    if (Lat<Q>::D == 3 && Lat<Q>::cz(i) != 0) {
      if (zs < 0) {
        const int b = p.bc[4];
        if (b == IBL_PERIODIC) zs += p.nz; else if (b == IBL_BOUNCEBACK) refl = 1; else unk = 4;
      } else if (zs >= p.nz) {
        const int b = p.bc[5];
        if (b == IBL_PERIODIC) zs -= p.nz; else if (b == IBL_BOUNCEBACK) refl = 1; else unk = 5;
      }
    }
    if (unk >= 0) {
      g[i] = R(0);
      zh_face = unk;
    } else if (refl) {
      g[i] = Store<T>::ld(src[opp(i) * N + cell]);
    } else {
      g[i] = Store<T>::ld(src[i * N + ((long long)zs * p.ny + ys) * p.nx + xs]);
    }
  }
  if (zh_face >= 0) zou_he<Q, R>(g, zh_face, p);
}

}  // namespace ibl
