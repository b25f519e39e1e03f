// Fluid kernels: fused streaming + face conditions + moments + BGK/Guo collision.
//
// One thread per cell, x fastest across a warp so that every population read
// and write is a coalesced 128-byte row segment (the +/-1 x-shifted pulls
// straddle one extra segment that the neighbouring warp also touches; L1/L2
// absorb it).  Per cell the kernel moves exactly Q loads and Q stores of the
// storage type: the bytes-per-cell roofline of a streaming stencil.
//
// Paper passages: Eq. 1 (BGK + streaming), Eq. 4 (equilibrium), Eqs. 7-8
// (Guo forcing), Eq. 9 (rho u = sum c_i f_i + F/2), Sec. 2.1 bounce-back,
// Sec. 3.1 Zou-He inlet / outlet.
#include <mutex>

#include "ibl_internal.cuh"
#include "lbm_gather.cuh"

namespace ibl {

// Velocity correction du of a cell from the band's fixed-point spreading sums
// (Eq. 15), zero elsewhere; the sums are cleared for the next step.
// Tile extents as compile-time constants of the lattice (16 x 4 x 4 in 3D,
// 16 x 16 in 2D), so that the lookups below are shifts and masks.
template <int Q> struct TileDim {
  static constexpr int X = TILE_X;
  static constexpr int Y = Lat<Q>::D == 3 ? TILE_Y : TILE_CELLS / TILE_X;
  static constexpr int Z = Lat<Q>::D == 3 ? TILE_Z3 : 1;
};

template <int Q, class R>
__device__ __forceinline__ int tile_index(int x, int y, int z, const FluidParams<R>& p) {
  using TD = TileDim<Q>;
  return ((z / TD::Z) * p.tg.nty + (y / TD::Y)) * p.tg.ntx + (x / TD::X);
}

template <int Q, class R>
__device__ __forceinline__ int band_du(int x, int y, int z, const FluidParams<R>& p, R du[3]) {
  using TD = TileDim<Q>;
  const int slot = p.tile_slot[tile_index<Q, R>(x, y, z, p)];
  if (slot < 0) return -1;
  const int local = ((z % TD::Z) * TD::Y + (y % TD::Y)) * TD::X + (x % TD::X);
  unsigned long long* a = p.band_acc + (long long)slot * 3 * TILE_CELLS + local;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    du[c] = (R)((double)(long long)a[c * TILE_CELLS] * (1.0 / FIX_SCALE));
    a[c * TILE_CELLS] = 0ull;
  }
  return slot * 3 * TILE_CELLS + local;
}

// ------------------------------------------------------------------ collision arithmetic
// Every operation of the collision is an explicit IEEE operation rounded on
// its own, so the result is fixed by the source.  Sc<R> runs it on one cell;
// Pk runs it on two cells at once with Blackwell's packed FP32 instructions
// (add/sub/mul/fma .rn.f32x2 round each lane exactly as the scalar
// instruction does), so the two-cell kernel and the one-cell kernels give
// bitwise the same populations.  One rule keeps that true: no product feeds
// an addition or subtraction.  The assembler fuses a packed multiply and a
// packed add that follows it into one FMA even with .rn on both (measured
// on sm_103a; the scalar .rn forms are left alone), so wherever a product
// meets a sum the collision uses an explicit FMA instead.
template <class R> struct Sc;
template <> struct Sc<float> {
  using R = float;
  using V = float;
  static __device__ __forceinline__ V splat(R s) { return s; }
  static __device__ __forceinline__ V add(V a, V b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ V sub(V a, V b) { return __fsub_rn(a, b); }
  static __device__ __forceinline__ V mul(V a, V b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ V fma(V a, V b, V c) { return __fmaf_rn(a, b, c); }
  static __device__ __forceinline__ V div(V a, V b) { return __fdiv_rn(a, b); }
};
template <> struct Sc<double> {
  using R = double;
  using V = double;
  static __device__ __forceinline__ V splat(R s) { return s; }
  static __device__ __forceinline__ V add(V a, V b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ V sub(V a, V b) { return __dsub_rn(a, b); }
  static __device__ __forceinline__ V mul(V a, V b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ V fma(V a, V b, V c) { return __fma_rn(a, b, c); }
  static __device__ __forceinline__ V div(V a, V b) { return __ddiv_rn(a, b); }
};

// Uniform coefficients (one rounded product, the same in every lane).
__device__ __forceinline__ float rn_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rn_mul(double a, double b) { return __dmul_rn(a, b); }

// Two FP32 lanes in one 64-bit register pair: lo = cell x, hi = cell x + 1.
struct F2 {
  unsigned long long v;
};
struct Pk {
  using R = float;
  using V = F2;
  static __device__ __forceinline__ V make(float lo, float hi) {
    V r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(lo), "f"(hi));
    return r;
  }
  static __device__ __forceinline__ float lo(V a) {
    float l, h;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(l), "=f"(h) : "l"(a.v));
    return l;
  }
  static __device__ __forceinline__ float hi(V a) {
    float l, h;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(l), "=f"(h) : "l"(a.v));
    return h;
  }
  static __device__ __forceinline__ V splat(R s) { return make(s, s); }
  static __device__ __forceinline__ V add(V a, V b) {
    V r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
  }
  static __device__ __forceinline__ V sub(V a, V b) {
    V r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
  }
  static __device__ __forceinline__ V mul(V a, V b) {
    V r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
  }
  static __device__ __forceinline__ V fma(V a, V b, V c) {
    V r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return r;
  }
  // no packed division: one IEEE division per lane
  static __device__ __forceinline__ V div(V a, V b) {
    return make(__fdiv_rn(lo(a), lo(b)), __fdiv_rn(hi(a), hi(b)));
  }
};

// c_a u_a + c_b u_b of the first member of a direction pair.  In both
// lattices the first member's first nonzero component is +1, so the sum is
// u_a, u_a + u_b or u_a - u_b: no negation.
template <int Q, class O>
__device__ __forceinline__ typename O::V dir_dot(int i, const typename O::V v[3]) {
  const int c[3] = {Lat<Q>::cx(i), Lat<Q>::cy(i), Lat<Q>::cz(i)};
  typename O::V s{};
  bool have = false;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (c[a] == 0) continue;
    if (!have) s = v[a];
    else s = c[a] > 0 ? O::add(s, v[a]) : O::sub(s, v[a]);
    have = true;
  }
  return s;
}

// BGK collision with the Guo source (Eqs. 7-8) in deviation form g = f - w.
// Pairs (c, -c) share |c.u| and |c.F|: the even part of f_eq and of the
// source is computed once per pair, the odd part flips sign.  rho = 1 + drho
// is never formed in the storage precision where it would drop drho's low
// bits: rho X = X + drho X and u = m - m drho/(1 + drho).  Returns drho.
// F is the uniform body force G plus, with IB, the IB force density
// 2 rho du (Eq. 26) formed here from this cell's own density; F is returned
// in F.  Without IB, du = 0 and F = G exactly (G carries no negative zero).
template <int Q, bool IB, class O>
__device__ __forceinline__ typename O::V collide_v(typename O::V g[Q], typename O::V F[3],
                                                   const typename O::V du[3],
                                                   const FluidParams<typename O::R>& p) {
  using V = typename O::V;
  using R = typename O::R;
  V drho = g[0];
  V m[3];
  bool have[3] = {false, false, false};
#pragma unroll
  for (int i = 1; i < Q; i += 2) {
    drho = O::add(drho, O::add(g[i], g[i + 1]));
    const V d = O::sub(g[i], g[i + 1]);
    const int c[3] = {Lat<Q>::cx(i), Lat<Q>::cy(i), Lat<Q>::cz(i)};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (c[a] == 0) continue;
      if (!have[a]) m[a] = c[a] > 0 ? d : O::sub(O::splat(R(0)), d);
      else m[a] = c[a] > 0 ? O::add(m[a], d) : O::sub(m[a], d);
      have[a] = true;
    }
  }
  if (Lat<Q>::D == 2) m[2] = O::splat(R(0));
  // 2 rho du = 2 du + drho (2 du) (rho = 1 + drho is not formed in low precision)
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (IB) {
      const V t = O::mul(O::splat(R(2)), du[a]);
      F[a] = O::add(O::splat(p.G[a]), O::fma(drho, t, t));
    } else {
      F[a] = O::splat(p.G[a]);
    }
  }
  // Eq. 9: rho u = sum c_i f_i + F/2, u = (m + F/2) - (m + F/2) drho/(1 + drho)
  const V nq = O::div(drho, O::sub(O::splat(R(-1)), drho));   // -drho/(1 + drho), exactly
  V u[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    u[a] = O::fma(O::splat(R(0.5)), F[a], m[a]);
    u[a] = O::fma(u[a], nq, u[a]);
  }
  const V usq = O::fma(u[2], u[2], O::fma(u[1], u[1], O::mul(u[0], u[0])));
  const V uF = O::fma(u[2], F[2], O::fma(u[1], F[1], O::mul(u[0], F[0])));
  const V X = O::mul(O::splat(R(-1.5)), usq);       // -1.5 u.u
  const V m3uF = O::mul(O::splat(R(-3)), uF);       // -3 u.F
  const V nom = O::splat(-p.omega);
  const R pref = p.pref;
  {
    // rest population: f_eq - w = w (drho - 1.5 rho u.u); source -3 pref w u.F
    //   g0 - omega (g0 - w E0) + (pref w) (-3 u.F)
    const R w = R(Lat<Q>::w(0));
    const V E0 = O::add(drho, O::fma(drho, X, X));
    const V t = O::fma(O::splat(-w), E0, g[0]);                        // g0 - w E0
    g[0] = O::fma(O::splat(rn_mul(pref, w)), m3uF, O::fma(nom, t, g[0]));
  }
#pragma unroll
  for (int i = 1; i < Q; i += 2) {
    const V cu = dir_dot<Q, O>(i, u);
    const V cF = dir_dot<Q, O>(i, F);
    const R w = R(Lat<Q>::w(i));
    const R wo = w3<Q, R>(i);
    const R pwo = rn_mul(pref, wo);
    // Eq. 4 (second-order expansion): even part rho w (4.5 cu^2 - 1.5 u.u),
    // odd part 3 w rho cu; f_eq - w = ge +/- wo (cu + drho cu)
    const V Xe = O::fma(O::mul(O::splat(R(4.5)), cu), cu, X);
    const V ge = O::mul(O::splat(w), O::add(drho, O::fma(drho, Xe, Xe)));
    const V Oc = O::fma(drho, cu, cu);
    const V eq_p = O::fma(O::splat(wo), Oc, ge);
    const V eq_m = O::fma(O::splat(-wo), Oc, ge);
    // Eq. 8: pref w [3 (c - u).F + 9 (c.u)(c.F)]: even pref w (9 cu cF - 3 uF),
    // odd +/- pref wo cF
    const V Se = O::mul(O::splat(rn_mul(pref, w)), O::fma(O::mul(O::splat(R(9)), cu), cF, m3uF));
    const V S_p = O::fma(O::splat(pwo), cF, Se);
    const V S_m = O::fma(O::splat(-pwo), cF, Se);
    const V a = g[i], b = g[i + 1];
    g[i] = O::add(O::fma(nom, O::sub(a, eq_p), a), S_p);
    g[i + 1] = O::add(O::fma(nom, O::sub(b, eq_m), b), S_m);
  }
  return drho;
}

template <int Q, bool IB, class R>
__device__ __forceinline__ R collide(R g[Q], R F[3], const R du[3], const FluidParams<R>& p) {
  return collide_v<Q, IB, Sc<R>>(g, F, du, p);
}

// Per-direction base pointers of the two population buffers (kernel
// parameters, so no 64-bit index arithmetic per load or store).
template <int Q, class T> struct DirPtrs {
  const T* s[Q];
  T* d[Q];
};

// True when the cell lies on a face that is not periodic (bounce-back or
// Zou-He), where the general gather applies.
template <class R>
__device__ __forceinline__ bool on_special_face(int x, int y, int z, int D, const FluidParams<R>& p) {
  return (x == 0 && p.bc[0] != IBL_PERIODIC) || (x == p.nx - 1 && p.bc[1] != IBL_PERIODIC) ||
         (y == 0 && p.bc[2] != IBL_PERIODIC) || (y == p.ny - 1 && p.bc[3] != IBL_PERIODIC) ||
         (D == 3 && ((z == 0 && p.bc[4] != IBL_PERIODIC) || (z == p.nz - 1 && p.bc[5] != IBL_PERIODIC)));
}

// Pull of an interior (or periodic-face) cell: neighbour rows and columns are
// wrapped once per thread; each direction then costs one add and one load.
template <int Q, class T, class R>
__device__ __forceinline__ void gather_fast(const DirPtrs<Q, T>& P, int x, int y, int z,
                                            const FluidParams<R>& p, R g[Q]) {
  int xs[3] = {x - 1, x, x + 1};
  if (xs[0] < 0) xs[0] += p.nx;
  if (xs[2] >= p.nx) xs[2] -= p.nx;
  int ys[3] = {y - 1, y, y + 1};
  if (ys[0] < 0) ys[0] += p.ny;
  if (ys[2] >= p.ny) ys[2] -= p.ny;
  int zs[3] = {z - 1, z, z + 1};
  if (Lat<Q>::D == 3) {
    if (zs[0] < 0) zs[0] += p.nz;
    if (zs[2] >= p.nz) zs[2] -= p.nz;
  }
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int dy = 1 - Lat<Q>::cy(i), dz = 1 - Lat<Q>::cz(i), dx = 1 - Lat<Q>::cx(i);
    const int src = (zs[dz] * p.ny + ys[dy]) * p.nx + xs[dx];
    g[i] = Store<T>::ld(P.s[i][src]);
  }
}

// One cell of the fused step: pull (with faces), IB velocity correction of
// band cells, collision with forcing, store; the same arithmetic whichever
// kernel runs it, so every launch split gives bitwise the same populations.
template <int Q, class T, bool PULL, bool IB>
__device__ __forceinline__ void collide_cell(const DirPtrs<Q, T>& P, const FluidParams<typename Store<T>::R>& p,
                                             int x, int y, int z) {
  using R = typename Store<T>::R;
  const int cell = (z * p.ny + y) * p.nx + x;
  R g[Q];
  if (!PULL) {
#pragma unroll
    for (int i = 0; i < Q; ++i) g[i] = Store<T>::ld(P.s[i][cell]);
  } else if (!on_special_face<R>(x, y, z, Lat<Q>::D, p)) {
    gather_fast<Q, T, R>(P, x, y, z, p, g);
  } else {
    gather_q<Q, T, true, R>(P.s[0], x, y, z, cell, p, g);
  }
  R F[3];
  R du[3] = {R(0), R(0), R(0)};
  int band = -1;
  if (IB) band = band_du<Q, R>(x, y, z, p, du);
  const R drho = collide<Q, IB, R>(g, F, du, p);
  if (!(drho > R(-1) && drho < R(99))) atomicOr(p.status, ST_DIVERGED);
#pragma unroll
  for (int i = 0; i < Q; ++i) P.d[i][cell] = Store<T>::st(g[i]);
  if (IB && band >= 0) {
    // the IB force density of this step, for ibl_get_field(IBL_FIELD_FORCE)
    p.band_F[band] = F[0] - p.G[0];
    p.band_F[band + TILE_CELLS] = F[1] - p.G[1];
    p.band_F[band + 2 * TILE_CELLS] = F[2] - p.G[2];
  }
}

// ---------------------------------------------------------------- 16-bit storage: two cells per thread
// With 2-byte populations one cell per thread keeps too few bytes in flight
// to cover HBM latency (the kernel then runs at ~0.56 of the bandwidth
// bound).  Here a thread takes the x-adjacent cells (x, x + 1), x even and nx
// even: every pull is an aligned 32-bit word, every store one 32-bit pair,
// and the two cells' collisions run as one stream of packed FP32 operations
// (Pk), which halves the instructions of the arithmetic that otherwise
// limits this kernel's issue rate.  Each lane computes exactly what the
// one-cell kernels compute, so the populations are bitwise theirs.
template <class T> struct __align__(4) Pair16 {
  T a, b;
};

// Two 16-bit values as one packed FP32 pair and back, with the scaling and
// rounding of Store<T>::ld and Store<T>::st (the scale is a power of two).
template <class T> struct Pack16;
template <> struct Pack16<__half> {
  static __device__ __forceinline__ F2 ld(__half a, __half b) {
    return Pk::mul(Pk::make(__half2float(a), __half2float(b)), Pk::splat(1.0f / 256.0f));
  }
  static __device__ __forceinline__ unsigned st(F2 v) {
    const F2 s = Pk::mul(v, Pk::splat(256.0f));
    const __half2 h = __floats2half2_rn(Pk::lo(s), Pk::hi(s));
    return *reinterpret_cast<const unsigned*>(&h);
  }
};
template <> struct Pack16<__nv_bfloat16> {
  static __device__ __forceinline__ F2 ld(__nv_bfloat16 a, __nv_bfloat16 b) {
    return Pk::make(__bfloat162float(a), __bfloat162float(b));
  }
  static __device__ __forceinline__ unsigned st(F2 v) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(Pk::lo(v), Pk::hi(v));
    return *reinterpret_cast<const unsigned*>(&h);
  }
};

// Pull of the cells (x, x + 1) with every load an aligned 32-bit word: per
// direction each thread loads the word (x, x + 1) of its source row; for
// c_x = +1 the value at x - 1 is the high half of the previous lane's word,
// for c_x = -1 the value at x + 2 the low half of the next lane's word (the
// lanes of a warp hold x, x + 2, ... of one row: blocks are a multiple of 32
// threads wide in x).  The first lane, the last lane and lanes at the row's
// ends load that value directly.  Every lane of the warp must call it
// (shuffles); lanes outside the grid pass clamped coordinates and discard
// the result.  g[i] holds the two cells' values of direction i, lo = x.
template <int Q, class T>
__device__ __forceinline__ void gather_pair_words(const DirPtrs<Q, T>& P, int x, int y, int z,
                                                  const FluidParams<float>& p, F2 g[Q]) {
  const int lane = threadIdx.x & 31;
  int xm = x - 1, xp = x + 2;
  if (xm < 0) xm += p.nx;
  if (xp >= p.nx) xp -= p.nx;
  const bool own_left = lane == 0 || x == 0;              // x - 1 not in the previous lane
  const bool own_right = lane == 31 || x + 2 >= p.nx;     // x + 2 not in the next lane
  int ys[3] = {y - 1, y, y + 1};
  if (ys[0] < 0) ys[0] += p.ny;
  if (ys[2] >= p.ny) ys[2] -= p.ny;
  int zs[3] = {z - 1, z, z + 1};
  if (Lat<Q>::D == 3) {
    if (zs[0] < 0) zs[0] += p.nz;
    if (zs[2] >= p.nz) zs[2] -= p.nz;
  }
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int dy = 1 - Lat<Q>::cy(i), dz = 1 - Lat<Q>::cz(i);
    const int row = (zs[dz] * p.ny + ys[dy]) * p.nx;
    const Pair16<T> w = *reinterpret_cast<const Pair16<T>*>(P.s[i] + row + x);
    const unsigned bits = *reinterpret_cast<const unsigned*>(&w);
    if (Lat<Q>::cx(i) == 0) {
      g[i] = Pack16<T>::ld(w.a, w.b);
    } else if (Lat<Q>::cx(i) > 0) {
      // sources x - 1, x
      const unsigned prev = __shfl_up_sync(0xffffffffu, bits, 1);
      Pair16<T> pw;
      *reinterpret_cast<unsigned*>(&pw) = prev;
      const T left = own_left ? P.s[i][row + xm] : pw.b;
      g[i] = Pack16<T>::ld(left, w.a);
    } else {
      // sources x + 1, x + 2
      const unsigned next = __shfl_down_sync(0xffffffffu, bits, 1);
      Pair16<T> nw;
      *reinterpret_cast<unsigned*>(&nw) = next;
      const T right = own_right ? P.s[i][row + xp] : nw.a;
      g[i] = Pack16<T>::ld(w.b, right);
    }
  }
}

// Band correction, collision and divergence check of the cells (x, x + 1)
// (the part of collide_cell between the pull and the store, on both lanes).
// x is even and tiles are 16 cells wide, so both cells lie in one tile.
template <int Q, bool IB>
__device__ __forceinline__ void collide_pair(F2 g[Q], const FluidParams<float>& p, int x, int y, int z) {
  F2 F[3], du[3];
  int band = -1;
  if (IB) {
    float da[3] = {0.0f, 0.0f, 0.0f}, db[3] = {0.0f, 0.0f, 0.0f};
    band = band_du<Q, float>(x, y, z, p, da);
    if (band >= 0) band_du<Q, float>(x + 1, y, z, p, db);
#pragma unroll
    for (int a = 0; a < 3; ++a) du[a] = Pk::make(da[a], db[a]);
  }
  const F2 drho = collide_v<Q, IB, Pk>(g, F, du, p);
  const float d0 = Pk::lo(drho), d1 = Pk::hi(drho);
  if (!(d0 > -1.0f && d0 < 99.0f) || !(d1 > -1.0f && d1 < 99.0f)) atomicOr(p.status, ST_DIVERGED);
  if (IB && band >= 0) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const F2 f = Pk::sub(F[a], Pk::splat(p.G[a]));
      p.band_F[band + a * TILE_CELLS] = Pk::lo(f);
      p.band_F[band + 1 + a * TILE_CELLS] = Pk::hi(f);
    }
  }
}

// The pair (x, x + 1) when either cell lies on a non-periodic face: the
// one-cell path with its face gathers, out of line so that its registers
// do not count against the two-cell kernels' hot path.
template <int Q, class T, bool IB>
__device__ __noinline__ void collide_face_pair(const DirPtrs<Q, T>& P, const FluidParams<float>& p, int x, int y,
                                               int z) {
  collide_cell<Q, T, true, IB>(P, p, x, y, z);
  collide_cell<Q, T, true, IB>(P, p, x + 1, y, z);
}

// Every cell of a grid with even nx: 2 x-adjacent cells per thread,
// blocks of up to 256 threads (the collide shape); IBL_PAIRS_MIN_BLOCKS blocks
// per SM without the band lookup, three with it.
#ifndef IBL_PAIRS_MIN_BLOCKS
#define IBL_PAIRS_MIN_BLOCKS 4
#endif
template <int Q, class T, bool IB>
__global__ void __launch_bounds__(256, IB ? 3 : IBL_PAIRS_MIN_BLOCKS) k_collide_pairs(DirPtrs<Q, T> P, FluidParams<float> p) {
  const int x = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  // every lane takes part in the word loads and shuffles; lanes outside the
  // grid read a clamped row and store nothing
  const bool inside = x < p.nx && y < p.ny;
  F2 g[Q];
  gather_pair_words<Q, T>(P, inside ? x : p.nx - 2, inside ? y : p.ny - 1, z, p, g);
  if (!inside) return;
  if (on_special_face<float>(x, y, z, Lat<Q>::D, p) || on_special_face<float>(x + 1, y, z, Lat<Q>::D, p)) {
    collide_face_pair<Q, T, IB>(P, p, x, y, z);
    return;
  }
  collide_pair<Q, IB>(g, p, x, y, z);
  const int cell = (z * p.ny + y) * p.nx + x;
#pragma unroll
  for (int i = 0; i < Q; ++i) *reinterpret_cast<unsigned*>(P.d[i] + cell) = Pack16<T>::st(g[i]);
}

// ---------------------------------------------------------------- 16-bit storage: planes in flight
// The two-cell kernel with each thread walking ZP planes in z: the 19 words
// of plane z + 1 (and the row-end halves its edge lanes need) are loaded
// before plane z collides, so a warp's loads for the next plane are in
// flight while it computes; the shuffles run once a plane's words have
// landed.
// Same pulls, same packed collision, same stores: bitwise the populations
// of the other kernels.
#ifndef IBL_ZP
#define IBL_ZP 8
#endif
constexpr int ZP = IBL_ZP;   // planes per thread

template <int Q, class T>
struct PairWords {
  unsigned w[Q];   // the word (x, x + 1) of each direction's source row
  T edge[Q];       // x - 1 (c_x = +1) or x + 2 (c_x = -1) where no neighbour lane holds it
};

template <int Q, class T>
__device__ __forceinline__ void load_pair_words(const DirPtrs<Q, T>& P, int x, int y, int z,
                                                const FluidParams<float>& p, PairWords<Q, T>& W) {
  const int lane = threadIdx.x & 31;
  int xm = x - 1, xp = x + 2;
  if (xm < 0) xm += p.nx;
  if (xp >= p.nx) xp -= p.nx;
  const bool own_left = lane == 0 || x == 0;
  const bool own_right = lane == 31 || x + 2 >= p.nx;
  int ys[3] = {y - 1, y, y + 1};
  if (ys[0] < 0) ys[0] += p.ny;
  if (ys[2] >= p.ny) ys[2] -= p.ny;
  int zs[3] = {z - 1, z, z + 1};
  if (Lat<Q>::D == 3) {
    if (zs[0] < 0) zs[0] += p.nz;
    if (zs[2] >= p.nz) zs[2] -= p.nz;
  }
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int dy = 1 - Lat<Q>::cy(i), dz = 1 - Lat<Q>::cz(i);
    const int row = (zs[dz] * p.ny + ys[dy]) * p.nx;
    W.w[i] = *reinterpret_cast<const unsigned*>(P.s[i] + row + x);
    if (Lat<Q>::cx(i) > 0) W.edge[i] = own_left ? P.s[i][row + xm] : T();
    else if (Lat<Q>::cx(i) < 0) W.edge[i] = own_right ? P.s[i][row + xp] : T();
  }
}

// The two cells' values per direction from a plane's words (every lane of
// the warp must call it: shuffles).
template <int Q, class T>
__device__ __forceinline__ void unpack_pair_words(const PairWords<Q, T>& W, int x, int nx, F2 g[Q]) {
  const int lane = threadIdx.x & 31;
  const bool own_left = lane == 0 || x == 0;
  const bool own_right = lane == 31 || x + 2 >= nx;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    Pair16<T> w;
    *reinterpret_cast<unsigned*>(&w) = W.w[i];
    if (Lat<Q>::cx(i) == 0) {
      g[i] = Pack16<T>::ld(w.a, w.b);
    } else if (Lat<Q>::cx(i) > 0) {
      Pair16<T> pw;
      *reinterpret_cast<unsigned*>(&pw) = __shfl_up_sync(0xffffffffu, W.w[i], 1);
      g[i] = Pack16<T>::ld(own_left ? W.edge[i] : pw.b, w.a);
    } else {
      Pair16<T> nw;
      *reinterpret_cast<unsigned*>(&nw) = __shfl_down_sync(0xffffffffu, W.w[i], 1);
      g[i] = Pack16<T>::ld(w.b, own_right ? W.edge[i] : nw.a);
    }
  }
}

#ifndef IBL_ZP_MIN_BLOCKS
#define IBL_ZP_MIN_BLOCKS 2
#endif
template <int Q, class T, bool IB>
__global__ void __launch_bounds__(256, IBL_ZP_MIN_BLOCKS) k_collide_pairs_zp(DirPtrs<Q, T> P, FluidParams<float> p) {
  const int x = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z0 = blockIdx.z * ZP, z1 = min(z0 + ZP, p.nz);
  // every lane loads and shuffles; lanes outside the grid read clamped rows
  const bool inside = x < p.nx && y < p.ny;
  const int xc = inside ? x : p.nx - 2, yc = inside ? y : p.ny - 1;
  PairWords<Q, T> next;
  load_pair_words<Q, T>(P, xc, yc, z0, p, next);
  for (int z = z0; z < z1; ++z) {
    // unpack this plane's words (landed during the previous plane's
    // collision), then put the next plane's loads in flight
    F2 g[Q];
    unpack_pair_words<Q, T>(next, xc, p.nx, g);
    if (z + 1 < z1) load_pair_words<Q, T>(P, xc, yc, z + 1, p, next);
    if (!inside) continue;
    if (on_special_face<float>(x, y, z, Lat<Q>::D, p) || on_special_face<float>(x + 1, y, z, Lat<Q>::D, p)) {
      collide_face_pair<Q, T, IB>(P, p, x, y, z);
      continue;
    }
    collide_pair<Q, IB>(g, p, x, y, z);
    const int cell = (z * p.ny + y) * p.nx + x;
#pragma unroll
    for (int i = 0; i < Q; ++i) *reinterpret_cast<unsigned*>(P.d[i] + cell) = Pack16<T>::st(g[i]);
  }
}

// ---------------------------------------------------------------- 16-bit storage: staged planes
// The two-cell kernel above keeps 19 words per thread in flight and then
// computes; at 4 blocks per SM the HBM then idles while most warps compute
// (long-scoreboard stalls lead, DRAM ~64 % busy).  Here a block of 64 x 4
// threads owns 128 x 4 cells of a column of SZ planes and walks it in z.
// While it collides plane z from shared memory, the source rows of plane
// z + 1 (for each direction i: the 4 rows y - c_y,i of plane z - c_z,i,
// cells x0 - 8 .. x0 + 135, one 288-byte segment each) arrive by bulk
// asynchronous copies (cp.async.bulk, completion counted in bytes on an
// mbarrier), so the loads of the next plane overlap the arithmetic of this
// one without holding registers.  Rows and planes wrap periodically; cells
// on non-periodic faces take the one-cell path (global pulls).  Every
// segment starts on a 16-byte boundary and is a multiple of 16 bytes long
// because nx is a multiple of 8.  The populations are bitwise those of the
// other kernels: the same values reach the same packed collision.
constexpr int SX = 128;                    // cells per block in x
constexpr int SY = 4;                      // rows per block
constexpr int SZ = 16;                     // planes per block
constexpr int SPAD = 8;                    // halo cells on each side (one 16-byte chunk)
constexpr int SROW = SX + 2 * SPAD;        // staged cells per row
constexpr long long STAGE_WAIT_LIMIT = 1LL << 26;   // mbarrier polls before giving up

__host__ __device__ constexpr size_t staged_smem_bytes(int Q) {
  return 2 * (size_t)Q * SY * SROW * 2 + 2 * sizeof(unsigned long long);
}

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

// One poll of the barrier's phase with the given parity; true once it completed.
__device__ __forceinline__ bool mbar_test(unsigned long long* bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// Bounded wait: false if the phase did not complete within the poll limit.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
  for (long long k = 0; k < STAGE_WAIT_LIMIT; ++k)
    if (mbar_test(bar, parity)) return true;
  return false;
}

// Order this thread's earlier shared-memory accesses before the async
// proxy's writes into the same buffer.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Thread t < Q * SY stages row t % SY of direction t / SY for plane z into
// buf: cells x0 - SPAD .. x0 + SX + SPAD - 1 of source row y0 + r - c_y of
// source plane z - c_z, both wrapped, as contiguous pieces split where the
// row wraps in x.
template <int Q, class T>
__device__ __forceinline__ void stage_plane(const DirPtrs<Q, T>& P, const FluidParams<float>& p, T* buf,
                                            unsigned long long* bar, int x0, int y0, int z, int tid) {
  if (tid >= Q * SY) return;
  const int i = tid / SY, r = tid % SY;
  int ys = y0 + r - Lat<Q>::cy(i);
  ys = ((ys % p.ny) + p.ny) % p.ny;
  int zs = z - Lat<Q>::cz(i);
  zs = ((zs % p.nz) + p.nz) % p.nz;
  // the direction's base P.s[i] is P.s[0] + i N (dir_ptrs), formed here so
  // that the parameter array is not indexed by a run-time value
  const T* row = P.s[0] + (long long)i * p.N + ((long long)zs * p.ny + ys) * p.nx;
  T* dst = buf + (i * SY + r) * SROW;
  fence_proxy_async();
  mbar_arrive_expect_tx(bar, SROW * (unsigned)sizeof(T));
  int done = 0;
  int xs = ((x0 - SPAD) % p.nx + p.nx) % p.nx;
  while (done < SROW) {
    const int len = min(SROW - done, p.nx - xs);
    bulk_copy_g2s(dst + done, row + xs, (unsigned)(len * sizeof(T)), bar);
    done += len;
    xs = 0;
  }
}

// One thread per cell pair (x, x + 1), 64 x 4 threads, SZ planes per block.
template <int Q, class T, bool IB>
__global__ void __launch_bounds__(256, IB ? 3 : 4) k_collide_pairs_staged(DirPtrs<Q, T> P, FluidParams<float> p) {
  extern __shared__ __align__(128) unsigned char stage_smem[];
  T* bufs = reinterpret_cast<T*>(stage_smem);
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(stage_smem + 2 * (size_t)Q * SY * SROW * sizeof(T));
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * blockDim.x + tx;
  const int x0 = blockIdx.x * SX, y0 = blockIdx.y * SY, z0 = blockIdx.z * SZ;
  const int planes = min(SZ, p.nz - z0);
  const int x = x0 + 2 * tx, y = y0 + ty;
  const bool inside = x < p.nx && y < p.ny;
  if (tid == 0) {
    mbar_init(&bar[0], Q * SY);
    mbar_init(&bar[1], Q * SY);
  }
  __syncthreads();
  stage_plane<Q, T>(P, p, bufs, &bar[0], x0, y0, z0, tid);
  for (int k = 0; k < planes; ++k) {
    const int b = k & 1;
    T* buf = bufs + (size_t)b * Q * SY * SROW;
    if (k + 1 < planes) stage_plane<Q, T>(P, p, bufs + (size_t)(b ^ 1) * Q * SY * SROW, &bar[b ^ 1], x0, y0,
                                          z0 + k + 1, tid);
    const bool ok = mbar_wait(&bar[b], (unsigned)((k >> 1) & 1));
    if (__syncthreads_or(!ok)) {
      // a copy did not land within the limit: report it, give the copies in
      // flight one more bounded wait, and leave this block's cells undone
      if (tid == 0) atomicOr(p.status, ST_TIMEOUT);
      mbar_wait(&bar[b], (unsigned)((k >> 1) & 1));
      if (k + 1 < planes) mbar_wait(&bar[b ^ 1], (unsigned)(((k + 1) >> 1) & 1));
      return;
    }
    const int z = z0 + k;
    if (inside) {
      if (on_special_face<float>(x, y, z, Lat<Q>::D, p) || on_special_face<float>(x + 1, y, z, Lat<Q>::D, p)) {
        collide_face_pair<Q, T, IB>(P, p, x, y, z);
      } else {
        F2 g[Q];
        const T* base = buf + ty * SROW + SPAD + 2 * tx;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          const T* s = base + i * SY * SROW;
          if (Lat<Q>::cx(i) == 0) {
            const Pair16<T> w = *reinterpret_cast<const Pair16<T>*>(s);
            g[i] = Pack16<T>::ld(w.a, w.b);
          } else {
            const int d = -Lat<Q>::cx(i);   // sources x - c_x, x + 1 - c_x
            g[i] = Pack16<T>::ld(s[d], s[d + 1]);
          }
        }
        collide_pair<Q, IB>(g, p, x, y, z);
        const int cell = (z * p.ny + y) * p.nx + x;
#pragma unroll
        for (int i = 0; i < Q; ++i) *reinterpret_cast<unsigned*>(P.d[i] + cell) = Pack16<T>::st(g[i]);
      }
    }
    __syncthreads();   // every thread is done with buf before it is staged again
  }
}

// Every cell, one per thread (blocks of the collide shape); IB selects the band lookup.
template <int Q, class T, bool PULL, bool IB>
__global__ void __launch_bounds__(256) k_collide(DirPtrs<Q, T> P, FluidParams<typename Store<T>::R> p) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= p.nx || y >= p.ny) return;
  collide_cell<Q, T, PULL, IB>(P, p, x, y, z);
}

// Cells outside the IB band, while the IB chain runs on other SMs: a
// persistent grid of 1024-thread blocks (one per SM: each holds the whole
// register file, so the SMs it does not take stay free for the solve), each
// walking 64 x 16-cell units of one z-plane; band tiles are skipped and
// left to k_collide_band.
constexpr int BULK_THREADS = 1024;
template <int Q, class T, bool PULL>
__global__ void __launch_bounds__(BULK_THREADS, 1) k_collide_bulk(DirPtrs<Q, T> P,
                                                                   FluidParams<typename Store<T>::R> p) {
  using R = typename Store<T>::R;
  const int ux = (p.nx + 63) >> 6, uy = (p.ny + 15) >> 4;
  const int lx = threadIdx.x & 63, ly = threadIdx.x >> 6;
  // unit u = blockIdx.x + k gridDim.x walked as (bx, by, z) with carries
  // instead of three divisions per unit
  const int G = gridDim.x;
  const int gx = G % ux, gy = (G / ux) % uy, gz = G / (ux * uy);
  int bx = blockIdx.x % ux, by = (blockIdx.x / ux) % uy, z = blockIdx.x / (ux * uy);
  while (z < p.nz) {
    const int x = (bx << 6) + lx, y = (by << 4) + ly;
    if (x < p.nx && y < p.ny && p.tile_slot[tile_index<Q, R>(x, y, z, p)] < 0)
      collide_cell<Q, T, PULL, false>(P, p, x, y, z);
    bx += gx;
    int carry = bx >= ux;
    bx -= carry ? ux : 0;
    by += gy + carry;
    carry = by >= uy;
    by -= carry ? uy : 0;
    z += gz + carry;
  }
}

// Cells of the IB band: one tile (TILE_CELLS cells) per block iteration over
// the assigned slots.
template <int Q, class T, bool PULL>
__global__ void __launch_bounds__(TILE_CELLS) k_collide_band(DirPtrs<Q, T> P, FluidParams<typename Store<T>::R> p,
                                                             const int* __restrict__ slot_tile,
                                                             const int* __restrict__ band_count, int cap) {
  const TileGeom& t = p.tg;
  const int n = min(*band_count, cap);
  const int lx = threadIdx.x % t.tx, ly = (threadIdx.x / t.tx) % t.ty, lz = threadIdx.x / (t.tx * t.ty);
  for (int s = blockIdx.x; s < n; s += gridDim.x) {
    const int tile = slot_tile[s];
    const int x = (tile % t.ntx) * t.tx + lx;
    const int y = ((tile / t.ntx) % t.nty) * t.ty + ly;
    const int z = (tile / (t.ntx * t.nty)) * t.tz + lz;
    if (x >= p.nx || y >= p.ny || z >= p.nz) continue;
    collide_cell<Q, T, PULL, true>(P, p, x, y, z);
  }
}

// rho, u = (sum c_i f_i + G/2)/rho and optionally f itself (FP64) of the
// current post-streaming populations.
template <int Q, class T, bool PULL>
__global__ void k_fields(const T* __restrict__ src, FluidParams<typename Store<T>::R> p,
                         double* __restrict__ rho_out, double* __restrict__ u_out,
                         double* __restrict__ pop_out) {
  using R = typename Store<T>::R;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= p.nx || y >= p.ny) return;
  const long long cell = ((long long)z * p.ny + y) * p.nx + x;
  R g[Q];
  gather_q<Q, T, PULL, R>(src, x, y, z, cell, p, g);
  double drho = 0, m[3] = {0, 0, 0};
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const double gi = (double)g[i];
    drho += gi;
    m[0] += Lat<Q>::cx(i) * gi;
    m[1] += Lat<Q>::cy(i) * gi;
    m[2] += Lat<Q>::cz(i) * gi;
    if (pop_out) pop_out[i * p.N + cell] = gi + Lat<Q>::w(i);
  }
  const double rho = 1.0 + drho;
  if (rho_out) rho_out[cell] = rho;
  if (u_out)
    for (int a = 0; a < Lat<Q>::D; ++a)
      u_out[a * p.N + cell] = (m[a] + 0.5 * (double)p.G[a]) / rho;
}

template <int Q, class T>
__global__ void k_init_eq(T* __restrict__ dst, long long N, const double* __restrict__ rho_in,
                          const double* __restrict__ u_in) {
  const long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= N) return;
  const double rho = rho_in ? rho_in[cell] : 1.0;
  double u[3] = {0, 0, 0};
  if (u_in)
    for (int a = 0; a < Lat<Q>::D; ++a) u[a] = u_in[a * N + cell];
  const double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const double cu = Lat<Q>::cx(i) * u[0] + Lat<Q>::cy(i) * u[1] + Lat<Q>::cz(i) * u[2];
    const double w = Lat<Q>::w(i);
    // f_eq - w, Eq. 4
    const double geq = w * ((rho - 1.0) + rho * (3.0 * cu + 4.5 * cu * cu - 1.5 * usq));
    dst[i * N + cell] = Store<T>::st((typename Store<T>::R)geq);
  }
}

template <int Q, class T>
__global__ void k_set_pop(T* __restrict__ dst, long long N, const double* __restrict__ f) {
  const long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= N) return;
#pragma unroll
  for (int i = 0; i < Q; ++i)
    dst[i * N + cell] = Store<T>::st((typename Store<T>::R)(f[i * N + cell] - Lat<Q>::w(i)));
}

// Fixed-order FP64 mass: block b sums cells [b*chunk, (b+1)*chunk) in a fixed
// strided pattern and a fixed tree; the host-side second pass is a fixed loop.
template <int Q, class T, bool PULL>
__global__ void k_mass(const T* __restrict__ src, FluidParams<typename Store<T>::R> p,
                       double* __restrict__ partials, long long chunk) {
  using R = typename Store<T>::R;
  __shared__ double sh[256];
  const long long start = (long long)blockIdx.x * chunk;
  long long end = start + chunk;
  if (end > p.N) end = p.N;
  double acc = 0;
  for (long long cell = start + threadIdx.x; cell < end; cell += blockDim.x) {
    const int x = (int)(cell % p.nx);
    const long long yz = cell / p.nx;
    const int y = (int)(yz % p.ny);
    const int z = (int)(yz / p.ny);
    R g[Q];
    gather_q<Q, T, PULL, R>(src, x, y, z, cell, p, g);
    double drho = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) drho += (double)g[i];
    acc += 1.0 + drho;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}

// Total of the mass partials in a fixed order (one warp) and the test of
// the periodic mass check.  mode 0 stores the total as the reference (at
// initialisation); mode 1 records it and flags divergence for a non-finite
// total or, when the faces conserve mass (no Zou-He face), a relative change
// from the reference above tol.  ref: [0] reference, [1] last total, [2] checks.
__global__ void k_mass_check(const double* __restrict__ partials, int nparts, double* __restrict__ ref, int mode,
                             double tol, int closed, int* status) {
  const int lane = threadIdx.x;
  double s = 0.0;
  for (int k = lane; k < nparts; k += 32) s += partials[k];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane != 0) return;
  if (mode == 0) {
    ref[0] = s;
    ref[1] = s;
    ref[2] = 0.0;
    return;
  }
  ref[1] = s;
  ref[2] += 1.0;
  if (!isfinite(s) || (closed && fabs(s - ref[0]) > tol * fabs(ref[0]))) atomicOr(status, ST_DIVERGED);
}

// ----------------------------------------------------------------- host side
template <class R>
FluidParams<R> make_params(ibl_ctx* c, bool with_ib) {
  FluidParams<R> p;
  p.nx = c->nx; p.ny = c->ny; p.nz = c->nz; p.N = c->N;
  for (int i = 0; i < 6; ++i) p.bc[i] = c->bc[i];
  for (int a = 0; a < 3; ++a) {
    p.u_in[a] = (R)c->u_in[a];
    p.G[a] = (R)c->G[a] + R(0);   // no negative zero: F = G exactly off the band
  }
  p.rho_out = (R)c->rho_out;
  p.omega = (R)(1.0 / c->tau);
  p.pref = (R)(1.0 - 0.5 / c->tau);
  p.tg = c->tg;
  p.tile_slot = with_ib ? c->d_tile_slot : nullptr;
  p.band_acc = with_ib ? c->d_acc : nullptr;
  p.band_F = with_ib ? (R*)c->d_band_F : nullptr;
  p.status = c->d_status;
  return p;
}

static dim3 cell_block(ibl_ctx* c) {
  return dim3(c->collide_bx, c->collide_by, 1);
}
static dim3 cell_grid(ibl_ctx* c, dim3 b) {
  return dim3((c->nx + b.x - 1) / b.x, (c->ny + b.y - 1) / b.y, c->nz);
}

template <int Q, class T>
DirPtrs<Q, T> dir_ptrs(ibl_ctx* c) {
  const T* src = (const T*)c->f[c->cur];
  T* dst = (T*)c->f[c->cur ^ 1];
  DirPtrs<Q, T> P;
  for (int i = 0; i < Q; ++i) {
    P.s[i] = src + (size_t)i * c->N;
    P.d[i] = dst + (size_t)i * c->N;
  }
  return P;
}

template <int Q, class T>
cudaError_t collide_q(ibl_ctx* c, bool with_ib) {
  using R = typename Store<T>::R;
  auto p = make_params<R>(c, with_ib);
  const DirPtrs<Q, T> P = dir_ptrs<Q, T>(c);
  dim3 b = cell_block(c), g = cell_grid(c, b);
  if constexpr (sizeof(T) == 2) {
    if constexpr (Q == 19) {
      if (!c->poststream && c->nx % 8 == 0 && c->collide_pairs == 2) {
        // 16-bit storage, nx a multiple of 8: staged planes (see k_collide_pairs_staged)
        const dim3 sb(SX / 2, SY, 1);
        const dim3 sg((c->nx + SX - 1) / SX, (c->ny + SY - 1) / SY, (c->nz + SZ - 1) / SZ);
        const size_t smem = staged_smem_bytes(Q);
        if (with_ib) k_collide_pairs_staged<Q, T, true><<<sg, sb, smem, c->stream>>>(P, p);
        else k_collide_pairs_staged<Q, T, false><<<sg, sb, smem, c->stream>>>(P, p);
        c->launches++;
        return cudaGetLastError();
      }
    }
    if (!c->poststream && c->nx % 2 == 0 && c->collide_pairs == 3) {
      // 16-bit storage: two cells per thread, ZP planes per thread
      const dim3 zb(b.x, b.y, 1);
      const dim3 zg((c->nx / 2 + zb.x - 1) / zb.x, (c->ny + zb.y - 1) / zb.y, (c->nz + ZP - 1) / ZP);
      if (with_ib) k_collide_pairs_zp<Q, T, true><<<zg, zb, 0, c->stream>>>(P, p);
      else k_collide_pairs_zp<Q, T, false><<<zg, zb, 0, c->stream>>>(P, p);
      c->launches++;
      return cudaGetLastError();
    }
    if (!c->poststream && c->nx % 2 == 0 && c->collide_pairs >= 1) {
      // 16-bit storage: two x-adjacent cells per thread
      g.x = (c->nx / 2 + b.x - 1) / b.x;
      if (with_ib) k_collide_pairs<Q, T, true><<<g, b, 0, c->stream>>>(P, p);
      else k_collide_pairs<Q, T, false><<<g, b, 0, c->stream>>>(P, p);
      c->launches++;
      return cudaGetLastError();
    }
  }
  if (c->poststream) {
    if (with_ib) k_collide<Q, T, false, true><<<g, b, 0, c->stream>>>(P, p);
    else k_collide<Q, T, false, false><<<g, b, 0, c->stream>>>(P, p);
  } else {
    if (with_ib) k_collide<Q, T, true, true><<<g, b, 0, c->stream>>>(P, p);
    else k_collide<Q, T, true, false><<<g, b, 0, c->stream>>>(P, p);
  }
  c->launches++;
  return cudaGetLastError();
}

template <int Q, class T>
cudaError_t collide_bulk_q(ibl_ctx* c, int blocks, cudaStream_t st) {
  using R = typename Store<T>::R;
  auto p = make_params<R>(c, true);
  const DirPtrs<Q, T> P = dir_ptrs<Q, T>(c);
  if (c->poststream) k_collide_bulk<Q, T, false><<<blocks, BULK_THREADS, 0, st>>>(P, p);
  else k_collide_bulk<Q, T, true><<<blocks, BULK_THREADS, 0, st>>>(P, p);
  c->launches++;
  return cudaGetLastError();
}

template <int Q, class T>
cudaError_t collide_band_q(ibl_ctx* c, int blocks) {
  using R = typename Store<T>::R;
  auto p = make_params<R>(c, true);
  const DirPtrs<Q, T> P = dir_ptrs<Q, T>(c);
  if (c->poststream)
    k_collide_band<Q, T, false><<<blocks, TILE_CELLS, 0, c->stream>>>(P, p, c->d_slot_tile, c->d_band_count,
                                                                       c->cap_slots);
  else
    k_collide_band<Q, T, true><<<blocks, TILE_CELLS, 0, c->stream>>>(P, p, c->d_slot_tile, c->d_band_count,
                                                                      c->cap_slots);
  c->launches++;
  return cudaGetLastError();
}

template <int Q, class T>
cudaError_t fields_q(ibl_ctx* c, double* d_rho, double* d_u, double* d_pop) {
  using R = typename Store<T>::R;
  auto p = make_params<R>(c, false);
  const T* src = (const T*)c->f[c->cur];
  dim3 b(64, 4, 1), g = cell_grid(c, b);
  if (c->poststream) k_fields<Q, T, false><<<g, b, 0, c->stream>>>(src, p, d_rho, d_u, d_pop);
  else k_fields<Q, T, true><<<g, b, 0, c->stream>>>(src, p, d_rho, d_u, d_pop);
  c->launches++;
  return cudaGetLastError();
}

template <int Q, class T>
cudaError_t mass_q(ibl_ctx* c, double* d_partials, int nparts) {
  using R = typename Store<T>::R;
  auto p = make_params<R>(c, false);
  const T* src = (const T*)c->f[c->cur];
  long long chunk = (c->N + nparts - 1) / nparts;
  if (c->poststream) k_mass<Q, T, false><<<nparts, 256, 0, c->stream>>>(src, p, d_partials, chunk);
  else k_mass<Q, T, true><<<nparts, 256, 0, c->stream>>>(src, p, d_partials, chunk);
  c->launches++;
  return cudaGetLastError();
}

template <int Q, class T>
cudaError_t init_q(ibl_ctx* c, const double* d_rho, const double* d_u) {
  const int bs = 256;
  const long long nb = (c->N + bs - 1) / bs;
  k_init_eq<Q, T><<<(unsigned)nb, bs, 0, c->stream>>>((T*)c->f[c->cur], c->N, d_rho, d_u);
  c->launches++;
  return cudaGetLastError();
}

template <int Q, class T>
cudaError_t setpop_q(ibl_ctx* c, const double* d_f) {
  const int bs = 256;
  const long long nb = (c->N + bs - 1) / bs;
  k_set_pop<Q, T><<<(unsigned)nb, bs, 0, c->stream>>>((T*)c->f[c->cur], c->N, d_f);
  c->launches++;
  return cudaGetLastError();
}

// Dispatch on (lattice, storage precision).
#define IBL_DISPATCH(FN, ...)                                                       \
  do {                                                                              \
    if (c->Q == 9) {                                                                \
      switch (c->prec) {                                                            \
        case IBL_FP64: return FN<9, double>(c, ##__VA_ARGS__);                      \
        case IBL_FP32: return FN<9, float>(c, ##__VA_ARGS__);                       \
        case IBL_FP16DEV: return FN<9, __half>(c, ##__VA_ARGS__);                  \
        default: return FN<9, __nv_bfloat16>(c, ##__VA_ARGS__);                     \
      }                                                                             \
    } else {                                                                        \
      switch (c->prec) {                                                            \
        case IBL_FP64: return FN<19, double>(c, ##__VA_ARGS__);                     \
        case IBL_FP32: return FN<19, float>(c, ##__VA_ARGS__);                      \
        case IBL_FP16DEV: return FN<19, __half>(c, ##__VA_ARGS__);                  \
        default: return FN<19, __nv_bfloat16>(c, ##__VA_ARGS__);                    \
      }                                                                             \
    }                                                                               \
  } while (0)

cudaError_t launch_collide(ibl_ctx* c, bool with_ib) { IBL_DISPATCH(collide_q, with_ib); }
cudaError_t launch_collide_bulk(ibl_ctx* c, int blocks, cudaStream_t st) { IBL_DISPATCH(collide_bulk_q, blocks, st); }
cudaError_t launch_collide_band(ibl_ctx* c, int blocks) { IBL_DISPATCH(collide_band_q, blocks); }
cudaError_t launch_fields(ibl_ctx* c, double* d_rho, double* d_u, double* d_pop) {
  IBL_DISPATCH(fields_q, d_rho, d_u, d_pop);
}
cudaError_t launch_mass(ibl_ctx* c, double* d_partials, int nparts, double* d_out) {
  (void)d_out;
  IBL_DISPATCH(mass_q, d_partials, nparts);
}
cudaError_t launch_mass_check(ibl_ctx* c, int mode) {
  cudaError_t e = launch_mass(c, c->d_mass_parts, MASS_PARTS, nullptr);
  if (e != cudaSuccess) return e;
  const double tol = c->mass_tol > 0 ? c->mass_tol
                                     : (c->prec == IBL_FP64 ? 1e-9 : (c->prec == IBL_FP32 ? 1e-4 : 1e-2));
  int closed = 1;
  for (int f = 0; f < 6; ++f) closed &= (c->bc[f] == IBL_PERIODIC || c->bc[f] == IBL_BOUNCEBACK) ? 1 : 0;
  k_mass_check<<<1, 32, 0, c->stream>>>(c->d_mass_parts, MASS_PARTS, c->d_mass_ref, mode, tol, closed, c->d_status);
  c->launches++;
  return cudaGetLastError();
}

cudaError_t launch_init_eq(ibl_ctx* c, const double* d_rho, const double* d_u) {
  IBL_DISPATCH(init_q, d_rho, d_u);
}
cudaError_t launch_set_pop(ibl_ctx* c, const double* d_f) { IBL_DISPATCH(setpop_q, d_f); }

}  // namespace ibl

// ----------------------------------------------------------------- allocation-free mass
// ibl_mass allocates its partial sums on every call.  For callers that may
// not allocate device memory, ibl_mass_noalloc keeps them in this file-scope
// array instead (32 KB, held by every GPU that loads the library until exit).
namespace {
constexpr int NOALLOC_MAX_PARTS = 4096;
__device__ __align__(256) double g_mass_partials[NOALLOC_MAX_PARTS];
constexpr int NOALLOC_MAX_DEVICES = 64;
double* g_mass_partials_addr[NOALLOC_MAX_DEVICES] = {nullptr};
std::mutex g_noalloc_mutex;
}  // namespace

extern "C" ibl_status ibl_mass_noalloc(ibl_ctx* c, int32_t nparts, double* mass) {
  using namespace ibl;
  if (!c) return IBL_EINVAL;
  if (!mass) return fail(c, IBL_EINVAL, "mass is NULL");
  if (nparts < 1 || nparts > NOALLOC_MAX_PARTS)
    return fail(c, IBL_EINVAL, "ibl_mass_noalloc: nparts must be in [1, 4096] (size of its static scratch)");
  if (!c->initialised) return fail(c, IBL_ESTATE, "fluid not initialised");
  if (c->device < 0 || c->device >= NOALLOC_MAX_DEVICES)
    return fail(c, IBL_EINVAL, "ibl_mass_noalloc supports device ordinals below 64");
  ibl_status s = sync_and_collect(c);
  if (s != IBL_OK && s != IBL_ENOTCONV) return s;
  // The array's name is a host-side stand-in: its device address is looked up
  // once per device, with that device current, on the first call.
  double* d_parts = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_mass_partials_addr[c->device]) {
      int prev = 0;
      cudaError_t e = cudaGetDevice(&prev);
      if (e == cudaSuccess && prev != c->device) e = cudaSetDevice(c->device);
      void* addr = nullptr;
      if (e == cudaSuccess) e = cudaGetSymbolAddress(&addr, g_mass_partials);
      if (prev != c->device) cudaSetDevice(prev);
      if (e != cudaSuccess) return cuda_check(c, e, "cudaGetSymbolAddress(g_mass_partials)");
      g_mass_partials_addr[c->device] = static_cast<double*>(addr);
    }
    d_parts = g_mass_partials_addr[c->device];
  }
  // every block writes its partial, so nothing needs clearing between calls
  cudaError_t e = launch_mass(c, d_parts, nparts, nullptr);
  double h[NOALLOC_MAX_PARTS];
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h, d_parts, sizeof(double) * nparts, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_check(c, e, "ibl_mass_noalloc");
  double acc = 0.0;
  for (int k = 0; k < nparts; ++k) acc += h[k];
  *mass = acc;
  return s;
}
