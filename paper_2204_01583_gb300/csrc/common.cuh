// Device helpers shared by the library's kernels: complex arithmetic, lattice
// neighbours, the Wilson stencil at one site and deterministic block reductions.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "ov_internal.h"

// ---------------------------------------------------------- double-float reals
// DF: a real carried as an unevaluated sum hi + lo of two FP32 numbers (|lo| <= ulp(hi)/2
// after each operation), giving ~48-bit significands from FP32 instructions alone.
// Sums use Knuth's error-free two-sum, products the FMA-based exact product; every
// operation renormalises with a fast two-sum.  On GB300, where FP64 runs at 1/58 of the
// FP32 rate, this carries FP64-class accuracy at FP32 throughput.
struct DF {
  float hi, lo;
  __host__ __device__ __forceinline__ DF() {}
  __host__ __device__ __forceinline__ DF(float h, float l) : hi(h), lo(l) {}
  __device__ __forceinline__ explicit DF(double x) {
    hi = __double2float_rn(x);
    lo = __double2float_rn(x - (double)hi);
  }
  __device__ __forceinline__ explicit DF(int x) : hi((float)x), lo(0.f) {}
  __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ DF df_quick_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return DF(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ void df_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ DF operator-(DF a) { return DF(-a.hi, -a.lo); }
__device__ __forceinline__ DF operator+(DF a, DF b) {
  float s, e;
  df_two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return df_quick_two_sum(s, e);
}
__device__ __forceinline__ DF operator-(DF a, DF b) { return a + (-b); }
__device__ __forceinline__ DF operator*(DF a, DF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_quick_two_sum(p, e);
}
// a * b + c with one renormalisation
__device__ __forceinline__ DF fma(DF a, DF b, DF c) {
  const float p = __fmul_rn(a.hi, b.hi);
  const float pe = __fmaf_rn(a.hi, b.hi, -p);
  float s, e;
  df_two_sum(c.hi, p, s, e);
  float t = __fadd_rn(__fadd_rn(e, pe), c.lo);
  t = __fmaf_rn(a.hi, b.lo, t);
  t = __fmaf_rn(a.lo, b.hi, t);
  return df_quick_two_sum(s, t);
}
// a * b + c without the final renormalisation (the result's low part may exceed half an
// ulp of its high part by a few units; fine for a running sum renormalised at the end)
__device__ __forceinline__ DF fma_unnormalised(DF a, DF b, DF c) {
  const float p = __fmul_rn(a.hi, b.hi);
  const float pe = __fmaf_rn(a.hi, b.hi, -p);
  float s, e;
  df_two_sum(c.hi, p, s, e);
  float t = __fadd_rn(__fadd_rn(e, pe), c.lo);
  t = __fmaf_rn(a.hi, b.lo, t);
  t = __fmaf_rn(a.lo, b.hi, t);
  return DF(s, t);
}
__device__ __forceinline__ DF& operator+=(DF& a, DF b) { return a = a + b; }
__device__ __forceinline__ DF& operator-=(DF& a, DF b) { return a = a - b; }

template <typename R>
struct Cx {
  R re, im;
};

// Storage type of one complex number and its (un)packing, per arithmetic type.
template <typename R> struct Store;
template <> struct Store<double> {
  using T = double2;
  __device__ __forceinline__ static Cx<double> unpack(double2 v) { return {v.x, v.y}; }
  __device__ __forceinline__ static double2 pack(Cx<double> c) { return make_double2(c.re, c.im); }
};
template <> struct Store<float> {
  using T = float2;
  __device__ __forceinline__ static Cx<float> unpack(float2 v) { return {v.x, v.y}; }
  __device__ __forceinline__ static float2 pack(Cx<float> c) { return make_float2(c.re, c.im); }
};
template <> struct Store<DF> {
  using T = float4;  // (re.hi, re.lo, im.hi, im.lo)
  __device__ __forceinline__ static Cx<DF> unpack(float4 v) { return {DF(v.x, v.y), DF(v.z, v.w)}; }
  __device__ __forceinline__ static float4 pack(Cx<DF> c) { return make_float4(c.re.hi, c.re.lo, c.im.hi, c.im.lo); }
};

// Loads: CG = false reads through the read-only (non-coherent) path, for data no block
// writes during the launch; CG = true reads from L2 (ld.global.cg), for data other blocks
// of a persistent launch wrote before a grid barrier.
template <typename R, bool CG = false>
__device__ __forceinline__ Cx<R> ld(const typename Store<R>::T* p) {
  return Store<R>::unpack(CG ? __ldcg(p) : __ldg(p));
}
template <typename R>
__device__ __forceinline__ void st(typename Store<R>::T* p, Cx<R> v) {
  *p = Store<R>::pack(v);
}
// complex from two doubles in the storage precision (exact split for DF)
template <typename R>
__device__ __forceinline__ Cx<R> cx_from(double re, double im) {
  return {(R)re, (R)im};
}

template <typename R> __device__ __forceinline__ Cx<R> cadd(Cx<R> a, Cx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <typename R> __device__ __forceinline__ Cx<R> csub(Cx<R> a, Cx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <typename R> __device__ __forceinline__ Cx<R> cscale(R s, Cx<R> a) { return {s * a.re, s * a.im}; }
// i * a and -i * a
template <typename R> __device__ __forceinline__ Cx<R> cmuli(Cx<R> a) { return {-a.im, a.re}; }
template <typename R> __device__ __forceinline__ Cx<R> cmulmi(Cx<R> a) { return {a.im, -a.re}; }
template <typename R> __device__ __forceinline__ Cx<R> cneg(Cx<R> a) { return {-a.re, -a.im}; }
// acc + a * b
template <typename R>
__device__ __forceinline__ Cx<R> cfma(Cx<R> a, Cx<R> b, Cx<R> acc) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
  return acc;
}
// acc + conj(a) * b
template <typename R>
__device__ __forceinline__ Cx<R> cfmaconj(Cx<R> a, Cx<R> b, Cx<R> acc) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(-a.im, b.re, acc.im);
  return acc;
}
template <typename R> __device__ __forceinline__ R cnorm2(Cx<R> a) { return a.re * a.re + a.im * a.im; }

// ------------------------------------------------------------ neighbours

__device__ __forceinline__ void site_coords(const Geom& g, int s, int c[4]) {
  c[0] = s % g.L[0];
  int q = s / g.L[0];
  c[1] = q % g.L[1];
  q /= g.L[1];
  c[2] = q % g.L[2];
  c[3] = q / g.L[2];
}

// site index of x + mu (fwd) or x - mu (bwd) and the boundary sign of that hop
__device__ __forceinline__ int nb_fwd(const Geom& g, int s, const int c[4], int mu, int* sgn) {
  if (c[mu] + 1 == g.L[mu]) {
    *sgn = (mu == 3) ? g.bc_t : 1;
    return s - (g.L[mu] - 1) * g.st[mu];
  }
  *sgn = 1;
  return s + g.st[mu];
}
__device__ __forceinline__ int nb_bwd(const Geom& g, int s, const int c[4], int mu, int* sgn) {
  if (c[mu] == 0) {
    *sgn = (mu == 3) ? g.bc_t : 1;
    return s + (g.L[mu] - 1) * g.st[mu];
  }
  *sgn = 1;
  return s - g.st[mu];
}

// ------------------------------------------------------- spin structure
// Chiral basis: gamma_mu = [[0, A_mu], [A_mu^dag, 0]] with
//   A_x = -i sigma_1, A_y = -i sigma_2, A_z = -i sigma_3, A_t = 1.
// (1 -+ gamma_mu) psi = (h, -+ A^dag h) with h = psi_up -+ A psi_lo  (A unitary).

template <int MU, typename R>
__device__ __forceinline__ void mulA(Cx<R> l0, Cx<R> l1, Cx<R>& a0, Cx<R>& a1) {
  if (MU == 0) { a0 = cmulmi(l1); a1 = cmulmi(l0); }
  else if (MU == 1) { a0 = cneg(l1); a1 = l0; }
  else if (MU == 2) { a0 = cmulmi(l0); a1 = cmuli(l1); }
  else { a0 = l0; a1 = l1; }
}
template <int MU, typename R>
__device__ __forceinline__ void mulAdag(Cx<R> h0, Cx<R> h1, Cx<R>& a0, Cx<R>& a1) {
  if (MU == 0) { a0 = cmuli(h1); a1 = cmuli(h0); }
  else if (MU == 1) { a0 = h1; a1 = cneg(h0); }
  else if (MU == 2) { a0 = cmuli(h0); a1 = cmulmi(h1); }
  else { a0 = h0; a1 = h1; }
}

// One direction of the hopping term, both hops, accumulated into acc[12]
// (acc -= 1/2 [(1 - g) U psi(x+mu) + (1 + g) U(x-mu)^dag psi(x-mu)]).
// in: spinor planes, element (k, site) at in[k * V + site]; U: link planes.
template <int MU, typename R, bool CG = false>
__device__ __forceinline__ void hop_dir(const typename Store<R>::T* __restrict__ in,
                                        const typename Store<R>::T* __restrict__ U, const Geom& g,
                                        int s, const int c[4], Cx<R> acc[12]) {
  const int V = g.V;
#pragma unroll
  for (int dir = 0; dir < 2; ++dir) {
    int sgn;
    const int sn = dir == 0 ? nb_fwd(g, s, c, MU, &sgn) : nb_bwd(g, s, c, MU, &sgn);
    const int sl = dir == 0 ? s : sn;  // link site
    // half spinor h[spin 2][colour 3]
    Cx<R> h0[3], h1[3];
#pragma unroll
    for (int col = 0; col < 3; ++col) {
      Cx<R> p0 = ld<R, CG>(in + (0 * 3 + col) * (size_t)V + sn);
      Cx<R> p1 = ld<R, CG>(in + (1 * 3 + col) * (size_t)V + sn);
      Cx<R> p2 = ld<R, CG>(in + (2 * 3 + col) * (size_t)V + sn);
      Cx<R> p3 = ld<R, CG>(in + (3 * 3 + col) * (size_t)V + sn);
      Cx<R> a0, a1;
      mulA<MU>(p2, p3, a0, a1);
      if (dir == 0) { h0[col] = csub(p0, a0); h1[col] = csub(p1, a1); }
      else { h0[col] = cadd(p0, a0); h1[col] = cadd(p1, a1); }
    }
    const R f = R(-0.5) * R(sgn);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      Cx<R> u0 = {R(0), R(0)}, u1 = {R(0), R(0)};
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        // forward: U[i][j]; backward: (U^dag)[i][j] = conj(U[j][i])
        const int e = dir == 0 ? (i * 3 + j) : (j * 3 + i);
        Cx<R> l = ld<R>(U + (MU * 9 + e) * (size_t)V + sl);
        if (dir == 0) { u0 = cfma(l, h0[j], u0); u1 = cfma(l, h1[j], u1); }
        else { u0 = cfmaconj(l, h0[j], u0); u1 = cfmaconj(l, h1[j], u1); }
      }
      Cx<R> b0, b1;
      mulAdag<MU>(u0, u1, b0, b1);
      // upper: += f * u ; lower: += f * (-+ A^dag u)
      acc[0 * 3 + i] = cadd(acc[0 * 3 + i], cscale(f, u0));
      acc[1 * 3 + i] = cadd(acc[1 * 3 + i], cscale(f, u1));
      if (dir == 0) {
        acc[2 * 3 + i] = csub(acc[2 * 3 + i], cscale(f, b0));
        acc[3 * 3 + i] = csub(acc[3 * 3 + i], cscale(f, b1));
      } else {
        acc[2 * 3 + i] = cadd(acc[2 * 3 + i], cscale(f, b0));
        acc[3 * 3 + i] = cadd(acc[3 * 3 + i], cscale(f, b1));
      }
    }
  }
}

// The lower spins of both hops of direction MU: A_mu^dag d with d_s = s_b u_b - s_f u_f
// = m2 uf_s + ub_s (m2 = -2 s_f, ub = s_f u_f + s_b u_b), each real output one FMA whose
// sign is folded into its operands (A_mu^dag is a permutation with unit phases).
template <int MU, typename R>
__device__ __forceinline__ void lower_from(Cx<R> uf0, Cx<R> ub0, Cx<R> uf1, Cx<R> ub1, R m2, Cx<R>& a0,
                                           Cx<R>& a1) {
  auto P = [m2](R f, R u) { return fma(m2, f, u); };    //  d
  auto N = [m2](R f, R u) { return fma(-m2, f, -u); };  // -d
  if (MU == 0) {         // A_x^dag d = (i d1, i d0)
    a0 = {N(uf1.im, ub1.im), P(uf1.re, ub1.re)};
    a1 = {N(uf0.im, ub0.im), P(uf0.re, ub0.re)};
  } else if (MU == 1) {  // A_y^dag d = (d1, -d0)
    a0 = {P(uf1.re, ub1.re), P(uf1.im, ub1.im)};
    a1 = {N(uf0.re, ub0.re), N(uf0.im, ub0.im)};
  } else if (MU == 2) {  // A_z^dag d = (i d0, -i d1)
    a0 = {N(uf0.im, ub0.im), P(uf0.re, ub0.re)};
    a1 = {P(uf1.im, ub1.im), N(uf1.re, ub1.re)};
  } else {               // A_t^dag d = d
    a0 = {P(uf0.re, ub0.re), P(uf0.im, ub0.im)};
    a1 = {P(uf1.re, ub1.re), P(uf1.im, ub1.im)};
  }
}

// Both hops of direction MU for one site, without the -1/2 and boundary-sign factors
// multiplied in: acc[12] = (upper: s_f u_f + s_b u_b, lower: A_mu^dag (s_b u_b - s_f u_f))
// with u_f = U_mu(x) h_f, h_f = psi_up(x+mu) - A_mu psi_lo(x+mu), u_b = U_mu(x-mu)^dag h_b,
// h_b = psi_up(x-mu) + A_mu psi_lo(x-mu) and s_f, s_b the boundary signs (applied as
// selects; SIGNED = false: the links carry them and both are +1).  The hop term of H_W
// is -1/2 acc (or the links carry the -1/2 as well).  The backward link products
// accumulate onto t u_f (t = s_f s_b), so C = t u_f + u_b comes out of the FMA chain:
// upper = s_b C, lower from s_b C - 2 s_f u_f (one FMA per real).  On GB300's FP64
// pipe every floating-point instruction saved is time: this form issues 72 + 72 FMAs,
// 24 projection adds and 12 FMAs per direction.
template <int MU, typename R, bool CG = false, bool SIGNED = true>
__device__ __forceinline__ void hop_dir_unscaled(const typename Store<R>::T* __restrict__ in,
                                                 const typename Store<R>::T* __restrict__ U, const Geom& g,
                                                 int s, const int c[4], Cx<R> acc[12]) {
  const int V = g.V;
  Cx<R> uf[6], ub[6];  // [spin * 3 + row]: u_f, then s_b C
  int sg[2];
#pragma unroll
  for (int dir = 0; dir < 2; ++dir) {
    const int sn = dir == 0 ? nb_fwd(g, s, c, MU, &sg[dir]) : nb_bwd(g, s, c, MU, &sg[dir]);
    if (!SIGNED) sg[dir] = 1;
    const int sl = dir == 0 ? s : sn;  // link site
    Cx<R> h0[3], h1[3];
#pragma unroll
    for (int col = 0; col < 3; ++col) {
      Cx<R> p0 = ld<R, CG>(in + (0 * 3 + col) * (size_t)V + sn);
      Cx<R> p1 = ld<R, CG>(in + (1 * 3 + col) * (size_t)V + sn);
      Cx<R> p2 = ld<R, CG>(in + (2 * 3 + col) * (size_t)V + sn);
      Cx<R> p3 = ld<R, CG>(in + (3 * 3 + col) * (size_t)V + sn);
      Cx<R> a0, a1;
      mulA<MU>(p2, p3, a0, a1);
      if (dir == 0) { h0[col] = csub(p0, a0); h1[col] = csub(p1, a1); }
      else { h0[col] = cadd(p0, a0); h1[col] = cadd(p1, a1); }
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      Cx<R> u0 = {R(0), R(0)}, u1 = {R(0), R(0)};
      if (dir == 1) {  // start from t u_f, t = s_f s_b
        const bool flip = SIGNED && sg[0] != sg[1];
        u0 = flip ? cneg(uf[i]) : uf[i];
        u1 = flip ? cneg(uf[3 + i]) : uf[3 + i];
      }
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const int e = dir == 0 ? (i * 3 + j) : (j * 3 + i);
        Cx<R> l = ld<R>(U + (MU * 9 + e) * (size_t)V + sl);
        if (dir == 0) { u0 = cfma(l, h0[j], u0); u1 = cfma(l, h1[j], u1); }
        else { u0 = cfmaconj(l, h0[j], u0); u1 = cfmaconj(l, h1[j], u1); }
      }
      if (dir == 0) {
        uf[i] = u0;
        uf[3 + i] = u1;
      } else {
        ub[i] = (SIGNED && sg[1] < 0) ? cneg(u0) : u0;
        ub[3 + i] = (SIGNED && sg[1] < 0) ? cneg(u1) : u1;
      }
    }
  }
  const R m2 = (SIGNED && sg[0] < 0) ? R(2) : R(-2);  // -2 s_f
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    acc[i] = ub[i];          // s_f u_f + s_b u_b
    acc[3 + i] = ub[3 + i];
    lower_from<MU, R>(uf[i], ub[i], uf[3 + i], ub[3 + i], m2, acc[6 + i], acc[9 + i]);
  }
}

// out[12] = (H_W in)(s) = gamma5 [ (4 + m) in(s) - 1/2 sum_mu hops ], r = 1.
template <typename R>
__device__ __forceinline__ void hw_site(const typename Store<R>::T* __restrict__ in,
                                        const typename Store<R>::T* __restrict__ U, const Geom& g,
                                        int s, R diag, Cx<R> out[12]) {
  int c[4];
  site_coords(g, s, c);
#pragma unroll
  for (int k = 0; k < 12; ++k) out[k] = cscale(diag, ld<R>(in + k * (size_t)g.V + s));
  hop_dir<0, R>(in, U, g, s, c, out);
  hop_dir<1, R>(in, U, g, s, c, out);
  hop_dir<2, R>(in, U, g, s, c, out);
  hop_dir<3, R>(in, U, g, s, c, out);
#pragma unroll
  for (int k = 6; k < 12; ++k) out[k] = cneg(out[k]);
}

// ------------------------------------------------------------ reductions

// Deterministic block sum of one double (fixed shuffle tree, fixed warp order).
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* sh /* >= NT/32 */) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < NT / 32; ++i) t += sh[i];
  }
  __syncthreads();
  return t;  // valid in thread 0
}

// Sum n partials (written by other blocks of this grid) in a fixed order, all threads of the block.
template <int NT>
__device__ __forceinline__ double sum_partials(const double* p, int n, double* sh) {
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += NT) v += __ldcg(p + i);
  return block_sum<NT>(v, sh);
}

// ------------------------------------------------- stencil, 4 threads per site
// A block of 128 threads handles 32 consecutive sites.  Phase 1: warp w computes the
// two hops of direction mu = w for the 32 sites (consecutive lanes, consecutive
// sites) and writes its 12 unscaled partial components to shared memory.  Phase 2:
// thread t owns site site0 + (t & 31) and components 3 (t >> 5) .. 3 (t >> 5) + 2 and
// forms the diagonal term minus 1/2 the four partials, then gamma5.  Four times the threads of
// hw_site for the same work, for small lattices where one thread per site leaves
// most of the GPU idle.  sm must hold 4 * 12 * 32 complex numbers.
constexpr int kSplitNT = 128;
constexpr int kSplitSites = 32;

// Unit phase: i^q a (q taken mod 4), by swaps and sign flips.
template <typename R>
__device__ __forceinline__ Cx<R> uphase(Cx<R> a, int q) {
  const Cx<R> t = (q & 1) ? Cx<R>{-a.im, a.re} : a;
  return (q & 2) ? Cx<R>{-t.re, -t.im} : t;
}

// The half-spinor operand of the link-row products of one hop, and the products
// u0 = sum_j l_j h0_j, u1 = sum_j l_j h1_j for a link row l (complex, 3 terms).
// Generic: complex FMAs.
template <typename R>
struct RowOperand {
  Cx<R> h0[3], h1[3];
  __device__ __forceinline__ void set(const Cx<R> a[3], const Cx<R> b[3]) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      h0[j] = a[j];
      h1[j] = b[j];
    }
  }
  __device__ __forceinline__ void products(const Cx<R> l[3], Cx<R>& u0, Cx<R>& u1) const {
    u0 = {R(0), R(0)};
    u1 = {R(0), R(0)};
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      u0 = cfma(l[j], h0[j], u0);
      u1 = cfma(l[j], h1[j], u1);
    }
  }
};

// Double-float: the two spins of a half spinor run lane-wise on FP32 pairs (lane 0:
// h0, lane 1: h1) with Blackwell's paired FP32 instructions (FMUL2/FFMA2/FADD2), so the
// six double-float products of each real output cost about half the instructions.  Each
// sum is a DFSum2 (value s - cn): leading products summed by error-free two-sum, all
// low-order terms negated in cn; link values enter as broadcast pairs.
__device__ __forceinline__ float2 bcast2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
struct DFSum2 {
  float2 s, cn;
};
// x y for x = (xh, xl) broadcast (given as XH, -XH, -XL) and y = (YH, YL) per lane
__device__ __forceinline__ DFSum2 dfs2_first(float2 XH, float2 NXH, float2 NXL, float2 YH, float2 YL) {
  const float2 p = __fmul2_rn(XH, YH);
  float2 cn = __ffma2_rn(NXH, YH, p);  // p - xh yh, exact
  cn = __ffma2_rn(NXH, YL, cn);        // - xh yl
  cn = __ffma2_rn(NXL, YH, cn);        // - xl yh
  return {p, cn};
}
__device__ __forceinline__ void dfs2_add(DFSum2& A, float2 XH, float2 NXH, float2 NXL, float2 YH, float2 YL) {
  const float2 p = __fmul2_rn(XH, YH);
  float2 cn = __fadd2_rn(A.cn, __ffma2_rn(NXH, YH, p));
  cn = __ffma2_rn(NXH, YL, cn);
  cn = __ffma2_rn(NXL, YH, cn);
  const float2 s = __fadd2_rn(A.s, p);  // two-sum of s + p
  const float2 bb = f2sub(s, A.s);
  const float2 err = __fadd2_rn(f2sub(A.s, f2sub(s, bb)), f2sub(p, bb));
  A.cn = f2sub(cn, err);
  A.s = s;
}
// s - cn normalised per lane: two-sum of s and -cn
__device__ __forceinline__ void dfs2_get(const DFSum2& A, float2& hi, float2& lo) {
  const float2 s = f2sub(A.s, A.cn);
  const float2 bb = f2sub(s, A.s);
  lo = f2sub(f2sub(A.s, f2sub(s, bb)), __fadd2_rn(A.cn, bb));
  hi = s;
}

template <>
struct RowOperand<DF> {
  float2 yh_re[3], yl_re[3], yh_im[3], yl_im[3];  // lane 0: h0, lane 1: h1
  __device__ __forceinline__ void set(const Cx<DF> a[3], const Cx<DF> b[3]) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      yh_re[j] = make_float2(a[j].re.hi, b[j].re.hi);
      yl_re[j] = make_float2(a[j].re.lo, b[j].re.lo);
      yh_im[j] = make_float2(a[j].im.hi, b[j].im.hi);
      yl_im[j] = make_float2(a[j].im.lo, b[j].im.lo);
    }
  }
  // re = sum_j (l.re h.re - l.im h.im), im = sum_j (l.re h.im + l.im h.re), both spins at once
  __device__ __forceinline__ void products(const Cx<DF> l[3], Cx<DF>& u0, Cx<DF>& u1) const {
    DFSum2 re, im;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const float2 xr = bcast2(l[j].re.hi), nxr = bcast2(-l[j].re.hi), nxrl = bcast2(-l[j].re.lo);
      const float2 xi = bcast2(l[j].im.hi), nxi = bcast2(-l[j].im.hi), nxil = bcast2(-l[j].im.lo);
      const float2 xil = bcast2(l[j].im.lo);
      if (j == 0) {
        re = dfs2_first(xr, nxr, nxrl, yh_re[j], yl_re[j]);
        im = dfs2_first(xr, nxr, nxrl, yh_im[j], yl_im[j]);
      } else {
        dfs2_add(re, xr, nxr, nxrl, yh_re[j], yl_re[j]);
        dfs2_add(im, xr, nxr, nxrl, yh_im[j], yl_im[j]);
      }
      dfs2_add(re, nxi, xi, xil, yh_im[j], yl_im[j]);  // x = -l.im
      dfs2_add(im, xi, nxi, nxil, yh_re[j], yl_re[j]);
    }
    float2 rh, rl, ih, il;
    dfs2_get(re, rh, rl);
    dfs2_get(im, ih, il);
    u0 = {DF(rh.x, rl.x), DF(ih.x, il.x)};
    u1 = {DF(rh.y, rl.y), DF(ih.y, il.y)};
  }
};

// Spin-projection sum psi_up + phase * psi_lo feeding the link-row products.  Double-float:
// the error-free sum of the leading parts with the low parts added, not renormalised
// (the products take hi and lo apart: hi * hi exactly, the cross terms rounded, so an
// unnormalised lo of at most a few ulp(hi) costs no accuracy and saves the final
// fast two-sum).  Other types: the plain sum.
template <typename R>
__device__ __forceinline__ Cx<R> proj_add(Cx<R> a, Cx<R> b) { return cadd(a, b); }
__device__ __forceinline__ DF df_add_unnormalised(DF a, DF b) {
  float s, e;
  df_two_sum(a.hi, b.hi, s, e);
  return DF(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}
template <>
__device__ __forceinline__ Cx<DF> proj_add<DF>(Cx<DF> a, Cx<DF> b) {
  return {df_add_unnormalised(a.re, b.re), df_add_unnormalised(a.im, b.im)};
}

// Phase 1 with one instruction stream for all directions and both hops: mu and the hop
// are runtime values, A_mu is applied as a permutation and unit phases, and the rows
// of the link product are a runtime loop that accumulates into shared memory.  Used
// for double-float arithmetic, where a complex FMA is ~60 FP32 instructions and the
// unrolled per-direction form (eight hop bodies live in one block) overflows the
// instruction cache.  Stores the hop sums unscaled (phase 2 applies the -1/2).
//   A_mu (l0, l1) = (i^qa0 l_{swap}, i^qa1 l_{1-swap}):  A_x = -i sigma_1 (swap, -i, -i),
//   A_y = -i sigma_2 (swap, -1, +1), A_z = -i sigma_3 (-i, +i), A_t = 1;
//   A_mu^dag is the transpose with conjugate phases.
// RAW (links carrying the boundary sign, !SIGNED): the partials hold the raw hop sums
// and differences and phase 2 applies the direction's phases (compile-time there).
template <typename R, bool CG, bool SIGNED = true>
__device__ __forceinline__ void hw_split_phase1_compact(const typename Store<R>::T* __restrict__ in,
                                                        const typename Store<R>::T* __restrict__ U, const Geom& g,
                                                        int site0, Cx<R>* sm) {
  constexpr bool RAW = !SIGNED;
  const int lane = threadIdx.x & 31, mu = threadIdx.x >> 5;
  const int s = site0 + lane;
  const int V = g.V;
  Cx<R>* acc = sm + mu * 12 * kSplitSites + lane;  // component k at acc[k * kSplitSites]
  if (s >= V) return;  // phase 2 reads no partial of a site beyond V
  const int Lm = g.L[mu], stm = g.st[mu];
  const int cm = (s / stm) % Lm;  // coordinate along mu
  const int bsg = (mu == 3) ? g.bc_t : 1;
  const bool swap = mu < 2;
  const int qa0 = (mu == 3) ? 0 : (mu == 1) ? 2 : 3;
  const int qa1 = (mu == 0) ? 3 : (mu == 2) ? 1 : 0;
  const int qb0 = (4 - (swap ? qa1 : qa0)) & 3, qb1 = (4 - (swap ? qa0 : qa1)) & 3;
  const int k2 = swap ? 3 : 2, k3 = swap ? 2 : 3;  // lower spin feeding row 0 / row 1 of A
#pragma unroll 1
  for (int dir = 0; dir < 2; ++dir) {
    const bool wrap = dir == 0 ? (cm + 1 == Lm) : (cm == 0);
    const int sgn = (SIGNED && wrap) ? bsg : 1;
    const int sn = dir == 0 ? (wrap ? s - (Lm - 1) * stm : s + stm) : (wrap ? s + (Lm - 1) * stm : s - stm);
    const int sl = dir == 0 ? s : sn;  // link site
    const int qd = dir == 0 ? 2 : 0;   // forward hop: h = psi_up - A psi_lo, lower gets -A^dag u
    const int qs = sgn < 0 ? 2 : 0;    // boundary sign
    // link rows are loaded one row ahead of their use (row 0 together with the spinor),
    // so that each load's latency is covered by the previous row's products; the
    // conjugation of the backward hop is applied when a row is taken into use
    const typename Store<R>::T* Ul = U + (size_t)mu * 9 * V + sl;
    // forward: U[i][j]; backward: (U^dag)[i][j] = conj(U[j][i])
    auto ld_row = [&](int i, Cx<R> l[3]) {
#pragma unroll
      for (int j = 0; j < 3; ++j) l[j] = ld<R>(Ul + (dir == 0 ? (i * 3 + j) : (j * 3 + i)) * (size_t)V);
    };
    Cx<R> ln[3];
    ld_row(0, ln);
    Cx<R> h0[3], h1[3];
#pragma unroll
    for (int col = 0; col < 3; ++col) {
      const Cx<R> p0 = ld<R, CG>(in + (0 * 3 + col) * (size_t)V + sn);
      const Cx<R> p1 = ld<R, CG>(in + (1 * 3 + col) * (size_t)V + sn);
      const Cx<R> pa = ld<R, CG>(in + (k2 * 3 + col) * (size_t)V + sn);
      const Cx<R> pb = ld<R, CG>(in + (k3 * 3 + col) * (size_t)V + sn);
      h0[col] = proj_add(p0, uphase(pa, qa0 + qd));
      h1[col] = proj_add(p1, uphase(pb, qa1 + qd));
    }
    RowOperand<R> hop;
    hop.set(h0, h1);
#pragma unroll 1
    for (int i = 0; i < 3; ++i) {
      Cx<R> l[3];
#pragma unroll
      for (int j = 0; j < 3; ++j) l[j] = dir ? Cx<R>{ln[j].re, -ln[j].im} : ln[j];
      if (i < 2) ld_row(i + 1, ln);
      Cx<R> u0, u1;
      hop.products(l, u0, u1);
      Cx<R>* a = acc + i * kSplitSites;
      if (RAW) {
        // raw hop sums and differences, no phases: the slots of spins 0, 1 receive
        // u_f + u_b per spin of the half spinor, those of spins 2, 3 receive u_b - u_f;
        // phase 2 applies A_mu^dag (a compile-time swap and phase per direction)
        if (dir == 0) {
          a[0 * 3 * kSplitSites] = u0;
          a[1 * 3 * kSplitSites] = u1;
        } else {
          const Cx<R> f0 = a[0 * 3 * kSplitSites], f1 = a[1 * 3 * kSplitSites];
          a[0 * 3 * kSplitSites] = proj_add(f0, u0);
          a[1 * 3 * kSplitSites] = proj_add(f1, u1);
          a[2 * 3 * kSplitSites] = proj_add(u0, cneg(f0));
          a[3 * 3 * kSplitSites] = proj_add(u1, cneg(f1));
        }
        continue;
      }
      const Cx<R> c0 = uphase(u0, qs), c1 = uphase(u1, qs);
      const Cx<R> c2 = uphase(swap ? u1 : u0, qb0 + qd + qs), c3 = uphase(swap ? u0 : u1, qb1 + qd + qs);
      if (dir == 0) {  // the first hop initialises the partials
        a[0 * 3 * kSplitSites] = c0;
        a[1 * 3 * kSplitSites] = c1;
        a[2 * 3 * kSplitSites] = c2;
        a[3 * 3 * kSplitSites] = c3;
      } else {
        // unnormalised (phase 2 sums the four partials with one renormalisation)
        a[0 * 3 * kSplitSites] = proj_add(a[0 * 3 * kSplitSites], c0);
        a[1 * 3 * kSplitSites] = proj_add(a[1 * 3 * kSplitSites], c1);
        a[2 * 3 * kSplitSites] = proj_add(a[2 * 3 * kSplitSites], c2);
        a[3 * 3 * kSplitSites] = proj_add(a[3 * 3 * kSplitSites], c3);
      }
    }
  }
}

// a + f (p0 + p1 + p2 + p3), f = -1/2 (HALF) or 1, in double-float with a single
// renormalisation: the (exactly) scaled leading parts enter an error-free two-sum chain,
// every low part and rounding error is summed in one float, then one two-sum.  Error a
// few units of 2^-48 of the largest term, as for the four separate additions it replaces.
template <bool HALF>
__device__ __forceinline__ DF df_sum5(DF a, DF p0, DF p1, DF p2, DF p3) {
  const DF p[4] = {p0, p1, p2, p3};
  float s = a.hi, lo = a.lo, e;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    df_two_sum(s, HALF ? -0.5f * p[k].hi : p[k].hi, s, e);
    lo = __fadd_rn(lo, HALF ? __fmaf_rn(-0.5f, p[k].lo, e) : __fadd_rn(p[k].lo, e));
  }
  float hi2, lo2;
  df_two_sum(s, lo, hi2, lo2);
  return DF(hi2, lo2);
}

// a - t / 2 (exact halving; one FMA per real for FP64 and FP32)
__device__ __forceinline__ Cx<DF> sub_half(Cx<DF> a, Cx<DF> t) {
  return csub(a, Cx<DF>{DF(0.5f * t.re.hi, 0.5f * t.re.lo), DF(0.5f * t.im.hi, 0.5f * t.im.lo)});
}
template <typename R>
__device__ __forceinline__ Cx<R> sub_half(Cx<R> a, Cx<R> t) {
  return {fma(R(-0.5), t.re, a.re), fma(R(-0.5), t.im, a.im)};
}

template <typename R, bool CG = false, bool SIGNED = true>
__device__ __forceinline__ void hw_split_phase1(const typename Store<R>::T* __restrict__ in,
                                                const typename Store<R>::T* __restrict__ U, const Geom& g,
                                                int site0, Cx<R>* sm) {
  if constexpr (std::is_same<R, DF>::value) {
    hw_split_phase1_compact<R, CG, SIGNED>(in, U, g, site0, sm);
    return;
  }
  const int lane = threadIdx.x & 31, mu = threadIdx.x >> 5;
  const int s = site0 + lane;
  Cx<R> acc[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = {R(0), R(0)};
  if (s < g.V) {
    int c[4];
    site_coords(g, s, c);
    switch (mu) {  // warp-uniform
      case 0: hop_dir_unscaled<0, R, CG, SIGNED>(in, U, g, s, c, acc); break;
      case 1: hop_dir_unscaled<1, R, CG, SIGNED>(in, U, g, s, c, acc); break;
      case 2: hop_dir_unscaled<2, R, CG, SIGNED>(in, U, g, s, c, acc); break;
      default: hop_dir_unscaled<3, R, CG, SIGNED>(in, U, g, s, c, acc); break;
    }
  }
#pragma unroll
  for (int k = 0; k < 12; ++k) sm[(mu * 12 + k) * kSplitSites + lane] = acc[k];
}

// Phase 2 for this thread's three components kk = 3 (t >> 5) + {0, 1, 2}; call after
// __syncthreads().  Returns false for sites beyond V.  HALVED: phase 1 ran on links
// scaled by -1/2, so its partials already carry the hop factor.
template <typename R, bool CG = false, bool HALVED = false>
__device__ __forceinline__ bool hw_split_phase2(const typename Store<R>::T* __restrict__ in, const Geom& g,
                                                int site0, R diag, const Cx<R>* sm, Cx<R> o[3], int* s_out,
                                                int* k0_out) {
  const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
  const int s = site0 + lane;
  *s_out = s;
  *k0_out = 3 * grp;
  if (s >= g.V) return false;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const int k = 3 * grp + q;
    // diagonal term minus 1/2 the sum of the four unscaled direction partials
    const Cx<R> x = ld<R, CG>(in + k * (size_t)g.V + s);
    Cx<R> t = sm[k * kSplitSites + lane];
    if constexpr (!std::is_same<R, DF>::value) {
#pragma unroll
      for (int mu = 1; mu < 4; ++mu) t = cadd(t, sm[(mu * 12 + k) * kSplitSites + lane]);
    }
    Cx<R> v;
    if constexpr (std::is_same<R, DF>::value) {
      // diag x + the four direction partials as one double-float sum of five terms: an
      // error-free two-sum chain of the leading parts, the low parts and errors in one
      // float, one renormalisation (instead of four double-float additions)
      const Cx<R> dv = cscale(diag, x);
      if constexpr (HALVED) {
        // raw partials (links carry -1/2 and the boundary sign): spins 0, 1 take the hop
        // sums as stored; spins 2, 3 take A_mu^dag of the differences, a fixed swap and
        // phase per direction
        const int i = k - 3 * grp;
        Cx<R> t[4];
        if (grp < 2) {
#pragma unroll
          for (int m = 0; m < 4; ++m) t[m] = sm[(m * 12 + k) * kSplitSites + lane];
        } else {
          // spin 2 of direction mu is i^{q2[mu]} d_{s2[mu]}, spin 3 is i^{q3[mu]} d_{s3[mu]},
          // d_s in slot 2 + s (A_x^dag = (i d1, i d0), A_y^dag = (d1, -d0),
          // A_z^dag = (i d0, -i d1), A_t^dag = (d0, d1))
          const bool sp2 = grp == 2;
          const Cx<R> d0x = sm[(0 * 12 + (sp2 ? 9 : 6) + i) * kSplitSites + lane];
          const Cx<R> d1y = sm[(1 * 12 + (sp2 ? 9 : 6) + i) * kSplitSites + lane];
          const Cx<R> d2z = sm[(2 * 12 + (sp2 ? 6 : 9) + i) * kSplitSites + lane];
          const Cx<R> d3t = sm[(3 * 12 + (sp2 ? 6 : 9) + i) * kSplitSites + lane];
          t[0] = cmuli(d0x);                       // x: i d1 (spin 2), i d0 (spin 3)
          t[1] = sp2 ? d1y : cneg(d1y);            // y: d1, -d0
          t[2] = sp2 ? cmuli(d2z) : cmulmi(d2z);   // z: i d0, -i d1
          t[3] = d3t;                              // t: d0, d1
        }
        v = {df_sum5<false>(dv.re, t[0].re, t[1].re, t[2].re, t[3].re),
             df_sum5<false>(dv.im, t[0].im, t[1].im, t[2].im, t[3].im)};
      } else {
        const Cx<R>* pp = sm + k * kSplitSites + lane;
        v = {df_sum5<true>(dv.re, pp[0].re, pp[12 * kSplitSites].re, pp[24 * kSplitSites].re,
                           pp[36 * kSplitSites].re),
             df_sum5<true>(dv.im, pp[0].im, pp[12 * kSplitSites].im, pp[24 * kSplitSites].im,
                           pp[36 * kSplitSites].im)};
      }
    } else if constexpr (HALVED) {
      v = {fma(diag, x.re, t.re), fma(diag, x.im, t.im)};
    } else {
      v = sub_half(cscale(diag, x), t);
    }
    o[q] = (k >= 6) ? cneg(v) : v;
  }
  return true;
}

