// FP32 fields in the right-hand-side-paired layout, and the H_W stencil on them.
//
// Layout: a set of nrhs spinors (padded to an even count) is stored as pairs; element
// (pair q, component k = 3 spin + colour, site) is one float4
//     (re[2q], re[2q+1], im[2q], im[2q+1])     at   (q * 12 + k) * V + site,
// so one 16-byte load brings one component of two right-hand sides, and every complex
// operation of the stencil acts lane-wise on (rhs 2q, rhs 2q+1) with Blackwell's paired
// FP32 instructions (__ffma2_rn, __fadd2_rn): half the FP32 instructions of a scalar
// stencil, and no lane shuffles, because the spin and colour algebra is the same on
// both lanes.  Links come in the spin-paired layout's float4 forms (dslash32.cu) and are
// broadcast to both lanes in registers.
#pragma once

#include "common.cuh"

struct P2 {
  float2 re, im;  // lanes: right-hand sides 2q and 2q + 1
};

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
// a - b
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }

__device__ __forceinline__ P2 ldp(const float4* p) {
  const float4 v = __ldg(p);
  return {make_float2(v.x, v.y), make_float2(v.z, v.w)};
}
__device__ __forceinline__ void stp(float4* p, P2 v) { *p = make_float4(v.re.x, v.re.y, v.im.x, v.im.y); }

// a + S b for a compile-time sign S = +-1 (one paired instruction)
template <int S>
__device__ __forceinline__ float2 pm(float2 a, float2 b) {
  return S > 0 ? add2(a, b) : sub2(a, b);
}

// h = psi_up + S A_mu psi_lo for one colour (S = -1: forward hop, +1: backward hop).
// A_x = -i s1, A_y = -i s2, A_z = -i s3, A_t = 1 (chiral basis, as in common.cuh):
//   A_x psi_lo = (-i p3, -i p2), A_y psi_lo = (-p3, p2), A_z psi_lo = (-i p2, i p3).
template <int MU, int S>
__device__ __forceinline__ void proj_pair(P2 p0, P2 p1, P2 p2, P2 p3, P2& h0, P2& h1) {
  if (MU == 0) {
    h0 = {pm<S>(p0.re, p3.im), pm<-S>(p0.im, p3.re)};
    h1 = {pm<S>(p1.re, p2.im), pm<-S>(p1.im, p2.re)};
  } else if (MU == 1) {
    h0 = {pm<-S>(p0.re, p3.re), pm<-S>(p0.im, p3.im)};
    h1 = {pm<S>(p1.re, p2.re), pm<S>(p1.im, p2.im)};
  } else if (MU == 2) {
    h0 = {pm<S>(p0.re, p2.im), pm<-S>(p0.im, p2.re)};
    h1 = {pm<-S>(p1.re, p3.im), pm<S>(p1.im, p3.re)};
  } else {
    h0 = {pm<S>(p0.re, p2.re), pm<S>(p0.im, p2.im)};
    h1 = {pm<S>(p1.re, p3.re), pm<S>(p1.im, p3.im)};
  }
}

// lower spins: acc_lo += F * A_mu^dag u with F (fl) and -F (nfl) given as lane pairs;
//   A_x^dag u = (i u1, i u0), A_y^dag u = (u1, -u0), A_z^dag u = (i u0, -i u1), A_t^dag u = u.
template <int MU>
__device__ __forceinline__ void acc_lower(P2& l0, P2& l1, P2 u0, P2 u1, float2 fl, float2 nfl) {
  if (MU == 0) {
    l0.re = fma2(nfl, u1.im, l0.re); l0.im = fma2(fl, u1.re, l0.im);
    l1.re = fma2(nfl, u0.im, l1.re); l1.im = fma2(fl, u0.re, l1.im);
  } else if (MU == 1) {
    l0.re = fma2(fl, u1.re, l0.re);  l0.im = fma2(fl, u1.im, l0.im);
    l1.re = fma2(nfl, u0.re, l1.re); l1.im = fma2(nfl, u0.im, l1.im);
  } else if (MU == 2) {
    l0.re = fma2(nfl, u0.im, l0.re); l0.im = fma2(fl, u0.re, l0.im);
    l1.re = fma2(fl, u1.im, l1.re);  l1.im = fma2(nfl, u1.re, l1.im);
  } else {
    l0.re = fma2(fl, u0.re, l0.re);  l0.im = fma2(fl, u0.im, l0.im);
    l1.re = fma2(fl, u1.re, l1.re);  l1.im = fma2(fl, u1.im, l1.im);
  }
}

// ------------------------------------------------------------------------------------
// The same stencil with 12-real links: rows 0 and 1 of U are read, row 2 is rebuilt as
// conj(row0 x row1) (U unitary with det U = 1) in paired arithmetic on lane-equal pairs,
// so one rebuild serves both right-hand sides of the pair (each element is rebuilt
// where it is used, which keeps one row fewer live).  The link form: the spin-paired
// layout's 3 float4 per link, (U00, U01), (U02, U10), (U11, U12) at (mu * 3 + k) * V +
// site (48 B per link, lanes broadcast in registers).
struct B2 {
  float2 re, im;  // both lanes hold the same complex number
};

__device__ __forceinline__ B2 bc2(float re, float im) { return {f2(re, re), f2(im, im)}; }

// rows 0 and 1 of a 12-real link as lane-equal pairs
__device__ __forceinline__ void link12_rows(const float4* __restrict__ L, int mu, int V, int site, B2 U[3][3]) {
  const float4* p = L + (size_t)mu * 3 * V + site;
  const float4 a = __ldg(p), b = __ldg(p + V), c = __ldg(p + 2 * (size_t)V);
  U[0][0] = bc2(a.x, a.y); U[0][1] = bc2(a.z, a.w); U[0][2] = bc2(b.x, b.y);
  U[1][0] = bc2(b.z, b.w); U[1][1] = bc2(c.x, c.y); U[1][2] = bc2(c.z, c.w);
}

// compact 12-real link with row 2 rebuilt once in scalar arithmetic (both lanes of a
// pair would compute the same value), then all 9 elements as lane-equal pairs
__device__ __forceinline__ void link12_scalar(const float4* __restrict__ L, int mu, int V, int site, B2 U[3][3]) {
  const float4* p = L + (size_t)mu * 3 * V + site;
  const float4 a = __ldg(p), b = __ldg(p + V), c = __ldg(p + 2 * (size_t)V);
  const Cx<float> u0[3] = {{a.x, a.y}, {a.z, a.w}, {b.x, b.y}};
  const Cx<float> u1[3] = {{b.z, b.w}, {c.x, c.y}, {c.z, c.w}};
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const int j1 = (j + 1) % 3, j2 = (j + 2) % 3;
    float re = u0[j1].re * u1[j2].re;
    re = fmaf(-u0[j1].im, u1[j2].im, re);
    re = fmaf(-u0[j2].re, u1[j1].re, re);
    re = fmaf(u0[j2].im, u1[j1].im, re);
    float im = u0[j1].re * u1[j2].im;
    im = fmaf(u0[j1].im, u1[j2].re, im);
    im = fmaf(-u0[j2].re, u1[j1].im, im);
    im = fmaf(-u0[j2].im, u1[j1].re, im);
    U[0][j] = bc2(u0[j].re, u0[j].im);
    U[1][j] = bc2(u1[j].re, u1[j].im);
    U[2][j] = bc2(re, -im);
  }
}

// row 2, column j of the link: conj(U0[j+1] U1[j+2] - U0[j+2] U1[j+1])
__device__ __forceinline__ B2 link12_row2(const B2 U[3][3], int j) {
  const int j1 = (j + 1) % 3, j2 = (j + 2) % 3;
  const B2 a = U[0][j1], b = U[1][j2], c = U[0][j2], d = U[1][j1];
  const float2 rp = fma2(a.re, b.re, mul2(c.im, d.im));
  const float2 rn = fma2(a.im, b.im, mul2(c.re, d.re));
  const float2 ip = fma2(a.re, b.im, mul2(a.im, b.re));
  const float2 iq = fma2(c.re, d.im, mul2(c.im, d.re));
  return {sub2(rp, rn), sub2(iq, ip)};
}

// Both hops of direction MU for one site and the two right-hand sides of a pair, with
// 12-real links.  Upper spins accumulate +f u, lower spins the NEGATED contribution
// (the caller applies gamma5 = -1 on them by adding -diag psi_lo at the end).
// LK 1: compact 12-real links, row 2 rebuilt element by element in paired arithmetic;
// 3: compact 12-real links with row 2 rebuilt once in scalar arithmetic.
template <int MU, int LK>
__device__ __forceinline__ void hop_pair12(const float4* __restrict__ in, const float4* __restrict__ L,
                                           const Geom& g, int s, const int c[4], P2 acc[12]) {
  const int V = g.V;
#pragma unroll
  for (int dir = 0; dir < 2; ++dir) {
    int sgn;
    const int sn = dir == 0 ? nb_fwd(g, s, c, MU, &sgn) : nb_bwd(g, s, c, MU, &sgn);
    const int sl = dir == 0 ? s : sn;
    P2 h0[3], h1[3];
#pragma unroll
    for (int col = 0; col < 3; ++col) {
      const P2 p0 = ldp(in + (0 * 3 + col) * (size_t)V + sn);
      const P2 p1 = ldp(in + (1 * 3 + col) * (size_t)V + sn);
      const P2 p2 = ldp(in + (2 * 3 + col) * (size_t)V + sn);
      const P2 p3 = ldp(in + (3 * 3 + col) * (size_t)V + sn);
      if (dir == 0)
        proj_pair<MU, -1>(p0, p1, p2, p3, h0[col], h1[col]);
      else
        proj_pair<MU, 1>(p0, p1, p2, p3, h0[col], h1[col]);
    }
    B2 U[3][3];
    if (LK == 3)
      link12_scalar(L, MU, V, sl, U);
    else
      link12_rows(L, MU, V, sl, U);
    const float f = -0.5f * (float)sgn;
    const float2 fu = f2(f, f);
    // lower spins (negated): +f forward (from 1 - gamma), -f backward (from 1 + gamma)
    const float2 fl = dir == 0 ? f2(f, f) : f2(-f, -f);
    const float2 nfl = dir == 0 ? f2(-f, -f) : f2(f, f);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      float2 a0 = f2(0.f, 0.f), c0 = f2(0.f, 0.f);
      float2 a1 = f2(0.f, 0.f), c1 = f2(0.f, 0.f);
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        // row 2 is rebuilt element by element where it is used
        const int r = dir == 0 ? i : j, q = dir == 0 ? j : i;
        const B2 l = (r < 2 || LK == 3) ? U[r][q] : link12_row2(U, q);
        const float2 nli = f2(-l.im.x, -l.im.y);
        a0 = fma2(l.re, h0[j].re, a0);
        a1 = fma2(l.re, h1[j].re, a1);
        c0 = fma2(l.re, h0[j].im, c0);
        c1 = fma2(l.re, h1[j].im, c1);
        if (dir == 0) {
          // U h: re = lr hr - li hi, im = lr hi + li hr (the minus in the operand)
          a0 = fma2(nli, h0[j].im, a0);
          a1 = fma2(nli, h1[j].im, a1);
          c0 = fma2(l.im, h0[j].re, c0);
          c1 = fma2(l.im, h1[j].re, c1);
        } else {
          // U^dag h: re = lr hr + li hi, im = lr hi - li hr
          a0 = fma2(l.im, h0[j].im, a0);
          a1 = fma2(l.im, h1[j].im, a1);
          c0 = fma2(nli, h0[j].re, c0);
          c1 = fma2(nli, h1[j].re, c1);
        }
      }
      const P2 u0 = {a0, c0}, u1 = {a1, c1};
      acc[0 * 3 + i].re = fma2(fu, u0.re, acc[0 * 3 + i].re);
      acc[0 * 3 + i].im = fma2(fu, u0.im, acc[0 * 3 + i].im);
      acc[1 * 3 + i].re = fma2(fu, u1.re, acc[1 * 3 + i].re);
      acc[1 * 3 + i].im = fma2(fu, u1.im, acc[1 * 3 + i].im);
      acc_lower<MU>(acc[2 * 3 + i], acc[3 * 3 + i], u0, u1, fl, nfl);
    }
  }
}

