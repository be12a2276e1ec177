// FP32 fields in the right-hand-side-paired layout, and the H_W stencil on them.
//
// Layout: a set of nrhs spinors (padded to an even count) is stored as pairs; element
// (pair q, component k = 3 spin + colour, site) is one float4
//     (re[2q], re[2q+1], im[2q], im[2q+1])     at   (q * 12 + k) * V + site,
// so one 16-byte load brings one component of two right-hand sides, and every complex
// operation of the stencil acts lane-wise on (rhs 2q, rhs 2q+1) with Blackwell's paired
// FP32 instructions (__ffma2_rn, __fadd2_rn): half the FP32 instructions of a scalar
// stencil, and no lane shuffles, because the spin and colour algebra is the same on
// both lanes.  Links are stored broadcast-ready: element (mu, 3i + j, site) is the
// float4 (re, re, im, im) of U_mu(site)[i][j].
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

// Both hops of direction MU for one site, two right-hand sides, accumulated into
// acc[12]: upper spins += f u, lower spins += -+ f A^dag u, f = -1/2 * boundary sign.
// in: pair base (component planes of V float4); L: broadcast links.
template <int MU>
__device__ __forceinline__ void hop_pair(const float4* __restrict__ in, const float4* __restrict__ L, const Geom& g,
                                         int s, const int c[4], P2 acc[12]) {
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
    const float f = -0.5f * (float)sgn;
    const float2 fu = f2(f, f);
    // lower spins carry -f (forward, from 1 - gamma) or +f (backward, from 1 + gamma)
    const float2 fl = dir == 0 ? f2(-f, -f) : f2(f, f);
    const float2 nfl = dir == 0 ? f2(f, f) : f2(-f, -f);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      // u_s[i] = sum_j M[i][j] h_s[j], M = U (forward) or U^dag (backward):
      //   forward:  re = sum lr hre - li him,  im = sum lr him + li hre
      //   backward: re = sum lr hre + li him,  im = sum lr him - li hre
      float2 a0 = f2(0.f, 0.f), b0 = f2(0.f, 0.f), c0 = f2(0.f, 0.f), e0 = f2(0.f, 0.f);
      float2 a1 = f2(0.f, 0.f), b1 = f2(0.f, 0.f), c1 = f2(0.f, 0.f), e1 = f2(0.f, 0.f);
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const int e = dir == 0 ? (i * 3 + j) : (j * 3 + i);
        const float4 l = __ldg(L + (MU * 9 + e) * (size_t)V + sl);
        const float2 lr = f2(l.x, l.y), li = f2(l.z, l.w);
        a0 = fma2(lr, h0[j].re, a0);
        b0 = fma2(li, h0[j].im, b0);
        c0 = fma2(lr, h0[j].im, c0);
        a1 = fma2(lr, h1[j].re, a1);
        b1 = fma2(li, h1[j].im, b1);
        c1 = fma2(lr, h1[j].im, c1);
        if (dir == 0) {
          c0 = fma2(li, h0[j].re, c0);
          c1 = fma2(li, h1[j].re, c1);
        } else {
          e0 = fma2(li, h0[j].re, e0);
          e1 = fma2(li, h1[j].re, e1);
        }
      }
      P2 u0, u1;
      if (dir == 0) {
        u0 = {sub2(a0, b0), c0};
        u1 = {sub2(a1, b1), c1};
      } else {
        u0 = {add2(a0, b0), sub2(c0, e0)};
        u1 = {add2(a1, b1), sub2(c1, e1)};
      }
      acc[0 * 3 + i].re = fma2(fu, u0.re, acc[0 * 3 + i].re);
      acc[0 * 3 + i].im = fma2(fu, u0.im, acc[0 * 3 + i].im);
      acc[1 * 3 + i].re = fma2(fu, u1.re, acc[1 * 3 + i].re);
      acc[1 * 3 + i].im = fma2(fu, u1.im, acc[1 * 3 + i].im);
      acc_lower<MU>(acc[2 * 3 + i], acc[3 * 3 + i], u0, u1, fl, nfl);
    }
  }
}

// out[12] = (H_W in)(s) for the two right-hand sides of one pair.
__device__ __forceinline__ void hw_pair_site(const float4* __restrict__ in, const float4* __restrict__ L,
                                             const Geom& g, int s, float diag, P2 out[12]) {
  int c[4];
  site_coords(g, s, c);
  const float2 d2 = f2(diag, diag);
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const P2 v = ldp(in + k * (size_t)g.V + s);
    out[k] = {mul2(d2, v.re), mul2(d2, v.im)};
  }
  hop_pair<0>(in, L, g, s, c, out);
  hop_pair<1>(in, L, g, s, c, out);
  hop_pair<2>(in, L, g, s, c, out);
  hop_pair<3>(in, L, g, s, c, out);
  const float2 m1 = f2(-1.f, -1.f);
#pragma unroll
  for (int k = 6; k < 12; ++k) out[k] = {mul2(m1, out[k].re), mul2(m1, out[k].im)};
}
