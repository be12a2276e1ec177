// SU(3) link force of L = Re <eta, S_N b> (the adjoint of Eqs. 4-7).
//
// Differentiating each resolvent, d(z - H)^-1 = (z - H)^-1 dH (z - H)^-1, gives
// dL = Re sum_j c_j xi_j^dag dH y_j with y_j = (z_j - H)^-1 b and
// xi_j = (conj z_j - H)^-1 eta.  For U_mu(x) -> exp(i omega_a lambda_a / 2) U_mu(x) the
// link enters the forward hop at x and (as U^dag) the backward hop at x + mu, and
//
//     dL / d omega_a = 1/4 Im tr( lambda_a M ),      M = s ( U Q - Q' U^dag ),
//     Q  = sum_j c_j sum_{u=0,1} h_u k_u^dag,   Q' = sum_j c_j sum_{u=0,1} h'_u k'_u^dag,
//
// where, with the chiral-basis blocks gamma_mu = [[0, A], [A^dag, 0]] and colour
// vectors per upper spin u:
//     h  = y(x+mu)_up  - A y(x+mu)_lo,     k  = xi(x)_up    + A xi(x)_lo,
//     h' = y(x)_up     + A y(x)_lo,        k' = xi(x+mu)_up - A xi(x+mu)_lo,
// and s = -1 on links that cross an antiperiodic t boundary.  (gamma5 (1 -+ gamma_mu)
// has rank two; the spin sums collapse to these two-component projections.)
// One thread per (site, mu) accumulates Q and Q' over the nodes in FP64.
#include "common.cuh"

namespace {

constexpr int kNT = 128;

template <int MU>
__device__ __forceinline__ void force_site(const double2* __restrict__ X, int nq, size_t n12,
                                           const double2* __restrict__ cq, const double2* __restrict__ U,
                                           const Geom& g, int s, const int c[4], double* __restrict__ F) {
  int sbc;
  const int sf = nb_fwd(g, s, c, MU, &sbc);
  const int V = g.V;
  Cx<double> Q[3][3], Qp[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) Q[a][b] = Qp[a][b] = {0.0, 0.0};
  for (int j = 0; j < nq; ++j) {
    const double2* Y = X + (size_t)j * n12;          // source 0: forward solutions
    const double2* Xi = X + ((size_t)nq + j) * n12;  // source 1: adjoint solutions
    const double2 cj2 = cq[j];
    const Cx<double> cj = {cj2.x, cj2.y};
    Cx<double> h[2][3], k[2][3], hp[2][3], kp[2][3];
#pragma unroll
    for (int col = 0; col < 3; ++col) {
      Cx<double> a0, a1;
      // h from y(x + mu): up - A lo
      Cx<double> y0 = ld<double>(Y + (0 * 3 + col) * (size_t)V + sf), y1 = ld<double>(Y + (1 * 3 + col) * (size_t)V + sf);
      Cx<double> y2 = ld<double>(Y + (2 * 3 + col) * (size_t)V + sf), y3 = ld<double>(Y + (3 * 3 + col) * (size_t)V + sf);
      mulA<MU>(y2, y3, a0, a1);
      h[0][col] = csub(y0, a0);
      h[1][col] = csub(y1, a1);
      // h' from y(x): up + A lo
      y0 = ld<double>(Y + (0 * 3 + col) * (size_t)V + s);
      y1 = ld<double>(Y + (1 * 3 + col) * (size_t)V + s);
      y2 = ld<double>(Y + (2 * 3 + col) * (size_t)V + s);
      y3 = ld<double>(Y + (3 * 3 + col) * (size_t)V + s);
      mulA<MU>(y2, y3, a0, a1);
      hp[0][col] = cadd(y0, a0);
      hp[1][col] = cadd(y1, a1);
      // k from xi(x): up + A lo
      Cx<double> x0 = ld<double>(Xi + (0 * 3 + col) * (size_t)V + s), x1 = ld<double>(Xi + (1 * 3 + col) * (size_t)V + s);
      Cx<double> x2 = ld<double>(Xi + (2 * 3 + col) * (size_t)V + s), x3 = ld<double>(Xi + (3 * 3 + col) * (size_t)V + s);
      mulA<MU>(x2, x3, a0, a1);
      k[0][col] = cadd(x0, a0);
      k[1][col] = cadd(x1, a1);
      // k' from xi(x + mu): up - A lo
      x0 = ld<double>(Xi + (0 * 3 + col) * (size_t)V + sf);
      x1 = ld<double>(Xi + (1 * 3 + col) * (size_t)V + sf);
      x2 = ld<double>(Xi + (2 * 3 + col) * (size_t)V + sf);
      x3 = ld<double>(Xi + (3 * 3 + col) * (size_t)V + sf);
      mulA<MU>(x2, x3, a0, a1);
      kp[0][col] = csub(x0, a0);
      kp[1][col] = csub(x1, a1);
    }
    // Q += c_j sum_u h_u k_u^dag, Q' += c_j sum_u h'_u k'_u^dag
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const Cx<double> ch0 = {cj.re * h[0][a].re - cj.im * h[0][a].im, cj.re * h[0][a].im + cj.im * h[0][a].re};
      const Cx<double> ch1 = {cj.re * h[1][a].re - cj.im * h[1][a].im, cj.re * h[1][a].im + cj.im * h[1][a].re};
      const Cx<double> cp0 = {cj.re * hp[0][a].re - cj.im * hp[0][a].im, cj.re * hp[0][a].im + cj.im * hp[0][a].re};
      const Cx<double> cp1 = {cj.re * hp[1][a].re - cj.im * hp[1][a].im, cj.re * hp[1][a].im + cj.im * hp[1][a].re};
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        Q[a][b] = cfmaconj(k[0][b], ch0, Q[a][b]);
        Q[a][b] = cfmaconj(k[1][b], ch1, Q[a][b]);
        Qp[a][b] = cfmaconj(kp[0][b], cp0, Qp[a][b]);
        Qp[a][b] = cfmaconj(kp[1][b], cp1, Qp[a][b]);
      }
    }
  }
  // M = s (U Q - Q' U^dag)
  Cx<double> L[3][3];
#pragma unroll
  for (int e = 0; e < 9; ++e) L[e / 3][e % 3] = ld<double>(U + (MU * 9 + e) * (size_t)V + s);
  Cx<double> M[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      Cx<double> m = {0.0, 0.0};
#pragma unroll
      for (int t = 0; t < 3; ++t) {
        m = cfma(L[a][t], Q[t][b], m);                                  // (U Q)_ab
        const Cx<double> ud = {L[b][t].re, -L[b][t].im};                 // (U^dag)_tb = conj(U_bt)
        m = cfma(cneg(Qp[a][t]), ud, m);                                // - (Q' U^dag)_ab
      }
      M[a][b] = cscale((double)sbc, m);
    }
  // 1/4 Im tr(lambda_a M), a = 1..8
  double* f = F + ((size_t)MU * V + s) * 8;
  const double r3 = 0.57735026918962576451;  // 1/sqrt(3)
  f[0] += 0.25 * (M[1][0].im + M[0][1].im);
  f[1] += 0.25 * (-M[1][0].re + M[0][1].re);
  f[2] += 0.25 * (M[0][0].im - M[1][1].im);
  f[3] += 0.25 * (M[2][0].im + M[0][2].im);
  f[4] += 0.25 * (-M[2][0].re + M[0][2].re);
  f[5] += 0.25 * (M[2][1].im + M[1][2].im);
  f[6] += 0.25 * (-M[2][1].re + M[1][2].re);
  f[7] += 0.25 * r3 * (M[0][0].im + M[1][1].im - 2.0 * M[2][2].im);
}

__global__ void __launch_bounds__(kNT) force_kernel(const double2* __restrict__ X, int nq,
                                                    const double2* __restrict__ cq, const double2* __restrict__ U,
                                                    Geom g, double* __restrict__ F) {
  const int idx = blockIdx.x * kNT + threadIdx.x;
  if (idx >= 4 * g.V) return;
  const int mu = idx / g.V, s = idx % g.V;
  int c[4];
  site_coords(g, s, c);
  const size_t n12 = (size_t)12 * g.V;
  switch (mu) {
    case 0: force_site<0>(X, nq, n12, cq, U, g, s, c, F); break;
    case 1: force_site<1>(X, nq, n12, cq, U, g, s, c, F); break;
    case 2: force_site<2>(X, nq, n12, cq, U, g, s, c, F); break;
    default: force_site<3>(X, nq, n12, cq, U, g, s, c, F); break;
  }
}

}  // namespace

// F[mu][site][8] += force from nq forward (X[0..nq)) and adjoint (X[nq..2nq)) solutions.
int launch_force(ov_ctx* ctx, const double2* X, int nq, const double2* cq, double* F, cudaStream_t s) {
  const int n = 4 * ctx->g.V;
  cudaEvent_t ev;
  kt_begin(ctx, KC_FORCE, s, &ev);
  force_kernel<<<(n + kNT - 1) / kNT, kNT, 0, s>>>(X, nq, cq, ctx->U64, ctx->g, F);
  kt_end(ctx, KC_FORCE, s, ev);
  OV_CHECK_LAUNCH(ctx, "force_kernel");
  return OV_OK;
}
