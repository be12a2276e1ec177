// Kernels of the mixed-precision solve (OV_MODE_MIXED) that are not Lanczos steps:
//
//  * basis combination: every node's FP32-phase solution y_j = sum_i w_ij U_i from the
//    stored (unnormalised) FP32 Lanczos basis, written in FP64;
//  * FP64 true residuals r_j = b - (z_j - H_W) y_j for every node and source, with the
//    FP64 stencil fused in, and their norms;
//  * accumulation y_j += e_j of the FP32 corrections (FP64 sum);
//  * the FP64 weighted sum s = c0 b + sum_j c_j y_j of Eq. 7.
#include "common.cuh"

namespace {

constexpr int kCombNT = 128;
constexpr int kCombNJ = 32;    // nodes per thread pass
constexpr int kCombKI = 32;    // basis vectors per shared-memory chunk
constexpr int kResNT = 128;

// Y[r][j][e] = sum_{i=1..k_r} W[r][j][i] * U_i[e] (basis slots 1..k_r of source r)
__global__ void __launch_bounds__(kCombNT) basis_combine_kernel(const float2* __restrict__ basis, int nslots,
                                                                const float2* __restrict__ W, int kmax,
                                                                const int* __restrict__ kr, double2* __restrict__ Y,
                                                                int nq, size_t n12) {
  __shared__ float2 wsh[kCombNJ][kCombKI];
  const int r = blockIdx.y;
  const int j0 = blockIdx.z * kCombNJ;
  const int nj = min(kCombNJ, nq - j0);
  const size_t e = (size_t)blockIdx.x * kCombNT + threadIdx.x;
  const int k = kr[r];
  const float2* B = basis + (size_t)r * nslots * n12;
  float2 acc[kCombNJ];
#pragma unroll
  for (int j = 0; j < kCombNJ; ++j) acc[j] = make_float2(0.f, 0.f);
  for (int i0 = 1; i0 <= k; i0 += kCombKI) {
    const int ni = min(kCombKI, k - i0 + 1);
    __syncthreads();
    for (int t = threadIdx.x; t < kCombNJ * kCombKI; t += kCombNT) {
      const int jj = t / kCombKI, ii = t % kCombKI;
      wsh[jj][ii] = (jj < nj && ii < ni) ? W[((size_t)r * nq + j0 + jj) * kmax + (i0 + ii - 1)] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    if (e < n12) {
      for (int ii = 0; ii < ni; ++ii) {
        const float2 u = __ldg(B + (size_t)(i0 + ii) * n12 + e);
#pragma unroll
        for (int j = 0; j < kCombNJ; ++j) {
          const float2 w = wsh[j][ii];
          acc[j].x = fmaf(w.x, u.x, fmaf(-w.y, u.y, acc[j].x));
          acc[j].y = fmaf(w.x, u.y, fmaf(w.y, u.x, acc[j].y));
        }
      }
    }
  }
  if (e < n12)
    for (int j = 0; j < nj; ++j)
      Y[((size_t)r * nq + j0 + j) * n12 + e] = make_double2((double)acc[j].x, (double)acc[j].y);
}

// R = b - z_j Y + H Y for (source r, node j) = blockIdx.y = r * nq + j; partial |R|^2 per block
__global__ void __launch_bounds__(kResNT) residual64_kernel(const double2* __restrict__ Y,
                                                            const double2* __restrict__ b,
                                                            const double2* __restrict__ z, const double2* U,
                                                            Geom g, double diag, double2* __restrict__ R,
                                                            double* __restrict__ part, int nq) {
  __shared__ double sh[kResNT / 32];
  const int rj = blockIdx.y;
  const int r = rj / nq, j = rj % nq;
  const size_t n12 = (size_t)12 * g.V;
  const double2* Yj = Y + (size_t)rj * n12;
  const double2* br = b + (size_t)r * n12;
  double2* Rj = R + (size_t)rj * n12;
  const double2 zj = z[j];
  const int s = blockIdx.x * kResNT + threadIdx.x;
  double nrm = 0.0;
  if (s < g.V) {
    Cx<double> o[12];
    hw_site<double>(Yj, U, g, s, diag, o);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const size_t e = k * (size_t)g.V + s;
      const double2 y = Yj[e], bb = br[e];
      // b - z y + H y
      const double re = bb.x - (zj.x * y.x - zj.y * y.y) + o[k].re;
      const double im = bb.y - (zj.x * y.y + zj.y * y.x) + o[k].im;
      Rj[e] = make_double2(re, im);
      nrm += re * re + im * im;
    }
  }
  const double t = block_sum<kResNT>(nrm, sh);
  if (threadIdx.x == 0) part[(size_t)rj * gridDim.x + blockIdx.x] = t;
}

__global__ void reduce_rows_kernel(const double* __restrict__ part, int nblk, double* __restrict__ out) {
  __shared__ double sh[256 / 32];
  const double t = sum_partials<256>(part + (size_t)blockIdx.x * nblk, nblk, sh);
  if (threadIdx.x == 0) out[blockIdx.x] = t;
}

__global__ void accumulate_kernel(double2* __restrict__ Y, const float2* __restrict__ X, size_t n) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const float2 x = X[t];
    double2 y = Y[t];
    y.x += (double)x.x;
    y.y += (double)x.y;
    Y[t] = y;
  }
}

// s[r][e] = c0 b[r][e] + sum_j c_j Y[r][j][e]
__global__ void weighted_sum_kernel(const double2* __restrict__ Y, const double2* __restrict__ b,
                                    const double2* __restrict__ c, double2 c0, double2* __restrict__ out, int nq,
                                    size_t n12, int nsrc) {
  const size_t n = n12 * nsrc;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const size_t r = t / n12, e = t % n12;
    const double2 bb = b[t];
    double re = c0.x * bb.x - c0.y * bb.y, im = c0.x * bb.y + c0.y * bb.x;
    for (int j = 0; j < nq; ++j) {
      const double2 y = Y[(r * nq + j) * n12 + e];
      const double2 cj = c[j];
      re += cj.x * y.x - cj.y * y.y;
      im += cj.x * y.y + cj.y * y.x;
    }
    out[t] = make_double2(re, im);
  }
}

int cap_grid(size_t n) {
  size_t b = (n + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  return (int)(b > 0 ? b : 1);
}

}  // namespace

int launch_basis_combine(ov_ctx* ctx, const float2* basis, int nslots, const float2* W, int kmax, const int* kr,
                         double2* Y, int nsrc, int nq, cudaStream_t s) {
  const size_t n12 = (size_t)12 * ctx->g.V;
  dim3 grid((unsigned)((n12 + kCombNT - 1) / kCombNT), nsrc, (nq + kCombNJ - 1) / kCombNJ);
  cudaEvent_t ev;
  kt_begin(ctx, KC_MISC, s, &ev);
  basis_combine_kernel<<<grid, kCombNT, 0, s>>>(basis, nslots, W, kmax, kr, Y, nq, n12);
  kt_end(ctx, KC_MISC, s, ev);
  OV_CHECK_LAUNCH(ctx, "basis_combine_kernel");
  return OV_OK;
}

int launch_residual64(ov_ctx* ctx, const double2* Y, const double2* b, const double2* z, double2* R, double* part,
                      double* rnorm2, int nsrc, int nq, cudaStream_t s) {
  const int nblk = (ctx->g.V + kResNT - 1) / kResNT;
  cudaEvent_t ev;
  kt_begin(ctx, KC_RESIDUAL, s, &ev);
  residual64_kernel<<<dim3(nblk, nsrc * nq), kResNT, 0, s>>>(Y, b, z, ctx->U64, ctx->g, 4.0 - ctx->m0, R, part, nq);
  reduce_rows_kernel<<<nsrc * nq, 256, 0, s>>>(part, nblk, rnorm2);
  kt_end(ctx, KC_RESIDUAL, s, ev);
  OV_CHECK_LAUNCH(ctx, "residual64_kernel");
  return OV_OK;
}

int residual64_partials(ov_ctx* ctx) { return (ctx->g.V + kResNT - 1) / kResNT; }

int launch_accumulate(ov_ctx* ctx, double2* Y, const float2* X, size_t n, cudaStream_t s) {
  accumulate_kernel<<<cap_grid(n), 256, 0, s>>>(Y, X, n);
  OV_CHECK_LAUNCH(ctx, "accumulate_kernel");
  return OV_OK;
}

int launch_weighted_sum(ov_ctx* ctx, const double2* Y, const double2* b, const double2* c, double2 c0, double2* out,
                        int nsrc, int nq, cudaStream_t s) {
  const size_t n12 = (size_t)12 * ctx->g.V;
  weighted_sum_kernel<<<cap_grid(n12 * nsrc), 256, 0, s>>>(Y, b, c, c0, out, nq, n12, nsrc);
  OV_CHECK_LAUNCH(ctx, "weighted_sum_kernel");
  return OV_OK;
}
