// Wilson operator H_W = gamma5 D_W(-m0) on structure-of-arrays fields, and the
// layout conversions between the canonical (array-of-structures) layout of the
// ABI and the site-major planes the kernels read.
//
// Structure of arrays: a spinor is 12 planes of V complex numbers (plane k =
// 3 * spin + colour), so consecutive threads (consecutive sites) read
// consecutive 8- or 16-byte words of a plane; a gauge field is 4 x 9 planes.
#include "common.cuh"

namespace {

constexpr int kNT = 128;

// canonical U[mu][site][i][j] -> planes (mu*9 + 3i + j), FP64 and FP32 copies, and the
// FP64 copy for the solver stencils: scaled by -1/2 (exact; the hop factor of D_W) and,
// on the time links of the last time slice, by the time boundary sign bc_t (a hop
// across the t boundary in either direction uses exactly that link, so the stencil
// applies no boundary sign of its own)
__global__ void gauge_ingest_kernel(const double2* __restrict__ aos, double2* __restrict__ u64,
                                    float2* __restrict__ u32, double2* __restrict__ u64h, int V, int Vt,
                                    double bc_t) {
  const size_t n = (size_t)4 * V * 9;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const size_t e = t % 9, q = t / 9;
    const size_t site = q % V, mu = q / V;
    const double2 v = aos[t];
    const size_t o = (mu * 9 + e) * V + site;
    u64[o] = v;
    u32[o] = make_float2((float)v.x, (float)v.y);
    const double f = (mu == 3 && site >= (size_t)(V - Vt)) ? -0.5 * bc_t : -0.5;
    u64h[o] = make_double2(f * v.x, f * v.y);
  }
}

template <typename T>
__global__ void pack_kernel(const T* __restrict__ aos, T* __restrict__ soa, int V, int nrhs) {
  const size_t n = (size_t)nrhs * V * 12;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const size_t k = t % 12, q = t / 12;
    const size_t site = q % V, r = q / V;
    soa[(r * 12 + k) * V + site] = aos[t];
  }
}

template <typename T>
__global__ void unpack_kernel(const T* __restrict__ soa, T* __restrict__ aos, int V, int nrhs) {
  const size_t n = (size_t)nrhs * V * 12;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const size_t k = t % 12, q = t / 12;
    const size_t site = q % V, r = q / V;
    aos[t] = soa[(r * 12 + k) * V + site];
  }
}

// out = (1+m)/2 b + (1-m)/2 gamma5 s ; b, out canonical; s structure of arrays
__global__ void overlap_epilogue_kernel(const double2* __restrict__ b, const double2* __restrict__ s,
                                        double2* __restrict__ out, double a, double c, int V, int nrhs) {
  const size_t n = (size_t)nrhs * V * 12;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const size_t k = t % 12, q = t / 12;
    const size_t site = q % V, r = q / V;
    const double2 sv = s[(r * 12 + k) * V + site];
    const double g = (k < 6) ? c : -c;  // gamma5 = diag(1, 1, -1, -1) on spin = k / 3
    const double2 bv = b[t];
    out[t] = make_double2(fma(a, bv.x, g * sv.x), fma(a, bv.y, g * sv.y));
  }
}

__global__ void gamma5_aos_kernel(const double2* __restrict__ in, double2* __restrict__ out, int V, int nrhs) {
  const size_t n = (size_t)nrhs * V * 12;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const double2 v = in[t];
    out[t] = ((t % 12) < 6) ? v : make_double2(-v.x, -v.y);
  }
}

template <typename R>
__global__ void __launch_bounds__(kNT) hw_kernel(const typename Store<R>::T* __restrict__ in,
                                                 typename Store<R>::T* __restrict__ out,
                                                 const typename Store<R>::T* __restrict__ U, Geom g, R diag) {
  const int s = blockIdx.x * kNT + threadIdx.x;
  if (s >= g.V) return;
  const size_t off = (size_t)blockIdx.y * 12 * g.V;
  Cx<R> o[12];
  hw_site<R>(in + off, U, g, s, diag, o);
#pragma unroll
  for (int k = 0; k < 12; ++k) st<R>(out + off + k * (size_t)g.V + s, o[k]);
}

// FP64 link planes -> double-float planes (hi, lo per real; float4 per complex)
__global__ void links_df_kernel(const double2* __restrict__ u64, float4* __restrict__ udf, size_t n) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const double2 v = u64[t];
    const float rh = __double2float_rn(v.x), ih = __double2float_rn(v.y);
    udf[t] = make_float4(rh, __double2float_rn(v.x - (double)rh), ih, __double2float_rn(v.y - (double)ih));
  }
}

int grid_for(size_t n, int nt) {
  size_t b = (n + nt - 1) / nt;
  if (b > 152 * 16) b = 152 * 16;
  return (int)(b > 0 ? b : 1);
}

}  // namespace

int launch_gauge_ingest(ov_ctx* ctx, const double2* U_aos, cudaStream_t s) {
  const size_t n = (size_t)4 * ctx->g.V * 9;
  cudaEvent_t ev;
  kt_begin(ctx, KC_LAYOUT, s, &ev);
  const int Vt = ctx->g.L[0] * ctx->g.L[1] * ctx->g.L[2];  // sites of one time slice
  gauge_ingest_kernel<<<grid_for(n, 256), 256, 0, s>>>(U_aos, ctx->U64, ctx->U32, ctx->U64h, ctx->g.V, Vt,
                                                       (double)ctx->g.bc_t);
  kt_end(ctx, KC_LAYOUT, s, ev);
  OV_CHECK_LAUNCH(ctx, "gauge_ingest_kernel");
  return OV_OK;
}

template <typename T>
static int pack_impl(ov_ctx* ctx, const T* aos, T* soa, int nrhs, cudaStream_t s, bool unpack) {
  const size_t n = (size_t)nrhs * ctx->g.V * 12;
  if (n == 0) return OV_OK;
  cudaEvent_t ev;
  kt_begin(ctx, KC_LAYOUT, s, &ev);
  if (unpack)
    unpack_kernel<T><<<grid_for(n, 256), 256, 0, s>>>(aos, soa, ctx->g.V, nrhs);
  else
    pack_kernel<T><<<grid_for(n, 256), 256, 0, s>>>(aos, soa, ctx->g.V, nrhs);
  kt_end(ctx, KC_LAYOUT, s, ev);
  OV_CHECK_LAUNCH(ctx, unpack ? "unpack_kernel" : "pack_kernel");
  return OV_OK;
}

int launch_pack64(ov_ctx* ctx, const double2* aos, double2* soa, int nrhs, cudaStream_t s) {
  return pack_impl<double2>(ctx, aos, soa, nrhs, s, false);
}
int launch_unpack64(ov_ctx* ctx, const double2* soa, double2* aos, int nrhs, cudaStream_t s) {
  return pack_impl<double2>(ctx, soa, aos, nrhs, s, true);
}
int launch_pack32(ov_ctx* ctx, const float2* aos, float2* soa, int nrhs, cudaStream_t s) {
  return pack_impl<float2>(ctx, aos, soa, nrhs, s, false);
}
int launch_unpack32(ov_ctx* ctx, const float2* soa, float2* aos, int nrhs, cudaStream_t s) {
  return pack_impl<float2>(ctx, soa, aos, nrhs, s, true);
}

int launch_hw64(ov_ctx* ctx, const double2* in, double2* out, int nrhs, cudaStream_t s) {
  dim3 grid((ctx->g.V + kNT - 1) / kNT, nrhs);
  cudaEvent_t ev;
  kt_begin(ctx, KC_DSLASH, s, &ev);
  hw_kernel<double><<<grid, kNT, 0, s>>>(in, out, ctx->U64, ctx->g, 4.0 - ctx->m0);
  kt_end(ctx, KC_DSLASH, s, ev);
  OV_CHECK_LAUNCH(ctx, "hw_kernel<double>");
  return OV_OK;
}

int launch_hw32(ov_ctx* ctx, const float2* in, float2* out, int nrhs, cudaStream_t s) {
  dim3 grid((ctx->g.V + kNT - 1) / kNT, nrhs);
  cudaEvent_t ev;
  kt_begin(ctx, KC_DSLASH, s, &ev);
  hw_kernel<float><<<grid, kNT, 0, s>>>(in, out, ctx->U32, ctx->g, (float)(4.0 - ctx->m0));
  kt_end(ctx, KC_DSLASH, s, ev);
  OV_CHECK_LAUNCH(ctx, "hw_kernel<float>");
  return OV_OK;
}

int launch_overlap_epilogue(ov_ctx* ctx, const double2* b_aos, const double2* s_soa, double2* out_aos,
                            double m_q, int nrhs, cudaStream_t s) {
  const size_t n = (size_t)nrhs * ctx->g.V * 12;
  cudaEvent_t ev;
  kt_begin(ctx, KC_LAYOUT, s, &ev);
  overlap_epilogue_kernel<<<grid_for(n, 256), 256, 0, s>>>(b_aos, s_soa, out_aos, 0.5 * (1.0 + m_q),
                                                           0.5 * (1.0 - m_q), ctx->g.V, nrhs);
  kt_end(ctx, KC_LAYOUT, s, ev);
  OV_CHECK_LAUNCH(ctx, "overlap_epilogue_kernel");
  return OV_OK;
}

int launch_gamma5_aos(ov_ctx* ctx, const double2* in, double2* out, int nrhs, cudaStream_t s) {
  const size_t n = (size_t)nrhs * ctx->g.V * 12;
  gamma5_aos_kernel<<<grid_for(n, 256), 256, 0, s>>>(in, out, ctx->g.V, nrhs);
  OV_CHECK_LAUNCH(ctx, "gamma5_aos_kernel");
  return OV_OK;
}

int ensure_links_df(ov_ctx* ctx, cudaStream_t s) {
  int st = OV_OK;
  const size_t n = (size_t)4 * 9 * ctx->g.V;
  ctx->Udf = (float4*)ws_get(ctx, "gauge.df", sizeof(float4) * n, &st);
  if (st != OV_OK) return st;
  if (!ctx->have_df) {
    links_df_kernel<<<grid_for(n, 256), 256, 0, s>>>(ctx->U64h, ctx->Udf, n);  // -1/2 U, signs baked in
    OV_CHECK_LAUNCH(ctx, "links_df_kernel");
    ctx->have_df = true;
  }
  return OV_OK;
}
