// Kernels on the right-hand-side-paired FP32 layout (see pair32.cuh): broadcast
// links, packing from and to the canonical layout, and H_W.
#include "pair32.cuh"

namespace {

constexpr int kNTP = 128;

// U32 planes (mu*9 + e, site) -> broadcast float4 (re, re, im, im)
__global__ void links_bcast_kernel(const float2* __restrict__ u32, float4* __restrict__ b, int V) {
  const size_t n = (size_t)4 * 9 * V;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const float2 v = u32[t];
    b[t] = make_float4(v.x, v.x, v.y, v.y);
  }
}

// canonical complex64 [rhs][site][12] -> pairs; a missing partner of an odd count is 0
__global__ void pack_pair_f32_kernel(const float2* __restrict__ aos, float4* __restrict__ pr, int V, int nrhs) {
  const int npair = (nrhs + 1) / 2;
  const size_t n = (size_t)npair * 12 * V;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const size_t site = t % V, q = t / V;
    const size_t k = q % 12, pq = q / 12;
    const int r0 = (int)(2 * pq), r1 = r0 + 1;
    const float2 a = aos[((size_t)r0 * V + site) * 12 + k];
    const float2 b = r1 < nrhs ? aos[((size_t)r1 * V + site) * 12 + k] : make_float2(0.f, 0.f);
    pr[t] = make_float4(a.x, b.x, a.y, b.y);
  }
}

__global__ void unpack_pair_f32_kernel(const float4* __restrict__ pr, float2* __restrict__ aos, int V, int nrhs) {
  const size_t n = (size_t)nrhs * V * 12;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const size_t k = t % 12, q = t / 12;
    const size_t site = q % V, r = q / V;
    const float4 v = pr[((r / 2) * 12 + k) * V + site];
    aos[t] = (r & 1) ? make_float2(v.y, v.w) : make_float2(v.x, v.z);
  }
}

// grid: x = pair, y = block of sites (consecutive blocks share links through L2)
__global__ void __launch_bounds__(kNTP) hw_pair_kernel(const float4* __restrict__ in, float4* __restrict__ out,
                                                       const float4* __restrict__ L, Geom g, float diag) {
  const int s = blockIdx.y * kNTP + threadIdx.x;
  if (s >= g.V) return;
  const size_t off = (size_t)blockIdx.x * 12 * g.V;
  P2 o[12];
  hw_pair_site(in + off, L, g, s, diag, o);
#pragma unroll
  for (int k = 0; k < 12; ++k) stp(out + off + k * (size_t)g.V + s, o[k]);
}

int cap_grid(size_t n) {
  size_t b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return (int)(b > 0 ? b : 1);
}

}  // namespace

const float4* pair_links(ov_ctx* ctx, cudaStream_t s, int* st) {
  float4* b = (float4*)ws_get(ctx, "gauge.b32", sizeof(float4) * 4 * 9 * (size_t)ctx->g.V, st);
  if (*st != OV_OK) return nullptr;
  if (!ctx->have_b32) {
    links_bcast_kernel<<<cap_grid((size_t)36 * ctx->g.V), 256, 0, s>>>(ctx->U32, b, ctx->g.V);
    ctx->have_b32 = true;
  }
  return b;
}

int launch_pack_pair32(ov_ctx* ctx, const float2* aos, float4* pr, int nrhs, cudaStream_t s) {
  const size_t n = (size_t)((nrhs + 1) / 2) * 12 * ctx->g.V;
  pack_pair_f32_kernel<<<cap_grid(n), 256, 0, s>>>(aos, pr, ctx->g.V, nrhs);
  OV_CHECK_LAUNCH(ctx, "pack_pair_f32_kernel");
  return OV_OK;
}

int launch_unpack_pair32(ov_ctx* ctx, const float4* pr, float2* aos, int nrhs, cudaStream_t s) {
  const size_t n = (size_t)nrhs * 12 * ctx->g.V;
  unpack_pair_f32_kernel<<<cap_grid(n), 256, 0, s>>>(pr, aos, ctx->g.V, nrhs);
  OV_CHECK_LAUNCH(ctx, "unpack_pair_f32_kernel");
  return OV_OK;
}

int launch_hw_pair(ov_ctx* ctx, const float4* in, float4* out, int npair, cudaStream_t s) {
  int st = OV_OK;
  const float4* L = pair_links(ctx, s, &st);
  if (st != OV_OK) return st;
  dim3 grid(npair, (ctx->g.V + kNTP - 1) / kNTP);
  cudaEvent_t ev;
  kt_begin(ctx, KC_DSLASH, s, &ev);
  hw_pair_kernel<<<grid, kNTP, 0, s>>>(in, out, L, ctx->g, (float)(4.0 - ctx->m0));
  kt_end(ctx, KC_DSLASH, s, ev);
  OV_CHECK_LAUNCH(ctx, "hw_pair_kernel");
  return OV_OK;
}
