// Kernels on the right-hand-side-paired FP32 layout (see pair32.cuh): packing from and
// to the canonical layout, and H_W.
#include "pair32.cuh"

namespace {

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

// H_W on the paired layout with 12-real links.  grid: x = pair, y = block of sites.
// At most 128 registers (4 blocks of 128 threads per SM): 12 accumulator pairs, the
// half spinor and the rebuilt link are live together.  The diagonal term is read before
// the hops, so that the x and y neighbours, which share its cache lines, follow it
// through L1.
template <int LK, int NT>
__global__ void __launch_bounds__(NT, 512 / NT) hw_pair12_kernel(const float4* __restrict__ in,
                                                                 float4* __restrict__ out,
                                                                 const float4* __restrict__ L, Geom g, float diag) {
  const int s = blockIdx.y * NT + threadIdx.x;
  if (s >= g.V) return;
  int c[4];
  site_coords(g, s, c);
  const size_t off = (size_t)blockIdx.x * 12 * g.V;
  const float4* inq = in + off;
  const float2 d2 = f2(diag, diag), nd2 = f2(-diag, -diag);
  P2 o[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const P2 v = ldp(inq + k * (size_t)g.V + s);
    const float2 d = k < 6 ? d2 : nd2;  // lower spins: gamma5 = -1, accumulated negated
    o[k] = {mul2(d, v.re), mul2(d, v.im)};
  }
  hop_pair12<0, LK>(inq, L, g, s, c, o);
  hop_pair12<1, LK>(inq, L, g, s, c, o);
  hop_pair12<2, LK>(inq, L, g, s, c, o);
  hop_pair12<3, LK>(inq, L, g, s, c, o);
#pragma unroll
  for (int k = 0; k < 12; ++k) stp(out + off + k * (size_t)g.V + s, o[k]);
}

int cap_grid(size_t n) {
  size_t b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return (int)(b > 0 ? b : 1);
}

}  // namespace

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

// form 2: compact 12-real links (the spin-paired layout's 3 float4 per link, 48 B), the
// centre read first, 128 threads per block; form 6: the same with row 2 rebuilt once in
// scalar arithmetic.
int launch_hw_pair12(ov_ctx* ctx, const float4* in, float4* out, int npair, int form, cudaStream_t s) {
  int st = OV_OK;
  const float4* L = s4_links(ctx, s, &st);
  if (st != OV_OK) return st;
  constexpr int NT = 128;
  dim3 grid(npair, (ctx->g.V + NT - 1) / NT);
  const float diag = (float)(4.0 - ctx->m0);
  cudaEvent_t ev;
  kt_begin(ctx, KC_DSLASH, s, &ev);
  if (form == 6)
    hw_pair12_kernel<3, NT><<<grid, NT, 0, s>>>(in, out, L, ctx->g, diag);
  else
    hw_pair12_kernel<1, NT><<<grid, NT, 0, s>>>(in, out, L, ctx->g, diag);
  kt_end(ctx, KC_DSLASH, s, ev);
  OV_CHECK_LAUNCH(ctx, "hw_pair12_kernel");
  return OV_OK;
}
