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

// 12-real links, broadcast form: U32 planes (mu*9 + e, site), e < 6 -> float4 (re, re, im, im)
__global__ void links_bcast12_kernel(const float2* __restrict__ u32, float4* __restrict__ b, int V) {
  const size_t n = (size_t)4 * 6 * V;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const size_t site = t % V, q = t / V;
    const float2 v = u32[((q / 6) * 9 + q % 6) * V + site];
    b[t] = make_float4(v.x, v.x, v.y, v.y);
  }
}

// H_W on the paired layout with 12-real links.  grid: x = pair, y = block of sites.
// At most 128 registers (4 blocks of 128 threads per SM): 12 accumulator pairs, the
// half spinor and the rebuilt link are live together.
// CF (centre first): the diagonal term is read before the hops, so that the x and y
// neighbours, which share its cache lines, follow it through L1.
// Ask L1 for one direction's neighbour data ahead of its use: the 12 component planes of
// the pair at x + mu and x - mu and the compact 12-real links U_mu(x), U_mu(x - mu)
// (prefetch.global.L1: no registers are held while the lines arrive).
__device__ __forceinline__ void pf_l1(const void* p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }
template <int MU>
__device__ __forceinline__ void prefetch_dir(const float4* __restrict__ in, const float4* __restrict__ L,
                                             const Geom& g, int s, const int c[4]) {
  int sg;
  const int sf = nb_fwd(g, s, c, MU, &sg), sb = nb_bwd(g, s, c, MU, &sg);
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    pf_l1(in + k * (size_t)g.V + sf);
    pf_l1(in + k * (size_t)g.V + sb);
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    pf_l1(L + ((size_t)MU * 3 + k) * g.V + s);
    pf_l1(L + ((size_t)MU * 3 + k) * g.V + sb);
  }
}

// PF: each direction's neighbour data is prefetched into L1 one direction ahead.
template <int LK, int NT, bool CF, bool PF = false>
__global__ void __launch_bounds__(NT, 512 / NT) hw_pair12_kernel(const float4* __restrict__ in,
                                                                 float4* __restrict__ out,
                                                                 const float4* __restrict__ L, Geom g, float diag) {
  const int s = blockIdx.y * NT + threadIdx.x;
  if (s >= g.V) return;
  int c[4];
  site_coords(g, s, c);
  const size_t off = (size_t)blockIdx.x * 12 * g.V;
  const float4* inq = in + off;
  if (PF) prefetch_dir<0>(inq, L, g, s, c);
  const float2 d2 = f2(diag, diag), nd2 = f2(-diag, -diag);
  P2 o[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    if (CF) {
      const P2 v = ldp(inq + k * (size_t)g.V + s);
      const float2 d = k < 6 ? d2 : nd2;  // lower spins: gamma5 = -1, accumulated negated
      o[k] = {mul2(d, v.re), mul2(d, v.im)};
    } else {
      o[k] = {f2(0.f, 0.f), f2(0.f, 0.f)};
    }
  }
  if (PF) prefetch_dir<1>(inq, L, g, s, c);
  hop_pair12<0, LK>(inq, L, g, s, c, o);
  if (PF) prefetch_dir<2>(inq, L, g, s, c);
  hop_pair12<1, LK>(inq, L, g, s, c, o);
  if (PF) prefetch_dir<3>(inq, L, g, s, c);
  hop_pair12<2, LK>(inq, L, g, s, c, o);
  hop_pair12<3, LK>(inq, L, g, s, c, o);
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    P2 r = o[k];
    if (!CF) {
      const P2 v = ldp(inq + k * (size_t)g.V + s);
      const float2 d = k < 6 ? d2 : nd2;
      r = {fma2(d, v.re, r.re), fma2(d, v.im, r.im)};
    }
    stp(out + off + k * (size_t)g.V + s, r);
  }
}

__device__ __forceinline__ void cp_async16(void* dst_shared, const void* src_global) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst_shared);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(__cvta_generic_to_global(src_global))
               : "memory");
}

// H_W on the paired layout with compact 12-real links, one tile of 128 consecutive sites
// per block: R = 128 / Lx whole rows of one xy-plane (R must divide Ly).  The tile's
// spinor rows -1..R and its x and y link rows -1..R-1 are copied into shared memory
// with asynchronous 16-byte copies while the z and t hops read global memory; the
// centre and the x and y hops then read shared memory (5 of the 9 spinor reads and 4 of
// the 8 link reads of a site).  Shared memory: (12 (R + 2) + 6 (R + 1)) Lx float4.
__global__ void __launch_bounds__(128, 4) hw_pair12_tile_kernel(const float4* __restrict__ in,
                                                                float4* __restrict__ out,
                                                                const float4* __restrict__ L, Geom g, float diag) {
  extern __shared__ float4 sm[];
  const int Lx = g.L[0], Ly = g.L[1], R = 128 / Lx;
  const int W = (R + 2) * Lx, WL = (R + 1) * Lx;
  float4* ssp = sm;           // [12][W]: spinor rows -1..R
  float4* slk = sm + 12 * W;  // [2 mu][3][WL]: x and y link rows -1..R-1
  const int t = threadIdx.x;
  const int s0 = blockIdx.y * 128, s = s0 + t;
  const int plane0 = s0 - s0 % (Lx * Ly);
  const int y0 = (s0 / Lx) % Ly;
  const float4* inq = in + (size_t)blockIdx.x * 12 * g.V;
  // staged position j (row j / Lx - 1, x = j % Lx) is the same site in both arrays
  for (int j = t; j < W; j += 128) {
    const int yy = (y0 + j / Lx - 1 + Ly) % Ly;
    const int src = plane0 + yy * Lx + j % Lx;
#pragma unroll
    for (int k = 0; k < 12; ++k) cp_async16(ssp + k * W + j, inq + (size_t)k * g.V + src);
    if (j < WL) {
#pragma unroll
      for (int mk = 0; mk < 6; ++mk) cp_async16(slk + mk * WL + j, L + (size_t)mk * g.V + src);  // mk = 3 mu + k
    }
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  P2 o[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) o[k] = {f2(0.f, 0.f), f2(0.f, 0.f)};
  int c[4];
  site_coords(g, s, c);
  hop_pair12<2, 1>(inq, L, g, s, c, o);
  hop_pair12<3, 1>(inq, L, g, s, c, o);
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();
  const int x = t % Lx, r = t / Lx;
  // both staged arrays start at row -1: (x, row r) is at (r + 1) Lx + x in each
  const int li = (r + 1) * Lx + x;
  const int xp = (r + 1) * Lx + (x + 1) % Lx, xm = (r + 1) * Lx + (x + Lx - 1) % Lx;
  hop_pair12_shared<0, 0>(ssp + xp, W, slk + 0 * WL + li, WL, o);       // U_x(x) psi(x + x^)
  hop_pair12_shared<0, 1>(ssp + xm, W, slk + 0 * WL + xm, WL, o);       // U_x(x - x^)^dag psi(x - x^)
  hop_pair12_shared<1, 0>(ssp + li + Lx, W, slk + 3 * WL + li, WL, o);  // U_y(x) psi(x + y^)
  hop_pair12_shared<1, 1>(ssp + li - Lx, W, slk + 3 * WL + li - Lx, WL, o);
  const float2 d2 = f2(diag, diag), nd2 = f2(-diag, -diag);
  float4* outq = out + (size_t)blockIdx.x * 12 * g.V;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const float4 v = ssp[k * W + li];
    const float2 d = k < 6 ? d2 : nd2;  // lower spins: gamma5 = -1, accumulated negated
    stp(outq + (size_t)k * g.V + s, P2{fma2(d, f2(v.x, v.y), o[k].re), fma2(d, f2(v.z, v.w), o[k].im)});
  }
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

const float4* pair_links12(ov_ctx* ctx, cudaStream_t s, int* st) {
  float4* b = (float4*)ws_get(ctx, "gauge.b12", sizeof(float4) * 4 * 6 * (size_t)ctx->g.V, st);
  if (*st != OV_OK) return nullptr;
  if (!ctx->have_b12) {
    links_bcast12_kernel<<<cap_grid((size_t)24 * ctx->g.V), 256, 0, s>>>(ctx->U32, b, ctx->g.V);
    ctx->have_b12 = true;
  }
  return b;
}

// form 5: tiles of 128 sites with the in-plane neighbours staged in shared memory
// (hw_pair12_tile_kernel; needs 128 % Lx == 0 and Ly % (128 / Lx) == 0).
static int launch_hw_pair12_tile(ov_ctx* ctx, const float4* in, float4* out, int npair, cudaStream_t s) {
  const int Lx = ctx->g.L[0], Ly = ctx->g.L[1];
  if (Lx > 128 || 128 % Lx != 0 || Ly % (128 / Lx) != 0)
    return ctx_fail(ctx, OV_ERR_INVALID_ARG, "shared-memory tiled stencil needs 128 % Lx == 0 and Ly % (128 / Lx) == 0");
  int st = OV_OK;
  const float4* L = s4_links(ctx, true, s, &st);
  if (st != OV_OK) return st;
  const int R = 128 / Lx;
  const size_t shm = sizeof(float4) * (size_t)(12 * (R + 2) + 6 * (R + 1)) * Lx;
  cudaError_t e = cudaFuncSetAttribute(hw_pair12_tile_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e == cudaSuccess && shm > 48 * 1024)
    e = cudaFuncSetAttribute(hw_pair12_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
  if (e != cudaSuccess) return ctx_cuda(ctx, e, "cudaFuncSetAttribute(hw_pair12_tile_kernel)");
  dim3 grid(npair, ctx->g.V / 128);
  cudaEvent_t ev;
  kt_begin(ctx, KC_DSLASH, s, &ev);
  hw_pair12_tile_kernel<<<grid, 128, shm, s>>>(in, out, L, ctx->g, (float)(4.0 - ctx->m0));
  kt_end(ctx, KC_DSLASH, s, ev);
  OV_CHECK_LAUNCH(ctx, "hw_pair12_tile_kernel");
  return OV_OK;
}

// form 0: broadcast 12-real links (96 B per link); 1: the spin-paired layout's 3 float4
// (48 B); 2 and 3: form 1 reading the centre first, 128 or 256 threads per block; 4: form
// 2 with all 9 link elements read (the spin-paired layout's padded 5 float4, 80 B), no
// rebuild; 5: hw_pair12_tile_kernel; 6: form 2 with row 2 rebuilt in scalar arithmetic;
// 7: form 6 with each direction's neighbour data prefetched into L1 one direction ahead
// (the carveout set to the smallest shared memory, so that L1 holds the prefetched lines).
int launch_hw_pair12(ov_ctx* ctx, const float4* in, float4* out, int npair, int form, cudaStream_t s) {
  if (form == 5) return launch_hw_pair12_tile(ctx, in, out, npair, s);
  int st = OV_OK;
  const float4* L = form == 0 ? pair_links12(ctx, s, &st) : s4_links(ctx, form != 4, s, &st);
  if (st != OV_OK) return st;
  const int NT = form == 3 ? 256 : 128;
  if (form == 7) {
    cudaError_t e = cudaFuncSetAttribute(hw_pair12_kernel<3, 128, true, true>,
                                         cudaFuncAttributePreferredSharedMemoryCarveout, 0);
    if (e != cudaSuccess) return ctx_cuda(ctx, e, "cudaFuncSetAttribute(hw_pair12_kernel)");
  }
  dim3 grid(npair, (ctx->g.V + NT - 1) / NT);
  const float diag = (float)(4.0 - ctx->m0);
  cudaEvent_t ev;
  kt_begin(ctx, KC_DSLASH, s, &ev);
  if (form == 0)
    hw_pair12_kernel<0, 128, false><<<grid, NT, 0, s>>>(in, out, L, ctx->g, diag);
  else if (form == 1)
    hw_pair12_kernel<1, 128, false><<<grid, NT, 0, s>>>(in, out, L, ctx->g, diag);
  else if (form == 2)
    hw_pair12_kernel<1, 128, true><<<grid, NT, 0, s>>>(in, out, L, ctx->g, diag);
  else if (form == 3)
    hw_pair12_kernel<1, 256, true><<<grid, NT, 0, s>>>(in, out, L, ctx->g, diag);
  else if (form == 4)
    hw_pair12_kernel<2, 128, true><<<grid, NT, 0, s>>>(in, out, L, ctx->g, diag);
  else if (form == 6)
    hw_pair12_kernel<3, 128, true><<<grid, NT, 0, s>>>(in, out, L, ctx->g, diag);
  else
    hw_pair12_kernel<3, 128, true, true><<<grid, NT, 0, s>>>(in, out, L, ctx->g, diag);
  kt_end(ctx, KC_DSLASH, s, ev);
  OV_CHECK_LAUNCH(ctx, "hw_pair12_kernel");
  return OV_OK;
}
