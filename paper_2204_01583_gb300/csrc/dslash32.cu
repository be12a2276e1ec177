// FP32 Wilson operator for many right-hand sides, and its autotuner.
//
// H_W is bandwidth bound in FP32 (1368 flop against 480 B per site and RHS with
// uncompressed links).  Two ways to cut bytes per RHS:
//  * RHS tiling: one thread applies the links it loads to RT right-hand sides, so
//    link traffic per RHS drops by RT (accumulators: 24 RT floats per thread);
//  * 12-real link compression: only rows 0 and 1 of each SU(3) link are stored;
//    row 2 = conj(row0 x row1) (unitarity and det U = 1), rebuilt in registers.
// With RT = 4 and compression the compulsory traffic is 192/4 + 192 = 240 B per site
// and RHS.  The autotuner times the variants on the live problem once per
// (lattice, nrhs) and keeps the fastest.
#include <vector>

#include "common.cuh"

namespace {

template <int MU, int RT, bool COMP>
__device__ __forceinline__ void hop_dir_tile(const float2* __restrict__ in, size_t rstride,
                                             const float2* __restrict__ U, const Geom& g, int s, const int c[4],
                                             Cx<float> acc[RT][12]) {
  const int V = g.V;
#pragma unroll
  for (int dir = 0; dir < 2; ++dir) {
    int sgn;
    const int sn = dir == 0 ? nb_fwd(g, s, c, MU, &sgn) : nb_bwd(g, s, c, MU, &sgn);
    const int sl = dir == 0 ? s : sn;
    // link in registers: L[i][j] = U[i][j]
    Cx<float> L[3][3];
    if (COMP) {
#pragma unroll
      for (int e = 0; e < 6; ++e) L[e / 3][e % 3] = ld<float>(U + (MU * 6 + e) * (size_t)V + sl);
      // row 2 = conj(row0 x row1)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const int j1 = (j + 1) % 3, j2 = (j + 2) % 3;
        Cx<float> t = {L[0][j1].re * L[1][j2].re - L[0][j1].im * L[1][j2].im,
                       L[0][j1].re * L[1][j2].im + L[0][j1].im * L[1][j2].re};
        t.re -= L[0][j2].re * L[1][j1].re - L[0][j2].im * L[1][j1].im;
        t.im -= L[0][j2].re * L[1][j1].im + L[0][j2].im * L[1][j1].re;
        L[2][j] = {t.re, -t.im};
      }
    } else {
#pragma unroll
      for (int e = 0; e < 9; ++e) L[e / 3][e % 3] = ld<float>(U + (MU * 9 + e) * (size_t)V + sl);
    }
    const float f = -0.5f * (float)sgn;
#pragma unroll
    for (int r = 0; r < RT; ++r) {
      const float2* inr = in + r * rstride;
      Cx<float> h0[3], h1[3];
#pragma unroll
      for (int col = 0; col < 3; ++col) {
        const Cx<float> p0 = ld<float>(inr + (0 * 3 + col) * (size_t)V + sn);
        const Cx<float> p1 = ld<float>(inr + (1 * 3 + col) * (size_t)V + sn);
        const Cx<float> p2 = ld<float>(inr + (2 * 3 + col) * (size_t)V + sn);
        const Cx<float> p3 = ld<float>(inr + (3 * 3 + col) * (size_t)V + sn);
        Cx<float> a0, a1;
        mulA<MU>(p2, p3, a0, a1);
        if (dir == 0) { h0[col] = csub(p0, a0); h1[col] = csub(p1, a1); }
        else { h0[col] = cadd(p0, a0); h1[col] = cadd(p1, a1); }
      }
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        Cx<float> u0 = {0.f, 0.f}, u1 = {0.f, 0.f};
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          if (dir == 0) { u0 = cfma(L[i][j], h0[j], u0); u1 = cfma(L[i][j], h1[j], u1); }
          else { u0 = cfmaconj(L[j][i], h0[j], u0); u1 = cfmaconj(L[j][i], h1[j], u1); }
        }
        Cx<float> b0, b1;
        mulAdag<MU>(u0, u1, b0, b1);
        acc[r][0 * 3 + i] = cadd(acc[r][0 * 3 + i], cscale(f, u0));
        acc[r][1 * 3 + i] = cadd(acc[r][1 * 3 + i], cscale(f, u1));
        if (dir == 0) {
          acc[r][2 * 3 + i] = csub(acc[r][2 * 3 + i], cscale(f, b0));
          acc[r][3 * 3 + i] = csub(acc[r][3 * 3 + i], cscale(f, b1));
        } else {
          acc[r][2 * 3 + i] = cadd(acc[r][2 * 3 + i], cscale(f, b0));
          acc[r][3 * 3 + i] = cadd(acc[r][3 * 3 + i], cscale(f, b1));
        }
      }
    }
  }
}

// out_r = H_W in_r for RT consecutive right-hand sides per thread (blockIdx.y = tile).
template <int RT, bool COMP, int NT>
__global__ void __launch_bounds__(NT) hw32_tile_kernel(const float2* __restrict__ in, float2* __restrict__ out,
                                                       const float2* __restrict__ U, Geom g, float diag, int nrhs) {
  const int s = blockIdx.x * NT + threadIdx.x;
  if (s >= g.V) return;
  const size_t rstride = (size_t)12 * g.V;
  const int r0 = blockIdx.y * RT;
  const int nr = min(RT, nrhs - r0);
  const float2* inb = in + r0 * rstride;
  float2* outb = out + r0 * rstride;
  Cx<float> acc[RT][12];
#pragma unroll
  for (int r = 0; r < RT; ++r)
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[r][k] = {0.f, 0.f};
  int c[4];
  site_coords(g, s, c);
  if (nr == RT) {
    hop_dir_tile<0, RT, COMP>(inb, rstride, U, g, s, c, acc);
    hop_dir_tile<1, RT, COMP>(inb, rstride, U, g, s, c, acc);
    hop_dir_tile<2, RT, COMP>(inb, rstride, U, g, s, c, acc);
    hop_dir_tile<3, RT, COMP>(inb, rstride, U, g, s, c, acc);
  } else {
    // ragged last tile: one RHS at a time (rare; keeps the full-tile path branch free)
    for (int r = 0; r < nr; ++r) {
      Cx<float> a1[1][12];
#pragma unroll
      for (int k = 0; k < 12; ++k) a1[0][k] = {0.f, 0.f};
      const float2* inr = inb + r * rstride;
      hop_dir_tile<0, 1, COMP>(inr, rstride, U, g, s, c, a1);
      hop_dir_tile<1, 1, COMP>(inr, rstride, U, g, s, c, a1);
      hop_dir_tile<2, 1, COMP>(inr, rstride, U, g, s, c, a1);
      hop_dir_tile<3, 1, COMP>(inr, rstride, U, g, s, c, a1);
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        Cx<float> v = cadd(cscale(diag, ld<float>(inr + k * (size_t)g.V + s)), a1[0][k]);
        if (k >= 6) v = cneg(v);
        st<float>(outb + r * rstride + k * (size_t)g.V + s, v);
      }
    }
    return;
  }
#pragma unroll
  for (int r = 0; r < RT; ++r)
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      Cx<float> v = cadd(cscale(diag, ld<float>(inb + r * rstride + k * (size_t)g.V + s)), acc[r][k]);
      if (k >= 6) v = cneg(v);
      st<float>(outb + r * rstride + k * (size_t)g.V + s, v);
    }
}

__global__ void compress_links_kernel(const float2* __restrict__ u32, float2* __restrict__ c32, int V) {
  const size_t n = (size_t)4 * 6 * V;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const size_t site = t % V, q = t / V;  // q = mu * 6 + e
    const size_t mu = q / 6, e = q % 6;
    c32[t] = u32[(mu * 9 + e) * V + site];
  }
}

template <int RT, bool COMP, int NT>
void launch_variant(const float2* in, float2* out, const float2* U, Geom g, float diag, int nrhs, cudaStream_t s) {
  dim3 grid((g.V + NT - 1) / NT, (nrhs + RT - 1) / RT);
  hw32_tile_kernel<RT, COMP, NT><<<grid, NT, 0, s>>>(in, out, U, g, diag, nrhs);
}

using LaunchFn = void (*)(const float2*, float2*, const float2*, Geom, float, int, cudaStream_t);

struct Cand {
  int rt;
  bool comp;
  int nt;
  LaunchFn fn;
};

const Cand kCands[] = {
    {1, false, 128, launch_variant<1, false, 128>}, {1, true, 128, launch_variant<1, true, 128>},
    {2, false, 128, launch_variant<2, false, 128>}, {2, true, 128, launch_variant<2, true, 128>},
    {4, true, 128, launch_variant<4, true, 128>},   {4, true, 64, launch_variant<4, true, 64>},
    {2, true, 256, launch_variant<2, true, 256>},   {1, true, 256, launch_variant<1, true, 256>},
};
constexpr int kNCands = sizeof(kCands) / sizeof(kCands[0]);

}  // namespace

// Compressed FP32 links (rows 0, 1), built lazily from the FP32 planes.
static float2* compressed_links(ov_ctx* ctx, cudaStream_t s, int* st) {
  float2* c = (float2*)ws_get(ctx, "gauge.c32", sizeof(float2) * 4 * 6 * (size_t)ctx->g.V, st);
  if (*st != OV_OK) return nullptr;
  if (!ctx->have_c32) {
    compress_links_kernel<<<1024, 256, 0, s>>>(ctx->U32, c, ctx->g.V);
    ctx->have_c32 = true;
  }
  return c;
}

// Time every structure-of-arrays variant on the live data (3 launches each after a
// warm-up); returns the best time per launch in ms and its index in *best.
float hw32_time_soa_variants(ov_ctx* ctx, const float2* in, float2* out, int nrhs, cudaStream_t s, int* best) {
  int st = OV_OK;
  const float2* Uc = compressed_links(ctx, s, &st);
  if (st != OV_OK) return 1e30f;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  const float diag = (float)(4.0 - ctx->m0);
  float best_ms = 1e30f;
  *best = 1;
  for (int k = 0; k < kNCands; ++k) {
    const Cand& c = kCands[k];
    const float2* U = c.comp ? Uc : ctx->U32;
    c.fn(in, out, U, ctx->g, diag, nrhs, s);  // warm
    cudaEventRecord(a, s);
    for (int rep = 0; rep < 3; ++rep) c.fn(in, out, U, ctx->g, diag, nrhs, s);
    cudaEventRecord(b, s);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    if (cudaGetLastError() == cudaSuccess && ms / 3 < best_ms) {
      best_ms = ms / 3;
      *best = k;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return best_ms;
}

int launch_hw32_tuned(ov_ctx* ctx, const float2* in, float2* out, int nrhs, cudaStream_t s, int force_variant,
                      int* used) {
  int st = OV_OK;
  const float2* Uc = compressed_links(ctx, s, &st);
  if (st != OV_OK) return st;
  int k = force_variant;
  if (k < 0 || k >= kNCands) hw32_time_soa_variants(ctx, in, out, nrhs, s, &k);
  const Cand& c = kCands[k];
  cudaEvent_t ev;
  kt_begin(ctx, KC_DSLASH, s, &ev);
  c.fn(in, out, c.comp ? Uc : ctx->U32, ctx->g, (float)(4.0 - ctx->m0), nrhs, s);
  kt_end(ctx, KC_DSLASH, s, ev);
  OV_CHECK_LAUNCH(ctx, "hw32_tile_kernel");
  if (used) *used = k;
  return OV_OK;
}

int hw32_variant_count() { return kNCands; }

void hw32_variant_info(int k, int* rt, int* comp, int* nt) {
  *rt = kCands[k].rt;
  *comp = kCands[k].comp;
  *nt = kCands[k].nt;
}
