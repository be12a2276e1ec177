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

// Four threads per site (one per direction), the partial hop sums combined through
// shared memory (hw_split_phase1/2): four times the threads of the tile kernel for the
// same work, so more loads are in flight per SM.  Uncompressed links.
__global__ void __launch_bounds__(kSplitNT) hw32_split_kernel(const float2* __restrict__ in, float2* __restrict__ out,
                                                             const float2* __restrict__ U, Geom g, float diag) {
  __shared__ Cx<float> sm[4 * 12 * kSplitSites];
  const size_t off = (size_t)blockIdx.y * 12 * g.V;
  const int site0 = blockIdx.x * kSplitSites;
  hw_split_phase1<float>(in + off, U, g, site0, sm);
  __syncthreads();
  Cx<float> o[3];
  int s, k0;
  if (hw_split_phase2<float>(in + off, g, site0, diag, sm, o, &s, &k0)) {
#pragma unroll
    for (int q = 0; q < 3; ++q) st<float>(out + off + (k0 + q) * (size_t)g.V + s, o[q]);
  }
}

void launch_split(const float2* in, float2* out, const float2* U, Geom g, float diag, int nrhs, cudaStream_t s) {
  dim3 grid((g.V + kSplitSites - 1) / kSplitSites, nrhs);
  hw32_split_kernel<<<grid, kSplitNT, 0, s>>>(in, out, U, g, diag);
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

// The structure-of-arrays variants kept: each is the fastest, or within 0.5% of it, for
// some lattice and right-hand-side count of a sweep over 8^4, 12^3 x 24, 16^4 and
// 16^3 x 32 with 1, 2, 3, 4, 6, 8 and 12 RHS (six others never were and were removed).
const Cand kCands[] = {
    {1, true, 128, launch_variant<1, true, 128>},
    {2, false, 128, launch_variant<2, false, 128>},
    {0, false, kSplitNT, launch_split},  // rhs tile 0: four threads per site
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

// ------------------------------------------------------------------------------------
// Spin-paired FP32 layout ("S4"): one float4 holds (psi[s][c], psi[s+2][c]) for an upper
// spin s in {0, 1}; element (rhs r, pair p = 3 s + c, site) at (r * 6 + p) * V + site.
// A neighbour spinor is 6 loads of 16 bytes (the float2 layout needs 12 of 8 bytes), and
// the addressing is 32-bit.  Links: 3 float4 per (mu, site) holding rows 0 and 1 of U
// (row 2 rebuilt as conj(row0 x row1)).
namespace {

// rows 0 and 1 of a 12-real S4 link (3 float4), row 2 rebuilt as conj(row0 x row1)
__device__ __forceinline__ void load_link_s4(const float4* __restrict__ L, int mu, int V, int site,
                                             Cx<float> U[3][3]) {
  const float4* p = L + (size_t)mu * 3 * V + site;
  const float4 a = __ldg(p), b = __ldg(p + V), c = __ldg(p + 2 * (size_t)V);
  U[0][0] = {a.x, a.y}; U[0][1] = {a.z, a.w}; U[0][2] = {b.x, b.y};
  U[1][0] = {b.z, b.w}; U[1][1] = {c.x, c.y}; U[1][2] = {c.z, c.w};
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const int j1 = (j + 1) % 3, j2 = (j + 2) % 3;
    Cx<float> t = {U[0][j1].re * U[1][j2].re - U[0][j1].im * U[1][j2].im,
                   U[0][j1].re * U[1][j2].im + U[0][j1].im * U[1][j2].re};
    t.re -= U[0][j2].re * U[1][j1].re - U[0][j2].im * U[1][j1].im;
    t.im -= U[0][j2].re * U[1][j1].im + U[0][j2].im * U[1][j1].re;
    U[2][j] = {t.re, -t.im};
  }
}

template <int MU>
__device__ __forceinline__ void hop_dir_s4(const float4* __restrict__ in, const float4* __restrict__ L, const Geom& g,
                                           int s, const int c[4], Cx<float> acc[12]) {
  const int V = g.V;
#pragma unroll
  for (int dir = 0; dir < 2; ++dir) {
    int sgn;
    const int sn = dir == 0 ? nb_fwd(g, s, c, MU, &sgn) : nb_bwd(g, s, c, MU, &sgn);
    const float4* pn = in + sn;
    Cx<float> h0[3], h1[3];
#pragma unroll
    for (int col = 0; col < 3; ++col) {
      const float4 a = __ldg(pn + col * V);        // (psi0, psi2) at colour col
      const float4 b = __ldg(pn + (3 + col) * V);  // (psi1, psi3)
      const Cx<float> p0 = {a.x, a.y}, p2 = {a.z, a.w}, p1 = {b.x, b.y}, p3 = {b.z, b.w};
      Cx<float> a0, a1;
      mulA<MU>(p2, p3, a0, a1);
      if (dir == 0) { h0[col] = csub(p0, a0); h1[col] = csub(p1, a1); }
      else { h0[col] = cadd(p0, a0); h1[col] = cadd(p1, a1); }
    }
    Cx<float> U[3][3];
    load_link_s4(L, MU, V, dir == 0 ? s : sn, U);
    const float f = -0.5f * (float)sgn;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      Cx<float> u0 = {0.f, 0.f}, u1 = {0.f, 0.f};
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        if (dir == 0) { u0 = cfma(U[i][j], h0[j], u0); u1 = cfma(U[i][j], h1[j], u1); }
        else { u0 = cfmaconj(U[j][i], h0[j], u0); u1 = cfmaconj(U[j][i], h1[j], u1); }
      }
      Cx<float> b0, b1;
      mulAdag<MU>(u0, u1, b0, b1);
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

// 7 resident blocks of 128 threads per SM (<= 72 registers): the kernel waits on L2
// latency, and the extra warps hide more of it (16^3x32, 12 RHS: 102.7 us at 80
// registers, 97.3 us here).  The diagonal term is read before the hops, so that the x
// and y neighbours, which share its cache lines, follow it through L1.
constexpr int kS4NT = 128;
__global__ void __launch_bounds__(kS4NT, 7) hw32_s4_kernel(const float4* __restrict__ in, float4* __restrict__ out,
                                                           const float4* __restrict__ L, Geom g, float diag) {
  const int s = blockIdx.x * kS4NT + threadIdx.x;
  if (s >= g.V) return;
  int c[4];
  site_coords(g, s, c);
  const int V = g.V;
  const float4* inr = in + (size_t)blockIdx.y * 6 * V;
  float4* outr = out + (size_t)blockIdx.y * 6 * V;
  Cx<float> acc[12];
#pragma unroll
  for (int p = 0; p < 6; ++p) {
    const int sp = p / 3, col = p % 3;
    const float4 v = __ldg(inr + p * V + s);
    acc[sp * 3 + col] = cscale(diag, Cx<float>{v.x, v.y});
    acc[(sp + 2) * 3 + col] = cscale(diag, Cx<float>{v.z, v.w});
  }
  hop_dir_s4<0>(inr, L, g, s, c, acc);
  hop_dir_s4<1>(inr, L, g, s, c, acc);
  hop_dir_s4<2>(inr, L, g, s, c, acc);
  hop_dir_s4<3>(inr, L, g, s, c, acc);
#pragma unroll
  for (int p = 0; p < 6; ++p) {
    const int sp = p / 3, col = p % 3;
    const Cx<float> up = acc[sp * 3 + col], lo = acc[(sp + 2) * 3 + col];
    // upper spin sp, lower spin sp + 2 (gamma5 = -1 on it)
    outr[p * V + s] = make_float4(up.re, up.im, -lo.re, -lo.im);
  }
}

// canonical complex64 [rhs][site][12] <-> S4
__global__ void pack_s4_kernel(const float2* __restrict__ aos, float4* __restrict__ s4, int V, int nrhs) {
  const size_t n = (size_t)nrhs * 6 * V;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const size_t site = t % V, q = t / V;
    const size_t p = q % 6, r = q / 6;
    const size_t sp = p / 3, col = p % 3;
    const float2* a = aos + ((size_t)r * V + site) * 12;
    const float2 u = a[sp * 3 + col], l = a[(sp + 2) * 3 + col];
    s4[t] = make_float4(u.x, u.y, l.x, l.y);
  }
}

__global__ void unpack_s4_kernel(const float4* __restrict__ s4, float2* __restrict__ aos, int V, int nrhs) {
  const size_t n = (size_t)nrhs * 6 * V;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const size_t site = t % V, q = t / V;
    const size_t p = q % 6, r = q / 6;
    const size_t sp = p / 3, col = p % 3;
    const float4 v = s4[t];
    float2* a = aos + ((size_t)r * V + site) * 12;
    a[sp * 3 + col] = make_float2(v.x, v.y);
    a[(sp + 2) * 3 + col] = make_float2(v.z, v.w);
  }
}

// U32 planes (mu*9 + e, site) -> 12-real S4 links: 3 float4 holding rows 0 and 1 in
// element pairs (U00, U01), (U02, U10), (U11, U12)
__global__ void links_s4_kernel(const float2* __restrict__ u32, float4* __restrict__ l3, int V) {
  const size_t n = (size_t)4 * V;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const size_t site = t % V, mu = t / V;
    float2 e[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) e[k] = u32[(mu * 9 + k) * V + site];
#pragma unroll
    for (int k = 0; k < 3; ++k) l3[(mu * 3 + k) * V + site] = make_float4(e[2 * k].x, e[2 * k].y, e[2 * k + 1].x, e[2 * k + 1].y);
  }
}

int cap_grid32(size_t n) {
  size_t b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return (int)(b > 0 ? b : 1);
}

}  // namespace

int launch_pack_s4(ov_ctx* ctx, const float2* aos, float4* s4, int nrhs, cudaStream_t s) {
  pack_s4_kernel<<<cap_grid32((size_t)nrhs * 6 * ctx->g.V), 256, 0, s>>>(aos, s4, ctx->g.V, nrhs);
  OV_CHECK_LAUNCH(ctx, "pack_s4_kernel");
  return OV_OK;
}

int launch_unpack_s4(ov_ctx* ctx, const float4* s4, float2* aos, int nrhs, cudaStream_t s) {
  unpack_s4_kernel<<<cap_grid32((size_t)nrhs * 6 * ctx->g.V), 256, 0, s>>>(s4, aos, ctx->g.V, nrhs);
  OV_CHECK_LAUNCH(ctx, "unpack_s4_kernel");
  return OV_OK;
}

// The 12-real S4 links (3 float4 per link, built on first use after set_gauge); the
// right-hand-side-paired kernels read the same form.
const float4* s4_links(ov_ctx* ctx, cudaStream_t s, int* st) {
  float4* l3 = (float4*)ws_get(ctx, "gauge.s4l3", sizeof(float4) * 4 * 3 * (size_t)ctx->g.V, st);
  if (*st != OV_OK) return nullptr;
  if (!ctx->have_s4) {
    links_s4_kernel<<<cap_grid32((size_t)4 * ctx->g.V), 256, 0, s>>>(ctx->U32, l3, ctx->g.V);
    ctx->have_s4 = true;
  }
  return l3;
}

// out = H_W in on the S4 layout with the 12-real links, one RHS per thread.
int launch_hw32_s4(ov_ctx* ctx, const float4* in, float4* out, int nrhs, cudaStream_t s) {
  int st = OV_OK;
  const float4* l3 = s4_links(ctx, s, &st);
  if (st != OV_OK) return st;
  const float diag = (float)(4.0 - ctx->m0);
  dim3 grid((ctx->g.V + kS4NT - 1) / kS4NT, nrhs);
  cudaEvent_t ev;
  kt_begin(ctx, KC_DSLASH, s, &ev);
  hw32_s4_kernel<<<grid, kS4NT, 0, s>>>(in, out, l3, ctx->g, diag);
  kt_end(ctx, KC_DSLASH, s, ev);
  OV_CHECK_LAUNCH(ctx, "hw32_s4_kernel");
  return OV_OK;
}
