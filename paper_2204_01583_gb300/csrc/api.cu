// The C ABI entry points declared in include/ov.h, and the context utilities.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"

const char* const kKernelClassNames[KC_COUNT] = {"hw_kernel",         "lanczos_hw_kernel", "lanczos_update_kernel",
                                                  "layout_kernels",    "init_kernels",      "force_kernel",
                                                  "residual_kernels",  "lanczos_regen_kernel", "lanczos_coop_kernel",
                                                  "basis_sum_kernel"};

// ------------------------------------------------------------ utilities

int ctx_fail(ov_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return code;
}

int ctx_cuda(ov_ctx* ctx, cudaError_t e, const char* what) {
  return ctx_fail(ctx, e == cudaErrorMemoryAllocation ? OV_ERR_OUT_OF_MEMORY : OV_ERR_CUDA,
                  std::string(what) + ": " + cudaGetErrorString(e));
}

void* ws_get(ov_ctx* ctx, const char* name, size_t bytes, int* status) {
  if (*status != OV_OK) return nullptr;
  DevBuf& b = ctx->bufs[name];
  if (b.bytes >= bytes && b.p) return b.p;
  if (b.p) {
    cudaDeviceSynchronize();
    cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    graphs_release(ctx);  // captured graphs may point at the old buffer
  }
  const size_t nb = std::max<size_t>(bytes, 256);
  cudaError_t e = cudaMalloc(&b.p, nb);
  if (e != cudaSuccess) {
    cudaGetLastError();
    // Out of memory: release the stored Krylov bases ("<tag>.ring" of the stored-basis
    // forms, the largest workspaces, rebuilt on demand) of every solver form other than the
    // requesting one -- those are idle -- and retry once.
    const std::string nm(name), tag = nm.substr(0, nm.find('.'));
    bool freed = false;
    for (auto& kv : ctx->bufs) {
      const std::string& k = kv.first;
      const bool ring = k.size() > 6 && k.compare(k.size() - 6, 6, "s.ring") == 0;
      if (kv.second.p && ring && k.substr(0, k.find('.')) != tag) {
        cudaDeviceSynchronize();
        cudaFree(kv.second.p);
        kv.second.p = nullptr;
        kv.second.bytes = 0;
        freed = true;
      }
    }
    if (freed) {
      graphs_release(ctx);
      e = cudaMalloc(&b.p, nb);
      if (e == cudaSuccess) {
        b.bytes = nb;
        return b.p;
      }
      cudaGetLastError();
    }
    b.p = nullptr;
    *status = ctx_fail(ctx, OV_ERR_OUT_OF_MEMORY,
                       std::string("cudaMalloc of workspace '") + name + "' (" + std::to_string(nb) + " bytes) failed");
    return nullptr;
  }
  b.bytes = nb;
  return b.p;
}

void ws_release_all(ov_ctx* ctx) {
  for (auto& kv : ctx->bufs)
    if (kv.second.p) cudaFree(kv.second.p);
  ctx->bufs.clear();
}

void graphs_release(ov_ctx* ctx) {
  for (auto& kv : ctx->graphs) cudaGraphExecDestroy(kv.second);
  ctx->graphs.clear();
}

void kt_begin(ov_ctx* ctx, int cls, cudaStream_t s, cudaEvent_t* a) {
  *a = nullptr;
  if (!ctx->timing) return;
  if (ctx->event_pool.empty()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    ctx->event_pool.push_back(e);
  }
  *a = ctx->event_pool.back();
  ctx->event_pool.pop_back();
  cudaEventRecord(*a, s);
  (void)cls;
}

void kt_end(ov_ctx* ctx, int cls, cudaStream_t s, cudaEvent_t a) {
  if (!ctx->timing || !a) return;
  cudaEvent_t b;
  if (ctx->event_pool.empty()) {
    if (cudaEventCreate(&b) != cudaSuccess) return;
  } else {
    b = ctx->event_pool.back();
    ctx->event_pool.pop_back();
  }
  cudaEventRecord(b, s);
  ctx->pending.push_back({cls, a, b});
}

void kt_collect(ov_ctx* ctx) {
  for (auto& p : ctx->pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      ctx->clocks[p.cls].launches += 1;
      ctx->clocks[p.cls].total_ms += ms;
    }
    ctx->event_pool.push_back(p.a);
    ctx->event_pool.push_back(p.b);
  }
  ctx->pending.clear();
}

// ------------------------------------------------ helpers of the entry points

ov_solve_opts resolve_opts(const ov_solve_opts* o) {
  ov_solve_opts r;
  r.mode = OV_MODE_FP64;
  r.tol = 1e-12;
  r.max_iter = 20000;
  r.host_io = 0;
  r.check_every = 32;
  r.use_graph = 1;
  r.node_chunk = 0;
  if (o) r = *o;
  if (r.check_every <= 0) r.check_every = 32;
  return r;
}

int check_opts(ov_ctx* ctx, const ov_solve_opts& o) {
  if (!(o.tol > 0.0) || !(o.tol < 1.0)) return ctx_fail(ctx, OV_ERR_INVALID_ARG, "tol must be in (0, 1)");
  if (o.max_iter < 1) return ctx_fail(ctx, OV_ERR_INVALID_ARG, "max_iter must be >= 1");
  if (o.mode != OV_MODE_FP64 && o.mode != OV_MODE_MIXED && o.mode != OV_MODE_FP64_2PASS &&
      o.mode != OV_MODE_FP64_REGEN && o.mode != OV_MODE_F32X2)
    return ctx_fail(ctx, OV_ERR_INVALID_ARG, "unknown solver mode");
  return OV_OK;
}

double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

namespace {
__global__ void copy16_kernel(const double2* __restrict__ src, double2* __restrict__ dst, size_t n) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    dst[t] = src[t];
}

// The device address of page-locked host memory (cudaHostAlloc, cudaHostRegister), or null
// for any other pointer.
const void* pinned_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // an unknown pointer: a non-sticky error, left to the copy below
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}
}  // namespace

// Device copy of a (possibly host) canonical spinor set; returns the device pointer.
// Page-locked host memory is read by a kernel over the host link: on GB300 the copy
// engine's host-to-device rate for a 302 MB set fell from ~210 GB/s to 15-60 GB/s in the
// course of repeated long solves, while a kernel reading the same buffer stayed at
// ~215 GB/s.  Other host memory goes through cudaMemcpyAsync.
const double2* stage_in(ov_ctx* ctx, const void* p, size_t bytes, int host_io, const char* name, cudaStream_t s,
                        int* st) {
  if (!host_io) return (const double2*)p;
  void* d = ws_get(ctx, name, bytes, st);
  if (*st != OV_OK) return nullptr;
  const void* hp = pinned_device_ptr(p);
  if (hp && ((uintptr_t)hp & 15) == 0 && bytes % 16 == 0) {
    const size_t n = bytes / 16;
    const unsigned grid = (unsigned)std::max<size_t>(1, std::min<size_t>((n + 255) / 256, 152 * 8));
    cudaEvent_t ev;
    kt_begin(ctx, KC_LAYOUT, s, &ev);
    copy16_kernel<<<grid, 256, 0, s>>>((const double2*)hp, (double2*)d, n);
    kt_end(ctx, KC_LAYOUT, s, ev);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) *st = ctx_cuda(ctx, e, "copy16_kernel");
    return (const double2*)d;
  }
  cudaError_t e = cudaMemcpyAsync(d, p, bytes, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) *st = ctx_cuda(ctx, e, "host-to-device copy");
  return (const double2*)d;
}

// Copy of a device result to host memory: written by a kernel when the destination is
// page-locked (as stage_in reads), else by cudaMemcpyAsync.
int stage_out(ov_ctx* ctx, void* host, const void* dev, size_t bytes, cudaStream_t s) {
  void* hp = const_cast<void*>(pinned_device_ptr(host));
  if (hp && ((uintptr_t)hp & 15) == 0 && ((uintptr_t)dev & 15) == 0 && bytes % 16 == 0) {
    const size_t n = bytes / 16;
    const unsigned grid = (unsigned)std::max<size_t>(1, std::min<size_t>((n + 255) / 256, 152 * 8));
    cudaEvent_t ev;
    kt_begin(ctx, KC_LAYOUT, s, &ev);
    copy16_kernel<<<grid, 256, 0, s>>>((const double2*)dev, (double2*)hp, n);
    kt_end(ctx, KC_LAYOUT, s, ev);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? OV_OK : ctx_cuda(ctx, e, "copy16_kernel");
  }
  const cudaError_t e = cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, s);
  return e == cudaSuccess ? OV_OK : ctx_cuda(ctx, e, "device-to-host copy");
}

namespace {
// out = c0 b: the quadrature with no nodes (a rank of a node-sharded sum that holds
// none of them contributes only its share of c0)
__global__ void cscale_kernel(const double2* __restrict__ in, double2* __restrict__ out, double2 c, size_t n) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const double2 v = in[t];
    out[t] = make_double2(c.x * v.x - c.y * v.y, c.x * v.y + c.y * v.x);
  }
}
}  // namespace

// Core of sgn / overlap: canonical b (device) -> S_N b (SoA, workspace).
int sign_core(ov_ctx* ctx, const double2* b_dev, int nrhs, const ov_solve_opts& o, SolveOut* so, cudaStream_t s,
              double2** s_soa_out, double2* xs) {
  NvtxRange nvtx_("sign_core");
  int st = OV_OK;
  const size_t n = (size_t)12 * ctx->g.V * nrhs;
  double2* b_soa = (double2*)ws_get(ctx, "api.b_soa", sizeof(double2) * n, &st);
  double2* s_soa = (double2*)ws_get(ctx, "api.s_soa", sizeof(double2) * n, &st);
  if (st != OV_OK) return st;
  st = launch_pack64(ctx, b_dev, b_soa, nrhs, s);
  if (st != OV_OK) return st;
  *s_soa_out = s_soa;
  if (ctx->z.empty()) {
    cscale_kernel<<<(unsigned)std::min<size_t>((n + 255) / 256, 152 * 8), 256, 0, s>>>(b_soa, s_soa, ctx->c0, n);
    OV_CHECK_LAUNCH(ctx, "cscale_kernel");
    *so = SolveOut();
    so->converged = 1;
    so->launches = 3.0;
    return OV_OK;
  }
  if (o.mode == OV_MODE_FP64 || xs) {
    st = solve_sign_soa(ctx, b_soa, s_soa, nrhs, o, so, s, xs);
  } else if (o.mode == OV_MODE_FP64_2PASS || o.mode == OV_MODE_FP64_REGEN || o.mode == OV_MODE_F32X2) {
    st = solve_sign_2pass(ctx, b_soa, s_soa, nrhs, o, so, s);
  } else if (o.mode == OV_MODE_MIXED) {
    st = solve_sign_mixed(ctx, b_soa, s_soa, nrhs, o, so, s);
  } else {
    return ctx_fail(ctx, OV_ERR_INVALID_ARG, "solver mode not available in this build");
  }
  *s_soa_out = s_soa;
  return st;
}

void fill_stats(ov_stats* st, const SolveOut& so, double ms) {
  if (!st) return;
  st->iterations = so.iterations;
  st->refine_rounds = so.refine_rounds;
  st->inner_iterations = so.inner_iterations;
  st->converged = so.converged;
  st->max_residual = so.max_residual;
  st->error_bound = so.error_bound;
  st->ms = ms;
  st->node_updates = so.node_updates;
  st->launches = so.launches;
}

// ------------------------------------------------------------------ ABI

extern "C" {

const char* ov_version(void) { return "ov-gb300 0.1 (sm_103a)"; }

int ov_create(ov_ctx** out, const int dims[4], int bc_t, double m0, double r, int device) {
  if (!out || !dims) return OV_ERR_INVALID_ARG;
  *out = nullptr;
  for (int k = 0; k < 4; ++k)
    if (dims[k] < 1) return OV_ERR_INVALID_ARG;
  if (bc_t != 1 && bc_t != -1) return OV_ERR_INVALID_ARG;
  if (r != 1.0) return OV_ERR_INVALID_ARG;
  if (!std::isfinite(m0)) return OV_ERR_INVALID_ARG;
  const long long V = (long long)dims[0] * dims[1] * dims[2] * dims[3];
  if (V > (1LL << 28)) return OV_ERR_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return OV_ERR_CUDA;
  }
  ov_ctx* ctx = new ov_ctx();
  ctx->device = device;
  DeviceGuard dg(device);
  for (int k = 0; k < 4; ++k) ctx->g.L[k] = dims[k];
  ctx->g.st[0] = 1;
  ctx->g.st[1] = dims[0];
  ctx->g.st[2] = dims[0] * dims[1];
  ctx->g.st[3] = dims[0] * dims[1] * dims[2];
  ctx->g.V = (int)V;
  ctx->g.bc_t = bc_t;
  ctx->m0 = m0;
  ctx->r = r;
  if (cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaHostAlloc((void**)&ctx->host_flag, sizeof(int) * 4, cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    ov_destroy(ctx);
    return OV_ERR_CUDA;
  }
  *out = ctx;
  return OV_OK;
}

int ov_destroy(ov_ctx* ctx) {
  if (!ctx) return OV_OK;
  DeviceGuard dg(ctx->device);
  cudaDeviceSynchronize();
  graphs_release(ctx);
  ws_release_all(ctx);
  if (ctx->U64) cudaFree(ctx->U64);
  if (ctx->U64h) cudaFree(ctx->U64h);
  if (ctx->U32) cudaFree(ctx->U32);
  for (auto& p : ctx->pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (auto e : ctx->event_pool) cudaEventDestroy(e);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  for (auto st : ctx->aux_streams) cudaStreamDestroy(st);
  for (auto e : ctx->cap_events) cudaEventDestroy(e);
  if (ctx->host_flag) cudaFreeHost(ctx->host_flag);
  delete ctx;
  return OV_OK;
}

const char* ov_last_error(const ov_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int ov_set_gauge(ov_ctx* ctx, const double* U, int on_device, void* stream) {
  NvtxRange nvtx_("ov_set_gauge");
  if (!ctx) return OV_ERR_INVALID_ARG;
  if (!U) return ctx_fail(ctx, OV_ERR_INVALID_ARG, "null gauge pointer");
  DeviceGuard dg(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n = (size_t)4 * ctx->g.V * 9;
  if (!ctx->U64) {
    if (cudaMalloc(&ctx->U64, sizeof(double2) * n) != cudaSuccess ||
        cudaMalloc(&ctx->U32, sizeof(float2) * n) != cudaSuccess ||
        cudaMalloc(&ctx->U64h, sizeof(double2) * n) != cudaSuccess) {
      cudaGetLastError();
      return ctx_fail(ctx, OV_ERR_OUT_OF_MEMORY, "gauge field allocation failed");
    }
  }
  int st = OV_OK;
  const double2* src = (const double2*)U;
  if (!on_device) {
    double2* tmp = (double2*)ws_get(ctx, "gauge.stage", sizeof(double2) * n, &st);
    if (st != OV_OK) return st;
    cudaError_t e = cudaMemcpyAsync(tmp, U, sizeof(double2) * n, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return ctx_cuda(ctx, e, "gauge copy");
    src = tmp;
  }
  st = launch_gauge_ingest(ctx, src, s);
  if (st != OV_OK) return st;
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return ctx_cuda(ctx, e, "ov_set_gauge");
  kt_collect(ctx);
  ctx->have_gauge = true;
  ctx->coef_iter_hint = 0;
  ctx->have_c32 = false;
  ctx->have_s4 = false;
  ctx->have_df = false;
  return OV_OK;
}

// FP32 stencil variants on float4 layouts, numbered after the structure-of-arrays ones:
// layout P (right-hand-side pairs, 12 float4 per site and pair) or S (spin pairs, 6
// float4 per site and RHS; its buffers alias the paired ones, 6 <= 12 per pair).
struct Float4Variant {
  bool paired;
  int form;              // P: launch_hw_pair12 form; S: unused (one S kernel)
  int rhs_tile, code, threads;  // as reported by ov_hw32_variants
};
constexpr Float4Variant kFloat4Variants[] = {
    {false, 0, 1, 8, 128},  // S, 12-real links, centre first
    {true, 2, 2, 9, 128},   // P, 12-real compact links, centre first
    {true, 6, 2, 12, 128},  // P, 12-real compact links, centre first, row 2 rebuilt in scalar
};
constexpr int kNFloat4Variants = sizeof(kFloat4Variants) / sizeof(kFloat4Variants[0]);

static int fp32_float4_pack(ov_ctx* ctx, int v, const float2* in, float4* buf, int nrhs, cudaStream_t s) {
  return kFloat4Variants[v].paired ? launch_pack_pair32(ctx, in, buf, nrhs, s) : launch_pack_s4(ctx, in, buf, nrhs, s);
}

static int fp32_float4_unpack(ov_ctx* ctx, int v, const float4* buf, float2* out, int nrhs, cudaStream_t s) {
  return kFloat4Variants[v].paired ? launch_unpack_pair32(ctx, buf, out, nrhs, s)
                                   : launch_unpack_s4(ctx, buf, out, nrhs, s);
}

static int fp32_float4_launch(ov_ctx* ctx, int v, const float4* in, float4* out, int nrhs, cudaStream_t s) {
  const Float4Variant& f = kFloat4Variants[v];
  const int npair = (nrhs + 1) / 2;
  if (!f.paired) return launch_hw32_s4(ctx, in, out, nrhs, s);
  return launch_hw_pair12(ctx, in, out, npair, f.form, s);
}

int ov_apply_HW(ov_ctx* ctx, const void* in, void* out, int nrhs, int precision, void* stream) {
  NvtxRange nvtx_("ov_apply_HW");
  if (!ctx) return OV_ERR_INVALID_ARG;
  if (!ctx->have_gauge) return ctx_fail(ctx, OV_ERR_NO_GAUGE, "ov_set_gauge has not been called");
  if (nrhs < 0 || (nrhs > 0 && (!in || !out)) || in == out)
    return ctx_fail(ctx, OV_ERR_INVALID_ARG, "bad vectors for ov_apply_HW");
  if (precision != OV_FP64 && precision != OV_FP32) return ctx_fail(ctx, OV_ERR_INVALID_ARG, "bad precision");
  if (nrhs == 0) return OV_OK;
  DeviceGuard dg(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n = (size_t)12 * ctx->g.V * nrhs;
  int st = OV_OK;
  if (precision == OV_FP64) {
    double2* a = (double2*)ws_get(ctx, "hw.a64", sizeof(double2) * n, &st);
    double2* b = (double2*)ws_get(ctx, "hw.b64", sizeof(double2) * n, &st);
    if (st != OV_OK) return st;
    if ((st = launch_pack64(ctx, (const double2*)in, a, nrhs, s))) return st;
    if ((st = launch_hw64(ctx, a, b, nrhs, s))) return st;
    if ((st = launch_unpack64(ctx, b, (double2*)out, nrhs, s))) return st;
  } else {
    const int npair = (nrhs + 1) / 2;
    const int kpair = hw32_variant_count();
    float2* a = (float2*)ws_get(ctx, "hw.a32", sizeof(float2) * n, &st);
    float2* b = (float2*)ws_get(ctx, "hw.b32", sizeof(float2) * n, &st);
    float4* pa = (float4*)ws_get(ctx, "hw.pa32", sizeof(float4) * 12 * (size_t)ctx->g.V * npair, &st);
    float4* pb = (float4*)ws_get(ctx, "hw.pb32", sizeof(float4) * 12 * (size_t)ctx->g.V * npair, &st);
    if (st != OV_OK) return st;
    int k = ctx->hw32_force;
    if (k < 0) {
      auto it = ctx->hw32_choice.find(nrhs);
      if (it != ctx->hw32_choice.end()) {
        k = it->second;
      } else {
        // autotune: every structure-of-arrays variant, then the paired and spin-paired
        // kernels, each timed on this data
        if ((st = launch_pack32(ctx, (const float2*)in, a, nrhs, s))) return st;
        int ksoa = 0;
        float best = hw32_time_soa_variants(ctx, a, b, nrhs, s, &ksoa);
        k = ksoa;
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        for (int kk = kpair; kk < kpair + kNFloat4Variants; ++kk) {
          if ((st = fp32_float4_pack(ctx, kk - kpair, (const float2*)in, pa, nrhs, s))) return st;
          st = fp32_float4_launch(ctx, kk - kpair, pa, pb, nrhs, s);  // warm (builds the links)
          if (st == OV_ERR_INVALID_ARG) {  // this lattice does not fit the variant
            st = OV_OK;
            continue;
          }
          if (st != OV_OK) return st;
          cudaEventRecord(e0, s);
          for (int rep = 0; rep < 3; ++rep) fp32_float4_launch(ctx, kk - kpair, pa, pb, nrhs, s);
          cudaEventRecord(e1, s);
          cudaEventSynchronize(e1);
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          if (ms / 3 < best) {
            best = ms / 3;
            k = kk;
          }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        ctx->hw32_choice[nrhs] = k;
      }
    }
    if (k >= kpair) {
      if ((st = fp32_float4_pack(ctx, k - kpair, (const float2*)in, pa, nrhs, s))) return st;
      if ((st = fp32_float4_launch(ctx, k - kpair, pa, pb, nrhs, s))) return st;
      if ((st = fp32_float4_unpack(ctx, k - kpair, pb, (float2*)out, nrhs, s))) return st;
    } else {
      if ((st = launch_pack32(ctx, (const float2*)in, a, nrhs, s))) return st;
      if ((st = launch_hw32_tuned(ctx, a, b, nrhs, s, k, nullptr))) return st;
      if ((st = launch_unpack32(ctx, b, (float2*)out, nrhs, s))) return st;
    }
  }
  return OV_OK;
}

int ov_set_contour(ov_ctx* ctx, int n, const double* z, const double* c, double c0_re, double c0_im) {
  if (!ctx) return OV_ERR_INVALID_ARG;
  if (n < 0 || (n > 0 && (!z || !c))) return ctx_fail(ctx, OV_ERR_INVALID_ARG, "bad contour arrays");
  if (!std::isfinite(c0_re) || !std::isfinite(c0_im)) return ctx_fail(ctx, OV_ERR_INVALID_ARG, "non-finite c0");
  std::vector<double2> zz(n), cc(n);
  for (int j = 0; j < n; ++j) {
    zz[j] = make_double2(z[2 * j], z[2 * j + 1]);
    cc[j] = make_double2(c[2 * j], c[2 * j + 1]);
    if (!std::isfinite(zz[j].x) || !std::isfinite(zz[j].y) || !std::isfinite(cc[j].x) || !std::isfinite(cc[j].y))
      return ctx_fail(ctx, OV_ERR_INVALID_ARG, "non-finite node or coefficient");
    if (zz[j].y == 0.0) return ctx_fail(ctx, OV_ERR_INVALID_ARG, "a node lies on the real axis");
  }
  ctx->z = zz;
  ctx->c = cc;
  ctx->c0 = make_double2(c0_re, c0_im);
  ctx->have_contour = true;
  ctx->coef_iter_hint = 0;
  return OV_OK;
}

int ov_set_contour_ellipse(ov_ctx* ctx, int n_q, double gamma, double rho, double alpha, int form) {
  if (!ctx) return OV_ERR_INVALID_ARG;
  if (n_q < 1 || !(rho > 0) || !(alpha > 0) || !std::isfinite(gamma) ||
      (form != OV_CONTOUR_SINGLE && form != OV_CONTOUR_PAIR))
    return ctx_fail(ctx, OV_ERR_INVALID_ARG, "bad ellipse parameters");
  std::vector<double2> z, c;
  double2 c0;
  ellipse_rule(n_q, gamma, rho, alpha, form, z, c, c0);
  for (auto& zz : z)
    if (zz.y == 0.0) return ctx_fail(ctx, OV_ERR_INVALID_ARG, "a node lies on the real axis");
  ctx->z = z;
  ctx->c = c;
  ctx->c0 = c0;
  ctx->have_contour = true;
  ctx->coef_iter_hint = 0;
  return OV_OK;
}

int ov_get_contour(const ov_ctx* ctx, int* n, double* z, double* c, double* c0) {
  if (!ctx || !n) return OV_ERR_INVALID_ARG;
  if (!ctx->have_contour) return OV_ERR_NO_CONTOUR;
  const int nn = (int)ctx->z.size();
  if (z && c) {
    if (*n < nn) return OV_ERR_INVALID_ARG;
    for (int j = 0; j < nn; ++j) {
      z[2 * j] = ctx->z[j].x;
      z[2 * j + 1] = ctx->z[j].y;
      c[2 * j] = ctx->c[j].x;
      c[2 * j + 1] = ctx->c[j].y;
    }
  }
  if (c0) {
    c0[0] = ctx->c0.x;
    c0[1] = ctx->c0.y;
  }
  *n = nn;
  return OV_OK;
}

// Spectral bounds from Lanczos on H and on H^2: extreme Ritz values lo, hi of H, an upper
// bound amax of |lambda| (Ritz value plus residual bound), the Ritz estimate gap of min
// |lambda| and gap_lo, a value below it by the residual bound of the H^2 Ritz value
// (at most 20% below).
static int spectral_bounds(ov_ctx* ctx, int steps, cudaStream_t s, double* lo, double* hi, double* amax,
                           double* gap, double* gap_lo, int* nsteps) {
  std::vector<double> a, b;
  int st = lanczos_tridiag(ctx, steps, 0, a, b, s);
  if (st != OV_OK) return st;
  double rlo, rhi;
  tridiag_extreme_eigs(a, b, lo, hi, &rlo, &rhi);
  *amax = std::max(std::fabs(*lo) + rlo, std::fabs(*hi) + rhi);
  std::vector<double> a2, b2;
  st = lanczos_tridiag(ctx, steps, 1, a2, b2, s);
  if (st != OV_OK) return st;
  double lo2, hi2, rlo2, rhi2;
  tridiag_extreme_eigs(a2, b2, &lo2, &hi2, &rlo2, &rhi2);
  *gap = std::max(std::sqrt(std::max(lo2, 0.0)), 1e-6 * *amax);
  *gap_lo = std::max(std::sqrt(std::max(lo2 - rlo2, 0.64 * lo2)), 1e-6 * *amax);
  *nsteps = (int)a.size();
  return OV_OK;
}

int ov_place_contour(ov_ctx* ctx, int n_q, int steps, ov_spectrum* out, void* stream) {
  NvtxRange nvtx_("ov_place_contour");
  if (!ctx) return OV_ERR_INVALID_ARG;
  if (!ctx->have_gauge) return ctx_fail(ctx, OV_ERR_NO_GAUGE, "ov_set_gauge has not been called");
  if (n_q < 2 || steps < 4) return ctx_fail(ctx, OV_ERR_INVALID_ARG, "need n_q >= 2 and steps >= 4");
  DeviceGuard dg(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  double lo, hi, amax, gap, gap_lo;
  int nsteps = 0;
  int st = spectral_bounds(ctx, steps, s, &lo, &hi, &amax, &gap, &gap_lo, &nsteps);
  if (st != OV_OK) return st;
  // single ellipse from 0 to 1.05 * amax; alpha minimises the predicted method error
  const double R = 1.05 * amax;
  const double gam = 0.5 * R, rho = 0.5 * R;
  std::vector<double> lam;
  const int nl = 200;
  for (int k = 0; k < nl; ++k) {
    const double t = (double)k / (nl - 1);
    const double l = gap * std::pow(amax / gap, t);
    lam.push_back(l);
    lam.push_back(-l);
  }
  double best_err = 1e300, best_alpha = 0.1;
  std::vector<double2> z, c;
  double2 c0;
  for (int k = 0; k <= 190; ++k) {
    const double al = 0.05 + 0.005 * k;
    ellipse_rule(n_q, gam, rho, al, OV_CONTOUR_SINGLE, z, c, c0);
    double err = 0.0;
    for (double l : lam) err = std::max(err, std::fabs(rational_value(l, z, c, c0) - (l > 0 ? 1.0 : -1.0)));
    if (err < best_err) {
      best_err = err;
      best_alpha = al;
    }
  }
  st = ov_set_contour_ellipse(ctx, n_q, gam, rho, best_alpha, OV_CONTOUR_SINGLE);
  if (st != OV_OK) return st;
  if (out) {
    out->lambda_min = lo;
    out->lambda_max = hi;
    out->abs_max_bound = amax;
    out->gap = gap;
    out->predicted_error = best_err;
    out->gamma = gam;
    out->rho = rho;
    out->alpha = best_alpha;
    out->steps = nsteps;
  }
  return OV_OK;
}

int ov_zolotarev_rule(int n_poles, double lambda_min, double lambda_max, double* z, double* c, double* delta) {
  if (!z || !c) return OV_ERR_INVALID_ARG;
  std::vector<double2> zz, cc;
  double2 c0;
  const int st = zolotarev_rule(n_poles, lambda_min, lambda_max, zz, cc, c0, delta);
  if (st != OV_OK) return st;
  for (size_t j = 0; j < zz.size(); ++j) {
    z[2 * j] = zz[j].x;
    z[2 * j + 1] = zz[j].y;
    c[2 * j] = cc[j].x;
    c[2 * j + 1] = cc[j].y;
  }
  return OV_OK;
}

int ov_set_contour_zolotarev(ov_ctx* ctx, int n_poles, double lambda_min, double lambda_max, double* delta) {
  if (!ctx) return OV_ERR_INVALID_ARG;
  std::vector<double2> z, c;
  double2 c0;
  if (zolotarev_rule(n_poles, lambda_min, lambda_max, z, c, c0, delta) != OV_OK)
    return ctx_fail(ctx, OV_ERR_INVALID_ARG, "need 1 <= n_poles <= 128 and 0 < lambda_min < lambda_max");
  ctx->z = z;
  ctx->c = c;
  ctx->c0 = c0;
  ctx->have_contour = true;
  ctx->coef_iter_hint = 0;
  return OV_OK;
}

int ov_place_zolotarev(ov_ctx* ctx, int n_poles, int steps, ov_spectrum* out, void* stream) {
  NvtxRange nvtx_("ov_place_zolotarev");
  if (!ctx) return OV_ERR_INVALID_ARG;
  if (!ctx->have_gauge) return ctx_fail(ctx, OV_ERR_NO_GAUGE, "ov_set_gauge has not been called");
  if (n_poles < 1 || n_poles > 128 || steps < 4)
    return ctx_fail(ctx, OV_ERR_INVALID_ARG, "need 1 <= n_poles <= 128 and steps >= 4");
  DeviceGuard dg(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  double lo, hi, amax, gap, gap_lo, delta = 0.0;
  int nsteps = 0;
  int st = spectral_bounds(ctx, steps, s, &lo, &hi, &amax, &gap, &gap_lo, &nsteps);
  if (st != OV_OK) return st;
  st = ov_set_contour_zolotarev(ctx, n_poles, gap_lo, amax, &delta);
  if (st != OV_OK) return st;
  if (out) {
    out->lambda_min = lo;
    out->lambda_max = hi;
    out->abs_max_bound = amax;
    out->gap = gap_lo;
    out->predicted_error = delta;
    out->gamma = 0.0;
    out->rho = 0.0;
    out->alpha = 0.0;
    out->steps = nsteps;
  }
  return OV_OK;
}

static int sign_or_overlap(ov_ctx* ctx, bool overlap, double m_q, const void* b, void* out, int nrhs,
                           const ov_solve_opts* opts, ov_stats* stats, void* stream) {
  const double t0 = now_ms();
  if (!ctx) return OV_ERR_INVALID_ARG;
  if (!ctx->have_gauge) return ctx_fail(ctx, OV_ERR_NO_GAUGE, "ov_set_gauge has not been called");
  if (!ctx->have_contour) return ctx_fail(ctx, OV_ERR_NO_CONTOUR, "no contour set");
  if (nrhs < 0 || (nrhs > 0 && (!b || !out))) return ctx_fail(ctx, OV_ERR_INVALID_ARG, "bad vectors");
  if (!std::isfinite(m_q)) return ctx_fail(ctx, OV_ERR_INVALID_ARG, "m_q is not finite");
  ov_solve_opts o = resolve_opts(opts);
  int st = check_opts(ctx, o);
  if (st != OV_OK) return st;
  if (nrhs == 0) return OV_OK;
  DeviceGuard dg(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n = (size_t)12 * ctx->g.V * nrhs;
  const double2* bd = stage_in(ctx, b, sizeof(double2) * n, o.host_io, "io.b", s, &st);
  if (st != OV_OK) return st;
  double2* od = o.host_io ? (double2*)ws_get(ctx, "io.out", sizeof(double2) * n, &st) : (double2*)out;
  if (st != OV_OK) return st;
  SolveOut so;
  double2* s_soa = nullptr;
  const int sst = sign_core(ctx, bd, nrhs, o, &so, s, &s_soa, nullptr);
  if (sst != OV_OK && sst != OV_ERR_NOT_CONVERGED) return sst;
  if (overlap)
    st = launch_overlap_epilogue(ctx, bd, s_soa, od, m_q, nrhs, s);
  else
    st = launch_unpack64(ctx, s_soa, od, nrhs, s);
  if (st != OV_OK) return st;
  if (o.host_io) {
    if ((st = stage_out(ctx, out, od, sizeof(double2) * n, s)) != OV_OK) return st;
    const cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return ctx_cuda(ctx, e, "sync");
  }
  kt_collect(ctx);
  fill_stats(stats, so, now_ms() - t0);
  return sst;
}

int ov_sgn_HW_apply(ov_ctx* ctx, const void* b, void* out, int nrhs, const ov_solve_opts* opts, ov_stats* stats,
                    void* stream) {
  NvtxRange nvtx_("ov_sgn_HW_apply");
  return sign_or_overlap(ctx, false, 0.0, b, out, nrhs, opts, stats, stream);
}

int ov_overlap_apply(ov_ctx* ctx, double m_q, const void* b, void* out, int nrhs, const ov_solve_opts* opts,
                     ov_stats* stats, void* stream) {
  NvtxRange nvtx_("ov_overlap_apply");
  return sign_or_overlap(ctx, true, m_q, b, out, nrhs, opts, stats, stream);
}

}  // extern "C"

namespace {

__global__ void axpy_c_kernel(double2* __restrict__ y, const double2* __restrict__ x, double2 c, size_t n) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const double2 v = x[t];
    double2 w = y[t];
    w.x += c.x * v.x - c.y * v.y;
    w.y += c.x * v.y + c.y * v.x;
    y[t] = w;
  }
}

__global__ void scale_kernel(double* __restrict__ p, double a, size_t n) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    p[t] *= a;
}

// Shared core of the two VJP entry points.  eta_s is the adjoint source of the sign
// function (eta, or gamma5 eta for the overlap operator); grad_b = a eta + gsc S_N^dag eta_s;
// force = fsc * dRe<eta_s, S_N b>/d omega.
int vjp_core(ov_ctx* ctx, double a_eta, double gsc, double fsc, bool gamma5_eta, const void* eta, const void* b,
             void* grad_b, double* grad_links, const ov_solve_opts* opts, ov_stats* stats, void* stream) {
  NvtxRange nvtx_("vjp_core");
  const double t0 = now_ms();
  if (!ctx) return OV_ERR_INVALID_ARG;
  if (!ctx->have_gauge) return ctx_fail(ctx, OV_ERR_NO_GAUGE, "ov_set_gauge has not been called");
  if (!ctx->have_contour) return ctx_fail(ctx, OV_ERR_NO_CONTOUR, "no contour set");
  if (!eta || !b) return ctx_fail(ctx, OV_ERR_INVALID_ARG, "null eta or b");
  ov_solve_opts o = resolve_opts(opts);
  int st = check_opts(ctx, o);
  if (st != OV_OK) return st;
  if (!grad_b && !grad_links) return OV_OK;
  DeviceGuard dg(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const int V = ctx->g.V;
  const size_t n12 = (size_t)12 * V;
  const int nq = (int)ctx->z.size();
  const int chunk = std::max(1, (o.node_chunk > 0 && o.node_chunk < nq) ? o.node_chunk : nq);
  const double2* etad = stage_in(ctx, eta, sizeof(double2) * n12, o.host_io, "vjp.eta", s, &st);
  const double2* bd = stage_in(ctx, b, sizeof(double2) * n12, o.host_io, "vjp.b", s, &st);
  double2* src2 = (double2*)ws_get(ctx, "vjp.src", sizeof(double2) * 2 * n12, &st);  // [b; eta_s] SoA
  double2* gb = (double2*)ws_get(ctx, "vjp.gb", sizeof(double2) * n12, &st);
  double2* gbo = (double2*)ws_get(ctx, "vjp.gbo", sizeof(double2) * n12, &st);
  double2* sums = (double2*)ws_get(ctx, "vjp.sums", sizeof(double2) * 2 * n12, &st);
  double2* X = (double2*)ws_get(ctx, "vjp.X", sizeof(double2) * 2 * n12 * chunk, &st);
  double* F = (double*)ws_get(ctx, "vjp.F", sizeof(double) * 4 * 8 * (size_t)V, &st);
  double2* cq = (double2*)ws_get(ctx, "vjp.c", sizeof(double2) * chunk, &st);
  double2* etag = (double2*)ws_get(ctx, "vjp.eta5", sizeof(double2) * n12, &st);
  if (st != OV_OK) return st;
  // sources in structure of arrays: b, and eta (or gamma5 eta)
  if ((st = launch_pack64(ctx, bd, src2, 1, s))) return st;
  const double2* es = etad;
  if (gamma5_eta) {
    if ((st = launch_gamma5_aos(ctx, etad, etag, 1, s))) return st;
    es = etag;
  }
  if ((st = launch_pack64(ctx, es, src2 + n12, 1, s))) return st;
  // grad_b starts as a_eta * eta (SoA) + gsc * conj(c0) eta_s
  double2* eta_soa = gb;  // reuse: pack eta into gb then scale
  if ((st = launch_pack64(ctx, etad, eta_soa, 1, s))) return st;
  scale_kernel<<<512, 256, 0, s>>>((double*)gb, a_eta, 2 * n12);
  axpy_c_kernel<<<512, 256, 0, s>>>(gb, src2 + n12, make_double2(gsc * ctx->c0.x, -gsc * ctx->c0.y), n12);
  cudaMemsetAsync(F, 0, sizeof(double) * 32 * (size_t)V, s);
  SolveOut tot;
  tot.converged = 1;
  // Coefficient-space forms: one stored-basis Lanczos pass for both sources, per-node
  // solutions formed from the basis chunk by chunk (no repeated solves).  Falls back to the
  // vector-space form when the basis does not fit.
  bool coef_done = nq == 0;  // no nodes: grad_b = a eta + gsc conj(c0) eta_s, no force
  if (!coef_done && (o.mode == OV_MODE_FP64_2PASS || o.mode == OV_MODE_FP64_REGEN || o.mode == OV_MODE_F32X2)) {
    std::vector<double2> zh(2 * (size_t)nq), ch(2 * (size_t)nq);
    for (int j = 0; j < nq; ++j) {
      const double2 z = ctx->z[j], c = ctx->c[j];
      zh[j] = z;
      ch[j] = c;
      zh[nq + j] = make_double2(z.x, -z.y);
      ch[nq + j] = make_double2(c.x, -c.y);
    }
    auto force_chunk = [&](int j0, int nc) -> int {
      if (!grad_links) return OV_OK;
      cudaError_t e = cudaMemcpyAsync(cq, ctx->c.data() + j0, sizeof(double2) * nc, cudaMemcpyHostToDevice, s);
      if (e != cudaSuccess) return ctx_cuda(ctx, e, "copy coefficients");
      return launch_force(ctx, X, nc, cq, F, s);
    };
    SolveOut so;
    st = solve_nodes_coef(ctx, src2, 2, nq, zh, ch, chunk, X, sums, o, &so, s, force_chunk);
    if (st == OV_OK || st == OV_ERR_NOT_CONVERGED) {
      coef_done = true;
      tot = so;
      axpy_c_kernel<<<512, 256, 0, s>>>(gb, sums + n12, make_double2(gsc, 0.0), n12);
    } else if (st != OV_ERR_INVALID_ARG) {
      return st;
    }
  }
  for (int j0 = 0; j0 < nq && !coef_done; j0 += chunk) {
    const int nc = std::min(chunk, nq - j0);
    // source 0 (b): nodes z_j; source 1 (eta_s): nodes conj(z_j), coefficients conj(c_j)
    std::vector<double2> zh(2 * (size_t)nc), ch(2 * (size_t)nc), cj(nc);
    for (int j = 0; j < nc; ++j) {
      const double2 z = ctx->z[j0 + j], c = ctx->c[j0 + j];
      zh[j] = z;
      ch[j] = c;
      zh[nc + j] = make_double2(z.x, -z.y);
      ch[nc + j] = make_double2(c.x, -c.y);
      cj[j] = c;
    }
    SolveOut so;
    st = o.mode == OV_MODE_F32X2 ? solve_nodes_soa_df(ctx, src2, 2, nc, zh, ch, make_double2(0, 0), sums, X, o, &so, s)
                                 : solve_nodes_soa(ctx, src2, 2, nc, zh, ch, make_double2(0, 0), sums, X, o, &so, s);
    if (st != OV_OK && st != OV_ERR_NOT_CONVERGED) return st;
    if (st == OV_ERR_NOT_CONVERGED) tot.converged = 0;
    tot.iterations += so.iterations;
    tot.max_residual = std::max(tot.max_residual, so.max_residual);
    tot.error_bound += so.error_bound;
    tot.node_updates += so.node_updates;
    tot.launches += so.launches;
    // grad_b += gsc * sum_j conj(c_j) xi_j (the second source's weighted sum)
    axpy_c_kernel<<<512, 256, 0, s>>>(gb, sums + n12, make_double2(gsc, 0.0), n12);
    if (grad_links) {
      cudaError_t e = cudaMemcpyAsync(cq, cj.data(), sizeof(double2) * nc, cudaMemcpyHostToDevice, s);
      if (e != cudaSuccess) return ctx_cuda(ctx, e, "copy coefficients");
      if ((st = launch_force(ctx, X, nc, cq, F, s))) return st;
    }
  }
  if (fsc != 1.0) scale_kernel<<<512, 256, 0, s>>>(F, fsc, 32 * (size_t)V);
  OV_CHECK_LAUNCH(ctx, "vjp kernels");
  cudaError_t e = cudaSuccess;
  if (grad_b) {
    double2* dst = o.host_io ? gbo : (double2*)grad_b;
    if ((st = launch_unpack64(ctx, gb, dst, 1, s))) return st;
    if (o.host_io && (st = stage_out(ctx, grad_b, gbo, sizeof(double2) * n12, s)) != OV_OK) return st;
  }
  if (grad_links) {
    if (o.host_io) {
      if ((st = stage_out(ctx, grad_links, F, sizeof(double) * 32 * (size_t)V, s)) != OV_OK) return st;
    } else {
      e = cudaMemcpyAsync(grad_links, F, sizeof(double) * 32 * (size_t)V, cudaMemcpyDeviceToDevice, s);
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return ctx_cuda(ctx, e, "VJP outputs");
  kt_collect(ctx);
  fill_stats(stats, tot, now_ms() - t0);
  if (!tot.converged) return ctx_fail(ctx, OV_ERR_NOT_CONVERGED, "VJP solves hit the iteration limit");
  return OV_OK;
}

}  // namespace

extern "C" {

int ov_sgn_vjp(ov_ctx* ctx, const void* eta, const void* b, void* grad_b, double* grad_links,
               const ov_solve_opts* opts, ov_stats* stats, void* stream) {
  return vjp_core(ctx, 0.0, 1.0, 1.0, false, eta, b, grad_b, grad_links, opts, stats, stream);
}

int ov_overlap_vjp(ov_ctx* ctx, double m_q, const void* eta, const void* b, void* grad_b, double* grad_links,
                   const ov_solve_opts* opts, ov_stats* stats, void* stream) {
  if (!std::isfinite(m_q)) return ctx_fail(ctx, OV_ERR_INVALID_ARG, "m_q is not finite");
  // L = Re<eta, (1+m)/2 b> + (1-m)/2 Re<gamma5 eta, S_N b>
  return vjp_core(ctx, 0.5 * (1.0 + m_q), 0.5 * (1.0 - m_q), 0.5 * (1.0 - m_q), true, eta, b, grad_b, grad_links,
                  opts, stats, stream);
}

int ov_set_hw32_variant(ov_ctx* ctx, int k) {
  if (!ctx) return OV_ERR_INVALID_ARG;
  if (k < -1 || k >= hw32_variant_count() + kNFloat4Variants) return ctx_fail(ctx, OV_ERR_INVALID_ARG, "no such FP32 stencil variant");
  ctx->hw32_force = k;
  return OV_OK;
}

int ov_hw32_variants(int k, int* rhs_tile, int* compressed, int* threads) {
  const int n = hw32_variant_count();
  if (k >= 0 && k < n && rhs_tile && compressed && threads) hw32_variant_info(k, rhs_tile, compressed, threads);
  if (k >= n && k < n + kNFloat4Variants && rhs_tile && compressed && threads) {
    const Float4Variant& f = kFloat4Variants[k - n];
    *rhs_tile = f.rhs_tile;
    *compressed = f.code;
    *threads = f.threads;
  }
  return n + kNFloat4Variants;
}

int ov_set_concurrency(ov_ctx* ctx, int groups) {
  if (!ctx) return OV_ERR_INVALID_ARG;
  if (groups < 0 || groups > 64) return ctx_fail(ctx, OV_ERR_INVALID_ARG, "groups must be in [0, 64]");
  ctx->groups = groups;
  return OV_OK;
}

int ov_set_persistent(ov_ctx* ctx, int enable) {
  if (!ctx) return OV_ERR_INVALID_ARG;
  ctx->no_coop = (enable == 0);
  return OV_OK;
}

int ov_set_kernel_timing(ov_ctx* ctx, int enable) {
  if (!ctx) return OV_ERR_INVALID_ARG;
  kt_collect(ctx);
  ctx->timing = enable != 0;
  for (auto& c : ctx->clocks) c = KernelClock{};
  return OV_OK;
}

int ov_kernel_times(ov_ctx* ctx, const char** names, long long* launches, double* total_ms, int cap) {
  if (!ctx) return OV_ERR_INVALID_ARG;
  kt_collect(ctx);
  for (int k = 0; k < KC_COUNT && k < cap; ++k) {
    if (names) names[k] = kKernelClassNames[k];
    if (launches) launches[k] = ctx->clocks[k].launches;
    if (total_ms) total_ms[k] = ctx->clocks[k].total_ms;
  }
  return KC_COUNT;
}

}  // extern "C"
