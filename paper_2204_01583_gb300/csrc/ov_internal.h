// Internal declarations of the overlap library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <functional>
#include <map>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "ov.h"

// Names the calls and phases of the library for a profiler's timeline (an NVTX range;
// header-only, and without a tool attached a push and a pop cost a function call each).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// ---------------------------------------------------------------- geometry

struct Geom {
  int L[4];    // Lx, Ly, Lz, Lt
  int st[4];   // site strides: 1, Lx, Lx*Ly, Lx*Ly*Lz
  int V;       // sites
  int bc_t;    // +1 / -1
};

// ---------------------------------------------------------------- workspace

// A device buffer that grows on demand and is reused across calls.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

// Per-kernel-class event timing (ov_set_kernel_timing).
struct KernelClock {
  long long launches = 0;
  double total_ms = 0.0;
};

struct PendingEvent {
  int cls;
  cudaEvent_t a, b;
};

enum KernelClass {
  KC_DSLASH = 0,     // H_W apply (plain)
  KC_LANCZOS_HW,     // dslash + Lanczos epilogue inside the solves
  KC_SHIFT_UPDATE,   // Lanczos vector update + per-node direction updates + weighted sum
  KC_LAYOUT,         // pack / unpack / epilogues
  KC_MISC,           // initialisation and small kernels
  KC_FORCE,          // link force
  KC_RESIDUAL,       // FP64 true residuals (mixed mode)
  KC_REGEN,          // regeneration pass of the two-pass mode
  KC_COOP,           // persistent cooperative Lanczos loop
  KC_BASIS_SUM,      // s = c0 b + sum_i g_i v_i from a stored basis
  KC_COUNT
};

extern const char* const kKernelClassNames[KC_COUNT];

// Graph cache entry for the per-iteration kernels of a solve: every pointer the
// captured launches read, plus the launch shape.
// Identity of a captured graph: the workspace pointers and every size that enters the
// captured kernel arguments (per-source offsets of grouped branches depend on the slot
// count and the history length).
struct GraphKey {
  const void* ptr[4];
  int nsrc, nshift, flavour, chunk;
  int nslots = 0, hist_len = 0;
  bool operator<(const GraphKey& o) const {
    for (int k = 0; k < 4; ++k)
      if (ptr[k] != o.ptr[k]) return ptr[k] < o.ptr[k];
    if (nsrc != o.nsrc) return nsrc < o.nsrc;
    if (nshift != o.nshift) return nshift < o.nshift;
    if (flavour != o.flavour) return flavour < o.flavour;
    if (chunk != o.chunk) return chunk < o.chunk;
    if (nslots != o.nslots) return nslots < o.nslots;
    return hist_len < o.hist_len;
  }
};

struct ov_ctx {
  int device = 0;
  Geom g{};
  double m0 = 0.0, r = 1.0;

  // gauge field, structure of arrays: element (mu, i, j, site) at [(mu*9 + 3i + j) * V + site]
  double2* U64 = nullptr;
  double2* U64h = nullptr;  // -1/2 U: the FP64 solver stencils take the hop factor from the links
  float2* U32 = nullptr;
  bool have_gauge = false;
  bool have_c32 = false;               // compressed FP32 links (workspace "gauge.c32") are current
  bool have_s4 = false;                // FP32 links for the spin-paired float4 layout
  float4* Udf = nullptr;               // double-float links (workspace "gauge.df") when have_df
  bool have_df = false;
  std::map<int, int> hw32_choice;      // nrhs -> autotuned FP32 stencil variant
  int hw32_force = -1;                 // ov_set_hw32_variant
  bool no_coop = true;                 // ov_set_persistent(ctx, 1) enables the persistent loop
  int groups = 0;                      // ov_set_concurrency: source groups per graph (0 = auto)
  int coef_iter_hint = 0;              // Krylov iterations of the last converged coefficient-space
                                       // solve (sizes the stored basis); reset with gauge or contour

  // quadrature S_N = c0 + sum_j c_j (z_j - H)^-1
  std::vector<double2> z, c;
  double2 c0{0.0, 0.0};
  bool have_contour = false;

  // named device workspace
  std::map<std::string, DevBuf> bufs;
  int* host_flag = nullptr;  // pinned host word for convergence reads
  cudaStream_t cap_stream = nullptr;
  std::vector<cudaStream_t> aux_streams;  // extra capture branches (source groups)
  std::vector<cudaEvent_t> cap_events;    // fork/join events of those branches
  std::map<GraphKey, cudaGraphExec_t> graphs;

  // kernel timing
  bool timing = false;
  KernelClock clocks[KC_COUNT];
  std::vector<PendingEvent> pending;
  std::vector<cudaEvent_t> event_pool;

  std::string err = "no error";
};

// ------------------------------------------------------------------ helpers

int ctx_fail(ov_ctx* ctx, int code, const std::string& msg);
int ctx_cuda(ov_ctx* ctx, cudaError_t e, const char* what);
void* ws_get(ov_ctx* ctx, const char* name, size_t bytes, int* status);
void ws_release_all(ov_ctx* ctx);
void graphs_release(ov_ctx* ctx);

// Kernel timing: bracket a launch with events when ctx->timing is set.
void kt_begin(ov_ctx* ctx, int cls, cudaStream_t s, cudaEvent_t* a);
void kt_end(ov_ctx* ctx, int cls, cudaStream_t s, cudaEvent_t a);
void kt_collect(ov_ctx* ctx);

#define OV_CHECK_LAUNCH(ctx, what)                                  \
  do {                                                              \
    cudaError_t e_ = cudaGetLastError();                            \
    if (e_ != cudaSuccess) return ctx_cuda((ctx), e_, (what));      \
  } while (0)

// ----------------------------------------------------------- launchers

// layout conversions (dslash.cu)
int launch_gauge_ingest(ov_ctx* ctx, const double2* U_aos, cudaStream_t s);
int launch_pack64(ov_ctx* ctx, const double2* aos, double2* soa, int nrhs, cudaStream_t s);
int launch_unpack64(ov_ctx* ctx, const double2* soa, double2* aos, int nrhs, cudaStream_t s);
int launch_pack32(ov_ctx* ctx, const float2* aos, float2* soa, int nrhs, cudaStream_t s);
int launch_unpack32(ov_ctx* ctx, const float2* soa, float2* aos, int nrhs, cudaStream_t s);
// out (SoA) = H_W in (SoA)
int launch_hw64(ov_ctx* ctx, const double2* in, double2* out, int nrhs, cudaStream_t s);
int launch_hw32(ov_ctx* ctx, const float2* in, float2* out, int nrhs, cudaStream_t s);
// FP32 multi-RHS stencil (dslash32.cu): variant -1 = autotuned
int launch_hw32_tuned(ov_ctx* ctx, const float2* in, float2* out, int nrhs, cudaStream_t s, int force_variant,
                      int* used);
int hw32_variant_count();  // SoA variants; index hw32_variant_count() is the paired kernel
void hw32_variant_info(int k, int* rt, int* comp, int* nt);
float hw32_time_soa_variants(ov_ctx* ctx, const float2* in, float2* out, int nrhs, cudaStream_t s, int* best);
// double-float links for the FP32-pair solve (dslash.cu)
int ensure_links_df(ov_ctx* ctx, cudaStream_t s);
// spin-paired float4 FP32 layout (dslash32.cu)
int launch_pack_s4(ov_ctx* ctx, const float2* aos, float4* s4, int nrhs, cudaStream_t s);
int launch_unpack_s4(ov_ctx* ctx, const float4* s4, float2* aos, int nrhs, cudaStream_t s);
int launch_hw32_s4(ov_ctx* ctx, const float4* in, float4* out, int nrhs, cudaStream_t s);
// paired FP32 layout (pair32.cu)
int launch_pack_pair32(ov_ctx* ctx, const float2* aos, float4* pr, int nrhs, cudaStream_t s);
int launch_unpack_pair32(ov_ctx* ctx, const float4* pr, float2* aos, int nrhs, cudaStream_t s);
int launch_hw_pair12(ov_ctx* ctx, const float4* in, float4* out, int npair, int form, cudaStream_t s);
const float4* s4_links(ov_ctx* ctx, cudaStream_t s, int* st);
// out(AoS) = (1+m)/2 b(AoS) + (1-m)/2 gamma5 s(SoA)
int launch_overlap_epilogue(ov_ctx* ctx, const double2* b_aos, const double2* s_soa, double2* out_aos,
                            double m_q, int nrhs, cudaStream_t s);
// gamma5 on an AoS spinor set (in place allowed)
int launch_gamma5_aos(ov_ctx* ctx, const double2* in, double2* out, int nrhs, cudaStream_t s);

// solves (solver.cu): out_soa = S_N b_soa for nrhs sources, contour from ctx
struct SolveOut {
  int iterations = 0;
  int converged = 0;
  double max_residual = 0.0;
  double error_bound = 0.0;
  int refine_rounds = 0;
  int inner_iterations = 0;
  double node_updates = 0.0;
  double launches = 0.0;
};
// Makes ctx's device current for the scope of an entry point.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// Helpers of the entry points (api.cu): defaults for null options, option checks, a
// host clock, staging of host input (host_io), the sign function of canonical device
// sources into a structure-of-arrays workspace, and the stats copy.
ov_solve_opts resolve_opts(const ov_solve_opts* o);
int check_opts(ov_ctx* ctx, const ov_solve_opts& o);
double now_ms();
const double2* stage_in(ov_ctx* ctx, const void* p, size_t bytes, int host_io, const char* name, cudaStream_t s,
                        int* st);
int stage_out(ov_ctx* ctx, void* host, const void* dev, size_t bytes, cudaStream_t s);
int sign_core(ov_ctx* ctx, const double2* b_dev, int nrhs, const ov_solve_opts& o, SolveOut* so, cudaStream_t s,
              double2** s_soa_out, double2* xs);
void fill_stats(ov_stats* st, const SolveOut& so, double ms);

int solve_sign_soa(ov_ctx* ctx, const double2* b_soa, double2* out_soa, int nrhs,
                   const ov_solve_opts& o, SolveOut* so, cudaStream_t s,
                   double2* xs_soa /* optional per-node solutions [src][node][12V] */);

int solve_nodes_soa(ov_ctx* ctx, const double2* b_soa, int nsrc, int ns, const std::vector<double2>& zh,
                    const std::vector<double2>& ch, double2 c0, double2* out_soa, double2* xs_soa,
                    const ov_solve_opts& o, SolveOut* so, cudaStream_t s);
// Per-node solutions X[src][node][12V] (FP64) of explicit per-source node lists through a
// stored Lanczos basis (FP64, or double-float for OV_MODE_F32X2), chunk nodes at a time
// (per_chunk(j0, nc) runs after each chunk), and the weighted sums sum_j c_j x_j into
// sums[src][12V].  OV_ERR_INVALID_ARG: the basis does not fit (use solve_nodes_soa).
int solve_nodes_coef(ov_ctx* ctx, const double2* b_soa, int nsrc, int ns, const std::vector<double2>& zh,
                     const std::vector<double2>& ch, int chunk, double2* X, double2* sums, const ov_solve_opts& o,
                     SolveOut* so, cudaStream_t s, const std::function<int(int, int)>& per_chunk);
// The same with double-float vectors (OV_MODE_F32X2); xs_soa receives FP64 copies.
int solve_nodes_soa_df(ov_ctx* ctx, const double2* b_soa, int nsrc, int ns, const std::vector<double2>& zh,
                    const std::vector<double2>& ch, double2 c0, double2* out_soa, double2* xs_soa,
                    const ov_solve_opts& o, SolveOut* so, cudaStream_t s);

// coefficient-space Lanczos (OV_MODE_FP64_2PASS / _REGEN in FP64, OV_MODE_F32X2 in
// double-float arithmetic)
int solve_sign_2pass(ov_ctx* ctx, const double2* b_soa, double2* out_soa, int nrhs, const ov_solve_opts& o,
                     SolveOut* so, cudaStream_t s);

// mixed-precision variant (OV_MODE_MIXED) and its kernels (mixed.cu)
int solve_sign_mixed(ov_ctx* ctx, const double2* b_soa, double2* out_soa, int nrhs, const ov_solve_opts& o,
                     SolveOut* so, cudaStream_t s);
int launch_basis_combine(ov_ctx* ctx, const float2* basis, int nslots, const float2* W, int kmax, const int* kr,
                         double2* Y, int nsrc, int nq, cudaStream_t s);
int launch_residual64(ov_ctx* ctx, const double2* Y, const double2* b, const double2* z, double2* R, double* part,
                      double* rnorm2, int nsrc, int nq, cudaStream_t s);
int residual64_partials(ov_ctx* ctx);
int launch_accumulate(ov_ctx* ctx, double2* Y, const float2* X, size_t n, cudaStream_t s);
int launch_weighted_sum(ov_ctx* ctx, const double2* Y, const double2* b, const double2* c, double2 c0, double2* out,
                        int nsrc, int nq, cudaStream_t s);

// Lanczos on H (or H^2) for spectral bounds (solver.cu); fills alpha[0..k), beta[0..k)
int lanczos_tridiag(ov_ctx* ctx, int steps, int squared, std::vector<double>& alpha,
                    std::vector<double>& beta, cudaStream_t s);

// force (force.cu): F[mu][site][8] += force from X = [forward y_j (nq); adjoint xi_j (nq)] (SoA)
int launch_force(ov_ctx* ctx, const double2* X, int nq, const double2* cq, double* F, cudaStream_t s);

// host-side contour math (contour.cpp)
void ellipse_rule(int n_q, double gamma, double rho, double alpha, int form, std::vector<double2>& z,
                  std::vector<double2>& c, double2& c0);
int zolotarev_rule(int n, double lmin, double lmax, std::vector<double2>& z, std::vector<double2>& c, double2& c0,
                   double* delta);
double rational_value(double lam, const std::vector<double2>& z, const std::vector<double2>& c,
                      double2 c0);
void tridiag_extreme_eigs(const std::vector<double>& a, const std::vector<double>& b, double* lo,
                          double* hi, double* lo_resid, double* hi_resid);
