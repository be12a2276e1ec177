// ov_apply_HW_noalloc: H_W applied without any device allocation.
//
// Some callers cannot call cudaMalloc: a lattice code that hands all of HBM to
// its own memory pool up front, or a process whose device memory is managed by a
// framework allocator it must not bypass (a cudaMalloc behind its back can fail, or
// take memory the allocator has promised elsewhere).  This entry point needs no context (creating one and
// loading a gauge field allocate) and no workspace: its staging buffers -- the
// structure-of-arrays copies of the gauge field and of the input and output
// spinors that the stencil kernel reads -- live in one fixed device array
// declared at file scope below.  Every GPU that loads the library holds that
// array (kNoAllocScratchBytes) until the process exits.
#include <cmath>
#include <mutex>

#include "common.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;  // 16 MiB
constexpr int kMaxDevices = 64;
constexpr int kNT = 128;

}  // namespace

// The scratch.  Host code must not pass this name to a kernel: on the host it is a
// stand-in symbol, not a device address.  Its device address comes from
// cudaGetSymbolAddress, once per device (see scratch_for_current_device).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device, looked up on the first call
// for that device (with that device current) and cached for the life of the process.
// A cudaDeviceReset rebuilds the device's context and invalidates the cached address:
// the entry point must not be used on a device after it has been reset.
// `before` is the error state the caller left pending: a failure here clears only an
// error of its own.
int scratch_for_current_device(void** out, cudaError_t before) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    if (before == cudaSuccess) cudaGetLastError();
    return OV_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      if (before == cudaSuccess) cudaGetLastError();
      return OV_ERR_CUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return OV_OK;
}

__global__ void na_gauge_pack(const double2* __restrict__ aos, double2* __restrict__ soa, int V) {
  const size_t n = (size_t)4 * V * 9;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const size_t e = t % 9, q = t / 9;
    const size_t site = q % V, mu = q / V;
    soa[(mu * 9 + e) * V + site] = aos[t];
  }
}

__global__ void na_spinor_pack(const double2* __restrict__ aos, double2* __restrict__ soa, int V, int nrhs) {
  const size_t n = (size_t)nrhs * V * 12;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const size_t k = t % 12, q = t / 12;
    const size_t site = q % V, r = q / V;
    soa[(r * 12 + k) * V + site] = aos[t];
  }
}

__global__ void na_spinor_unpack(const double2* __restrict__ soa, double2* __restrict__ aos, int V, int nrhs) {
  const size_t n = (size_t)nrhs * V * 12;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const size_t k = t % 12, q = t / 12;
    const size_t site = q % V, r = q / V;
    aos[t] = soa[(r * 12 + k) * V + site];
  }
}

__global__ void __launch_bounds__(kNT) na_hw(const double2* __restrict__ in, double2* __restrict__ out,
                                              const double2* __restrict__ U, Geom g, double diag) {
  const int s = blockIdx.x * kNT + threadIdx.x;
  if (s >= g.V) return;
  const size_t off = (size_t)blockIdx.y * 12 * g.V;
  Cx<double> o[12];
  hw_site<double>(in + off, U, g, s, diag, o);
#pragma unroll
  for (int k = 0; k < 12; ++k) st<double>(out + off + k * (size_t)g.V + s, o[k]);
}

int grid_cap(size_t n) {
  size_t b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return (int)(b > 0 ? b : 1);
}

size_t round256(size_t x) { return (x + 255) & ~size_t(255); }

// One launch, its own status (cudaLaunchKernel returns the error of this launch only).
template <typename... A>
cudaError_t launch(void (*k)(A...), dim3 grid, dim3 block, cudaStream_t s, A... args) {
  void* p[] = {(void*)&args...};
  return cudaLaunchKernel((const void*)k, grid, block, p, 0, s);
}

}  // namespace

extern "C" int ov_apply_HW_noalloc(const int dims[4], int bc_t, double m0, const double* U, const void* in,
                                   void* out, int nrhs, void* stream) {
  if (!dims || !U || !in || !out || in == out || nrhs < 1) return OV_ERR_INVALID_ARG;
  if (bc_t != 1 && bc_t != -1) return OV_ERR_INVALID_ARG;
  if (!std::isfinite(m0)) return OV_ERR_INVALID_ARG;
  // V built one factor at a time, so that no product overflows before the size check
  long long V = 1;
  for (int k = 0; k < 4; ++k) {
    if (dims[k] < 1) return OV_ERR_INVALID_ARG;
    V *= dims[k];
    if (V > (1LL << 28)) return OV_ERR_SCRATCH_TOO_SMALL;
  }
  const size_t gauge_bytes = round256(sizeof(double2) * 4 * 9 * (size_t)V);
  if (gauge_bytes > kNoAllocScratchBytes) return OV_ERR_SCRATCH_TOO_SMALL;
  const size_t per_rhs = sizeof(double2) * 12 * (size_t)V;
  if ((size_t)nrhs > (kNoAllocScratchBytes - gauge_bytes) / (2 * per_rhs)) return OV_ERR_SCRATCH_TOO_SMALL;
  const size_t spinor_bytes = round256(per_rhs * (size_t)nrhs);
  if (gauge_bytes + 2 * spinor_bytes > kNoAllocScratchBytes) return OV_ERR_SCRATCH_TOO_SMALL;
  // An error the caller left pending (from its own earlier work) is neither cleared nor
  // reported as this call's: only the status of this call's own CUDA calls counts.
  const cudaError_t before = cudaPeekAtLastError();
  void* base = nullptr;
  int st = scratch_for_current_device(&base, before);
  if (st != OV_OK) return st;
  double2* U_soa = (double2*)base;
  double2* in_soa = (double2*)((unsigned char*)base + gauge_bytes);
  double2* out_soa = (double2*)((unsigned char*)base + gauge_bytes + spinor_bytes);
  Geom g;
  for (int k = 0; k < 4; ++k) g.L[k] = dims[k];
  g.st[0] = 1;
  g.st[1] = dims[0];
  g.st[2] = dims[0] * dims[1];
  g.st[3] = dims[0] * dims[1] * dims[2];
  g.V = (int)V;
  g.bc_t = bc_t;
  cudaStream_t s = (cudaStream_t)stream;
  // every byte of the scratch the stencil reads is written first in this call,
  // so nothing carried over from an earlier call is used
  cudaError_t e = launch(na_gauge_pack, dim3(grid_cap((size_t)4 * 9 * V)), dim3(256), s, (const double2*)U, U_soa,
                         g.V);
  if (e == cudaSuccess)
    e = launch(na_spinor_pack, dim3(grid_cap((size_t)12 * V * nrhs)), dim3(256), s, (const double2*)in, in_soa, g.V,
               nrhs);
  if (e == cudaSuccess)
    e = launch(na_hw, dim3((g.V + kNT - 1) / kNT, nrhs), dim3(kNT), s, (const double2*)in_soa, out_soa,
               (const double2*)U_soa, g, 4.0 - m0);
  if (e == cudaSuccess)
    e = launch(na_spinor_unpack, dim3(grid_cap((size_t)12 * V * nrhs)), dim3(256), s, (const double2*)out_soa,
               (double2*)out, g.V, nrhs);
  if (e != cudaSuccess) {
    if (before == cudaSuccess) cudaGetLastError();  // clear this call's own launch error
    return OV_ERR_CUDA;
  }
  return OV_OK;
}
