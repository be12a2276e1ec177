// Shifted Krylov solve for every quadrature node at once, and the weighted sum.
//
// The paper solves (z_j - H_W) y_j = b for all nodes with a shift solver seeded at
// z_seed (the shift-solver remark after Eq. 7; shifted BiCG in its numerical
// section).  For hermitian H_W, BiCG with shadow vector equal to the initial
// residual produces at step k, for every shift, the Galerkin iterate in the Krylov
// space K_k(H_W, b): y_{k,j} = V_k (z_j - T_k)^-1 e_1 ||b||, where H_W V_k = V_k T_k +
// beta_k v_{k+1} e_k^T is the hermitian Lanczos relation with real tridiagonal T_k
// (alpha_i on the diagonal, beta_i off it).  These iterates do not depend on the seed.
// We compute exactly them:
//
//   * one Lanczos process on H_W per source (kernels K1, K2 below);
//   * for every node, the LDL^T factorisation of the complex-symmetric tridiagonal
//     z_j - T_k, updated one row per step:
//       d_1 = z - alpha_1,  d_i = z - alpha_i - beta_{i-1}^2 / d_{i-1},
//       l_i = -beta_i / d_i,  omega_1 = ||b||,  omega_i = -l_{i-1} omega_{i-1},
//       zeta_i = omega_i / d_i
//     (1 / d_i is kept, so each step costs one real division per node);
//     |Im d_i| >= |Im z| > 0, so no pivot ever vanishes (no breakdown);
//   * per node the direction p_i = v_i - l_{i-1} p_{i-1} and y += zeta_i p_i, so that
//     the weighted sum of Eq. 7, s = c0 b + sum_j c_j y_j, is accumulated directly;
//   * the FOM residual of node j after step i is beta_i |zeta_i| v_{i+1}, so its norm
//     is known from scalars; a node stops updating once it is below tol ||b||.
//
// Lanczos vectors are kept unnormalised, U_i = beta_{i-1} v_i (U_1 = b), in a ring
// of three buffers; each consumer scales by 1/||U_i||.  All recurrence scalars are
// FP64 and live on the device; the last block of each kernel (per source) reduces
// the block partials in a fixed order, so reruns are bit-identical, and updates the
// scalars.  The host only reads a done counter every few iterations, and replays
// the per-iteration kernels from a CUDA graph.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <string>
#include <cstring>
#include <functional>
#include <type_traits>
#include <vector>

#include <cooperative_groups.h>

#include "common.cuh"

namespace {

constexpr int NT1 = 128;  // K1: stencil + Lanczos epilogue; K3: regeneration pass
constexpr int NT2 = 256;  // K2: vector updates
// Resident blocks per SM the stencil kernels are compiled for: 4 (<= 128 registers) for
// FP64; 7 (<= 72 registers) for double-float (16^3x32, 12 sources, double-float solve:
// 467 / 421 / 457 ms at 6 / 7 / 8 blocks per SM -- at 8 the 64-register limit spills
// and the shared-memory partials leave L1 almost no room; with the link rows loaded one
// row ahead, 414 / 407.5 ms at 6 / 7).
template <typename R>
constexpr int k1_min_blocks() { return std::is_same<R, DF>::value ? 7 : 4; }
// FP64 and double-float solves read the link copy scaled by -1/2 (the hop factor of D_W) with the time
// boundary sign on the last time slice's time links, so phase 1 applies no boundary sign
// and phase 2 adds the partials to the diagonal term without a multiplication
template <typename R>
constexpr bool kHalvedLinks = std::is_same<R, double>::value || std::is_same<R, DF>::value;

struct SrcState {
  double bnorm;   // ||b||
  double inv_b2;  // 1 / ||b||^2
  double n_prev;  // ||U_{i-1}||
  double n_cur;   // ||U_i||
  double alpha;   // alpha_i
  int iter;       // i
  int done;
  int status;     // OV_OK, OV_ERR_NOT_CONVERGED, OV_ERR_BREAKDOWN
  int n_act;
  double node_updates;  // sum over iterations of n_act
  int k_final;    // second pass: number of Lanczos vectors to regenerate
  int pad_;
  // derived once per iteration by the block that updates the norms (not per thread):
  double inv_n;   // 1 / ||U_i||
  double cm;      // ||U_i|| / ||U_{i-1}|| (0 at i = 1)
  double alpha_n; // alpha_i / ||U_i||: U_{i+1} = w - alpha_n U_i in one FMA per real
  float df[8];    // inv_n, cm, alpha, alpha_n as double-float (hi, lo) pairs
};

// exact double-float split of an FP64 value: hi = rn(x), lo = rn(x - hi)
__device__ __forceinline__ void df_split(double x, float* d) {
  d[0] = __double2float_rn(x);
  d[1] = __double2float_rn(x - (double)d[0]);
}

// inv_n, cm and (double-float vectors only) their double-float forms from n_cur, n_prev
// and iter.  These run in one thread on the path between two launches, where every FP64
// instruction waits for the previous one (GB300's FP64 rate is 1/64 of FP32): the
// reciprocal is the correctly rounded one (the same value as 1.0 / n_cur), and the FP64
// solve skips the splits it does not read.
template <typename R>
__device__ __forceinline__ void set_norm_scalars(SrcState* S) {
  S->inv_n = __drcp_rn(S->n_cur);
  S->cm = (S->iter > 1) ? S->n_cur / S->n_prev : 0.0;
  if constexpr (std::is_same<R, DF>::value) {
    df_split(S->inv_n, S->df + 0);
    df_split(S->cm, S->df + 2);
  }
}

// An FP64 recurrence scalar in the vector arithmetic type; for double-float, from its
// stored split (no per-thread FP64 conversion).
template <typename R>
__device__ __forceinline__ R scal(double v, const float*) { return (R)v; }
template <>
__device__ __forceinline__ DF scal<DF>(double, const float* d) { return DF(d[0], d[1]); }

// Per-iteration scalars of the regeneration pass, in the vector arithmetic type.
template <typename R>
struct RegenRec {
  R inv_n, cm, alpha, alpha_n;
  Cx<R> g;
};

struct ShiftState {
  double2 invd, omega, zeta;  // 1 / d_i, omega_i, zeta_i of the LDL^T recurrence
  double res2;                // |beta_i zeta_i|^2 / ||b||^2 (squared relative FOM residual)
  int active;
  int last_iter;
};

struct SolveParams {
  double tol;
  int max_iter;
  int nshift;
  int vec_shifts;  // 1: per-node direction vectors and the weighted sum in K2; 0: scalars only
  int nslots;      // Lanczos vector slots per source: 3 (ring, slot i % 3) or a stored basis (slot i)
  int store;       // 1: slot i holds U_i for every i (basis kept for a later combination)
  // 1 (scalar-only forms): the per-node LDL^T rows and stopping tests run in
  // node_check_kernel every kNodeCheck iterations from the recorded alpha_i, beta_i,
  // not in the last blocks of K1 and K2 (which then only form alpha_i and beta_i)
  int defer_nodes;
};

// Iterations between per-node stopping checks of the scalar-only forms: a source runs at
// most kNodeCheck - 1 iterations past the one where its last node met tol.
constexpr int kNodeCheck = 8;

// Per-node coefficients l_{i-1}, c_j zeta_i, zeta_i of the vector-space update, stored
// per iteration by K1's last block: FP64 for FP64 and FP32 vectors (converted where
// used), double-float splits for double-float vectors (no per-element FP64 conversion).
template <typename R>
struct Coef {
  using T = double2;
  __device__ __forceinline__ static T make(double2 v) { return v; }
  __device__ __forceinline__ static Cx<R> get(const T* p) {
    const double2 v = __ldg(p);
    return {(R)v.x, (R)v.y};
  }
};
template <>
struct Coef<DF> {
  using T = float4;
  __device__ __forceinline__ static T make(double2 v) { return Store<DF>::pack(cx_from<DF>(v.x, v.y)); }
  __device__ __forceinline__ static Cx<DF> get(const T* p) { return Store<DF>::unpack(__ldg(p)); }
};

// Device pointers of one solve (all in workspace owned by the context).
template <typename R>
struct SolveArgs {
  using T = typename Store<R>::T;
  T* ring;            // [src][3][12V]
  T* p;               // [src][nshift][12V]
  T* x;               // [src][nshift][12V] or null
  double2* sacc;      // [src][12V] weighted sum (FP64) or null
  T* ssum;            // [src][12V] regeneration-pass sum in the vector type (double-float) or null
  const T* stencil;   // optional pre-applied H U_i for K1 ([src][12V]) or null
  SrcState* src;
  ShiftState* sh;     // [src][nshift]
  const double2* z;   // [src][nshift]
  const double2* c;   // [src][nshift]
  int* act_idx;       // [src][nshift]
  typename Coef<R>::T* act_l;   // [src][nshift] l_{i-1}
  typename Coef<R>::T* act_cz;  // [src][nshift] c_j zeta_i
  typename Coef<R>::T* act_z;   // [src][nshift] zeta_i
  double* part1;      // [src][nblk1]
  double* part2;      // [src][nblk2]
  unsigned* cnt;      // [src][2]
  int* done_count;
  double* hist_a;     // [src][max_iter] or null
  double* hist_b;
  const double2* gco; // [src][max_iter] second-pass coefficients or null
  const RegenRec<R>* rrec;  // [src][max_iter] regeneration-pass scalars or null
  const double* tol_src;  // [src] per-source tolerance or null (then SolveParams::tol)
  const SolveParams* prm;
  const T* U;         // links
  Geom g;
  R diag;
};

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Lanczos vector slot of iteration index i: a ring of three, or the stored basis.
__device__ __forceinline__ size_t lz_slot(const SolveParams* p, int i) {
  return p->store ? (size_t)i : (size_t)(i % 3);
}

// The Lanczos vector arithmetic, written with explicitly rounded operations so that
// every kernel that performs it (K1/K2 of the solve, K3 of the second pass) produces
// the same bits: the second pass of OV_MODE_FP64_2PASS regenerates the first pass's
// basis exactly.
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rfma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float rfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ DF rmul(DF a, DF b) { return a * b; }
__device__ __forceinline__ DF rfma(DF a, DF b, DF c) { return fma(a, b, c); }

// w = (H U_i) / n_i - (n_i / n_{i-1}) U_{i-1}   (second term absent at i = 1)
template <typename R>
__device__ __forceinline__ Cx<R> lz_w(Cx<R> o, Cx<R> um, R inv_n, R cm, bool first) {
  Cx<R> w = {rmul(inv_n, o.re), rmul(inv_n, o.im)};
  if (!first) {
    w.re = rfma(-cm, um.re, w.re);
    w.im = rfma(-cm, um.im, w.im);
  }
  return w;
}
// v_i = U_i / n_i
template <typename R>
__device__ __forceinline__ Cx<R> lz_v(Cx<R> u, R inv_n) {
  return {rmul(inv_n, u.re), rmul(inv_n, u.im)};
}
// U_{i+1} = w - alpha_i v_i = w - (alpha_i / ||U_i||) U_i, one FMA per real with the
// scalar alpha_n = alpha_i / ||U_i|| (the FP64 pipe bounds these kernels)
template <typename R>
__device__ __forceinline__ Cx<R> lz_next(Cx<R> w, Cx<R> u, R alpha_n) {
  return {rfma(-alpha_n, u.re, w.re), rfma(-alpha_n, u.im, w.im)};
}

// Per-thread partial of an inner product.  FP64 and FP32 vectors: an FP64 sum.
// Double-float vectors: a double-float sum (FP32 instructions only), converted to FP64
// once per thread -- per-element FP64 conversions would put the kernel on the FP64 pipe.
template <typename R>
struct Acc {
  using T = double;
  __device__ __forceinline__ static T zero() { return 0.0; }
  // FP64 vectors: two FMAs per complex (the FP64 pipe is the bound); FP32 vectors: the
  // products in FP64
  __device__ __forceinline__ static T dot(T acc, Cx<R> u, Cx<R> w) {
    if constexpr (std::is_same<R, double>::value) return fma(u.im, w.im, fma(u.re, w.re, acc));
    return acc + ((double)u.re * (double)w.re + (double)u.im * (double)w.im);
  }
  __device__ __forceinline__ static double get(T acc) { return acc; }
  template <int NT>
  __device__ __forceinline__ static double total(T acc, double* sh) { return block_sum<NT>(acc, sh); }
};
template <>
struct Acc<DF> {
  using T = DF;
  __device__ __forceinline__ static T zero() { return DF(0.f, 0.f); }
  // running sum unnormalised (renormalised by the block sum)
  __device__ __forceinline__ static T dot(T acc, Cx<DF> u, Cx<DF> w) {
    return fma_unnormalised(u.im, w.im, fma_unnormalised(u.re, w.re, acc));
  }
  __device__ __forceinline__ static double get(T acc) { return (double)acc; }
  // block sum in double-float (fixed tree), one FP64 conversion per block; sh >= NT/32 doubles
  template <int NT>
  __device__ __forceinline__ static double total(T v, double* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
      v = v + DF(__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o));
    DF* shd = reinterpret_cast<DF*>(sh);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) shd[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0) {
      DF u = shd[0];
#pragma unroll
      for (int k = 1; k < NT / 32; ++k) u = u + shd[k];
      t = (double)u;
    }
    __syncthreads();
    return t;  // valid in thread 0
  }
};

// s += g v in the regeneration pass.  FP64 and FP32 vectors: into the FP64 sum.
// Double-float vectors: into a double-float sum (a.ssum), folded into the FP64 sum
// after the last iteration.  The element is read and written by this thread only.
template <typename R>
struct SumAdd {
  __device__ __forceinline__ static void add(const SolveArgs<R>& a, size_t idx, Cx<R> g, Cx<R> v) {
    double2 sv = a.sacc[idx];
    sv.x += (double)g.re * (double)v.re - (double)g.im * (double)v.im;
    sv.y += (double)g.re * (double)v.im + (double)g.im * (double)v.re;
    a.sacc[idx] = sv;
  }
};
template <>
struct SumAdd<DF> {
  __device__ __forceinline__ static void add(const SolveArgs<DF>& a, size_t idx, Cx<DF> g, Cx<DF> v) {
    const Cx<DF> sv = Store<DF>::unpack(a.ssum[idx]);
    a.ssum[idx] = Store<DF>::pack(cfma(g, v, sv));
  }
};

__device__ void mark_done(SrcState* S, int* done_count, int status) {
  S->done = 1;
  S->status = status;
  atomicAdd(done_count, 1);
}

// Block-wide ordered compaction helper: returns this thread's slot among the
// threads with flag set (in thread order) and the block total in *total.
template <int NT>
__device__ __forceinline__ int block_rank(bool flag, int* total, int* wsh) {
  const unsigned bal = __ballot_sync(0xffffffffu, flag);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) wsh[wid] = __popc(bal);
  __syncthreads();
  int off = 0, tot = 0;
#pragma unroll
  for (int w = 0; w < NT / 32; ++w) {
    if (w < wid) off += wsh[w];
    tot += wsh[w];
  }
  __syncthreads();
  *total = tot;
  return off + __popc(bal & ((1u << lane) - 1u));
}

// K1: w = H U_i / n_i - (n_i / n_{i-1}) U_{i-1};  alpha_i = Re <U_i, w> / n_i; then,
// in the last block, row i of every active node's LDL^T and the active list for K2.
// The stencil runs 4 threads per site (hw_split_*): a block covers 32 sites.
// 4 blocks per SM (<= 128 registers): an 8^4 x 4-source grid (512 blocks) fits one wave
template <typename R>
__global__ void __launch_bounds__(NT1, k1_min_blocks<R>()) lanczos_hw_kernel(SolveArgs<R> a) {
  using T = typename Store<R>::T;
  __shared__ double sh[NT1 / 32];
  __shared__ int wsh[NT1 / 32];
  __shared__ bool last;
  __shared__ double alpha_sh;
  __shared__ Cx<R> sm[4 * 12 * kSplitSites];
  // one-dimensional grid, the sources of a site tile in consecutive blocks (k1_grid)
  const int nb = (a.g.V + kSplitSites - 1) / kSplitSites;  // site tiles per source
  const int nsl = gridDim.x / nb;                           // sources in this launch
  const int r = blockIdx.x % nsl, tb = blockIdx.x / nsl;
  SrcState* S = a.src + r;
  if (S->done) return;
  const int V = a.g.V;
  const size_t n12 = (size_t)12 * V;
  const int i = S->iter;
  T* base = a.ring + (size_t)r * a.prm->nslots * n12;
  const T* Ui = base + lz_slot(a.prm, i) * n12;
  const T* Um = base + (a.prm->store ? (size_t)(i - 1) : (size_t)((i + 2) % 3)) * n12;  // U_{i-1}
  T* W = base + lz_slot(a.prm, i + 1) * n12;
  const double inv_n = S->inv_n;
  const R inv_nR = scal<R>(inv_n, S->df + 0), cmR = scal<R>(S->cm, S->df + 2);
  const int site0 = tb * kSplitSites;
  typename Acc<R>::T dot = Acc<R>::zero();
  if (a.stencil) {
    // pre-applied operator (H^2 Lanczos for the spectral gap): one thread per (site, 3 components)
    const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5, s = site0 + lane;
    if (s < V) {
      const T* Hs = a.stencil + (size_t)r * n12;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const size_t e = (3 * grp + q) * (size_t)V + s;
        const Cx<R> u = ld<R>(Ui + e);
        const Cx<R> um = (i > 1) ? ld<R>(Um + e) : Cx<R>{R(0), R(0)};
        const Cx<R> w = lz_w<R>(ld<R>(Hs + e), um, inv_nR, cmR, i == 1);
        st<R>(W + e, w);
        dot = Acc<R>::dot(dot, u, w);
      }
    }
  } else {
    hw_split_phase1<R, false, !kHalvedLinks<R>>(Ui, a.U, a.g, site0, sm);
    __syncthreads();
    Cx<R> o[3];
    int s, k0;
    if (hw_split_phase2<R, false, kHalvedLinks<R>>(Ui, a.g, site0, a.diag, sm, o, &s, &k0)) {
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const size_t e = (k0 + q) * (size_t)V + s;
        const Cx<R> u = ld<R>(Ui + e);
        const Cx<R> um = (i > 1) ? ld<R>(Um + e) : Cx<R>{R(0), R(0)};
        const Cx<R> w = lz_w<R>(o[q], um, inv_nR, cmR, i == 1);
        st<R>(W + e, w);
        dot = Acc<R>::dot(dot, u, w);
      }
    }
  }
  double bs = Acc<R>::template total<NT1>(dot, sh);
  if (threadIdx.x == 0) {
    a.part1[(size_t)r * nb + tb] = bs;
    __threadfence();
    last = (atomicAdd(a.cnt + 2 * r, 1u) == (unsigned)nb - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  const double tot = sum_partials<NT1>(a.part1 + (size_t)r * nb, nb, sh);
  if (threadIdx.x == 0) {
    a.cnt[2 * r] = 0;
    const double alpha = tot * inv_n;
    S->alpha = alpha;
    S->alpha_n = alpha * inv_n;
    if constexpr (std::is_same<R, DF>::value) {
      df_split(alpha, S->df + 4);
      df_split(S->alpha_n, S->df + 6);
    }
    alpha_sh = alpha;
    if (a.hist_a) a.hist_a[(size_t)r * a.prm->max_iter + (i - 1)] = alpha;
    if (!isfinite(alpha)) {
      S->n_act = 0;
      mark_done(S, a.done_count, OV_ERR_BREAKDOWN);
    }
  }
  __syncthreads();
  const double alpha = alpha_sh;
  if (!isfinite(alpha) || a.prm->defer_nodes) return;
  // per-node LDL^T row i (one thread per node) and the ordered active list
  const int ns = a.prm->nshift;
  const double beta_prev = S->n_cur;  // beta_{i-1} = ||U_i|| (i >= 2)
  int na = 0;
  for (int j0 = 0; j0 < ns; j0 += NT1) {
    const int j = j0 + threadIdx.x;
    bool act = false;
    double2 lprev = make_double2(0.0, 0.0), zeta = make_double2(0.0, 0.0);
    if (j < ns) {
      ShiftState& q = a.sh[(size_t)r * ns + j];
      act = q.active != 0;
      if (act) {
        const double2 zj = a.z[(size_t)r * ns + j];
        double2 d, om;
        if (i == 1) {
          d = make_double2(zj.x - alpha, zj.y);
          om = make_double2(S->bnorm, 0.0);
        } else {
          const double2 ip = q.invd;  // 1 / d_{i-1}
          lprev = make_double2(-beta_prev * ip.x, -beta_prev * ip.y);
          const double b2 = beta_prev * beta_prev;
          d = make_double2(zj.x - alpha - b2 * ip.x, zj.y - b2 * ip.y);
          om = cmul(make_double2(-lprev.x, -lprev.y), q.omega);
        }
        const double inv = __drcp_rn(d.x * d.x + d.y * d.y);  // = 1.0 / |d|^2
        const double2 invd = make_double2(d.x * inv, -d.y * inv);
        zeta = cmul(om, invd);
        q.invd = invd;
        q.omega = om;
        q.zeta = zeta;
      }
    }
    int cnt;
    const int slot = block_rank<NT1>(act, &cnt, wsh);
    if (act) {
      const size_t o = (size_t)r * ns + na + slot;
      a.act_idx[o] = j;
      a.act_l[o] = Coef<R>::make(lprev);
      a.act_cz[o] = Coef<R>::make(cmul(a.c[(size_t)r * ns + j], zeta));
      a.act_z[o] = Coef<R>::make(zeta);
    }
    na += cnt;
  }
  if (threadIdx.x == 0) {
    S->n_act = na;
    S->node_updates += (a.prm->vec_shifts ? na : 0);
  }
}

// K2: U_{i+1} = w - alpha_i U_i / n_i (in place over w), beta_i = ||U_{i+1}||,
// per active node p = v_i - l_{i-1} p, x += zeta_i p, s += c_j zeta_i p (vec_shifts),
// then per-node residuals |beta_i zeta_i| and l_i = -beta_i / d_i in the last block.
template <typename R>
__global__ void __launch_bounds__(NT2) lanczos_update_kernel(SolveArgs<R> a) {
  using T = typename Store<R>::T;
  __shared__ double sh[NT2 / 32];
  __shared__ bool last;
  __shared__ double nrm2_sh;
  const int r = blockIdx.y;
  SrcState* S = a.src + r;
  if (S->done) return;
  const int V = a.g.V;
  const size_t n12 = (size_t)12 * V;
  const int i = S->iter;
  const int ns = a.prm->nshift;
  T* base = a.ring + (size_t)r * a.prm->nslots * n12;
  const T* Ui = base + lz_slot(a.prm, i) * n12;
  T* W = base + lz_slot(a.prm, i + 1) * n12;
  const int na = a.prm->vec_shifts ? S->n_act : 0;
  const R inv_nR = scal<R>(S->inv_n, S->df + 0), anR = scal<R>(S->alpha_n, S->df + 6);
  typename Acc<R>::T nrm = Acc<R>::zero();
  double nrm_im = 0.0;  // FP64 vectors: the imaginary parts in a second, independent FMA chain
  size_t e0 = (size_t)blockIdx.x * NT2 + threadIdx.x;
  const size_t gs = (size_t)gridDim.x * NT2;
  if constexpr (!std::is_same<R, float>::value) {
    // scalar-only forms (no per-node vectors): four elements per thread in flight, their
    // loads issued before any arithmetic (the arithmetic and HBM overlap across them)
    if (na == 0) {
      constexpr int B = 4;
      for (; e0 + (B - 1) * gs < n12; e0 += B * gs) {
        Cx<R> ub[B], wb[B];
#pragma unroll
        for (int k = 0; k < B; ++k) {
          ub[k] = ld<R>(Ui + e0 + k * gs);
          wb[k] = ld<R>(W + e0 + k * gs);
        }
#pragma unroll
        for (int k = 0; k < B; ++k) {
          const Cx<R> u = lz_next<R>(wb[k], ub[k], anR);
          st<R>(W + e0 + k * gs, u);
          if constexpr (std::is_same<R, double>::value) {
            nrm = fma(u.re, u.re, nrm);
            nrm_im = fma(u.im, u.im, nrm_im);
          } else {
            nrm = Acc<R>::dot(nrm, u, u);
          }
        }
      }
    }
  }
  // grid-stride: a few blocks per source (fewer partials and atomics than one block per chunk)
  for (size_t e = e0; e < n12; e += gs) {
    const Cx<R> ui = ld<R>(Ui + e);
    const Cx<R> u = lz_next<R>(ld<R>(W + e), ui, anR);
    st<R>(W + e, u);
    if constexpr (std::is_same<R, double>::value) {
      nrm = fma(u.re, u.re, nrm);
      nrm_im = fma(u.im, u.im, nrm_im);
    } else {
      nrm = Acc<R>::dot(nrm, u, u);
    }
    Cx<R> v = ui;  // v_i = U_i / ||U_i||, read only by the per-node direction updates
    if (na > 0) v = lz_v<R>(ui, inv_nR);
    double sre = 0.0, sim = 0.0;      // weighted sum over nodes: FP64 (FP64, FP32 vectors)
    Cx<R> sdf = {R(0), R(0)};          // or double-float (double-float vectors)
    const int* idx = a.act_idx + (size_t)r * ns;
    const typename Coef<R>::T* al = a.act_l + (size_t)r * ns;
    const typename Coef<R>::T* acz = a.act_cz + (size_t)r * ns;
    const typename Coef<R>::T* az = a.act_z + (size_t)r * ns;
    for (int k = 0; k < na; ++k) {
      const int j = __ldg(idx + k);
      T* P = a.p + ((size_t)r * ns + j) * n12 + e;
      Cx<R> pv = v;
      if (i > 1) pv = cfma(cneg(Coef<R>::get(al + k)), ld<R>(P), v);  // v - l p
      st<R>(P, pv);
      if constexpr (std::is_same<R, DF>::value) {
        sdf = cfma(Coef<R>::get(acz + k), pv, sdf);
      } else {
        const double2 cz = __ldg(acz + k);
        sre += cz.x * (double)pv.re - cz.y * (double)pv.im;
        sim += cz.x * (double)pv.im + cz.y * (double)pv.re;
      }
      if (a.x) {
        T* X = a.x + ((size_t)r * ns + j) * n12 + e;
        const Cx<R> xo = (i > 1) ? ld<R>(X) : Cx<R>{R(0), R(0)};
        st<R>(X, cfma(Coef<R>::get(az + k), pv, xo));
      }
    }
    if (a.sacc && na > 0) {
      if constexpr (std::is_same<R, DF>::value) {
        sre = (double)sdf.re;
        sim = (double)sdf.im;
      }
      double2* Sx = a.sacc + (size_t)r * n12 + e;
      double2 sv = *Sx;
      sv.x += sre;
      sv.y += sim;
      *Sx = sv;
    }
  }
  if constexpr (std::is_same<R, double>::value) nrm += nrm_im;
  double bs = Acc<R>::template total<NT2>(nrm, sh);
  if (threadIdx.x == 0) {
    a.part2[(size_t)r * gridDim.x + blockIdx.x] = bs;
    __threadfence();
    last = (atomicAdd(a.cnt + 2 * r + 1, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // ||u||^2 goes to every thread before the square root is taken: the node tests need
  // only beta^2, and sqrt sits on one thread's serial FP64 path
  const double tot = sum_partials<NT2>(a.part2 + (size_t)r * gridDim.x, gridDim.x, sh);
  if (threadIdx.x == 0) {
    a.cnt[2 * r + 1] = 0;
    nrm2_sh = tot;
    if (!isfinite(tot)) {
      if (a.hist_b) a.hist_b[(size_t)r * a.prm->max_iter + (i - 1)] = sqrt(tot);
      mark_done(S, a.done_count, OV_ERR_BREAKDOWN);
    }
  }
  __syncthreads();
  const double nrm2 = nrm2_sh;
  if (!isfinite(nrm2)) return;
  const double tol = a.tol_src ? a.tol_src[r] : a.prm->tol;
  const double tol2 = tol * tol;
  const double b2n = nrm2 * S->inv_b2;
  const bool defer = a.prm->defer_nodes != 0;
  int still = 0;
  for (int j0 = 0; j0 < ns && !defer; j0 += NT2) {
    const int j = j0 + threadIdx.x;
    bool act = false;
    if (j < ns) {
      ShiftState& q = a.sh[(size_t)r * ns + j];
      if (q.active) {
        q.res2 = b2n * (q.zeta.x * q.zeta.x + q.zeta.y * q.zeta.y);
        q.last_iter = i;
        if (q.res2 <= tol2 || nrm2 == 0.0) {
          q.active = 0;
          if (nrm2 == 0.0) q.res2 = 0.0;
        } else {
          act = true;
        }
      }
    }
    still += __syncthreads_count(act);
  }
  if (threadIdx.x != 0) return;
  const double beta = sqrt(nrm2);
  if (a.hist_b) a.hist_b[(size_t)r * a.prm->max_iter + (i - 1)] = beta;
  S->n_prev = S->n_cur;
  S->n_cur = beta;
  S->iter = i + 1;
  set_norm_scalars<R>(S);
  if (beta == 0.0) {
    mark_done(S, a.done_count, OV_OK);
  } else if (ns > 0 && still == 0 && !defer) {
    mark_done(S, a.done_count, OV_OK);
  } else if (i >= a.prm->max_iter || (a.prm->store && i + 2 >= a.prm->nslots)) {
    mark_done(S, a.done_count, ns > 0 ? OV_ERR_NOT_CONVERGED : OV_OK);
  }
}

// Per-node LDL^T rows and stopping tests of the scalar-only forms (defer_nodes), caught up
// from the recorded alpha_i, beta_i over the iterations completed since the last check:
// one thread per node, the same recurrence K1 and K2 run per iteration otherwise,
//   d_1 = z - alpha_1, omega_1 = ||b||;  l_{i-1} = -beta_{i-1} / d_{i-1},
//   d_i = z - alpha_i - beta_{i-1}^2 / d_{i-1},  omega_i = -l_{i-1} omega_{i-1};
//   zeta_i = omega_i / d_i,  node residual |beta_i zeta_i| / ||b||.
// A node stops at the first iteration that meets tol; a source whose nodes have all
// stopped is marked done (also one K2 stopped at its iteration limit in that same
// iteration: its status becomes OV_OK).  Off the per-iteration critical path: K1 and K2
// keep only their two reductions in the last block.
template <typename R>
__global__ void __launch_bounds__(NT1) node_check_kernel(SolveArgs<R> a) {
  const int r = blockIdx.y;
  SrcState* S = a.src + r;
  const int ns = a.prm->nshift;
  const int mi = a.prm->max_iter;
  const int upto = S->iter - 1;  // iterations whose alpha_i and beta_i are recorded
  const double tol = a.tol_src ? a.tol_src[r] : a.prm->tol;
  const double tol2 = tol * tol;
  const double* ha = a.hist_a + (size_t)r * mi;
  const double* hb = a.hist_b + (size_t)r * mi;
  int still = 0;
  for (int j0 = 0; j0 < ns; j0 += NT1) {
    const int j = j0 + threadIdx.x;
    bool act = false;
    if (j < ns) {
      ShiftState& q = a.sh[(size_t)r * ns + j];
      if (q.active) {
        const double2 zj = a.z[(size_t)r * ns + j];
        double2 invd = q.invd, om = q.omega, zeta = q.zeta;
        double res2 = q.res2;
        int i = q.last_iter + 1;
        act = true;
        for (; i <= upto; ++i) {
          const double alpha = ha[i - 1], beta = hb[i - 1];
          double2 d;
          if (i == 1) {
            d = make_double2(zj.x - alpha, zj.y);
            om = make_double2(S->bnorm, 0.0);
          } else {
            const double bp = hb[i - 2];  // beta_{i-1} = ||U_i||
            const double2 lprev = make_double2(-bp * invd.x, -bp * invd.y);
            const double b2 = bp * bp;
            d = make_double2(zj.x - alpha - b2 * invd.x, zj.y - b2 * invd.y);
            om = cmul(make_double2(-lprev.x, -lprev.y), om);
          }
          const double inv = __drcp_rn(d.x * d.x + d.y * d.y);
          invd = make_double2(d.x * inv, -d.y * inv);
          zeta = cmul(om, invd);
          res2 = beta * beta * S->inv_b2 * (zeta.x * zeta.x + zeta.y * zeta.y);
          if (res2 <= tol2 || beta == 0.0) {
            if (beta == 0.0) res2 = 0.0;
            act = false;
            break;
          }
        }
        q.invd = invd;
        q.omega = om;
        q.zeta = zeta;
        q.res2 = res2;
        q.last_iter = act ? upto : i;
        q.active = act ? 1 : 0;
      }
    }
    still += __syncthreads_count(act);
  }
  if (threadIdx.x == 0 && ns > 0 && still == 0) {
    if (!S->done)
      mark_done(S, a.done_count, OV_OK);
    else if (S->status == OV_ERR_NOT_CONVERGED)
      S->status = OV_OK;
  }
}

// K3 (second pass of OV_MODE_FP64_2PASS): regenerate U_{i+1} from the recorded
// alpha_i and ||U_i|| with the first pass's arithmetic, and add g_i v_i to the sum.
// One kernel per iteration; the last block advances the iteration counter.
template <typename R>
__global__ void __launch_bounds__(NT1, k1_min_blocks<R>()) lanczos_regen_kernel(SolveArgs<R> a) {
  using T = typename Store<R>::T;
  __shared__ bool last;
  __shared__ Cx<R> sm[4 * 12 * kSplitSites];
  const int r = blockIdx.y;
  SrcState* S = a.src + r;
  const int i = S->iter;
  if (i > S->k_final) return;
  const int V = a.g.V;
  const size_t n12 = (size_t)12 * V;
  const int mi = a.prm->max_iter;
  T* base = a.ring + (size_t)r * a.prm->nslots * n12;
  const T* Ui = base + (size_t)(i % 3) * n12;
  const T* Um = base + (size_t)((i + 2) % 3) * n12;
  T* W = base + (size_t)((i + 1) % 3) * n12;
  const RegenRec<R> rc = a.rrec[(size_t)r * mi + i - 1];
  const R inv_nR = rc.inv_n, cmR = rc.cm, anR = rc.alpha_n;
  const int site0 = blockIdx.x * kSplitSites;
  hw_split_phase1<R, false, !kHalvedLinks<R>>(Ui, a.U, a.g, site0, sm);
  __syncthreads();
  Cx<R> o[3];
  int s, k0;
  if (hw_split_phase2<R, false, kHalvedLinks<R>>(Ui, a.g, site0, a.diag, sm, o, &s, &k0)) {
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const int k = k0 + q;
      const size_t e = k * (size_t)V + s;
      const Cx<R> um = (i > 1) ? ld<R>(Um + e) : Cx<R>{R(0), R(0)};
      const Cx<R> w = lz_w<R>(o[q], um, inv_nR, cmR, i == 1);
      const Cx<R> ui = ld<R>(Ui + e);
      const Cx<R> v = lz_v<R>(ui, inv_nR);
      st<R>(W + e, lz_next<R>(w, ui, anR));
      SumAdd<R>::add(a, (size_t)r * n12 + e, rc.g, v);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = (atomicAdd(a.cnt + 2 * r, 1u) == gridDim.x - 1);
    if (last) {
      a.cnt[2 * r] = 0;
      S->iter = i + 1;
    }
  }
}

// The whole Lanczos loop of the scalar-only forms (vec_shifts = 0) as one cooperative
// persistent launch.  Per iteration: stencil phase (w and <U_i, w> partials), grid
// barrier, every block reduces the same partials in the same order (so every block
// holds the same alpha_i: no serial last-block step), vector update (U_{i+1} and
// ||U_{i+1}||^2 partials), grid barrier, beta_i, and each thread of the grid advances
// at most one node's LDL^T recurrence.  A source whose nodes have all met tol is
// retired at the next barrier (it spends one extra stencil phase).  Data that other
// blocks write during the launch is read through L2 (ld.global.cg).
constexpr int kCoopMaxSrc = 16;

template <typename R>
__global__ void __launch_bounds__(NT1, 4) lanczos_coop_kernel(SolveArgs<R> a, int nsrc) {
  namespace cg = cooperative_groups;
  using T = typename Store<R>::T;
  cg::grid_group grid = cg::this_grid();
  __shared__ Cx<R> sm[4 * 12 * kSplitSites];
  __shared__ double sh[NT1 / 32];
  __shared__ double s_part[kCoopMaxSrc], s_alpha[kCoopMaxSrc], s_beta[kCoopMaxSrc];
  __shared__ double s_ncur[kCoopMaxSrc], s_nprev[kCoopMaxSrc];
  __shared__ int s_done[kCoopMaxSrc];
  __shared__ int s_stop;
  const int G = gridDim.x, b = blockIdx.x, tid = threadIdx.x;
  const int V = a.g.V;
  const size_t n12 = (size_t)12 * V;
  const int ntile = (V + kSplitSites - 1) / kSplitSites;
  const int nwork = ntile * nsrc;
  const int ns = a.prm->nshift, mi = a.prm->max_iter;
  const size_t nsl = (size_t)a.prm->nslots;
  const int lane = tid & 31, grp = tid >> 5;
  if (tid < nsrc) {
    s_ncur[tid] = a.src[tid].n_cur;
    s_nprev[tid] = a.src[tid].n_prev;
    s_done[tid] = a.src[tid].done;
  }
  __syncthreads();
  for (int i = 1;; ++i) {
    // ---- phase 1: w = H U_i / n_i - (n_i / n_{i-1}) U_{i-1}, partial <U_i, w>
    if (tid < kCoopMaxSrc) s_part[tid] = 0.0;
    __syncthreads();
    if (i <= mi) {
      for (int wk = b; wk < nwork; wk += G) {
        const int r = wk / ntile, site0 = (wk % ntile) * kSplitSites;
        if (s_done[r]) continue;
        const T* base = a.ring + (size_t)r * nsl * n12;
        const T* Ui = base + lz_slot(a.prm, i) * n12;
        const T* Um = base + (a.prm->store ? (size_t)(i - 1) : (size_t)((i + 2) % 3)) * n12;
        T* W = (T*)base + lz_slot(a.prm, i + 1) * n12;
        const double inv_n = 1.0 / s_ncur[r];
        const double cm = (i > 1) ? s_ncur[r] / s_nprev[r] : 0.0;
        const R inv_nR = (R)inv_n, cmR = (R)cm;
        hw_split_phase1<R, true, !kHalvedLinks<R>>(Ui, a.U, a.g, site0, sm);
        __syncthreads();
        Cx<R> o[3];
        int s, k0;
        typename Acc<R>::T dot = Acc<R>::zero();
        if (hw_split_phase2<R, true, kHalvedLinks<R>>(Ui, a.g, site0, a.diag, sm, o, &s, &k0)) {
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            const size_t e = (k0 + q) * (size_t)V + s;
            const Cx<R> u = ld<R, true>(Ui + e);
            const Cx<R> um = (i > 1) ? ld<R, true>(Um + e) : Cx<R>{R(0), R(0)};
            const Cx<R> w = lz_w<R>(o[q], um, inv_nR, cmR, i == 1);
            st<R>(W + e, w);
            dot = Acc<R>::dot(dot, u, w);
          }
        }
        const double bs = block_sum<NT1>(Acc<R>::get(dot), sh);
        if (tid == 0) s_part[r] += bs;
        __syncthreads();
      }
    }
    if (tid < nsrc) a.part1[(size_t)tid * G + b] = s_part[tid];
    grid.sync();
    // ---- retire sources whose nodes all met tol at iteration i - 1
    if (i > 1) {
      for (int r = 0; r < nsrc; ++r) {
        if (s_done[r]) continue;
        int act = 0;
        for (int j0 = 0; j0 < ns; j0 += NT1) {
          const int j = j0 + tid;
          const int f = (j < ns) ? __ldcg(&a.sh[(size_t)r * ns + j].active) : 0;
          act += __syncthreads_count(f);
        }
        const bool beta0 = (s_ncur[r] == 0.0);
        if (act == 0 || beta0 || i > mi) {
          if (tid == 0) {
            s_done[r] = 1;
            if (b == 0) {
              SrcState* S = a.src + r;
              S->iter = i;
              S->n_cur = s_ncur[r];
              S->n_prev = s_nprev[r];
              set_norm_scalars<R>(S);
              S->status = (act > 0 && !beta0) ? OV_ERR_NOT_CONVERGED : OV_OK;
              S->done = 1;
            }
          }
        }
        __syncthreads();
      }
    }
    if (tid == 0) {
      int all = 1;
      for (int r = 0; r < nsrc; ++r) all &= s_done[r];
      s_stop = all;
    }
    __syncthreads();
    if (s_stop) break;
    // ---- alpha_i for every source (same order in every block)
    for (int r = 0; r < nsrc; ++r) {
      const double t = sum_partials<NT1>(a.part1 + (size_t)r * G, G, sh);
      if (tid == 0) s_alpha[r] = t / s_ncur[r];
    }
    __syncthreads();
    // ---- phase 2: U_{i+1} = w - alpha_i v_i (in place), partial ||U_{i+1}||^2
    if (tid < kCoopMaxSrc) s_part[tid] = 0.0;
    __syncthreads();
    for (int wk = b; wk < nwork; wk += G) {
      const int r = wk / ntile, site0 = (wk % ntile) * kSplitSites;
      if (s_done[r]) continue;
      const T* base = a.ring + (size_t)r * nsl * n12;
      const T* Ui = base + lz_slot(a.prm, i) * n12;
      T* W = (T*)base + lz_slot(a.prm, i + 1) * n12;
      const double inv_n = 1.0 / s_ncur[r];
      const int s = site0 + lane;
      typename Acc<R>::T nrm = Acc<R>::zero();
      const R anR = (R)(s_alpha[r] * inv_n);
      if (s < V) {
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const size_t e = (3 * grp + q) * (size_t)V + s;
          const Cx<R> u = lz_next<R>(ld<R, true>(W + e), ld<R, true>(Ui + e), anR);
          st<R>(W + e, u);
          nrm = Acc<R>::dot(nrm, u, u);
        }
      }
      const double bs = block_sum<NT1>(Acc<R>::get(nrm), sh);
      if (tid == 0) s_part[r] += bs;
      __syncthreads();
    }
    if (tid < nsrc) a.part2[(size_t)tid * G + b] = s_part[tid];
    grid.sync();
    for (int r = 0; r < nsrc; ++r) {
      const double t = sum_partials<NT1>(a.part2 + (size_t)r * G, G, sh);
      if (tid == 0) s_beta[r] = sqrt(t);
    }
    __syncthreads();
    // ---- node recurrences (one node per thread of the grid) and history
    for (int q = b * NT1 + tid; q < nsrc * ns; q += G * NT1) {
      const int r = q / ns;
      if (s_done[r]) continue;
      ShiftState& st8 = a.sh[q];
      if (!st8.active) continue;
      const double alpha = s_alpha[r], beta = s_beta[r], beta_prev = s_ncur[r];
      const double2 zj = a.z[q];
      double2 d, om;
      if (i == 1) {
        d = make_double2(zj.x - alpha, zj.y);
        om = make_double2(a.src[r].bnorm, 0.0);
      } else {
        const double2 ip = st8.invd;
        const double b2 = beta_prev * beta_prev;
        d = make_double2(zj.x - alpha - b2 * ip.x, zj.y - b2 * ip.y);
        om = cmul(make_double2(beta_prev * ip.x, beta_prev * ip.y), st8.omega);
      }
      const double inv = 1.0 / (d.x * d.x + d.y * d.y);
      const double2 invd = make_double2(d.x * inv, -d.y * inv);
      const double2 zeta = cmul(om, invd);
      st8.invd = invd;
      st8.omega = om;
      st8.zeta = zeta;
      const double tol = a.tol_src ? a.tol_src[r] : a.prm->tol;
      st8.res2 = beta * beta * a.src[r].inv_b2 * (zeta.x * zeta.x + zeta.y * zeta.y);
      st8.last_iter = i;
      if (st8.res2 <= tol * tol || beta == 0.0) {
        st8.active = 0;
        if (beta == 0.0) st8.res2 = 0.0;
      }
    }
    if (tid < nsrc && !s_done[tid]) {
      if (b == 0 && a.hist_a) {
        a.hist_a[(size_t)tid * mi + (i - 1)] = s_alpha[tid];
        a.hist_b[(size_t)tid * mi + (i - 1)] = s_beta[tid];
      }
      s_nprev[tid] = s_ncur[tid];
      s_ncur[tid] = s_beta[tid];
      if (!isfinite(s_alpha[tid]) || !isfinite(s_beta[tid])) {
        s_done[tid] = 1;
        if (b == 0) {
          a.src[tid].iter = i + 1;
          a.src[tid].status = OV_ERR_BREAKDOWN;
          a.src[tid].done = 1;
        }
      }
    }
    __syncthreads();
  }
}

// Per-iteration scalars of the regeneration pass from the recorded alpha_i, beta_i and
// the coefficients g_i, in the vector type -- with the same FP64 expressions (and
// double-float splits) as the first pass, so the regenerated basis is bit-identical.
template <typename R>
__global__ void regen_scalars_kernel(SolveArgs<R> a, RegenRec<R>* rec, int nsrc) {
  const int mi = a.prm->max_iter;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nsrc * mi; t += gridDim.x * blockDim.x) {
    const int r = t / mi, i = t % mi + 1;
    const SrcState* S = a.src + r;
    if (i > S->k_final) continue;
    const double n_i = (i == 1) ? S->bnorm : a.hist_b[(size_t)r * mi + i - 2];
    const double n_m = (i <= 2) ? S->bnorm : a.hist_b[(size_t)r * mi + i - 3];
    float d[8];
    const double inv_n = __drcp_rn(n_i), cm = (i > 1) ? n_i / n_m : 0.0, alpha = a.hist_a[(size_t)r * mi + i - 1];
    const double alpha_n = alpha * inv_n;  // as K1 forms it
    df_split(inv_n, d + 0);
    df_split(cm, d + 2);
    df_split(alpha, d + 4);
    df_split(alpha_n, d + 6);
    const double2 g = a.gco[(size_t)r * mi + i - 1];
    RegenRec<R> o;
    o.inv_n = scal<R>(inv_n, d + 0);
    o.cm = scal<R>(cm, d + 2);
    o.alpha = scal<R>(alpha, d + 4);
    o.alpha_n = scal<R>(alpha_n, d + 6);
    o.g = cx_from<R>(g.x, g.y);
    rec[t] = o;
  }
}

// Stored-basis variant of the second pass: sum[r][e] += sum_{i=1..k_r} gw[r][i-1] U_i[e],
// gw = g_i / ||U_i|| (the basis is stored unnormalised), in the arithmetic of the basis
// (FP64, or double-float with gw split into double-float pairs on the host); one read
// of the basis and one FP64 update of the sum per element.  REAL: the coefficients are
// real (a node list closed under conjugation, z_j and conj(z_j) with conj(c_j): T_k is
// real, so (conj z - T_k)^-1 e_1 = conj((z - T_k)^-1 e_1) and g = sum_j c_j y^j is real),
// two FMAs per element and basis vector instead of four.
template <typename R, bool REAL = false>
__global__ void basis_sum_kernel(const typename Store<R>::T* __restrict__ basis, int nslots,
                                 const typename Store<R>::T* __restrict__ gw, int ldg, const int* __restrict__ kr,
                                 double2* __restrict__ sum, size_t n12) {
  const int r = blockIdx.y;
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n12) return;
  const typename Store<R>::T* B = basis + (size_t)r * nslots * n12 + e;
  const typename Store<R>::T* w = gw + (size_t)r * ldg;
  Cx<R> acc = {R(0), R(0)};
  const int k = kr[r];
  for (int i = 1; i <= k; ++i) {
    const Cx<R> wi = ld<R>(w + i - 1), b = ld<R>(B + (size_t)i * n12);
    if constexpr (REAL) {
      acc.re = fma(wi.re, b.re, acc.re);
      acc.im = fma(wi.re, b.im, acc.im);
    } else {
      acc = cfma(wi, b, acc);
    }
  }
  double2 sv = sum[(size_t)r * n12 + e];
  sv.x += (double)acc.re;
  sv.y += (double)acc.im;
  sum[(size_t)r * n12 + e] = sv;
}

// Per-node solutions from a stored basis: X[r][jj][e] = sum_{i=1..k_r} Y[r][j0 + jj][i-1] U_i[e]
// for the nc nodes of a chunk (Y holds the FOM coefficients folded with 1 / ||U_i||), JT
// nodes per thread so that one read of the basis serves JT outputs; FP64 output.
template <typename R, int JT>
__global__ void basis_nodes_kernel(const typename Store<R>::T* __restrict__ basis, int nslots,
                                   const typename Store<R>::T* __restrict__ Y, int ns, int ldy,
                                   const int* __restrict__ kr, int j0, int nc, double2* __restrict__ X,
                                   size_t n12) {
  const int r = blockIdx.y, jt = blockIdx.z * JT;
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n12 || jt >= nc) return;
  const typename Store<R>::T* B = basis + (size_t)r * nslots * n12 + e;
  const typename Store<R>::T* Yr = Y + ((size_t)r * ns + j0 + jt) * ldy;
  const int k = kr[r], nj = min(JT, nc - jt);
  Cx<R> acc[JT];
#pragma unroll
  for (int q = 0; q < JT; ++q) acc[q] = {R(0), R(0)};
  for (int i = 1; i <= k; ++i) {
    const Cx<R> u = ld<R>(B + (size_t)i * n12);
#pragma unroll
    for (int q = 0; q < JT; ++q)
      if (q < nj) acc[q] = cfma(ld<R>(Yr + (size_t)q * ldy + (i - 1)), u, acc[q]);
  }
#pragma unroll
  for (int q = 0; q < JT; ++q)
    if (q < nj) X[((size_t)r * nc + jt + q) * n12 + e] = make_double2((double)acc[q].re, (double)acc[q].im);
}

// sum += (double) ssum: the double-float regeneration-pass sum into the FP64 sum
__global__ void fold_df_sum_kernel(const float4* __restrict__ ssum, double2* __restrict__ sum, size_t n) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const float4 v = ssum[t];
    double2 sv = sum[t];
    sv.x += (double)v.x + (double)v.y;
    sv.y += (double)v.z + (double)v.w;
    sum[t] = sv;
  }
}

// Init: U_1 = b (ring slot 1), ||b|| per source, s = c0 b, node states reset.
template <typename R>
__global__ void __launch_bounds__(NT2) lanczos_init_kernel(SolveArgs<R> a, const double2* __restrict__ b,
                                                           double2 c0) {
  using T = typename Store<R>::T;
  __shared__ double sh[NT2 / 32];
  __shared__ bool last;
  const int r = blockIdx.y;
  const size_t n12 = (size_t)12 * a.g.V;
  T* U1 = a.ring + (size_t)r * a.prm->nslots * n12 + n12;
  const size_t e = (size_t)blockIdx.x * NT2 + threadIdx.x;
  double nrm = 0.0;
  if (e < n12) {
    const double2 bv = b[(size_t)r * n12 + e];
    st<R>(U1 + e, cx_from<R>(bv.x, bv.y));
    nrm = bv.x * bv.x + bv.y * bv.y;
    if (a.sacc) a.sacc[(size_t)r * n12 + e] = make_double2(c0.x * bv.x - c0.y * bv.y, c0.x * bv.y + c0.y * bv.x);
  }
  double bs = block_sum<NT2>(nrm, sh);
  if (threadIdx.x == 0) {
    a.part2[(size_t)r * gridDim.x + blockIdx.x] = bs;
    __threadfence();
    last = (atomicAdd(a.cnt + 2 * r + 1, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double tot = sum_partials<NT2>(a.part2 + (size_t)r * gridDim.x, gridDim.x, sh);
  if (threadIdx.x != 0) return;
  a.cnt[2 * r + 1] = 0;
  SrcState* S = a.src + r;
  S->bnorm = sqrt(tot);
  S->inv_b2 = tot > 0.0 ? 1.0 / tot : 0.0;
  S->n_cur = S->bnorm;
  S->n_prev = 1.0;
  S->alpha = 0.0;
  S->iter = 1;
  set_norm_scalars<R>(S);
  S->status = OV_OK;
  S->n_act = 0;
  S->node_updates = 0.0;
  S->k_final = 0;
  S->done = 0;
  const int ns = a.prm->nshift;
  for (int j = 0; j < ns; ++j) {
    ShiftState& q = a.sh[(size_t)r * ns + j];
    q.invd = q.omega = q.zeta = make_double2(0.0, 0.0);
    q.res2 = 1.0;
    q.active = 1;
    q.last_iter = 0;
  }
  // a source whose tolerance is >= 1 needs no work (a correction right-hand side that
  // already meets tol): done before the first step, which could otherwise enlarge it
  const bool skip = a.tol_src && a.tol_src[r] >= 1.0;
  if (skip || !(S->bnorm > 0.0) || !isfinite(S->bnorm)) {
    for (int j = 0; j < ns; ++j) {
      a.sh[(size_t)r * ns + j].active = 0;
      a.sh[(size_t)r * ns + j].res2 = 0.0;
    }
    mark_done(S, a.done_count, (skip || isfinite(S->bnorm)) ? OV_OK : OV_ERR_BREAKDOWN);
  }
}

// second pass: U_1 = b again in ring slot 1 (the first pass overwrote the ring)
template <typename R>
__global__ void ring_reset_kernel(SolveArgs<R> a, const double2* __restrict__ b, int nsrc, int nslots) {
  using T = typename Store<R>::T;
  const size_t n12 = (size_t)12 * a.g.V;
  const size_t n = n12 * nsrc;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const size_t r = t / n12, e = t % n12;
    const double2 bv = b[t];
    st<R>(a.ring + r * nslots * n12 + n12 + e, cx_from<R>(bv.x, bv.y));
  }
}

// zero the per-node solution buffers (first update writes them, but a node that is
// converged at init must still read as zero)
template <typename R>
__global__ void zero_kernel(typename Store<R>::T* p, size_t n) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    st<R>(p + t, Cx<R>{R(0), R(0)});
}

}  // namespace

// ------------------------------------------------------------------ host side

namespace {

// workspace name prefix per arithmetic type of the coefficient-space forms
template <typename R> const char* coef_tag();
template <> const char* coef_tag<double>() { return "fp64"; }
template <> const char* coef_tag<DF>() { return "df"; }

// a complex coefficient in the storage type of the vectors (host side)
inline double2 host_store(double2 v, double2*) { return v; }
inline float4 host_store(double2 v, float4*) {
  const float rh = (float)v.x, ih = (float)v.y;
  return make_float4(rh, (float)(v.x - (double)rh), ih, (float)(v.y - (double)ih));
}

// link planes and host-side scalar conversion per arithmetic type
template <typename R> const typename Store<R>::T* solver_links(ov_ctx* ctx);
template <> const double2* solver_links<double>(ov_ctx* ctx) { return ctx->U64h; }  // -1/2 U
template <> const float2* solver_links<float>(ov_ctx* ctx) { return ctx->U32; }
template <> const float4* solver_links<DF>(ov_ctx* ctx) { return ctx->Udf; }
template <typename R> R solver_real(double x) { return (R)x; }
template <> DF solver_real<DF>(double x) {
  const float h = (float)x;
  return DF(h, (float)(x - (double)h));
}

template <typename R>
struct SolveWs {
  SolveArgs<R> a{};
  int nblk1 = 0, nblk2 = 0, nblk2u = 0;
  int nslots = 3;
  int nshift = 0;
  int max_iter = 0;  // row length of the per-source histories
  SolveParams* prm_dev = nullptr;
  bool defer = false;  // per-node recurrences in node_check_kernel (SolveParams::defer_nodes)
};

// The arguments of sources r0, r0 + 1, ... as a launch of their own sees them: every
// per-source array offset by r0 (kernels index sources by blockIdx.y, K1 by its
// position within a tile's group of blocks).
template <typename R>
SolveArgs<R> args_for_sources(const SolveWs<R>& w, int r0) {
  SolveArgs<R> a = w.a;
  const size_t n12 = (size_t)12 * w.a.g.V, ns = (size_t)w.nshift, r = (size_t)r0;
  a.ring += r * w.nslots * n12;
  if (a.p) a.p += r * ns * n12;
  if (a.x) a.x += r * ns * n12;
  if (a.sacc) a.sacc += r * n12;
  if (a.ssum) a.ssum += r * n12;
  if (a.stencil) a.stencil += r * n12;
  a.src += r;
  a.sh += r * ns;
  a.z += r * ns;
  a.c += r * ns;
  a.act_idx += r * ns;
  a.act_l += r * ns;
  a.act_cz += r * ns;
  a.act_z += r * ns;
  a.part1 += r * w.nblk1;
  a.part2 += r * w.nblk2u;
  a.cnt += 2 * r;
  if (a.hist_a) a.hist_a += r * w.max_iter;
  if (a.hist_b) a.hist_b += r * w.max_iter;
  if (a.gco) a.gco += r * w.max_iter;
  if (a.rrec) a.rrec += r * w.max_iter;
  if (a.tol_src) a.tol_src += r;
  return a;
}

// Source groups of a replayed graph.  Sources are independent, so the per-iteration
// kernels of G groups can run as parallel branches of one graph: on small lattices, where
// a launch leaves SMs idle through its tail, its serial last-block step and the next
// launch's ramp, each branch fills the other's gaps; on large ones one branch's update
// kernel (bound by HBM) runs beside the other's stencil kernel (bound by the FP64 pipe or
// FP32 issue).  Auto: one group per source, at most four, when the stencil grid of all
// sources fits two waves (152 SMs x 4 blocks); else two, or six for double-float.
// (8^4, 4 sources, FP64 two-pass: 23.8 / 22.6 / 22.0 ms per apply with 1 / 2 / 4 groups;
// 16^3 x 32, 12 sources in batches of 6, 1 / 2 / 3 / 6 groups: FP64 two-pass 1385 / 1373
// / 1374 / 1375 ms, double-float 407 / 390 / 390 / 386 ms; 16^4: 533.6 / 529.8 ms.)
template <typename R>
int source_groups(const ov_ctx* ctx, int nsrc, int nblk1) {
  int g = ctx->groups;
  if (g <= 0) g = ((size_t)nblk1 * nsrc <= (size_t)2 * 152 * 4) ? 4 : (std::is_same<R, DF>::value ? 6 : 2);
  return std::max(1, std::min(g, nsrc));
}

// Capture body(stream, args, sources) once per source group, each group on its own branch
// (forked from and joined back to the capture stream), and instantiate the graph.
template <typename R, typename F>
int capture_groups(ov_ctx* ctx, const SolveWs<R>& w, int nsrc, int G, F body, cudaGraphExec_t* exec) {
  while ((int)ctx->aux_streams.size() < G) {
    cudaStream_t st = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess) return ctx_cuda(ctx, e, "cudaStreamCreate");
    ctx->aux_streams.push_back(st);
  }
  while ((int)ctx->cap_events.size() < G) {
    cudaEvent_t ev = nullptr;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return ctx_cuda(ctx, e, "cudaEventCreate");
    ctx->cap_events.push_back(ev);
  }
  cudaError_t e = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return ctx_cuda(ctx, e, "cudaStreamBeginCapture");
  if (G > 1) {
    cudaEventRecord(ctx->cap_events[0], ctx->cap_stream);
    for (int g = 1; g < G; ++g) cudaStreamWaitEvent(ctx->aux_streams[g], ctx->cap_events[0], 0);
  }
  for (int g = 0; g < G; ++g) {
    const int lo = (int)((long long)nsrc * g / G), hi = (int)((long long)nsrc * (g + 1) / G);
    body(g == 0 ? ctx->cap_stream : ctx->aux_streams[g], args_for_sources(w, lo), hi - lo);
  }
  if (G > 1) {
    for (int g = 1; g < G; ++g) {
      cudaEventRecord(ctx->cap_events[g], ctx->aux_streams[g]);
      cudaStreamWaitEvent(ctx->cap_stream, ctx->cap_events[g], 0);
    }
  }
  cudaGraph_t gph = nullptr;
  e = cudaStreamEndCapture(ctx->cap_stream, &gph);
  if (e != cudaSuccess) return ctx_cuda(ctx, e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(exec, gph, 0);
  cudaGraphDestroy(gph);
  if (e != cudaSuccess) return ctx_cuda(ctx, e, "cudaGraphInstantiate");
  return OV_OK;
}

template <typename R>
int setup_ws(ov_ctx* ctx, int nsrc, int ns, bool want_x, bool want_sacc, bool want_hist, int max_iter,
             SolveWs<R>* w, const char* tag, int nslots = 3, bool want_p = true) {
  using T = typename Store<R>::T;
  const int V = ctx->g.V;
  const size_t n12 = (size_t)12 * V;
  int st = OV_OK;
  std::string t(tag);
  w->nblk1 = (V + kSplitSites - 1) / kSplitSites;
  // K1's one-dimensional grid holds every (tile, source) pair of a launch
  if ((size_t)w->nblk1 * (size_t)nsrc > (size_t)0x7fffffff)
    return ctx_fail(ctx, OV_ERR_INVALID_ARG, "too many sources for one stencil launch at this volume");
  w->nshift = ns;
  w->max_iter = max_iter;
  // the init kernel uses the K2 partial buffer with up to ceil(12V / NT2) blocks
  w->nblk2 = (int)((n12 + NT2 - 1) / NT2);
  // K2 is a grid-stride loop: about two blocks per SM in total when the vectors are small
  // (fewer partials, short tail), up to eight (full occupancy, enough loads in flight for
  // HBM) when every thread would otherwise stride over more than 8 elements
  const size_t want = std::min<size_t>(8 * 152, std::max<size_t>(2 * 152, (size_t)nsrc * n12 / (NT2 * 8)));
  w->nblk2u = (int)std::min<size_t>(w->nblk2, std::max<size_t>(8, want / (size_t)nsrc));
  auto& a = w->a;
  w->nslots = nslots;
  a.ring = (T*)ws_get(ctx, (t + ".ring").c_str(), sizeof(T) * (size_t)nslots * n12 * nsrc, &st);
  // per-node direction vectors: only the vector-space form (coefficient-space: none)
  a.p = (ns && want_p) ? (T*)ws_get(ctx, (t + ".p").c_str(), sizeof(T) * n12 * (size_t)nsrc * ns, &st) : nullptr;
  a.x = (want_x && ns) ? (T*)ws_get(ctx, (t + ".x").c_str(), sizeof(T) * n12 * (size_t)nsrc * ns, &st) : nullptr;
  a.sacc = want_sacc ? (double2*)ws_get(ctx, (t + ".sacc").c_str(), sizeof(double2) * n12 * nsrc, &st) : nullptr;
  a.src = (SrcState*)ws_get(ctx, (t + ".src").c_str(), sizeof(SrcState) * nsrc, &st);
  const size_t nsh = (size_t)nsrc * (ns > 0 ? ns : 1);
  a.sh = (ShiftState*)ws_get(ctx, (t + ".sh").c_str(), sizeof(ShiftState) * nsh, &st);
  a.z = (const double2*)ws_get(ctx, (t + ".z").c_str(), sizeof(double2) * nsh, &st);
  a.c = (const double2*)ws_get(ctx, (t + ".c").c_str(), sizeof(double2) * nsh, &st);
  a.act_idx = (int*)ws_get(ctx, (t + ".aidx").c_str(), sizeof(int) * nsh, &st);
  using CT = typename Coef<R>::T;
  a.act_l = (CT*)ws_get(ctx, (t + ".al").c_str(), sizeof(CT) * nsh, &st);
  a.act_cz = (CT*)ws_get(ctx, (t + ".acz").c_str(), sizeof(CT) * nsh, &st);
  a.act_z = (CT*)ws_get(ctx, (t + ".az").c_str(), sizeof(CT) * nsh, &st);
  a.part1 = (double*)ws_get(ctx, (t + ".part1").c_str(), sizeof(double) * (size_t)w->nblk1 * nsrc, &st);
  a.part2 = (double*)ws_get(ctx, (t + ".part2").c_str(), sizeof(double) * (size_t)w->nblk2 * nsrc, &st);
  a.cnt = (unsigned*)ws_get(ctx, (t + ".cnt").c_str(), sizeof(unsigned) * 2 * nsrc, &st);
  a.done_count = (int*)ws_get(ctx, (t + ".done").c_str(), sizeof(int), &st);
  if (want_hist) {
    a.hist_a = (double*)ws_get(ctx, (t + ".ha").c_str(), sizeof(double) * (size_t)nsrc * max_iter, &st);
    a.hist_b = (double*)ws_get(ctx, (t + ".hb").c_str(), sizeof(double) * (size_t)nsrc * max_iter, &st);
  } else {
    a.hist_a = a.hist_b = nullptr;
  }
  a.gco = nullptr;
  a.tol_src = nullptr;
  w->prm_dev = (SolveParams*)ws_get(ctx, (t + ".prm").c_str(), sizeof(SolveParams), &st);
  a.prm = w->prm_dev;
  a.stencil = nullptr;
  a.g = ctx->g;
  a.diag = solver_real<R>(4.0 - ctx->m0);
  a.U = solver_links<R>(ctx);
  return st;
}

// K1's grid for n sources: one dimension, the n sources of a site tile in consecutive
// blocks, so that they run side by side and the tile's links come from DRAM once for
// all of them (L2 serves the rest).  With the sources in a second grid dimension each
// source swept the whole lattice in turn and re-read the link field from DRAM (16^3 x
// 32, 6 sources: 522 MB of DRAM traffic per launch here, about 850 MB that way).  The
// time hardly moves, since neither stencil is DRAM-bound: FP64 1386 ms per 12-source
// solve either way, double-float 424.4 vs 421.7 ms.
template <typename R>
dim3 k1_grid(const SolveWs<R>& w, int n) {
  return dim3((unsigned)w.nblk1 * (unsigned)n);
}

template <typename R>
void launch_node_check(const SolveWs<R>& w, const SolveArgs<R>& a, int nsrc, cudaStream_t s) {
  node_check_kernel<R><<<dim3(1, nsrc), NT1, 0, s>>>(a);
}

// One Lanczos iteration (K1, K2); `it` counts iterations from 0 within the loop, and a
// scalar-only form with deferred node recurrences checks its nodes after every
// kNodeCheck-th.
template <typename R>
int launch_iteration(ov_ctx* ctx, const SolveWs<R>& w, int nsrc, cudaStream_t s, int it) {
  cudaEvent_t ev;
  kt_begin(ctx, KC_LANCZOS_HW, s, &ev);
  lanczos_hw_kernel<R><<<k1_grid(w, nsrc), NT1, 0, s>>>(w.a);
  kt_end(ctx, KC_LANCZOS_HW, s, ev);
  kt_begin(ctx, KC_SHIFT_UPDATE, s, &ev);
  lanczos_update_kernel<R><<<dim3(w.nblk2u, nsrc), NT2, 0, s>>>(w.a);
  kt_end(ctx, KC_SHIFT_UPDATE, s, ev);
  if (w.defer && (it + 1) % kNodeCheck == 0) launch_node_check<R>(w, w.a, nsrc, s);
  return OV_OK;
}

// Run iterations until every source is done or max_iter is reached.
template <typename R>
int run_iterations(ov_ctx* ctx, const SolveWs<R>& w, int nsrc, int nshift, int flavour, int max_iter,
                   const ov_solve_opts& o, cudaStream_t s, double* launches) {
  NvtxRange nvtx_("lanczos iterations");
  int chunk = o.check_every > 0 ? o.check_every : 32;
  // deferred node checks run after every kNodeCheck-th iteration counted from the start,
  // whatever the chunking: a replayed chunk must span whole check intervals
  if (w.defer) chunk = (chunk + kNodeCheck - 1) / kNodeCheck * kNodeCheck;
  const bool graph = o.use_graph && !ctx->timing;
  cudaGraphExec_t exec = nullptr;
  if (graph) {
    const int G = source_groups<R>(ctx, nsrc, w.nblk1);
    GraphKey key{{(const void*)w.a.ring, (const void*)w.a.p, (const void*)w.a.x, (const void*)w.a.sacc},
                 nsrc, nshift, flavour * 128 + G, chunk, w.nslots, w.max_iter};
    auto it = ctx->graphs.find(key);
    if (it != ctx->graphs.end()) {
      exec = it->second;
    } else {
      // the graph replays identical launches: every argument is a workspace pointer
      // and all per-iteration state lives in device memory
      const int st = capture_groups<R>(
          ctx, w, nsrc, G,
          [&](cudaStream_t cs, const SolveArgs<R>& a, int n) {
            for (int k = 0; k < chunk; ++k) {
              lanczos_hw_kernel<R><<<k1_grid(w, n), NT1, 0, cs>>>(a);
              lanczos_update_kernel<R><<<dim3(w.nblk2u, n), NT2, 0, cs>>>(a);
              if (w.defer && (k + 1) % kNodeCheck == 0) launch_node_check<R>(w, a, n, cs);
            }
          },
          &exec);
      if (st != OV_OK) return st;
      ctx->graphs[key] = exec;
    }
  }
  const int G = graph ? source_groups<R>(ctx, nsrc, w.nblk1) : 1;
  int done_iters = 0;
  while (done_iters < max_iter) {
    const int n = std::min(chunk, max_iter - done_iters);
    const int nchecks = w.defer ? (done_iters + n) / kNodeCheck - done_iters / kNodeCheck : 0;
    if (graph && n == chunk) {
      cudaError_t e = cudaGraphLaunch(exec, s);
      if (e != cudaSuccess) return ctx_cuda(ctx, e, "cudaGraphLaunch");
      *launches += (2.0 * n + nchecks) * G;
    } else {
      for (int k = 0; k < n; ++k) launch_iteration<R>(ctx, w, nsrc, s, done_iters + k);
      OV_CHECK_LAUNCH(ctx, "lanczos kernels");
      *launches += 2.0 * n + nchecks;
    }
    done_iters += n;
    cudaError_t e = cudaMemcpyAsync(ctx->host_flag, w.a.done_count, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return ctx_cuda(ctx, e, "cudaMemcpyAsync(done)");
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return ctx_cuda(ctx, e, "cudaStreamSynchronize");
    kt_collect(ctx);
    if (*ctx->host_flag >= nsrc) break;
  }
  if (w.defer) {  // the iterations since the last check (final node residuals and status)
    launch_node_check<R>(w, w.a, nsrc, s);
    OV_CHECK_LAUNCH(ctx, "node_check_kernel");
    *launches += 1.0;
  }
  return OV_OK;
}

// The persistent form of the iteration loop (lanczos_coop_kernel) when it applies:
// scalar-only node recurrences, at most kCoopMaxSrc sources, and a grid that is
// co-resident (one block per 32-site tile and source, capped by occupancy).  Returns
// OV_ERR_INVALID_ARG (nothing launched) when it does not apply.
template <typename R>
int run_coop(ov_ctx* ctx, SolveWs<R>& w, int nsrc, cudaStream_t s, double* launches) {
  if (nsrc > kCoopMaxSrc || ctx->no_coop) return OV_ERR_INVALID_ARG;
  int dev = 0, coop = 0, nsm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (!coop) return OV_ERR_INVALID_ARG;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lanczos_coop_kernel<R>, NT1, 0) != cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    return OV_ERR_INVALID_ARG;
  }
  const int ntile = (ctx->g.V + kSplitSites - 1) / kSplitSites;
  const int G = std::min(per_sm * nsm, ntile * nsrc);
  SolveArgs<R> a = w.a;
  // block partials, indexed source * G + block
  int st = OV_OK;
  a.part1 = (double*)ws_get(ctx, "coop.part1", sizeof(double) * (size_t)G * nsrc, &st);
  a.part2 = (double*)ws_get(ctx, "coop.part2", sizeof(double) * (size_t)G * nsrc, &st);
  if (st != OV_OK) return st;
  void* args[] = {(void*)&a, (void*)&nsrc};
  cudaEvent_t ev;
  kt_begin(ctx, KC_COOP, s, &ev);
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)lanczos_coop_kernel<R>, dim3(G), dim3(NT1), args, 0, s);
  kt_end(ctx, KC_COOP, s, ev);
  if (e != cudaSuccess) return ctx_cuda(ctx, e, "cudaLaunchCooperativeKernel");
  *launches += 1.0;
  return OV_OK;
}

template <typename R>
int init_solve(ov_ctx* ctx, SolveWs<R>& w, const double2* b_soa, int nsrc, int ns,
               const std::vector<double2>& zh, const std::vector<double2>& ch, double2 c0,
               double tol, int max_iter, cudaStream_t s, int vec_shifts = 1) {
  // scalar-only forms with nodes defer the per-node recurrences (they record alpha, beta)
  w.defer = (vec_shifts == 0 && ns > 0 && w.a.hist_a && w.a.hist_b);
  SolveParams prm{tol, max_iter, ns, vec_shifts, w.nslots, w.nslots > 3 ? 1 : 0, w.defer ? 1 : 0};
  cudaError_t e = cudaMemcpyAsync(w.prm_dev, &prm, sizeof(prm), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return ctx_cuda(ctx, e, "copy params");
  if (ns > 0) {
    e = cudaMemcpyAsync((void*)w.a.z, zh.data(), sizeof(double2) * zh.size(), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return ctx_cuda(ctx, e, "copy nodes");
    e = cudaMemcpyAsync((void*)w.a.c, ch.data(), sizeof(double2) * ch.size(), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return ctx_cuda(ctx, e, "copy coefficients");
  }
  cudaMemsetAsync(w.a.cnt, 0, sizeof(unsigned) * 2 * nsrc, s);
  cudaMemsetAsync(w.a.done_count, 0, sizeof(int), s);
  if (w.a.x) {
    const size_t n = (size_t)12 * ctx->g.V * nsrc * ns;
    zero_kernel<R><<<1024, 256, 0, s>>>(w.a.x, n);
  }
  cudaEvent_t ev;
  kt_begin(ctx, KC_MISC, s, &ev);
  lanczos_init_kernel<R><<<dim3(w.nblk2, nsrc), NT2, 0, s>>>(w.a, b_soa, c0);
  kt_end(ctx, KC_MISC, s, ev);
  OV_CHECK_LAUNCH(ctx, "lanczos_init_kernel");
  return OV_OK;
}

template <typename R>
int finish_solve(ov_ctx* ctx, SolveWs<R>& w, int nsrc, int ns, const std::vector<double2>& zh,
                 const std::vector<double2>& ch, SolveOut* so, cudaStream_t s) {
  std::vector<SrcState> S(nsrc);
  std::vector<ShiftState> Q((size_t)nsrc * (ns > 0 ? ns : 1));
  cudaError_t e = cudaMemcpyAsync(S.data(), w.a.src, sizeof(SrcState) * nsrc, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && ns > 0)
    e = cudaMemcpyAsync(Q.data(), w.a.sh, sizeof(ShiftState) * (size_t)nsrc * ns, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return ctx_cuda(ctx, e, "read solver state");
  int status = OV_OK;
  so->iterations = 0;
  so->converged = 1;
  so->max_residual = 0.0;
  so->error_bound = 0.0;
  so->node_updates = 0.0;
  for (int r = 0; r < nsrc; ++r) {
    so->node_updates += S[r].node_updates;
    so->iterations = std::max(so->iterations, S[r].iter - 1);
    if (!S[r].done) S[r].status = OV_ERR_NOT_CONVERGED;
    if (S[r].status != OV_OK) {
      so->converged = 0;
      if (status == OV_OK || S[r].status == OV_ERR_BREAKDOWN) status = S[r].status;
    }
    double bound = 0.0;
    for (int j = 0; j < ns; ++j) {
      const ShiftState& q = Q[(size_t)r * ns + j];
      const double res = std::sqrt(q.res2);
      so->max_residual = std::max(so->max_residual, res);
      const double2 zz = zh[(size_t)r * ns + j], cc = ch[(size_t)r * ns + j];
      bound += std::hypot(cc.x, cc.y) * res / std::fabs(zz.y);
    }
    so->error_bound = std::max(so->error_bound, bound);
  }
  if (status == OV_ERR_NOT_CONVERGED)
    return ctx_fail(ctx, status, "shifted solve hit the iteration limit before every node met tol");
  if (status == OV_ERR_BREAKDOWN) return ctx_fail(ctx, status, "non-finite Lanczos scalar (NaN/Inf in input?)");
  return OV_OK;
}

}  // namespace

// Shifted FP64 solve with an explicit node list per source (zh, ch: nsrc x ns): the
// weighted sum c0 b + sum_j c_j y_j goes to out_soa (if not null) and, if xs_soa is
// not null, every node's solution y_j to xs_soa[src][j][12V].
// The vector-space shifted solve for explicit nodes (per source), optionally keeping every
// node's solution (xs, in the vector storage type): FP64 or double-float vectors.
template <typename R>
static int solve_nodes_t(ov_ctx* ctx, const double2* b_soa, int nsrc, int ns, const std::vector<double2>& zh,
                         const std::vector<double2>& ch, double2 c0, double2* out_soa, typename Store<R>::T* xs,
                         const ov_solve_opts& o, SolveOut* so, cudaStream_t s, const char* tag) {
  SolveWs<R> w;
  int st = setup_ws<R>(ctx, nsrc, ns, false, true, false, o.max_iter, &w, tag);
  if (st != OV_OK) return st;
  w.a.x = xs;
  st = init_solve<R>(ctx, w, b_soa, nsrc, ns, zh, ch, c0, o.tol, o.max_iter, s);
  if (st != OV_OK) return st;
  double launches = 1.0 + (xs ? 1.0 : 0.0);  // init (+ zeroing)
  st = run_iterations<R>(ctx, w, nsrc, ns, xs ? 1 : 0, o.max_iter, o, s, &launches);
  if (st != OV_OK) return st;
  st = finish_solve<R>(ctx, w, nsrc, ns, zh, ch, so, s);
  so->launches = launches + 2.0;  // pack + unpack/epilogue issued by the caller
  if (out_soa) {
    // the weighted sum, even when not converged (best iterate)
    cudaError_t e = cudaMemcpyAsync(out_soa, w.a.sacc, sizeof(double2) * 12 * (size_t)ctx->g.V * nsrc,
                                    cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return ctx_cuda(ctx, e, "copy sum");
  }
  return st;
}

int solve_nodes_soa(ov_ctx* ctx, const double2* b_soa, int nsrc, int ns, const std::vector<double2>& zh,
                    const std::vector<double2>& ch, double2 c0, double2* out_soa, double2* xs_soa,
                    const ov_solve_opts& o, SolveOut* so, cudaStream_t s) {
  return solve_nodes_t<double>(ctx, b_soa, nsrc, ns, zh, ch, c0, out_soa, xs_soa, o, so, s, "fp64");
}

namespace {
__global__ void df_to_double_kernel(const float4* __restrict__ in, double2* __restrict__ out, size_t n) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const float4 v = in[t];
    out[t] = make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
  }
}
}  // namespace

int solve_nodes_soa_df(ov_ctx* ctx, const double2* b_soa, int nsrc, int ns, const std::vector<double2>& zh,
                       const std::vector<double2>& ch, double2 c0, double2* out_soa, double2* xs_soa,
                       const ov_solve_opts& o, SolveOut* so, cudaStream_t s) {
  int st = ensure_links_df(ctx, s);
  if (st != OV_OK) return st;
  const size_t nx = (size_t)12 * ctx->g.V * nsrc * ns;
  float4* xd = xs_soa ? (float4*)ws_get(ctx, "dfn.xs", sizeof(float4) * nx, &st) : nullptr;
  if (st != OV_OK) return st;
  st = solve_nodes_t<DF>(ctx, b_soa, nsrc, ns, zh, ch, c0, out_soa, xd, o, so, s, "dfn");
  if (xs_soa && (st == OV_OK || st == OV_ERR_NOT_CONVERGED)) {
    df_to_double_kernel<<<152 * 8, 256, 0, s>>>(xd, xs_soa, nx);
    OV_CHECK_LAUNCH(ctx, "df_to_double_kernel");
  }
  return st;
}

int solve_sign_soa(ov_ctx* ctx, const double2* b_soa, double2* out_soa, int nsrc, const ov_solve_opts& o,
                   SolveOut* so, cudaStream_t s, double2* xs_soa) {
  NvtxRange nvtx_("solve: vector-space form");
  const int ns = (int)ctx->z.size();
  std::vector<double2> zh((size_t)nsrc * ns), ch((size_t)nsrc * ns);
  for (int r = 0; r < nsrc; ++r)
    for (int j = 0; j < ns; ++j) {
      zh[(size_t)r * ns + j] = ctx->z[j];
      ch[(size_t)r * ns + j] = ctx->c[j];
    }
  return solve_nodes_soa(ctx, b_soa, nsrc, ns, zh, ch, ctx->c0, out_soa, xs_soa, o, so, s);
}

// FOM coefficients y = (z - T_k)^-1 e_1 ||b|| of one node from the recorded Lanczos
// scalars al[0..k), be[0..k): forward LDL^T sweep (d_i, l_i = -beta_i / d_i, zeta_i =
// omega_i / d_i) and back substitution y_i = zeta_i - l_i y_{i+1}.
struct FomScratch {
  std::vector<std::complex<double>> dd, ll, zt;
};
static void fom_coefficients(const double* al, const double* be, int k, double bnorm, std::complex<double> z,
                             FomScratch& sc, std::vector<std::complex<double>>& yy) {
  sc.dd.assign(k, 0.0);
  sc.ll.assign(k, 0.0);
  sc.zt.assign(k, 0.0);
  yy.assign(k, 0.0);
  if (k < 1) return;
  std::complex<double> om = bnorm;
  for (int i = 0; i < k; ++i) {
    if (i == 0) {
      sc.dd[0] = z - al[0];
    } else {
      sc.dd[i] = z - al[i] - be[i - 1] * be[i - 1] / sc.dd[i - 1];
      om = -sc.ll[i - 1] * om;
    }
    sc.ll[i] = -be[i] / sc.dd[i];
    sc.zt[i] = om / sc.dd[i];
  }
  yy[k - 1] = sc.zt[k - 1];
  for (int i = k - 2; i >= 0; --i) yy[i] = sc.zt[i] - sc.ll[i] * yy[i + 1];
}

// g = sum_j c_j (z_j - T_k)^-1 e_1 ||b|| per source, from the recorded alpha (ha) and beta
// (hb), leading dimension ld.
static void lanczos_sum_coefficients(const ov_ctx* ctx, int nsrc, const std::vector<int>& kr,
                                     const std::vector<double>& bnorm, const std::vector<double>& ha,
                                     const std::vector<double>& hb, int ld, std::vector<double2>& g) {
  const int ns = (int)ctx->z.size();
  g.assign((size_t)nsrc * ld, make_double2(0.0, 0.0));
  FomScratch sc;
  std::vector<std::complex<double>> yy;
  for (int r = 0; r < nsrc; ++r) {
    const int k = kr[r];
    if (k < 1) continue;
    for (int j = 0; j < ns; ++j) {
      const std::complex<double> zj(ctx->z[j].x, ctx->z[j].y), cj(ctx->c[j].x, ctx->c[j].y);
      fom_coefficients(ha.data() + (size_t)r * ld, hb.data() + (size_t)r * ld, k, bnorm[r], zj, sc, yy);
      for (int i = 0; i < k; ++i) {
        const std::complex<double> t = cj * yy[i];
        g[(size_t)r * ld + i].x += t.real();
        g[(size_t)r * ld + i].y += t.imag();
      }
    }
  }
}

// Stored-basis form of OV_MODE_FP64_2PASS: pass 1 keeps U_1 .. U_k (slot i), then
// s = c0 b + sum_i (g_i / ||U_i||) U_i in one read of the basis.
template <typename R>
static int solve_sign_stored(ov_ctx* ctx, const double2* b_soa, double2* out_soa, int nsrc,
                             const ov_solve_opts& o, SolveOut* so, cudaStream_t s, int cap) {
  NvtxRange nvtx_("solve: stored basis");
  const int ns = (int)ctx->z.size();
  const size_t n12 = (size_t)12 * ctx->g.V;
  SolveWs<R> w;
  const std::string tag = std::string(coef_tag<R>()) + "s";
  int st = setup_ws<R>(ctx, nsrc, ns, false, true, true, cap, &w, tag.c_str(), cap + 3, false);
  if (st != OV_OK) return st;
  std::vector<double2> zh((size_t)nsrc * ns), ch((size_t)nsrc * ns);
  for (int r = 0; r < nsrc; ++r)
    for (int j = 0; j < ns; ++j) {
      zh[(size_t)r * ns + j] = ctx->z[j];
      ch[(size_t)r * ns + j] = ctx->c[j];
    }
  st = init_solve<R>(ctx, w, b_soa, nsrc, ns, zh, ch, ctx->c0, o.tol, cap, s, 0);
  if (st != OV_OK) return st;
  double launches = 1.0;
  st = run_coop<R>(ctx, w, nsrc, s, &launches);
  if (st == OV_ERR_INVALID_ARG) st = run_iterations<R>(ctx, w, nsrc, ns, 6, cap, o, s, &launches);
  if (st != OV_OK) return st;
  const int fst = finish_solve<R>(ctx, w, nsrc, ns, zh, ch, so, s);
  // not converged within the store: the caller regenerates, unless the store already
  // spans max_iter (then the best iterate is returned with OV_ERR_NOT_CONVERGED)
  if (fst != OV_OK && !(fst == OV_ERR_NOT_CONVERGED && cap >= o.max_iter)) return fst;
  std::vector<SrcState> S(nsrc);
  std::vector<double> ha((size_t)nsrc * cap), hb((size_t)nsrc * cap);
  cudaError_t e = cudaMemcpyAsync(S.data(), w.a.src, sizeof(SrcState) * nsrc, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ha.data(), w.a.hist_a, sizeof(double) * ha.size(), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hb.data(), w.a.hist_b, sizeof(double) * hb.size(), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return ctx_cuda(ctx, e, "read Lanczos history");
  std::vector<int> kr(nsrc);
  std::vector<double> bn(nsrc);
  for (int r = 0; r < nsrc; ++r) {
    kr[r] = std::max(0, S[r].iter - 1);
    bn[r] = S[r].bnorm;
  }
  std::vector<double2> g;
  lanczos_sum_coefficients(ctx, nsrc, kr, bn, ha, hb, cap, g);
  for (int r = 0; r < nsrc; ++r)
    for (int i = 0; i < kr[r]; ++i) {  // fold in 1 / ||U_i||
      const double ni = (i == 0) ? bn[r] : hb[(size_t)r * cap + i - 1];
      g[(size_t)r * cap + i].x /= ni;
      g[(size_t)r * cap + i].y /= ni;
    }
  // a node list closed under conjugation gives real coefficients (up to rounding):
  // then the sum takes half the multiplications
  bool real = true;
  for (int r = 0; r < nsrc && real; ++r) {
    double gmax = 0.0, imax = 0.0;
    for (int i = 0; i < kr[r]; ++i) {
      const double2 v = g[(size_t)r * cap + i];
      gmax = std::max(gmax, std::hypot(v.x, v.y));
      imax = std::max(imax, std::fabs(v.y));
    }
    real = std::isfinite(gmax) && imax <= 1e-14 * gmax;
  }
  using T = typename Store<R>::T;
  std::vector<T> gs(g.size());
  for (size_t t = 0; t < g.size(); ++t) gs[t] = host_store(g[t], (T*)nullptr);
  T* gd = (T*)ws_get(ctx, (tag + ".g").c_str(), sizeof(T) * gs.size(), &st);
  int* krd = (int*)ws_get(ctx, (tag + ".kr").c_str(), sizeof(int) * nsrc, &st);
  if (st != OV_OK) return st;
  e = cudaMemcpyAsync(gd, gs.data(), sizeof(T) * gs.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(krd, kr.data(), sizeof(int) * nsrc, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return ctx_cuda(ctx, e, "copy coefficients");
  cudaEvent_t ev;
  kt_begin(ctx, KC_BASIS_SUM, s, &ev);
  const dim3 gsum((unsigned)((n12 + 255) / 256), nsrc);
  if (real)
    basis_sum_kernel<R, true><<<gsum, 256, 0, s>>>(w.a.ring, cap + 3, gd, cap, krd, w.a.sacc, n12);
  else
    basis_sum_kernel<R, false><<<gsum, 256, 0, s>>>(w.a.ring, cap + 3, gd, cap, krd, w.a.sacc, n12);
  kt_end(ctx, KC_BASIS_SUM, s, ev);
  OV_CHECK_LAUNCH(ctx, "basis_sum_kernel");
  so->launches = launches + 3.0;
  e = cudaMemcpyAsync(out_soa, w.a.sacc, sizeof(double2) * n12 * nsrc, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return ctx_cuda(ctx, e, "copy sum");
  return fst;
}

// OV_MODE_FP64_2PASS.  Pass 1: the Lanczos process with every node's LDL^T scalar
// recurrence (for the stopping test) but no per-node vectors; alpha_i and beta_i
// are recorded.  Host: for every node the FOM coefficients y^j = (z_j - T_k)^-1 e_1 ||b||
// (forward LDL^T sweep, back substitution), summed as g = sum_j c_j y^j.  Pass 2:
// regenerate v_1 .. v_k with bit-identical arithmetic and accumulate
// s = c0 b + sum_i g_i v_i.  Same result as OV_MODE_FP64 up to rounding; the vector
// work no longer grows with the number of nodes.
template <typename R>
static int solve_sign_regen(ov_ctx* ctx, const double2* b_soa, double2* out_soa, int nsrc,
                            const ov_solve_opts& o, SolveOut* so, cudaStream_t s);

// Fold the statistics of one batch of sources into the call's.
void merge_stats(SolveOut* tot, const SolveOut& b, bool first) {
  if (first) {
    *tot = b;
    return;
  }
  tot->iterations = std::max(tot->iterations, b.iterations);
  tot->converged = tot->converged && b.converged;
  tot->max_residual = std::max(tot->max_residual, b.max_residual);
  tot->error_bound = std::max(tot->error_bound, b.error_bound);
  tot->refine_rounds += b.refine_rounds;
  tot->inner_iterations += b.inner_iterations;
  tot->node_updates += b.node_updates;
  tot->launches += b.launches;
}

// Coefficient-space solve.  Preferred: keep the Lanczos basis in HBM (pass 2 is one read
// of it instead of a second Lanczos pass), for as many sources at a time as fit the store
// budget -- 40% of device memory, and no more than what is free beyond a 10% reserve (a
// store this context already holds counts as free).  The store depth is min(max_iter,
// 1024) vectors, or 1.25x the iterations of the previous batch or call (plus 32) once
// those are known; a batch that outgrows its store, or that cannot be allocated, is
// solved by regenerating the basis instead.  OV_MODE_FP64_REGEN always regenerates.
template <typename R>
static int solve_sign_coef(ov_ctx* ctx, const double2* b_soa, double2* out_soa, int nsrc, const ov_solve_opts& o,
                           SolveOut* so, cudaStream_t s) {
  NvtxRange nvtx_("solve: coefficient space");
  if (o.mode == OV_MODE_FP64_REGEN) return solve_sign_regen<R>(ctx, b_soa, out_soa, nsrc, o, so, s);
  size_t freeb = 0, totalb = 0;
  cudaMemGetInfo(&freeb, &totalb);
  const std::string ring = std::string(coef_tag<R>()) + "s.ring";
  auto it = ctx->bufs.find(ring);
  const double held = it != ctx->bufs.end() ? (double)it->second.bytes : 0.0;
  const double budget = std::min(0.40 * (double)totalb, (double)freeb + held - 0.10 * (double)totalb);
  const size_t n12 = (size_t)12 * ctx->g.V;
  const double per_vec = (double)n12 * sizeof(double2);
  int cap = std::min(o.max_iter, ctx->coef_iter_hint > 0 ? std::max(64, ctx->coef_iter_hint * 5 / 4 + 32) : 1024);
  int r0 = 0, worst = OV_OK;
  bool first = true;
  while (r0 < nsrc) {
    const int rem = nsrc - r0;
    const int nb_max = (int)std::min<double>(rem, std::floor(budget / ((cap + 3) * per_vec)));
    const int nbat = nb_max >= 1 ? (rem + nb_max - 1) / nb_max : 1;
    const int nb = nb_max >= 1 ? (rem + nbat - 1) / nbat : rem;  // even batches
    SolveOut sb;
    int st = OV_ERR_OUT_OF_MEMORY;
    if (nb_max >= 1) st = solve_sign_stored<R>(ctx, b_soa + r0 * n12, out_soa + r0 * n12, nb, o, &sb, s, cap);
    if (st == OV_ERR_OUT_OF_MEMORY || (st == OV_ERR_NOT_CONVERGED && cap < o.max_iter)) {
      cudaGetLastError();
      sb = SolveOut();
      st = solve_sign_regen<R>(ctx, b_soa + r0 * n12, out_soa + r0 * n12, nb, o, &sb, s);
    }
    if (st != OV_OK && st != OV_ERR_NOT_CONVERGED) return st;
    if (st == OV_ERR_NOT_CONVERGED) worst = st;
    merge_stats(so, sb, first);
    first = false;
    if (sb.converged) {
      ctx->coef_iter_hint = sb.iterations;
      cap = std::min(o.max_iter, std::max(64, sb.iterations * 5 / 4 + 32));
    }
    r0 += nb;
  }
  return worst;
}

// OV_MODE_FP64_REGEN and the fallback of the stored form: pass 1 records alpha_i, beta_i,
// pass 2 regenerates v_1 .. v_k with bit-identical arithmetic and sums g_i v_i.
template <typename R>
static int solve_sign_regen(ov_ctx* ctx, const double2* b_soa, double2* out_soa, int nsrc,
                            const ov_solve_opts& o, SolveOut* so, cudaStream_t s) {
  const int ns = (int)ctx->z.size();
  SolveWs<R> w;
  const std::string tag = coef_tag<R>();
  int st = setup_ws<R>(ctx, nsrc, ns, false, true, true, o.max_iter, &w, tag.c_str(), 3, false);
  if (st != OV_OK) return st;
  double2* gco = (double2*)ws_get(ctx, (tag + ".gco").c_str(), sizeof(double2) * (size_t)nsrc * o.max_iter, &st);
  if (st != OV_OK) return st;
  const size_t n12 = (size_t)12 * ctx->g.V;
  float4* ssum = nullptr;
  if (std::is_same<R, DF>::value) {
    ssum = (float4*)ws_get(ctx, "df.ssum", sizeof(float4) * n12 * nsrc, &st);
    if (st != OV_OK) return st;
  }
  w.a.p = nullptr;
  std::vector<double2> zh((size_t)nsrc * ns), ch((size_t)nsrc * ns);
  for (int r = 0; r < nsrc; ++r)
    for (int j = 0; j < ns; ++j) {
      zh[(size_t)r * ns + j] = ctx->z[j];
      ch[(size_t)r * ns + j] = ctx->c[j];
    }
  st = init_solve<R>(ctx, w, b_soa, nsrc, ns, zh, ch, ctx->c0, o.tol, o.max_iter, s, 0);
  if (st != OV_OK) return st;
  double launches = 1.0;
  st = run_iterations<R>(ctx, w, nsrc, ns, 2, o.max_iter, o, s, &launches);
  if (st != OV_OK) return st;
  const int fst = finish_solve<R>(ctx, w, nsrc, ns, zh, ch, so, s);
  if (fst != OV_OK && fst != OV_ERR_NOT_CONVERGED) return fst;
  // coefficients of the sum in the Lanczos basis
  std::vector<SrcState> S(nsrc);
  cudaError_t e = cudaMemcpyAsync(S.data(), w.a.src, sizeof(SrcState) * nsrc, cudaMemcpyDeviceToHost, s);
  std::vector<double> ha((size_t)nsrc * o.max_iter), hb((size_t)nsrc * o.max_iter);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ha.data(), w.a.hist_a, sizeof(double) * ha.size(), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(hb.data(), w.a.hist_b, sizeof(double) * hb.size(), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return ctx_cuda(ctx, e, "read Lanczos history");
  int kmax = 0;
  std::vector<int> kr(nsrc);
  std::vector<double> bn(nsrc);
  for (int r = 0; r < nsrc; ++r) {
    kr[r] = std::max(0, S[r].iter - 1);
    bn[r] = S[r].bnorm;
    S[r].k_final = kr[r];
    kmax = std::max(kmax, kr[r]);
    if (kr[r] >= 1) {
      S[r].iter = 1;
      S[r].done = 0;
    }
  }
  std::vector<double2> g;
  lanczos_sum_coefficients(ctx, nsrc, kr, bn, ha, hb, o.max_iter, g);
  e = cudaMemcpyAsync(gco, g.data(), sizeof(double2) * g.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(w.a.src, S.data(), sizeof(SrcState) * nsrc, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(w.a.cnt, 0, sizeof(unsigned) * 2 * nsrc, s);
  if (e != cudaSuccess) return ctx_cuda(ctx, e, "second-pass setup");
  w.a.gco = gco;
  w.a.ssum = (typename Store<R>::T*)ssum;
  RegenRec<R>* rrec =
      (RegenRec<R>*)ws_get(ctx, (tag + ".rrec").c_str(), sizeof(RegenRec<R>) * (size_t)nsrc * o.max_iter, &st);
  if (st != OV_OK) return st;
  w.a.rrec = rrec;
  regen_scalars_kernel<R><<<64, 256, 0, s>>>(w.a, rrec, nsrc);
  OV_CHECK_LAUNCH(ctx, "regen_scalars_kernel");
  ring_reset_kernel<R><<<256, 256, 0, s>>>(w.a, b_soa, nsrc, 3);
  launches += 2.0;
  if (ssum) {
    e = cudaMemsetAsync(ssum, 0, sizeof(float4) * n12 * nsrc, s);
    if (e != cudaSuccess) return ctx_cuda(ctx, e, "clear double-float sum");
  }
  // pass 2: kmax regeneration launches (no host reads), replayed from a graph
  const int chunk = o.check_every > 0 ? o.check_every : 32;
  const bool graph = o.use_graph && !ctx->timing;
  cudaGraphExec_t exec = nullptr;
  if (graph && kmax >= chunk) {
    const int G = source_groups<R>(ctx, nsrc, w.nblk1);
    GraphKey key{{(const void*)w.a.ring, (const void*)gco, (const void*)w.a.sacc, (const void*)w.a.hist_a},
                 nsrc, ns, 3 * 128 + G, chunk, w.nslots, w.max_iter};
    auto it = ctx->graphs.find(key);
    if (it != ctx->graphs.end()) {
      exec = it->second;
    } else {
      st = capture_groups<R>(
          ctx, w, nsrc, G,
          [&](cudaStream_t cs, const SolveArgs<R>& a, int n) {
            for (int k = 0; k < chunk; ++k) lanczos_regen_kernel<R><<<dim3(w.nblk1, n), NT1, 0, cs>>>(a);
          },
          &exec);
      if (st != OV_OK) return st;
      ctx->graphs[key] = exec;
    }
  }
  const int Gr = exec ? source_groups<R>(ctx, nsrc, w.nblk1) : 1;
  int done = 0;
  while (done < kmax) {
    const int n = std::min(chunk, kmax - done);
    if (exec && n == chunk) {
      e = cudaGraphLaunch(exec, s);
      if (e != cudaSuccess) return ctx_cuda(ctx, e, "cudaGraphLaunch");
      launches += (double)n * (Gr - 1);  // the other branches' launches
    } else {
      for (int k = 0; k < n; ++k) {
        cudaEvent_t ev;
        kt_begin(ctx, KC_REGEN, s, &ev);
        lanczos_regen_kernel<R><<<dim3(w.nblk1, nsrc), NT1, 0, s>>>(w.a);
        kt_end(ctx, KC_REGEN, s, ev);
      }
      OV_CHECK_LAUNCH(ctx, "lanczos_regen_kernel");
    }
    done += n;
    launches += n;
  }
  if (ssum) {
    fold_df_sum_kernel<<<152 * 8, 256, 0, s>>>(ssum, w.a.sacc, n12 * nsrc);
    OV_CHECK_LAUNCH(ctx, "fold_df_sum_kernel");
    launches += 1.0;
  }
  so->launches = launches + 2.0;
  e = cudaMemcpyAsync(out_soa, w.a.sacc, sizeof(double2) * n12 * nsrc, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return ctx_cuda(ctx, e, "copy sum");
  return fst;
}

// Per-node solutions of explicit per-source node lists through the coefficient space:
// one stored-basis Lanczos pass for all sources (no per-node vectors), the FOM coefficient
// vector of every node on the host, then x_j = V y^j for one chunk of nodes at a time
// (each chunk handed to per_chunk) and the weighted sums sum_j c_j x_j.  The Lanczos
// work does not repeat per chunk.  Returns OV_ERR_INVALID_ARG when the basis does not fit
// the store budget or the solve outgrows it (the caller uses the vector-space form).
template <typename R>
static int nodes_coef(ov_ctx* ctx, const double2* b_soa, int nsrc, int ns, const std::vector<double2>& zh,
                      const std::vector<double2>& ch, int chunk, double2* X, double2* sums, const ov_solve_opts& o,
                      SolveOut* so, cudaStream_t s, const std::function<int(int, int)>& per_chunk) {
  const size_t n12 = (size_t)12 * ctx->g.V;
  size_t freeb = 0, totalb = 0;
  cudaMemGetInfo(&freeb, &totalb);
  const std::string tag = std::string(coef_tag<R>()) + "s";
  auto it = ctx->bufs.find(tag + ".ring");
  const double held = it != ctx->bufs.end() ? (double)it->second.bytes : 0.0;
  const double budget = std::min(0.40 * (double)totalb, (double)freeb + held - 0.10 * (double)totalb);
  const int cap = std::min(o.max_iter, ctx->coef_iter_hint > 0 ? std::max(64, ctx->coef_iter_hint * 5 / 4 + 32) : 1024);
  if ((double)(cap + 3) * nsrc * n12 * sizeof(double2) > budget) return OV_ERR_INVALID_ARG;
  SolveWs<R> w;
  int st = setup_ws<R>(ctx, nsrc, ns, false, true, true, cap, &w, tag.c_str(), cap + 3, false);
  if (st != OV_OK) return st;
  st = init_solve<R>(ctx, w, b_soa, nsrc, ns, zh, ch, make_double2(0.0, 0.0), o.tol, cap, s, 0);
  if (st != OV_OK) return st;
  double launches = 1.0;
  st = run_iterations<R>(ctx, w, nsrc, ns, 7, cap, o, s, &launches);
  if (st != OV_OK) return st;
  const int fst = finish_solve<R>(ctx, w, nsrc, ns, zh, ch, so, s);
  if (fst != OV_OK && !(fst == OV_ERR_NOT_CONVERGED && cap >= o.max_iter)) return OV_ERR_INVALID_ARG;
  std::vector<SrcState> S(nsrc);
  std::vector<double> ha((size_t)nsrc * cap), hb((size_t)nsrc * cap);
  cudaError_t e = cudaMemcpyAsync(S.data(), w.a.src, sizeof(SrcState) * nsrc, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ha.data(), w.a.hist_a, sizeof(double) * ha.size(), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hb.data(), w.a.hist_b, sizeof(double) * hb.size(), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return ctx_cuda(ctx, e, "read Lanczos history");
  // FOM coefficients y^j = (z_j - T_k)^-1 e_1 ||b|| per source and node (forward LDL^T sweep,
  // back substitution), folded with 1 / ||U_i||; g_r = sum_j c_j y^j for the sums
  using T = typename Store<R>::T;
  std::vector<T> Yh((size_t)nsrc * ns * cap);
  std::vector<T> gh((size_t)nsrc * cap);
  std::vector<int> kr(nsrc);
  FomScratch sc;
  std::vector<std::complex<double>> yy, gs;
  for (int r = 0; r < nsrc; ++r) {
    const int k = kr[r] = std::max(0, S[r].iter - 1);
    const double* al = ha.data() + (size_t)r * cap;
    const double* be = hb.data() + (size_t)r * cap;
    gs.assign(k, 0.0);
    for (int j = 0; j < ns && k > 0; ++j) {
      const std::complex<double> zj(zh[(size_t)r * ns + j].x, zh[(size_t)r * ns + j].y);
      const std::complex<double> cj(ch[(size_t)r * ns + j].x, ch[(size_t)r * ns + j].y);
      fom_coefficients(al, be, k, S[r].bnorm, zj, sc, yy);
      for (int i = 0; i < k; ++i) {
        const double ni = (i == 0) ? S[r].bnorm : be[i - 1];
        const std::complex<double> y = yy[i] / ni;
        Yh[((size_t)r * ns + j) * cap + i] = host_store(make_double2(y.real(), y.imag()), (T*)nullptr);
        gs[i] += cj * y;
      }
    }
    for (int i = 0; i < k; ++i) gh[(size_t)r * cap + i] = host_store(make_double2(gs[i].real(), gs[i].imag()), (T*)nullptr);
  }
  T* Yd = (T*)ws_get(ctx, (tag + ".Y").c_str(), sizeof(T) * Yh.size(), &st);
  T* gd = (T*)ws_get(ctx, (tag + ".g").c_str(), sizeof(T) * gh.size(), &st);
  int* krd = (int*)ws_get(ctx, (tag + ".kr").c_str(), sizeof(int) * nsrc, &st);
  if (st != OV_OK) return st;
  e = cudaMemcpyAsync(Yd, Yh.data(), sizeof(T) * Yh.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(gd, gh.data(), sizeof(T) * gh.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(krd, kr.data(), sizeof(int) * nsrc, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(sums, 0, sizeof(double2) * n12 * nsrc, s);
  if (e != cudaSuccess) return ctx_cuda(ctx, e, "copy node coefficients");
  cudaEvent_t ev;
  kt_begin(ctx, KC_BASIS_SUM, s, &ev);
  basis_sum_kernel<R><<<dim3((unsigned)((n12 + 255) / 256), nsrc), 256, 0, s>>>(w.a.ring, cap + 3, gd, cap, krd,
                                                                             sums, n12);
  kt_end(ctx, KC_BASIS_SUM, s, ev);
  OV_CHECK_LAUNCH(ctx, "basis_sum_kernel");
  constexpr int JT = 8;
  for (int j0 = 0; j0 < ns; j0 += chunk) {
    const int nc = std::min(chunk, ns - j0);
    basis_nodes_kernel<R, JT><<<dim3((unsigned)((n12 + 255) / 256), nsrc, (nc + JT - 1) / JT), 256, 0, s>>>(
        w.a.ring, cap + 3, Yd, ns, cap, krd, j0, nc, X, n12);
    OV_CHECK_LAUNCH(ctx, "basis_nodes_kernel");
    if ((st = per_chunk(j0, nc)) != OV_OK) return st;
  }
  so->launches = launches + 2.0 + (ns + chunk - 1) / chunk;
  if (so->converged) ctx->coef_iter_hint = so->iterations;
  return fst;
}

int solve_nodes_coef(ov_ctx* ctx, const double2* b_soa, int nsrc, int ns, const std::vector<double2>& zh,
                     const std::vector<double2>& ch, int chunk, double2* X, double2* sums, const ov_solve_opts& o,
                     SolveOut* so, cudaStream_t s, const std::function<int(int, int)>& per_chunk) {
  if (o.mode == OV_MODE_F32X2) {
    const int st = ensure_links_df(ctx, s);
    if (st != OV_OK) return st;
    return nodes_coef<DF>(ctx, b_soa, nsrc, ns, zh, ch, chunk, X, sums, o, so, s, per_chunk);
  }
  return nodes_coef<double>(ctx, b_soa, nsrc, ns, zh, ch, chunk, X, sums, o, so, s, per_chunk);
}

int solve_sign_2pass(ov_ctx* ctx, const double2* b_soa, double2* out_soa, int nsrc, const ov_solve_opts& o,
                     SolveOut* so, cudaStream_t s) {
  if (o.mode == OV_MODE_F32X2) {
    const int st = ensure_links_df(ctx, s);
    if (st != OV_OK) return st;
    return solve_sign_coef<DF>(ctx, b_soa, out_soa, nsrc, o, so, s);
  }
  return solve_sign_coef<double>(ctx, b_soa, out_soa, nsrc, o, so, s);
}

// OV_MODE_MIXED.
//  Phase A (FP32): one Lanczos process per source with FP32 vectors and FP64 scalars;
//    every node's LDL^T recurrence runs on scalars (for the stopping test) and the basis
//    is kept (slot i = U_i; GB300's HBM holds hundreds of basis vectors per source).  The
//    host forms each node's FOM coefficients (z_j - T_k)^-1 e_1 ||b|| and a combination
//    kernel writes y_j = sum_i w_ij U_i in FP64.
//  Rounds: FP64 true residuals r_j = b - (z_j - H_W) y_j (FP64 stencil fused) for every
//    node and source; if any exceeds tol ||b||, one batched FP32 correction solve over
//    all nodes x sources (each right-hand side its own Lanczos process with its single
//    shift z_j, per-RHS tolerance, converged ones leave the batch), y_j += e_j in FP64.
//  Finally the FP64 weighted sum s = c0 b + sum_j c_j y_j.
int solve_sign_mixed(ov_ctx* ctx, const double2* b_soa, double2* out_soa, int nsrc, const ov_solve_opts& o,
                     SolveOut* so, cudaStream_t s) {
  NvtxRange nvtx_("solve: mixed precision");
  const int nq = (int)ctx->z.size();
  const size_t n12 = (size_t)12 * ctx->g.V;
  const int nrhs = nsrc * nq;
  int st = OV_OK;
  cudaError_t e;
  // basis capacity: at most 600 vectors per source, a third of device memory and max_iter
  size_t freeb = 0, totalb = 0;
  cudaMemGetInfo(&freeb, &totalb);
  const size_t per_slot = (size_t)nsrc * n12 * sizeof(float2);
  long long cap = (long long)(0.33 * (double)totalb / (double)per_slot) - 2;
  const int kcap = (int)std::max<long long>(8, std::min<long long>(std::min<long long>(cap, 600), o.max_iter));
  double launches = 0.0;

  // ---- phase A
  std::vector<double2> zh((size_t)nsrc * nq), ch((size_t)nsrc * nq);
  for (int r = 0; r < nsrc; ++r)
    for (int j = 0; j < nq; ++j) {
      zh[(size_t)r * nq + j] = ctx->z[j];
      ch[(size_t)r * nq + j] = ctx->c[j];
    }
  SolveWs<float> wA;
  st = setup_ws<float>(ctx, nsrc, nq, false, false, true, kcap, &wA, "mxA", kcap + 2, false);
  if (st != OV_OK) return st;
  const double tolA = std::max(o.tol, 1e-6);
  st = init_solve<float>(ctx, wA, b_soa, nsrc, nq, zh, ch, make_double2(0, 0), tolA, kcap, s, 0);
  if (st != OV_OK) return st;
  launches += 1;
  st = run_iterations<float>(ctx, wA, nsrc, nq, 4, kcap, o, s, &launches);
  if (st != OV_OK) return st;
  SolveOut soA;
  const int fa = finish_solve<float>(ctx, wA, nsrc, nq, zh, ch, &soA, s);
  if (fa == OV_ERR_BREAKDOWN) return fa;
  std::vector<SrcState> S(nsrc);
  std::vector<double> ha((size_t)nsrc * kcap), hb((size_t)nsrc * kcap);
  e = cudaMemcpyAsync(S.data(), wA.a.src, sizeof(SrcState) * nsrc, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ha.data(), wA.a.hist_a, sizeof(double) * ha.size(), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hb.data(), wA.a.hist_b, sizeof(double) * hb.size(), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return ctx_cuda(ctx, e, "read phase-A history");
  int kmax = 1;
  std::vector<int> kr(nsrc);
  for (int r = 0; r < nsrc; ++r) {
    kr[r] = std::max(0, S[r].iter - 1);
    kmax = std::max(kmax, kr[r]);
  }
  // w_ij = [(z_j - T_k)^-1 e_1 ||b||]_i / ||U_i||  (the basis is stored unnormalised)
  std::vector<float2> W((size_t)nsrc * nq * kmax, make_float2(0.f, 0.f));
  std::vector<std::complex<double>> dd, ll, zt, yy;
  for (int r = 0; r < nsrc; ++r) {
    const int k = kr[r];
    if (k < 1) continue;
    const double* al = ha.data() + (size_t)r * kcap;
    const double* be = hb.data() + (size_t)r * kcap;
    dd.assign(k, 0.0);
    ll.assign(k, 0.0);
    zt.assign(k, 0.0);
    yy.assign(k, 0.0);
    for (int j = 0; j < nq; ++j) {
      const std::complex<double> zj(ctx->z[j].x, ctx->z[j].y);
      std::complex<double> om = S[r].bnorm;
      for (int i = 0; i < k; ++i) {
        if (i == 0) {
          dd[0] = zj - al[0];
        } else {
          dd[i] = zj - al[i] - be[i - 1] * be[i - 1] / dd[i - 1];
          om = -ll[i - 1] * om;
        }
        ll[i] = -be[i] / dd[i];
        zt[i] = om / dd[i];
      }
      yy[k - 1] = zt[k - 1];
      for (int i = k - 2; i >= 0; --i) yy[i] = zt[i] - ll[i] * yy[i + 1];
      for (int i = 0; i < k; ++i) {
        const double ni = (i == 0) ? S[r].bnorm : be[i - 1];
        const std::complex<double> w = yy[i] / ni;
        W[((size_t)r * nq + j) * kmax + i] = make_float2((float)w.real(), (float)w.imag());
      }
    }
  }
  float2* Wd = (float2*)ws_get(ctx, "mx.W", sizeof(float2) * W.size(), &st);
  int* krd = (int*)ws_get(ctx, "mx.kr", sizeof(int) * nsrc, &st);
  double2* Y = (double2*)ws_get(ctx, "mx.Y", sizeof(double2) * n12 * nrhs, &st);
  double2* R = (double2*)ws_get(ctx, "mx.R", sizeof(double2) * n12 * nrhs, &st);
  double* part = (double*)ws_get(ctx, "mx.part", sizeof(double) * (size_t)residual64_partials(ctx) * nrhs, &st);
  double* rn2 = (double*)ws_get(ctx, "mx.rn2", sizeof(double) * nrhs, &st);
  double2* zd = (double2*)ws_get(ctx, "mx.z", sizeof(double2) * nq, &st);
  double2* cd = (double2*)ws_get(ctx, "mx.c", sizeof(double2) * nq, &st);
  double* told = (double*)ws_get(ctx, "mx.tol", sizeof(double) * nrhs, &st);
  if (st != OV_OK) return st;
  e = cudaMemcpyAsync(Wd, W.data(), sizeof(float2) * W.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(krd, kr.data(), sizeof(int) * nsrc, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(zd, ctx->z.data(), sizeof(double2) * nq, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(cd, ctx->c.data(), sizeof(double2) * nq, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return ctx_cuda(ctx, e, "phase-A coefficients");
  st = launch_basis_combine(ctx, wA.a.ring, kcap + 2, Wd, kmax, krd, Y, nsrc, nq, s);
  if (st != OV_OK) return st;
  launches += 1;

  // ---- FP64 residuals and FP32 corrections
  std::vector<double> rn(nrhs), tol_h(nrhs);
  const int max_rounds = 4;
  so->refine_rounds = 0;
  so->inner_iterations = 0;
  so->node_updates = soA.node_updates;
  double maxres = 0.0, bound = 0.0;
  std::string hist;
  for (int round = 0;; ++round) {
    st = launch_residual64(ctx, Y, b_soa, zd, R, part, rn2, nsrc, nq, s);
    if (st != OV_OK) return st;
    launches += 2;
    e = cudaMemcpyAsync(rn.data(), rn2, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return ctx_cuda(ctx, e, "read residual norms");
    maxres = 0.0;
    bound = 0.0;
    bool bad = false;
    for (int r = 0; r < nsrc; ++r) {
      const double bn = S[r].bnorm > 0 ? S[r].bnorm : 1.0;
      double bd = 0.0;
      for (int j = 0; j < nq; ++j) {
        const double res = std::sqrt(rn[(size_t)r * nq + j]) / bn;
        if (!std::isfinite(res)) bad = true;
        maxres = std::max(maxres, res);
        bd += std::hypot(ctx->c[j].x, ctx->c[j].y) * res / std::fabs(ctx->z[j].y);
        // FP32 corrections reach ~1e-6 relative: ask for that, or what tol needs
        tol_h[(size_t)r * nq + j] = res <= o.tol ? 1e30 : std::max(0.3 * o.tol / res, 2e-6);
      }
      bound = std::max(bound, bd);
    }
    if (bad) return ctx_fail(ctx, OV_ERR_BREAKDOWN, "non-finite residual in the mixed-precision solve");
    char buf[64];
    snprintf(buf, sizeof buf, "%s%.3g", round ? ", " : "", maxres);
    hist += buf;
    if (maxres <= o.tol || round >= max_rounds) break;
    ++so->refine_rounds;
    std::vector<double2> zc(nrhs), cc(nrhs, make_double2(1.0, 0.0));
    for (int r = 0; r < nsrc; ++r)
      for (int j = 0; j < nq; ++j) zc[(size_t)r * nq + j] = ctx->z[j];
    SolveWs<float> wC;
    st = setup_ws<float>(ctx, nrhs, 1, true, false, false, o.max_iter, &wC, "mxC");
    if (st != OV_OK) return st;
    e = cudaMemcpyAsync(told, tol_h.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return ctx_cuda(ctx, e, "copy tolerances");
    wC.a.tol_src = told;
    st = init_solve<float>(ctx, wC, R, nrhs, 1, zc, cc, make_double2(0, 0), 0.5, o.max_iter, s, 1);
    if (st != OV_OK) return st;
    launches += 2;
    st = run_iterations<float>(ctx, wC, nrhs, 1, 5, o.max_iter, o, s, &launches);
    if (st != OV_OK) return st;
    SolveOut soC;
    const int fc = finish_solve<float>(ctx, wC, nrhs, 1, zc, cc, &soC, s);
    if (fc == OV_ERR_BREAKDOWN) return fc;
    so->inner_iterations += soC.iterations;
    so->node_updates += soC.node_updates;
    st = launch_accumulate(ctx, Y, wC.a.x, n12 * nrhs, s);
    if (st != OV_OK) return st;
    launches += 1;
  }
  st = launch_weighted_sum(ctx, Y, b_soa, cd, ctx->c0, out_soa, nsrc, nq, s);
  if (st != OV_OK) return st;
  so->iterations = soA.iterations;
  so->max_residual = maxres;
  so->error_bound = bound;
  so->converged = maxres <= o.tol;
  so->launches = launches + 3;
  if (!so->converged)
    return ctx_fail(ctx, OV_ERR_NOT_CONVERGED,
                    "mixed-precision refinement did not reach tol; max relative FP64 residual after phase A and "
                    "each correction round: " + hist);
  return OV_OK;
}

// Lanczos tridiagonal of H_W (squared = 0) or H_W^2 (squared = 1) from a fixed
// pseudo-random start vector; returns alpha[0..k), beta[0..k).
namespace {
__global__ void start_vector_kernel(double2* v, size_t n) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    // splitmix64 of the element index: a fixed, reproducible start vector
    unsigned long long x = t + 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    x ^= x >> 31;
    const double a = (double)(x & 0xFFFFFFFFull) / 4294967296.0 - 0.5;
    const double b = (double)(x >> 32) / 4294967296.0 - 0.5;
    v[t] = make_double2(a, b);
  }
}
}  // namespace

int lanczos_tridiag(ov_ctx* ctx, int steps, int squared, std::vector<double>& alpha, std::vector<double>& beta,
                    cudaStream_t s) {
  SolveWs<double> w;
  int st = setup_ws<double>(ctx, 1, 0, false, false, true, steps, &w, "lz");
  if (st != OV_OK) return st;
  const size_t n12 = (size_t)12 * ctx->g.V;
  double2* b = (double2*)ws_get(ctx, "lz.b", sizeof(double2) * n12, &st);
  double2* tmp = squared ? (double2*)ws_get(ctx, "lz.tmp", sizeof(double2) * n12, &st) : nullptr;
  double2* tmp2 = squared ? (double2*)ws_get(ctx, "lz.tmp2", sizeof(double2) * n12, &st) : nullptr;
  if (st != OV_OK) return st;
  start_vector_kernel<<<256, 256, 0, s>>>(b, n12);
  std::vector<double2> none;
  st = init_solve<double>(ctx, w, b, 1, 0, none, none, make_double2(0, 0), 0.0, steps, s);
  if (st != OV_OK) return st;
  for (int it = 0; it < steps; ++it) {
    SolveArgs<double> a = w.a;
    if (squared) {
      // H^2: apply H twice to U_i (ring slot i % 3, i = it + 1); K1 reads the result
      const double2* Ui = w.a.ring + (size_t)((it + 1) % 3) * n12;
      st = launch_hw64(ctx, Ui, tmp, 1, s);
      if (st == OV_OK) st = launch_hw64(ctx, tmp, tmp2, 1, s);
      if (st != OV_OK) return st;
      a.stencil = tmp2;
    }
    lanczos_hw_kernel<double><<<k1_grid(w, 1), NT1, 0, s>>>(a);
    lanczos_update_kernel<double><<<dim3(w.nblk2u, 1), NT2, 0, s>>>(a);
  }
  OV_CHECK_LAUNCH(ctx, "lanczos bound kernels");
  SrcState S;
  cudaError_t e = cudaMemcpyAsync(&S, w.a.src, sizeof(S), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return ctx_cuda(ctx, e, "lanczos state");
  const int k = S.iter - 1;
  if (S.status == OV_ERR_BREAKDOWN || k < 1) return ctx_fail(ctx, OV_ERR_BREAKDOWN, "Lanczos bound breakdown");
  alpha.resize(k);
  beta.resize(k);
  e = cudaMemcpy(alpha.data(), w.a.hist_a, sizeof(double) * k, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(beta.data(), w.a.hist_b, sizeof(double) * k, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return ctx_cuda(ctx, e, "lanczos history");
  return OV_OK;
}
