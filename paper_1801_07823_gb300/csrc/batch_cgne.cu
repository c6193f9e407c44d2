// Coarsest-level CGNE for a batch of right-hand sides in one persistent
// cooperative kernel (batched solves of a mixed-precision hierarchy).
//
// Same iteration as the single-RHS kernel (cgne.cu) for every right-hand side,
// each with its own alpha, beta, stopping test and iteration count; a
// right-hand side that has stopped is no longer updated while the others go
// on.
//
// A stencil application is a batched block contraction: for every coarse site
// X, out[X] (nc x K) = sum_d Z[X][d] (nc x nc) v[nb(X, d)] (nc x K), where Z is
// the forward stencil (A v) or the adjoint stencil (A^dag v).  Both are FP32
// copies in which each (site, direction) block is one contiguous column-major
// nc x nc array; the adjoint copy holds Y[nb(X, d)][opp(d)]^dag explicitly, so
// the two products read their blocks the same way.  A CTA owns the sites
// X = blockIdx + gridDim * m (m = 0, 1, ...).  One thread copies each
// (block, neighbour vector) pair into shared memory with bulk asynchronous
// copies that complete on an mbarrier, a few stages ahead of the threads that
// use them.  A thread owns one row of a site for four right-hand sides and sums
// the five blocks' columns in order, so an output is computed the same way for
// every batch width K.
//
// Stencil products and their sums are FP32 (the coarsest solve of a batch is a
// 0.2-tolerance preconditioner); iterates, residuals and Krylov scalars stay
// FP64, and FP32 copies of r and p feed the stencil.  Norms are summed per site
// over its rows in a fixed tree, per CTA over its sites in order, and over the
// CTAs in a fixed order with one CTA per SM for every K, so a right-hand side's
// scalars, and hence its result, do not depend on its batch-mates.
//
// Layout inside the kernel: right-hand-side-minor.  FP64 vectors hold element
// (dof, rhs) at dof * K + rhs; the FP32 copies that feed the stencil are
// planar per dof (K real parts, then K imaginary parts), so a neighbour's
// nc x K block is contiguous and two right-hand sides' parts form the operand
// pairs of one paired FP32 FMA (__ffma2_rn, each lane rounded like fmaf).
#include <string>

#include "sw_internal.h"

namespace {

constexpr long kSpinLimit = 1L << 24;      // grid barrier polls
constexpr long kCopySpinLimit = 1L << 22;  // mbarrier polls per stage
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

// Tiling of one batch width: kS sites in flight per CTA, kStages stages of
// kS (block, vector) pairs each in dynamic shared memory.
template <int NC, int K>
struct Tile {
  static constexpr int kGroups = K / 4;              // four right-hand sides per thread
  // rows per thread: two when one row per thread would need the whole CTA for one site
  static constexpr int kR = NC * kGroups > kThreads / 2 ? 2 : 1;
  static constexpr int kRowsT = NC / kR;             // row slots per site
  static constexpr int kTps = kRowsT * kGroups;      // threads per site
  static constexpr int kSiteF2 = NC * NC + NC * K;   // float2 per site and stage
  static constexpr int kSThr = kThreads / kTps;
  static constexpr int kSPair = kThreads / (4 * K);  // per-site norm tree: four threads per pair
  static constexpr int kSMem0 = (100 * 1024) / (kSiteF2 * 8);
  static constexpr int kSMem = kSMem0 > 0 ? kSMem0 : 1;
  static constexpr int kS0 = kSThr < kSMem ? kSThr : kSMem;
  static constexpr int kS = kS0 < kSPair ? kS0 : kSPair;
  static constexpr int kStageF2 = kS * kSiteF2;
  static constexpr int kStagesMem = (200 * 1024) / (kStageF2 * 8);
  static constexpr int kStages = kStagesMem < 4 ? kStagesMem : 4;
  static constexpr int kSmem = kStages * kStageF2 * 8;
  static_assert(NC % 4 == 0 && K % 4 == 0 && NC % kR == 0, "rows and right-hand sides in fours");
  static_assert(kTps <= kThreads && kS >= 1 && kStages >= 2, "tile does not fit");
  static_assert(kS * K * 4 <= kThreads, "per-site norm tree needs four threads per pair");
};

__device__ __forceinline__ int nbr(int X, int d, int E0, int E1) {
  int X0 = X % E0, X1 = X / E0;
  if (d == 1) X0 = (X0 + 1 == E0) ? 0 : X0 + 1;
  if (d == 2) X0 = (X0 == 0) ? E0 - 1 : X0 - 1;
  if (d == 3) X1 = (X1 + 1 == E1) ? 0 : X1 + 1;
  if (d == 4) X1 = (X1 == 0) ? E1 - 1 : X1 - 1;
  return X0 + E0 * X1;
}
__device__ __forceinline__ int opp(int d) {
  return d == 0 ? 0 : (d == 1 ? 2 : (d == 2 ? 1 : (d == 3 ? 4 : 3)));
}

// ------------------------------------------------ mbarrier and bulk copies
__device__ __forceinline__ unsigned su32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect(unsigned long long* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long* b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(su32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase with the given parity; false when it gave up.
__device__ bool mbar_wait(unsigned long long* b, unsigned parity) {
  for (long k = 0; k < kCopySpinLimit; ++k)
    if (mbar_test(b, parity)) return true;
  return false;
}
// Global -> shared bulk copy (16-byte aligned addresses, size a multiple of 16)
// completing as transaction bytes on mbarrier b.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes,
                                          unsigned long long* b) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(su32(dst)),
      "l"(src), "r"(bytes), "r"(su32(b))
      : "memory");
}
__device__ __forceinline__ void fence_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}
__device__ __forceinline__ void fence_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

struct BatchArgs {
  const float2* Yf;        // forward stencil blocks (FP32, column-major per (site, direction))
  const float2* Yd;        // adjoint stencil blocks, same layout
  const double2* const* b; // [K] right-hand sides (entries beyond nb unused)
  double2* const* xout;    // [K] solutions
  double2* X;              // [n][K] FP64 iterates
  double2* R;              // [n][K] FP64 residuals
  double2* P;              // [n][K] FP64 directions
  float* Rf;               // [n][2][K] FP32 copies read by the stencil (planar per dof)
  float* Pf;
  double* partials;        // [2][K][gridDim.x]
  unsigned* bar;           // grid barrier state (2 words)
  int* status;             // [0] wait timeout or misaligned buffer, [1] non-finite,
                           // [2 + r] iterations
  int nb, E0, E1, maxit;
  double tol;
};

__device__ bool grid_barrier(unsigned* bar, int* status) {
  __shared__ int ok;
  // this thread's generic writes of the phase before the next phase's bulk reads
  fence_async_global();
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    unsigned g = *gen;
    __threadfence();
    unsigned arrived = atomicAdd(bar, 1u);
    if (arrived == gridDim.x - 1) {
      bar[0] = 0u;
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long spins = 0;
      while (*gen == g) {
        if (++spins > kSpinLimit) {
          atomicExch(status, 1);
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
    ok = *((volatile int*)status) == 0;
  }
  __syncthreads();
  return ok;
}

// Per-CTA partial sums of K values (thread-owned v[r]) into part[r * G + blockIdx].
template <int K>
__device__ void cta_partials(const double* v, double (*red)[kWarps], double* part) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int r = 0; r < K; ++r) {
    double s = v[r];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) red[r][w] = s;
  }
  __syncthreads();
  if (threadIdx.x < K) {
    double s = 0.0;
    for (int q = 0; q < kWarps; ++q) s += red[threadIdx.x][q];
    part[threadIdx.x * gridDim.x + blockIdx.x] = s;
    __threadfence();
  }
}
// All K grid sums, same order in every CTA; result in out[K] (shared).
template <int K>
__device__ void grid_sums(const double* part, double* out) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int G = gridDim.x;
  for (int r = w; r < K; r += kWarps) {
    // all loads first, then the adds in the order of the lane-strided loop
    const double* pr = part + r * G;
    double v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = lane + 32 * k < G ? __ldcg(pr + lane + 32 * k) : 0.0;
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (lane + 32 * k < G) s += v[k];
    for (int q = lane + 256; q < G; q += 32) s += __ldcg(pr + q);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[r] = s;
  }
  __syncthreads();
}

// re += y v and im += y v for two right-hand sides at once: re and im hold the
// real (imaginary) parts of the two sums, vr and vi the two right-hand sides'
// real and imaginary parts.  Each lane runs fmaf(y.x, vx, .), fmaf(-y.y, vy, .)
// for the real part and fmaf(y.x, vy, .), fmaf(y.y, vx, .) for the imaginary
// part, the same sequence for every row and right-hand side.
__device__ __forceinline__ void cmac2(float2& re, float2& im, float2 y, float2 vr, float2 vi) {
  const float2 yx = make_float2(y.x, y.x), yy = make_float2(y.y, y.y);
  const float2 nyy = make_float2(-y.y, -y.y);
  re = __ffma2_rn(yx, vr, re);
  re = __ffma2_rn(nyy, vi, re);
  im = __ffma2_rn(yx, vi, im);
  im = __ffma2_rn(yy, vr, im);
}

enum { kModeInit = 0, kModeXR = 1, kModeP = 2 };

// Shared state of the kernel beyond the stage buffers.
template <int NC, int K>
struct Smem {
  unsigned long long full[Tile<NC, K>::kStages];
  double sq[Tile<NC, K>::kS * K * NC];  // per-row squared norms of the sites in flight
  double siteval[Tile<NC, K>::kS * K];  // per-site sums
  double cta_sum[K];                    // this CTA's sum over its sites, in order
  double red[K][kWarps];
  double sum[K], rr[K], stop[K], coef[K];
  int state[K];                         // 0 active, 1 stopped, 2 non-finite
  int iters[K];
  int any;
  int copy_timeout;
};

// One stencil application over this CTA's sites fused with the update of its
// mode, leaving this CTA's per-right-hand-side norm sum in sm.cta_sum:
//   kModeInit: p = A^dag r (all right-hand sides), |p|^2
//   kModeXR:   w = A p; x += alpha p; r -= alpha w (active ones), |r|^2
//   kModeP:    p = A^dag r + beta p (active ones), |p|^2
// qbase counts the stages this CTA has used so far (buffer and mbarrier parity).
template <int NC, int K, int MODE>
__device__ void stencil_phase(const BatchArgs& a, float2* stage, Smem<NC, K>& sm,
                              unsigned& qbase) {
  using T = Tile<NC, K>;
  constexpr int R = T::kR;
  const int t = threadIdx.x;
  const int s = t / T::kTps, w = t - s * T::kTps;
  const int g = w % T::kGroups, i = w / T::kGroups;  // rows i + k * kRowsT, k < R
  const bool act = s < T::kS;
  const int G = gridDim.x, cta = blockIdx.x;
  const int nsites = a.E0 * a.E1;
  const int nmine = cta < nsites ? (nsites - 1 - cta) / G + 1 : 0;
  const int nchunks = (nmine + T::kS - 1) / T::kS;
  const int nst = nchunks * 5;
  const float2* Z = MODE == kModeXR ? a.Yf : a.Yd;
  const float* V = MODE == kModeXR ? a.Pf : a.Rf;

  // stage q of this phase: chunk q / 5 of this CTA's sites, direction q % 5
  auto issue = [&](int q) {
    const int c = q / 5, d = q - c * 5;
    const unsigned Q = qbase + q;
    float2* buf = stage + (size_t)(Q % T::kStages) * T::kStageF2;
    unsigned long long* mb = sm.full + Q % T::kStages;
    const int nv = min(T::kS, nmine - c * T::kS);
    mbar_arrive_expect(mb, (unsigned)(nv * T::kSiteF2 * 8));
    for (int ss = 0; ss < nv; ++ss) {
      const int Xs = cta + G * (c * T::kS + ss);
      const int nbs = nbr(Xs, d, a.E0, a.E1);
      bulk_load(buf + ss * NC * NC, Z + ((size_t)Xs * 5 + d) * NC * NC, NC * NC * 8, mb);
      bulk_load(buf + T::kS * NC * NC + ss * NC * K, V + (size_t)nbs * NC * 2 * K, NC * K * 8,
                mb);
    }
  };

  if (t == 0) {
    fence_async_global();  // other CTAs' writes, acquired at the grid barrier, before bulk reads
    const int pre = nst < T::kStages ? nst : T::kStages;
    for (int q = 0; q < pre; ++q) issue(q);
  }
  if (t < K) sm.cta_sum[t] = 0.0;
  for (int c = 0; c < nchunks; ++c) {
    const int m = c * T::kS + s;
    const bool valid = act && m < nmine;
    const int X = cta + G * m;
    // real / imaginary parts of the sums of right-hand sides (4g, 4g+1) and (4g+2, 4g+3)
    float2 re01[R], re23[R], im01[R], im23[R];
#pragma unroll
    for (int k = 0; k < R; ++k)
      re01[k] = re23[k] = im01[k] = im23[k] = make_float2(0.f, 0.f);
    for (int d = 0; d < 5; ++d) {
      const int q = c * 5 + d;
      const unsigned Q = qbase + q;
      const int bi = (int)(Q % T::kStages);
      if (!mbar_wait(sm.full + bi, (Q / T::kStages) & 1u)) {
        sm.copy_timeout = 1;
        atomicExch(a.status, 1);
      }
      if (valid) {
        const float2* Ys = stage + (size_t)bi * T::kStageF2 + s * NC * NC + i;
        const float* Vs = reinterpret_cast<const float*>(stage + (size_t)bi * T::kStageF2 +
                                                         T::kS * NC * NC + s * NC * K) +
                          4 * g;
#pragma unroll 4
        for (int j = 0; j < NC; ++j) {
          const float4 vr = *reinterpret_cast<const float4*>(Vs + j * 2 * K);
          const float4 vi = *reinterpret_cast<const float4*>(Vs + j * 2 * K + K);
#pragma unroll
          for (int k = 0; k < R; ++k) {
            const float2 y = Ys[j * NC + k * T::kRowsT];
            cmac2(re01[k], im01[k], y, make_float2(vr.x, vr.y), make_float2(vi.x, vi.y));
            cmac2(re23[k], im23[k], y, make_float2(vr.z, vr.w), make_float2(vi.z, vi.w));
          }
        }
      }
      __syncthreads();  // every thread is done with this buffer
      if (t == 0 && q + T::kStages < nst) {
        fence_async_shared();
        issue(q + T::kStages);
      }
    }
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int row = i + k * T::kRowsT;
      const float accx[4] = {re01[k].x, re01[k].y, re23[k].x, re23[k].y};
      const float accy[4] = {im01[k].x, im01[k].y, im23[k].x, im23[k].y};
      double q2[4] = {0.0, 0.0, 0.0, 0.0};
      if (valid) {
        const size_t e = ((size_t)X * NC + row) * K + 4 * g;          // FP64, interleaved
        float* vf = (MODE == kModeXR ? a.Rf : a.Pf) + ((size_t)X * NC + row) * 2 * K + 4 * g;
        float fr[4], fi[4];
        if (MODE == kModeInit) {
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const double2 pv = make_double2((double)accx[u], (double)accy[u]);
            a.P[e + u] = pv;
            fr[u] = accx[u];
            fi[u] = accy[u];
            q2[u] = fma(pv.x, pv.x, pv.y * pv.y);
          }
        } else if (MODE == kModeXR) {
          double2 pv[4], xv[4], rv[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {  // all loads first
            pv[u] = __ldcg(a.P + e + u);
            xv[u] = __ldcg(a.X + e + u);
            rv[u] = __ldcg(a.R + e + u);
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int r = 4 * g + u;
            if (sm.state[r] == 0) {
              const double al = sm.coef[r];
              xv[u].x = fma(al, pv[u].x, xv[u].x);
              xv[u].y = fma(al, pv[u].y, xv[u].y);
              rv[u].x = fma(-al, (double)accx[u], rv[u].x);
              rv[u].y = fma(-al, (double)accy[u], rv[u].y);
              a.X[e + u] = xv[u];
              a.R[e + u] = rv[u];
              q2[u] = fma(rv[u].x, rv[u].x, rv[u].y * rv[u].y);
            }
            // a stopped right-hand side keeps r, so this rewrites the same FP32 value
            fr[u] = (float)rv[u].x;
            fi[u] = (float)rv[u].y;
          }
        } else {
          double2 pv[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) pv[u] = __ldcg(a.P + e + u);
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int r = 4 * g + u;
            if (sm.state[r] == 0) {
              const double be = sm.coef[r];
              pv[u].x = fma(be, pv[u].x, (double)accx[u]);
              pv[u].y = fma(be, pv[u].y, (double)accy[u]);
              a.P[e + u] = pv[u];
              q2[u] = fma(pv[u].x, pv[u].x, pv[u].y * pv[u].y);
            }
            fr[u] = (float)pv[u].x;
            fi[u] = (float)pv[u].y;
          }
        }
        *reinterpret_cast<float4*>(vf) = make_float4(fr[0], fr[1], fr[2], fr[3]);
        *reinterpret_cast<float4*>(vf + K) = make_float4(fi[0], fi[1], fi[2], fi[3]);
      }
      // per-site sums over rows: four threads per (site, rhs) pair, NC/4 rows each
      if (act) {
#pragma unroll
        for (int u = 0; u < 4; ++u) sm.sq[(s * K + 4 * g + u) * NC + row] = q2[u];
      }
    }
    __syncthreads();
    {
      const int pair = t >> 2, part = t & 3;
      double v = 0.0;
      if (pair < T::kS * K) {
        const double* src = sm.sq + pair * NC + part * (NC / 4);
        for (int k = 0; k < NC / 4; ++k) v += src[k];
      }
      v += __shfl_xor_sync(0xffffffffu, v, 1);
      v += __shfl_xor_sync(0xffffffffu, v, 2);
      if (part == 0 && pair < T::kS * K) sm.siteval[pair] = v;
    }
    __syncthreads();
    if (t < K) {
      for (int ss = 0; ss < T::kS; ++ss)
        if (c * T::kS + ss < nmine) sm.cta_sum[t] += sm.siteval[ss * K + t];
    }
  }
  qbase += (unsigned)nst;
}

// Thread 0 waits once more for the last stages of every buffer after a copy
// wait gave up, so that no copy is in flight when the CTA exits.
template <int NC, int K>
__device__ void drain_copies(Smem<NC, K>& sm, unsigned qbase) {
  using T = Tile<NC, K>;
  __syncthreads();
  if (threadIdx.x == 0 && sm.copy_timeout) {
    for (unsigned Q = qbase >= (unsigned)T::kStages ? qbase - T::kStages : 0u; Q < qbase; ++Q)
      mbar_wait(sm.full + Q % T::kStages, (Q / T::kStages) & 1u);
  }
}

template <int NC, int K>
__device__ void publish(Smem<NC, K>& sm, double* part) {
  if (threadIdx.x < K) {
    part[threadIdx.x * gridDim.x + blockIdx.x] = sm.cta_sum[threadIdx.x];
    __threadfence();
  }
}

template <int NC, int K>
__global__ void __launch_bounds__(kThreads, 1) k_cgne_batch(BatchArgs a) {
  extern __shared__ __align__(128) float2 stage[];
  __shared__ Smem<NC, K> sm;
  const long n = (long)a.E0 * a.E1 * NC;
  const long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long nthr = (long)gridDim.x * blockDim.x;
  unsigned qbase = 0;
  double nrm[K];

  if (threadIdx.x == 0) {
    for (int k = 0; k < Tile<NC, K>::kStages; ++k) mbar_init(sm.full + k, 1);
    sm.copy_timeout = 0;
    fence_mbar_init();
    fence_async_shared();
    // bulk copies need 16-byte aligned ends: refuse (status, then every CTA
    // returns at the first grid barrier, before any copy) rather than issue one
    const size_t gl = (size_t)a.Yf | (size_t)a.Yd | (size_t)a.Rf | (size_t)a.Pf;
    if (((su32(stage) & 15u) | (unsigned)(gl & 15)) != 0) atomicExch(a.status, 1);
  }
  // gather: X = 0, R = b, Rf = float(b), ||r||^2 per right-hand side
#pragma unroll
  for (int r = 0; r < K; ++r) nrm[r] = 0.0;
  for (long dof = tid; dof < n; dof += nthr) {
#pragma unroll
    for (int r = 0; r < K; ++r) {
      long e = dof * K + r;
      double2 v = r < a.nb ? a.b[r][dof] : make_double2(0.0, 0.0);
      a.X[e] = make_double2(0.0, 0.0);
      a.R[e] = v;
      a.Rf[dof * 2 * K + r] = (float)v.x;
      a.Rf[dof * 2 * K + K + r] = (float)v.y;
      nrm[r] = fma(v.x, v.x, fma(v.y, v.y, nrm[r]));
    }
  }
  int ph = 0;
  cta_partials<K>(nrm, sm.red, a.partials + ph * K * gridDim.x);
  if (!grid_barrier(a.bar, a.status)) return;
  grid_sums<K>(a.partials + ph * K * gridDim.x, sm.sum);
  if (threadIdx.x < K) {
    int r = threadIdx.x;
    double rr0 = sm.sum[r];
    sm.rr[r] = rr0;
    sm.stop[r] = a.tol * sqrt(rr0);
    sm.iters[r] = 0;
    sm.state[r] = !isfinite(rr0) ? 2 : ((a.maxit <= 0 || !(sqrt(rr0) > sm.stop[r])) ? 1 : 0);
  }
  __syncthreads();
  ph ^= 1;
  // P = A^dag R, ||p||^2
  stencil_phase<NC, K, kModeInit>(a, stage, sm, qbase);
  publish<NC, K>(sm, a.partials + ph * K * gridDim.x);
  if (!grid_barrier(a.bar, a.status)) return drain_copies<NC, K>(sm, qbase);
  grid_sums<K>(a.partials + ph * K * gridDim.x, sm.sum);
  if (threadIdx.x < K) sm.coef[threadIdx.x] = sm.rr[threadIdx.x] / sm.sum[threadIdx.x];  // alpha
  if (threadIdx.x == 0) {
    int any = 0;
    for (int r = 0; r < K; ++r) any |= sm.state[r] == 0;
    sm.any = any;
  }
  __syncthreads();
  ph ^= 1;
  while (sm.any) {
    // w = A p; x += alpha p; r -= alpha w (right-hand sides still active)
    stencil_phase<NC, K, kModeXR>(a, stage, sm, qbase);
    publish<NC, K>(sm, a.partials + ph * K * gridDim.x);
    if (!grid_barrier(a.bar, a.status)) return drain_copies<NC, K>(sm, qbase);
    grid_sums<K>(a.partials + ph * K * gridDim.x, sm.sum);
    if (threadIdx.x < K) {
      int r = threadIdx.x;
      if (sm.state[r] == 0) {
        double rr_new = sm.sum[r];
        int k = ++sm.iters[r];
        if (!isfinite(rr_new))
          sm.state[r] = 2;
        else if (!(k < a.maxit && sqrt(rr_new) > sm.stop[r]))
          sm.state[r] = 1;
        sm.coef[r] = rr_new / sm.rr[r];  // beta
        sm.rr[r] = rr_new;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int any = 0;
      for (int r = 0; r < K; ++r) any |= sm.state[r] == 0;
      sm.any = any;
    }
    __syncthreads();
    ph ^= 1;
    if (!sm.any) break;
    // p = A^dag r + beta p (right-hand sides still active)
    stencil_phase<NC, K, kModeP>(a, stage, sm, qbase);
    publish<NC, K>(sm, a.partials + ph * K * gridDim.x);
    if (!grid_barrier(a.bar, a.status)) return drain_copies<NC, K>(sm, qbase);
    grid_sums<K>(a.partials + ph * K * gridDim.x, sm.sum);
    if (threadIdx.x < K && sm.state[threadIdx.x] == 0)
      sm.coef[threadIdx.x] = sm.rr[threadIdx.x] / sm.sum[threadIdx.x];  // alpha
    __syncthreads();
    ph ^= 1;
  }
  // scatter the solutions
  for (long dof = tid; dof < n; dof += nthr)
    for (int r = 0; r < a.nb; ++r) a.xout[r][dof] = __ldcg(a.X + dof * K + r);
  if (blockIdx.x == 0 && threadIdx.x < K) {
    if (sm.state[threadIdx.x] == 2) atomicExch(a.status + 1, 1);
    a.status[2 + threadIdx.x] = sm.iters[threadIdx.x];
  }
}

// Adjoint blocks: Yd[X][d] = Y[nb(X, d)][opp(d)]^dag in FP32, one CTA per block.
__global__ void k_adjoint_f32(const double2* __restrict__ Y, float2* __restrict__ Yd, int E0,
                              int E1, int nc) {
  const int X = blockIdx.x / 5, d = blockIdx.x - 5 * (blockIdx.x / 5);
  const size_t src = ((size_t)nbr(X, d, E0, E1) * 5 + opp(d)) * nc * nc;
  const size_t dst = ((size_t)X * 5 + d) * nc * nc;
  for (int e = threadIdx.x; e < nc * nc; e += blockDim.x) {
    const int i = e % nc, j = e / nc;  // (row i, column j) of the adjoint block
    const double2 y = Y[src + (size_t)i * nc + j];  // (row j, column i) of the neighbour's block
    Yd[dst + e] = make_float2((float)y.x, (float)-y.y);
  }
}

template <int NC, int K>
bool launch_b(const BatchArgs& args, int device, cudaStream_t s, int sms_use) {
  using T = Tile<NC, K>;
  static int cached_sms[64] = {0};
  int& sms = cached_sms[device & 63];
  if (sms == 0) {
    int occ = 0, coop = 0, n = 0;
    SW_CUDA(cudaFuncSetAttribute((const void*)k_cgne_batch<NC, K>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, T::kSmem));
    SW_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cgne_batch<NC, K>, kThreads,
                                                          T::kSmem));
    SW_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, device));
    SW_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device));
    if (!coop || occ < 1)
      throw SwError{SW_ERR_CUDA, "batched CGNE cannot be launched cooperatively (occupancy " +
                                     std::to_string(occ) + ", cooperative " +
                                     std::to_string(coop) + ")"};
    sms = n;
  }
  // one CTA per SM it may use, for every batch width (see the header note)
  const int grid = sms_use < sms ? (sms_use > 0 ? sms_use : 1) : sms;
  BatchArgs a = args;
  void* params[] = {&a};
  SW_CUDA(cudaLaunchCooperativeKernel((const void*)k_cgne_batch<NC, K>, dim3(grid),
                                      dim3(kThreads), params, T::kSmem, s));
  sw_count_launch();
  return true;
}

}  // namespace

int cgne_batch_width(int nb) { return nb <= 4 ? 4 : (nb <= 8 ? 8 : 16); }

void launch_adjoint_f32(const CoarseGeom& g, const double2* Y, float2* Yd, cudaStream_t s) {
  k_adjoint_f32<<<g.E0 * g.E1 * 5, 256, 0, s>>>(Y, Yd, g.E0, g.E1, g.nc);
  SW_LAUNCH_CHECK();
}

bool launch_cgne_batch(const CoarseGeom& g, const float2* Yf, const float2* Yd, int nb,
                       const double2* const* b, double2* const* x, double2* X, double2* R,
                       double2* P, float2* Rf, float2* Pf, double* partials, unsigned* bar,
                       int* status, int maxit, double tol, int device, cudaStream_t s,
                       int sms_use) {
  if (nb < 1 || nb > 16) return false;
  SW_CUDA(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s));
  SW_CUDA(cudaMemsetAsync(status, 0, 18 * sizeof(int), s));
  BatchArgs a{Yf, Yd, b, x, X, R, P, reinterpret_cast<float*>(Rf), reinterpret_cast<float*>(Pf),
              partials, bar, status, nb, g.E0, g.E1, maxit, tol};
  int K = cgne_batch_width(nb);
#define SW_CASE(NCV)                                   \
  case NCV:                                            \
    if (K == 4) return launch_b<NCV, 4>(a, device, s, sms_use); \
    if (K == 8) return launch_b<NCV, 8>(a, device, s, sms_use); \
    return launch_b<NCV, 16>(a, device, s, sms_use);
  switch (g.nc) {
    SW_CASE(16)
    SW_CASE(24)
    SW_CASE(64)
    default: return false;
  }
#undef SW_CASE
}
