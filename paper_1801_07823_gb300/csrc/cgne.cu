// Coarsest-level CGNE (CG on the normal error, Sec. IV and Table kcycle) as
// one persistent cooperative kernel.
//
// The coarsest level is small (16^2 sites x 64 dof at 256^2) and its solve
// runs hundreds of iterations, each two stencil applications and two norms.
// As separate launches every iteration pays launch latency and a grid tail
// twice; here all CTAs stay resident, every stencil row is updated where it
// is computed, and two grid barriers per iteration order the phases:
//   P1  w = A p (row by row), x += alpha p, r -= alpha w, partial ||r||^2
//   --- barrier: every CTA adds the partials in the same order -> rr_new;
//       all CTAs take the same stopping decision
//   P2  p = A^dag r + beta p (row by row), partial ||p||^2
//   --- barrier -> pp, alpha = rr_new / pp
// Work items are (site, 8 consecutive rows), one warp each: four lanes share
// a row, each summing a quarter of the columns of all five blocks, and a
// fixed shuffle tree adds the quarters, so items need no block-wide barrier.  Items
// are dealt round-robin over CTAs first, so every SM gets the same number to
// within one.  The per-CTA partials alternate between two arrays, so a CTA
// that runs ahead never overwrites partials a slower CTA has still to read.
// A^dag is read from the same stencil storage as A (transposed access), so
// one copy of the coarsest stencil serves both and stays in L2.  Vectors
// written inside the kernel are read with ld.global.cg (L2), never from a
// possibly stale L1 line.  The iterates are those of the sequential loop;
// only the order of the partial sums differs.
//
// Barrier waits are bounded: a CTA that waits longer than kSpinLimit polls
// records an error and every CTA leaves at its next barrier; the host
// reports SW_ERR_TIMEOUT.
#include "sw_internal.h"

namespace {

constexpr long kSpinLimit = 1L << 24;    // ~0.3-1.5 s of polling

__device__ __forceinline__ void cfma(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
__device__ __forceinline__ void cfmac(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}
// Double-float ("df64") arithmetic on the FP32 pipes (Dekker 1971; Knuth's
// two-sum): a value is hi + lo with two floats, 48 significant bits.
// GB300 issues FP32 FMAs at 62x the FP64 rate, so the coarsest stencil in
// df64 costs about 48 FP32 operations per complex multiply-add instead of 4
// FP64 FMAs.
struct df2 {  // accumulator of a real number in df64
  float hi, lo;
};
__device__ __forceinline__ void df_mac(df2& acc, float ah, float al, float bh, float bl) {
  float p = ah * bh;
  float e = fmaf(ah, bh, -p);  // exact low part of ah * bh
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);         // al * bl is below the df64 precision
  float s = acc.hi + p;        // two-sum of acc.hi and p
  float z = s - acc.hi;
  float t = (acc.hi - (s - z)) + (p - z);
  acc.hi = s;
  acc.lo += t + e;
}
__device__ __forceinline__ float4 to_df(double2 v) {  // (re_hi, re_lo, im_hi, im_lo)
  float rh = (float)v.x, ih = (float)v.y;
  return make_float4(rh, (float)(v.x - (double)rh), ih, (float)(v.y - (double)ih));
}
// acc += a * b (DAG: conj(a) * b) for df64 complex a (stencil entry), b (vector)
template <bool DAG>
__device__ __forceinline__ void df_cmac(df2& re, df2& im, float4 a, float4 b) {
  if (!DAG) {
    df_mac(re, a.x, a.y, b.x, b.y);
    df_mac(re, -a.z, -a.w, b.z, b.w);
    df_mac(im, a.x, a.y, b.z, b.w);
    df_mac(im, a.z, a.w, b.x, b.y);
  } else {
    df_mac(re, a.x, a.y, b.x, b.y);
    df_mac(re, a.z, a.w, b.z, b.w);
    df_mac(im, a.x, a.y, b.z, b.w);
    df_mac(im, -a.z, -a.w, b.x, b.y);
  }
}

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

struct CgneArgs {
  const void* Y;      // complex128 stencil, or df64 float4 stencil for the DF variant
  const double2* b;
  double2* x;
  double2* r;
  double2* p;
  float4* rdf;        // DF variant: df64 copies of r and p that the stencil reads
  float4* pdf;
  double* partials;   // [2][gridDim.x], alternating by phase
  unsigned* bar;      // [0] arrival count, [1] generation
  int* status;        // [0] iterations, [1] barrier timeout, [2] non-finite residual
  int E0, E1, maxit;
  double tol;
  int stall_test;     // 1: CTA 0 never arrives at the first barrier (timeout test)
};

// Grid barrier (all CTAs co-resident: cooperative launch).  Returns false if
// this CTA gave up waiting or another CTA already did.
__device__ bool grid_barrier(unsigned* bar, int* status) {
  __shared__ int ok;
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
          atomicExch(status + 1, 1);
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
    ok = *((volatile int*)(status + 1)) == 0;
  }
  __syncthreads();
  return ok;
}

// Sum of one double per thread into partials[blockIdx.x] (fixed order).
__device__ void cta_partial(double v, double* red, double* partials) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[q];
    partials[blockIdx.x] = s;
    __threadfence();
  }
}
// Every CTA adds all partials in the same order (lane-strided, then a fixed
// shuffle tree), so all CTAs hold the same sum.
__device__ double grid_sum(const double* partials, double* bcast) {
  if (threadIdx.x < 32) {
    double s = 0.0;
    for (int q = threadIdx.x; q < (int)gridDim.x; q += 32) s += __ldcg(partials + q);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) *bcast = s;
  }
  __syncthreads();
  return *bcast;
}

constexpr int kWarps = 8;  // warps per CTA
constexpr int kRows = 8;   // rows per work item (one warp, 4 lanes per row)

// Row i of (A v)_X (dagger: (A^dag v)_X) summed by the 4 lanes of the row:
// lane q takes columns j in [q nc/4, (q+1) nc/4) of all five blocks.  Every
// lane of the row returns the same value.
template <int NC, bool DF>
__device__ __forceinline__ double2 stencil_row(const void* __restrict__ Yv,
                                               const double2* __restrict__ v,
                                               const float4* __restrict__ vdf, int X, int i,
                                               int q, int E0, int E1, bool dagger) {
  constexpr int QJ = NC / 4;  // columns per lane and direction
  const int j0 = q * QJ;
  double2 acc = make_double2(0.0, 0.0);
  df2 re{0.f, 0.f}, im{0.f, 0.f};
#pragma unroll
  for (int d = 0; d < 5; ++d) {
    const long nb = nbr(X, d, E0, E1);
    const long ybase = dagger ? ((nb * 5 + opp(d)) * NC + i) * NC + j0
                              : (((long)X * 5 + d) * NC + j0) * NC + i;
    const long ystep = dagger ? 1 : NC;
    const long xbase = nb * NC + j0;
    if (!DF) {
      const double2* Y = (const double2*)Yv + ybase;
#pragma unroll 8
      for (int t = 0; t < QJ; ++t) {
        double2 y = __ldg(Y + t * ystep);
        double2 xv = __ldcg(v + xbase + t);
        if (dagger)
          cfmac(acc, y, xv);
        else
          cfma(acc, y, xv);
      }
    } else {
      const float4* Y = (const float4*)Yv + ybase;
#pragma unroll 8
      for (int t = 0; t < QJ; ++t) {
        float4 y = __ldg(Y + t * ystep);
        float4 xv = __ldcg(vdf + xbase + t);
        if (dagger)
          df_cmac<true>(re, im, y, xv);
        else
          df_cmac<false>(re, im, y, xv);
      }
    }
  }
  if (DF) acc = make_double2((double)re.hi + (double)re.lo, (double)im.hi + (double)im.lo);
  // quarters of the row: butterfly over lanes q = 0..3 (exactly commutative)
  acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 1);
  acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 1);
  acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 2);
  acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 2);
  return acc;
}

template <int NC, bool DF>
__global__ void __launch_bounds__(kWarps * 32, 2) k_cgne(CgneArgs a) {
  __shared__ double red[32];
  __shared__ double bcast;
  __shared__ double sh_rr, sh_stop, sh_coef;
  __shared__ int sh_state;  // 0: continue, 1: converged / cap, 2: non-finite
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rr8 = lane >> 2, q = lane & 3;
  const int nsites = a.E0 * a.E1;
  const long n = (long)nsites * NC;
  const int chunks = NC / kRows;
  const int nitems = nsites * chunks;
  const int nwarps = gridDim.x * kWarps;
  const int rounds = (nitems + nwarps - 1) / nwarps;
  const long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long nthr = (long)gridDim.x * blockDim.x;

  // x = 0, r = b, ||r||^2
  double acc = 0.0;
  for (long e = tid; e < n; e += nthr) {
    double2 v = a.b[e];
    a.x[e] = make_double2(0.0, 0.0);
    a.r[e] = v;
    if (DF) a.rdf[e] = to_df(v);
    acc = fma(v.x, v.x, fma(v.y, v.y, acc));
  }
  int ph = 0;  // which partials array this phase writes
  cta_partial(acc, red, a.partials + ph * gridDim.x);
  if (a.stall_test && blockIdx.x == 0) return;  // the others' first wait must run out
  if (!grid_barrier(a.bar, a.status)) return;
  {
    double rr0 = grid_sum(a.partials + ph * gridDim.x, &bcast);
    if (threadIdx.x == 0) {
      sh_rr = rr0;
      sh_stop = a.tol * sqrt(rr0);
      sh_state = !isfinite(rr0) ? 2 : ((a.maxit <= 0 || !(sqrt(rr0) > sh_stop)) ? 1 : 0);
    }
    __syncthreads();
  }
  ph ^= 1;
  if (sh_state) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      a.status[0] = 0;
      if (sh_state == 2) a.status[2] = 1;
    }
    return;
  }
  // p = A^dag r, ||p||^2
  acc = 0.0;
  for (int rd = 0; rd < rounds; ++rd) {
    int item = rd * nwarps + warp * gridDim.x + blockIdx.x;
    if (item >= nitems) break;  // warp-uniform
    int X = item / chunks, i = (item - X * chunks) * kRows + rr8;
    double2 w = stencil_row<NC, DF>(a.Y, a.r, a.rdf, X, i, q, a.E0, a.E1, true);
    if (q == 0) {
      long e = (long)X * NC + i;
      a.p[e] = w;
      if (DF) a.pdf[e] = to_df(w);
      acc = fma(w.x, w.x, fma(w.y, w.y, acc));
    }
  }
  cta_partial(acc, red, a.partials + ph * gridDim.x);
  if (!grid_barrier(a.bar, a.status)) return;
  {
    double pp = grid_sum(a.partials + ph * gridDim.x, &bcast);
    if (threadIdx.x == 0) sh_coef = sh_rr / pp;  // alpha
    __syncthreads();
  }
  ph ^= 1;
  int k = 0;
  for (;;) {
    double alpha = sh_coef;
    // P1: w = A p; x += alpha p; r -= alpha w
    acc = 0.0;
    for (int rd = 0; rd < rounds; ++rd) {
      int item = rd * nwarps + warp * gridDim.x + blockIdx.x;
      if (item >= nitems) break;
      int X = item / chunks, i = (item - X * chunks) * kRows + rr8;
      double2 w = stencil_row<NC, DF>(a.Y, a.p, a.pdf, X, i, q, a.E0, a.E1, false);
      if (q == 0) {
        long e = (long)X * NC + i;
        double2 pv = __ldcg(a.p + e), xv = __ldcg(a.x + e), rv = __ldcg(a.r + e);
        xv.x = fma(alpha, pv.x, xv.x);
        xv.y = fma(alpha, pv.y, xv.y);
        rv.x = fma(-alpha, w.x, rv.x);
        rv.y = fma(-alpha, w.y, rv.y);
        a.x[e] = xv;
        a.r[e] = rv;
        if (DF) a.rdf[e] = to_df(rv);
        acc = fma(rv.x, rv.x, fma(rv.y, rv.y, acc));
      }
    }
    cta_partial(acc, red, a.partials + ph * gridDim.x);
    if (!grid_barrier(a.bar, a.status)) return;
    ++k;
    {
      double rr_new = grid_sum(a.partials + ph * gridDim.x, &bcast);
      if (threadIdx.x == 0) {
        if (!isfinite(rr_new))
          sh_state = 2;
        else if (!(k < a.maxit && sqrt(rr_new) > sh_stop))
          sh_state = 1;
        sh_coef = rr_new / sh_rr;  // beta
        sh_rr = rr_new;
      }
      __syncthreads();
    }
    ph ^= 1;
    if (sh_state) break;
    double beta = sh_coef;
    // P2: p = A^dag r + beta p
    acc = 0.0;
    for (int rd = 0; rd < rounds; ++rd) {
      int item = rd * nwarps + warp * gridDim.x + blockIdx.x;
      if (item >= nitems) break;
      int X = item / chunks, i = (item - X * chunks) * kRows + rr8;
      double2 w = stencil_row<NC, DF>(a.Y, a.r, a.rdf, X, i, q, a.E0, a.E1, true);
      if (q == 0) {
        long e = (long)X * NC + i;
        double2 pv = __ldcg(a.p + e);
        pv.x = fma(beta, pv.x, w.x);
        pv.y = fma(beta, pv.y, w.y);
        a.p[e] = pv;
        if (DF) a.pdf[e] = to_df(pv);
        acc = fma(pv.x, pv.x, fma(pv.y, pv.y, acc));
      }
    }
    cta_partial(acc, red, a.partials + ph * gridDim.x);
    if (!grid_barrier(a.bar, a.status)) return;
    {
      double pp = grid_sum(a.partials + ph * gridDim.x, &bcast);
      if (threadIdx.x == 0) sh_coef = sh_rr / pp;  // alpha
      __syncthreads();
    }
    ph ^= 1;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.status[0] = k;
    if (sh_state == 2) a.status[2] = 1;
  }
}

// One double-float stencil application (test access; the solver uses the
// persistent kernel); df64 sums per direction, added in FP64.
template <bool DAG>
__global__ void k_coarse_apply_df(const float4* __restrict__ Y, const double2* __restrict__ in,
                                  double2* __restrict__ out, int E0, int E1, int nc) {
  long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long)E0 * E1 * nc) return;
  int X = (int)(e / nc), i = (int)(e - (long)X * nc);
  double2 tot = make_double2(0.0, 0.0);
  for (int d = 0; d < 5; ++d) {
    int Z = nbr(X, d, E0, E1);
    df2 re{0.f, 0.f}, im{0.f, 0.f};
    for (int j = 0; j < nc; ++j) {
      float4 b = to_df(in[(long)Z * nc + j]);
      if (!DAG)
        df_cmac<false>(re, im, Y[(((long)X * 5 + d) * nc + j) * nc + i], b);
      else
        df_cmac<true>(re, im, Y[(((long)Z * 5 + opp(d)) * nc + i) * nc + j], b);
    }
    tot.x += (double)re.hi + (double)re.lo;
    tot.y += (double)im.hi + (double)im.lo;
  }
  out[e] = tot;
}

template <int NC, bool DF>
bool launch_cgne_t(const CgneArgs& args, int device, cudaStream_t s, int sms_use) {
  static int cached_per_sm[64] = {0}, cached_sms[64] = {0};
  int& per_sm = cached_per_sm[device & 63];
  int& sms = cached_sms[device & 63];
  if (per_sm == 0) {
    int occ = 0, coop = 0;
    SW_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cgne<NC, DF>, kWarps * 32, 0));
    SW_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    SW_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device));
    if (!coop || occ < 1) return false;
    per_sm = occ < 2 ? occ : 2;
  }
  const int grid = (sms_use < sms ? (sms_use > 0 ? sms_use : 1) : sms) * per_sm;
  CgneArgs a = args;
  void* params[] = {&a};
  SW_CUDA(cudaLaunchCooperativeKernel((const void*)k_cgne<NC, DF>, dim3(grid), dim3(kWarps * 32),
                                      params, 0, s));
  sw_count_launch();
  return true;
}

}  // namespace

void launch_coarse_apply_df(const CoarseGeom& g, const float4* Y, int dagger, const double2* in,
                            double2* out, cudaStream_t s) {
  long n = (long)g.E0 * g.E1 * g.nc;
  int blocks = (int)((n + 127) / 128);
  if (dagger)
    k_coarse_apply_df<true><<<blocks, 128, 0, s>>>(Y, in, out, g.E0, g.E1, g.nc);
  else
    k_coarse_apply_df<false><<<blocks, 128, 0, s>>>(Y, in, out, g.E0, g.E1, g.nc);
  SW_LAUNCH_CHECK();
}

// Runs the whole coarsest CGNE on the device.  Returns false (nothing
// launched) when nc has no compiled variant; then the caller uses the
// host-driven loop.  partials needs 2 x grid doubles (grid <= 2 x SMs), bar 2 unsigned
// (zeroed here), status 3 ints.
bool launch_cgne_persistent(const CoarseGeom& g, const void* Y, int df64, const double2* b,
                            double2* x, double2* r, double2* p, float4* rdf, float4* pdf,
                            double* partials, unsigned* bar, int* status, int maxit, double tol,
                            int device, cudaStream_t s, int stall_test, int sms_use) {
  SW_CUDA(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s));
  SW_CUDA(cudaMemsetAsync(status, 0, 3 * sizeof(int), s));
  CgneArgs a{Y, b, x, r, p, rdf, pdf, partials, bar, status, g.E0, g.E1, maxit, tol, stall_test};
  if (df64) {
    if (!rdf || !pdf) return false;
    switch (g.nc) {
      case 16: return launch_cgne_t<16, true>(a, device, s, sms_use);
      case 24: return launch_cgne_t<24, true>(a, device, s, sms_use);
      case 32: return launch_cgne_t<32, true>(a, device, s, sms_use);
      case 48: return launch_cgne_t<48, true>(a, device, s, sms_use);
      case 64: return launch_cgne_t<64, true>(a, device, s, sms_use);
      default: return false;
    }
  }
  switch (g.nc) {
    case 16: return launch_cgne_t<16, false>(a, device, s, sms_use);
    case 24: return launch_cgne_t<24, false>(a, device, s, sms_use);
    case 32: return launch_cgne_t<32, false>(a, device, s, sms_use);
    case 48: return launch_cgne_t<48, false>(a, device, s, sms_use);
    case 64: return launch_cgne_t<64, false>(a, device, s, sms_use);
    default: return false;
  }
}
