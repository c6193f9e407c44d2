// Coarsest-level CGNE for a batch of right-hand sides in one persistent
// cooperative kernel (batched solves of a mixed-precision hierarchy).
//
// Same iteration as the single-RHS kernel (cgne.cu) for every right-hand side,
// each with its own alpha, beta, stopping test and iteration count; a
// right-hand side that has stopped is no longer updated while the others go
// on.  The stencil is read once per batch: a lane owns one row for all K
// right-hand sides, so each FP32 stencil entry feeds K complex products.
// Stencil products and their sums are FP32 (the coarsest solve of a batch is
// a 0.2-tolerance preconditioner); the iterates, residuals and Krylov scalars
// stay FP64, and FP32 copies of r and p feed the stencil.
//
// Layout inside the kernel: right-hand-side-minor, element (dof, rhs) at
// dof * K + rhs, so the K values a stencil column needs are contiguous.  The
// grid is one CTA per SM for every batch width and each thread takes the same
// dofs and rows whatever K is, so a right-hand side's sums run in the same
// order whatever its batch-mates are: its result does not depend on them.
#include <string>

#include "sw_internal.h"

namespace {

constexpr long kSpinLimit = 1L << 24;
constexpr int kWarps = 8;
constexpr int kRows = 8;

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

struct BatchArgs {
  const float2* Y;         // FP32 copy of the coarsest stencil (column-major blocks)
  const double2* const* b; // [K] right-hand sides (entries beyond nb unused)
  double2* const* xout;    // [K] solutions
  double2* X;              // [n][K] FP64 iterates
  double2* R;              // [n][K] FP64 residuals
  double2* P;              // [n][K] FP64 directions
  float2* Rf;              // [n][K] FP32 copies read by the stencil
  float2* Pf;
  double* partials;        // [2][K][gridDim.x]
  unsigned* bar;           // grid barrier state (2 words)
  int* status;             // [0] barrier timeout, [1] non-finite, [2 + r] iterations of rhs r
  int nb, E0, E1, maxit;
  double tol;
};

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
  for (int r = w; r < K; r += kWarps) {
    double s = 0.0;
    for (int q = lane; q < (int)gridDim.x; q += 32) s += __ldcg(part + r * gridDim.x + q);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[r] = s;
  }
  __syncthreads();
}

// Row i of (A v) or (A^dag v) for all K right-hand sides (FP32), summed over
// the 4 lanes of the row (lane q takes columns [q nc/4, (q+1) nc/4) of all
// five blocks); every lane of the row holds the totals.
template <int NC, int K>
__device__ __forceinline__ void stencil_row_b(const float2* __restrict__ Y,
                                              const float2* __restrict__ v, int X, int i, int q,
                                              int E0, int E1, bool dagger, float2* acc) {
  constexpr int QJ = NC / 4;
  const int j0 = q * QJ;
#pragma unroll
  for (int r = 0; r < K; ++r) acc[r] = make_float2(0.f, 0.f);
#pragma unroll
  for (int d = 0; d < 5; ++d) {
    const long nb = nbr(X, d, E0, E1);
    const long ybase = dagger ? ((nb * 5 + opp(d)) * NC + i) * NC + j0
                              : (((long)X * 5 + d) * NC + j0) * NC + i;
    const long ystep = dagger ? 1 : NC;
    const float2* xb = v + (nb * NC + j0) * K;
#pragma unroll 2
    for (int t = 0; t < QJ; ++t) {
      float2 y = __ldg(Y + ybase + t * ystep);
      if (dagger) y.y = -y.y;
      const float4* xv = reinterpret_cast<const float4*>(xb + t * K);
#pragma unroll
      for (int r2 = 0; r2 < K / 2; ++r2) {
        float4 x2 = __ldcg(xv + r2);
        float2& a0 = acc[2 * r2];
        float2& a1 = acc[2 * r2 + 1];
        a0.x = fmaf(y.x, x2.x, a0.x);
        a0.x = fmaf(-y.y, x2.y, a0.x);
        a0.y = fmaf(y.x, x2.y, a0.y);
        a0.y = fmaf(y.y, x2.x, a0.y);
        a1.x = fmaf(y.x, x2.z, a1.x);
        a1.x = fmaf(-y.y, x2.w, a1.x);
        a1.y = fmaf(y.x, x2.w, a1.y);
        a1.y = fmaf(y.y, x2.z, a1.y);
      }
    }
  }
#pragma unroll
  for (int r = 0; r < K; ++r) {
    acc[r].x += __shfl_xor_sync(0xffffffffu, acc[r].x, 1);
    acc[r].y += __shfl_xor_sync(0xffffffffu, acc[r].y, 1);
    acc[r].x += __shfl_xor_sync(0xffffffffu, acc[r].x, 2);
    acc[r].y += __shfl_xor_sync(0xffffffffu, acc[r].y, 2);
  }
}

template <int NC, int K>
__global__ void __launch_bounds__(kWarps * 32, 1) k_cgne_batch(BatchArgs a) {
  __shared__ double red[K][kWarps];
  __shared__ double sh_sum[K], sh_rr[K], sh_stop[K], sh_coef[K];
  __shared__ int sh_state[K];  // 0 active, 1 stopped, 2 non-finite
  __shared__ int sh_iters[K];
  __shared__ int sh_any;
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
  double nrm[K];
  float2 acc[K];

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
      a.Rf[e] = make_float2((float)v.x, (float)v.y);
      nrm[r] = fma(v.x, v.x, fma(v.y, v.y, nrm[r]));
    }
  }
  int ph = 0;
  cta_partials<K>(nrm, red, a.partials + ph * K * gridDim.x);
  if (!grid_barrier(a.bar, a.status)) return;
  grid_sums<K>(a.partials + ph * K * gridDim.x, sh_sum);
  if (threadIdx.x < K) {
    int r = threadIdx.x;
    double rr0 = sh_sum[r];
    sh_rr[r] = rr0;
    sh_stop[r] = a.tol * sqrt(rr0);
    sh_iters[r] = 0;
    sh_state[r] = !isfinite(rr0) ? 2 : ((a.maxit <= 0 || !(sqrt(rr0) > sh_stop[r])) ? 1 : 0);
  }
  __syncthreads();
  ph ^= 1;
  // P = A^dag R, ||p||^2
#pragma unroll
  for (int r = 0; r < K; ++r) nrm[r] = 0.0;
  for (int rd = 0; rd < rounds; ++rd) {
    int item = rd * nwarps + warp * gridDim.x + blockIdx.x;
    if (item >= nitems) break;  // warp-uniform
    int X = item / chunks, i = (item - X * chunks) * kRows + rr8;
    stencil_row_b<NC, K>(a.Y, a.Rf, X, i, q, a.E0, a.E1, true, acc);
    if (q == 0) {
      long e = ((long)X * NC + i) * K;
#pragma unroll
      for (int r = 0; r < K; ++r) {
        double2 w = make_double2((double)acc[r].x, (double)acc[r].y);
        a.P[e + r] = w;
        a.Pf[e + r] = acc[r];
        nrm[r] = fma(w.x, w.x, fma(w.y, w.y, nrm[r]));
      }
    }
  }
  cta_partials<K>(nrm, red, a.partials + ph * K * gridDim.x);
  if (!grid_barrier(a.bar, a.status)) return;
  grid_sums<K>(a.partials + ph * K * gridDim.x, sh_sum);
  if (threadIdx.x < K) sh_coef[threadIdx.x] = sh_rr[threadIdx.x] / sh_sum[threadIdx.x];  // alpha
  if (threadIdx.x == 0) {
    int any = 0;
    for (int r = 0; r < K; ++r) any |= sh_state[r] == 0;
    sh_any = any;
  }
  __syncthreads();
  ph ^= 1;
  while (sh_any) {
    // P1: w = A p; x += alpha p; r -= alpha w (right-hand sides still active)
#pragma unroll
    for (int r = 0; r < K; ++r) nrm[r] = 0.0;
    for (int rd = 0; rd < rounds; ++rd) {
      int item = rd * nwarps + warp * gridDim.x + blockIdx.x;
      if (item >= nitems) break;
      int X = item / chunks, i = (item - X * chunks) * kRows + rr8;
      stencil_row_b<NC, K>(a.Y, a.Pf, X, i, q, a.E0, a.E1, false, acc);
      if (q == 0) {
        long e = ((long)X * NC + i) * K;
#pragma unroll
        for (int r = 0; r < K; ++r) {
          if (sh_state[r] != 0) continue;
          double al = sh_coef[r];
          double2 pv = __ldcg(a.P + e + r), xv = __ldcg(a.X + e + r), rv = __ldcg(a.R + e + r);
          xv.x = fma(al, pv.x, xv.x);
          xv.y = fma(al, pv.y, xv.y);
          rv.x = fma(-al, (double)acc[r].x, rv.x);
          rv.y = fma(-al, (double)acc[r].y, rv.y);
          a.X[e + r] = xv;
          a.R[e + r] = rv;
          a.Rf[e + r] = make_float2((float)rv.x, (float)rv.y);
          nrm[r] = fma(rv.x, rv.x, fma(rv.y, rv.y, nrm[r]));
        }
      }
    }
    cta_partials<K>(nrm, red, a.partials + ph * K * gridDim.x);
    if (!grid_barrier(a.bar, a.status)) return;
    grid_sums<K>(a.partials + ph * K * gridDim.x, sh_sum);
    if (threadIdx.x < K) {
      int r = threadIdx.x;
      if (sh_state[r] == 0) {
        double rr_new = sh_sum[r];
        int k = ++sh_iters[r];
        if (!isfinite(rr_new))
          sh_state[r] = 2;
        else if (!(k < a.maxit && sqrt(rr_new) > sh_stop[r]))
          sh_state[r] = 1;
        sh_coef[r] = rr_new / sh_rr[r];  // beta
        sh_rr[r] = rr_new;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int any = 0;
      for (int r = 0; r < K; ++r) any |= sh_state[r] == 0;
      sh_any = any;
    }
    __syncthreads();
    ph ^= 1;
    if (!sh_any) break;
    // P2: p = A^dag r + beta p (right-hand sides still active)
#pragma unroll
    for (int r = 0; r < K; ++r) nrm[r] = 0.0;
    for (int rd = 0; rd < rounds; ++rd) {
      int item = rd * nwarps + warp * gridDim.x + blockIdx.x;
      if (item >= nitems) break;
      int X = item / chunks, i = (item - X * chunks) * kRows + rr8;
      stencil_row_b<NC, K>(a.Y, a.Rf, X, i, q, a.E0, a.E1, true, acc);
      if (q == 0) {
        long e = ((long)X * NC + i) * K;
#pragma unroll
        for (int r = 0; r < K; ++r) {
          if (sh_state[r] != 0) continue;
          double be = sh_coef[r];
          double2 pv = __ldcg(a.P + e + r);
          pv.x = fma(be, pv.x, (double)acc[r].x);
          pv.y = fma(be, pv.y, (double)acc[r].y);
          a.P[e + r] = pv;
          a.Pf[e + r] = make_float2((float)pv.x, (float)pv.y);
          nrm[r] = fma(pv.x, pv.x, fma(pv.y, pv.y, nrm[r]));
        }
      }
    }
    cta_partials<K>(nrm, red, a.partials + ph * K * gridDim.x);
    if (!grid_barrier(a.bar, a.status)) return;
    grid_sums<K>(a.partials + ph * K * gridDim.x, sh_sum);
    if (threadIdx.x < K && sh_state[threadIdx.x] == 0)
      sh_coef[threadIdx.x] = sh_rr[threadIdx.x] / sh_sum[threadIdx.x];  // alpha
    __syncthreads();
    ph ^= 1;
  }
  // scatter the solutions
  for (long dof = tid; dof < n; dof += nthr)
    for (int r = 0; r < a.nb; ++r) a.xout[r][dof] = __ldcg(a.X + dof * K + r);
  if (blockIdx.x == 0 && threadIdx.x < K) {
    if (sh_state[threadIdx.x] == 2) atomicExch(a.status + 1, 1);
    a.status[2 + threadIdx.x] = sh_iters[threadIdx.x];
  }
}

template <int NC, int K>
bool launch_b(const BatchArgs& args, int device, cudaStream_t s) {
  static int cached_grid[64] = {0};
  int& grid = cached_grid[device & 63];
  if (grid == 0) {
    int occ = 0, sms = 0, coop = 0;
    SW_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cgne_batch<NC, K>, kWarps * 32,
                                                          0));
    SW_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    SW_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device));
    if (!coop || occ < 1)
      throw SwError{SW_ERR_CUDA, "batched CGNE cannot be launched cooperatively (occupancy " +
                                     std::to_string(occ) + ", cooperative " +
                                     std::to_string(coop) + ")"};
    grid = sms;  // one CTA per SM for every batch width (see the header note)
  }
  BatchArgs a = args;
  void* params[] = {&a};
  SW_CUDA(cudaLaunchCooperativeKernel((const void*)k_cgne_batch<NC, K>, dim3(grid),
                                      dim3(kWarps * 32), params, 0, s));
  sw_count_launch();
  return true;
}

}  // namespace

int cgne_batch_width(int nb) { return nb <= 4 ? 4 : (nb <= 8 ? 8 : 16); }

bool launch_cgne_batch(const CoarseGeom& g, const float2* Yf, int nb, const double2* const* b,
                       double2* const* x, double2* X, double2* R, double2* P, float2* Rf,
                       float2* Pf, double* partials, unsigned* bar, int* status, int maxit,
                       double tol, int device, cudaStream_t s) {
  if (nb < 1 || nb > 16) return false;
  SW_CUDA(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s));
  SW_CUDA(cudaMemsetAsync(status, 0, 18 * sizeof(int), s));
  BatchArgs a{Yf, b, x, X, R, P, Rf, Pf, partials, bar, status, nb, g.E0, g.E1, maxit, tol};
  int K = cgne_batch_width(nb);
#define SW_CASE(NCV)                                   \
  case NCV:                                            \
    if (K == 4) return launch_b<NCV, 4>(a, device, s); \
    if (K == 8) return launch_b<NCV, 8>(a, device, s); \
    return launch_b<NCV, 16>(a, device, s);
  switch (g.nc) {
    SW_CASE(16)
    SW_CASE(24)
    SW_CASE(64)
    default: return false;
  }
#undef SW_CASE
}
