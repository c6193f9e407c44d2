// BLAS-1 on complex128 vectors with device-resident Krylov coefficients.
//
// Reductions are single launches with a fixed grid (at most kReduceBlocks
// CTAs, chosen from n only): each CTA sums a grid-stride slice with a warp
// shuffle tree, writes one partial, and the last CTA to finish (atomic
// counter) adds the partials in index order.  The summation order therefore
// depends on n alone, so every result is bitwise reproducible.
#include "sw_internal.h"

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// Block-wide sum of two values; result valid in thread 0.
__device__ __forceinline__ void block_sum2(double& a, double& b) {
  __shared__ double sa[32], sb[32];
  a = warp_sum(a);
  b = warp_sum(b);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) { sa[w] = a; sb[w] = b; }
  __syncthreads();
  int nw = blockDim.x >> 5;
  if (w == 0) {
    a = lane < nw ? sa[lane] : 0.0;
    b = lane < nw ? sb[lane] : 0.0;
    a = warp_sum(a);
    b = warp_sum(b);
  }
}

template <int MODE>  // 0: <a, b> = sum conj(a) b;  1: ||a||^2
__global__ void __launch_bounds__(kThreads) k_reduce(const double2* __restrict__ a,
                                                     const double2* __restrict__ b, long n,
                                                     double* partials, unsigned* counter,
                                                     double2* slots, int slot,
                                                     const int* __restrict__ skip) {
  if (skip && *skip) return;
  double re = 0.0, im = 0.0;
  long stride = (long)gridDim.x * blockDim.x;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    double2 x = a[i];
    if (MODE == 0) {
      double2 y = b[i];
      re = fma(x.x, y.x, re); re = fma(x.y, y.y, re);
      im = fma(x.x, y.y, im); im = fma(-x.y, y.x, im);
    } else {
      re = fma(x.x, x.x, re); re = fma(x.y, x.y, re);
    }
  }
  block_sum2(re, im);
  __shared__ bool last;
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = re;
    partials[2 * blockIdx.x + 1] = im;
    __threadfence();
    unsigned t = atomicAdd(counter, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (last) {
    __threadfence();
    double r2 = 0.0, i2 = 0.0;
    const volatile double* vp = partials;
    for (int j = threadIdx.x; j < (int)gridDim.x; j += blockDim.x) {
      r2 += vp[2 * j];
      i2 += vp[2 * j + 1];
    }
    block_sum2(r2, i2);
    if (threadIdx.x == 0) {
      slots[slot] = make_double2(r2, i2);
      *counter = 0u;
    }
  }
}

__global__ void k_axpy(double2* __restrict__ y, const double2* __restrict__ x, long n,
                       const double2* __restrict__ S, Coef c, const int* __restrict__ skip) {
  if (skip && *skip) return;
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double2 a = coef_eval(S, c);
  double2 v = x[i], o = y[i];
  o.x = fma(a.x, v.x, o.x); o.x = fma(-a.y, v.y, o.x);
  o.y = fma(a.x, v.y, o.y); o.y = fma(a.y, v.x, o.y);
  y[i] = o;
}
__global__ void k_xpay(double2* __restrict__ y, const double2* __restrict__ x, long n,
                       const double2* __restrict__ S, Coef c, const int* __restrict__ skip) {
  if (skip && *skip) return;
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double2 a = coef_eval(S, c);
  double2 v = y[i], o = x[i];
  o.x = fma(a.x, v.x, o.x); o.x = fma(-a.y, v.y, o.x);
  o.y = fma(a.x, v.y, o.y); o.y = fma(a.y, v.x, o.y);
  y[i] = o;
}
__global__ void k_scale(double2* __restrict__ y, long n, const double2* __restrict__ S, Coef c) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double2 a = coef_eval(S, c);
  double2 v = y[i];
  y[i] = make_double2(a.x * v.x - a.y * v.y, a.x * v.y + a.y * v.x);
}
__global__ void k_sub(double2* __restrict__ o, const double2* __restrict__ a,
                      const double2* __restrict__ b, long n) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double2 u = a[i], v = b[i];
  o[i] = make_double2(u.x - v.x, u.y - v.y);
}
__global__ void k_add3(double2* __restrict__ o, const double2* __restrict__ a,
                       const double2* __restrict__ b, const double2* __restrict__ d, long n) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double2 u = a[i], v = b[i], w = d[i];
  o[i] = make_double2((u.x + v.x) + w.x, (u.y + v.y) + w.y);
}

inline int grid_for(long n) { return (int)((n + kThreads - 1) / kThreads); }
inline int reduce_grid(long n) {
  long g = (n + kThreads - 1) / kThreads;
  if (g > kReduceBlocks) g = kReduceBlocks;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

void blas_dot(sw_ctx* c, const double2* a, const double2* b, long n, int slot, const int* skip) {
  k_reduce<0><<<reduce_grid(n), kThreads, 0, c->stream>>>(a, b, n, c->partials, c->counter,
                                                          c->slots, slot, skip);
  SW_LAUNCH_CHECK();
}
void blas_norm2(sw_ctx* c, const double2* a, long n, int slot, const int* skip) {
  k_reduce<1><<<reduce_grid(n), kThreads, 0, c->stream>>>(a, nullptr, n, c->partials, c->counter,
                                                          c->slots, slot, skip);
  SW_LAUNCH_CHECK();
}
void blas_axpy(sw_ctx* c, double2* y, const double2* x, long n, Coef a, const int* skip) {
  if (n <= 0) return;
  k_axpy<<<grid_for(n), kThreads, 0, c->stream>>>(y, x, n, c->slots, a, skip);
  SW_LAUNCH_CHECK();
}
void blas_xpay(sw_ctx* c, double2* y, const double2* x, long n, Coef a, const int* skip) {
  if (n <= 0) return;
  k_xpay<<<grid_for(n), kThreads, 0, c->stream>>>(y, x, n, c->slots, a, skip);
  SW_LAUNCH_CHECK();
}
void blas_scale(sw_ctx* c, double2* y, long n, Coef a) {
  if (n <= 0) return;
  k_scale<<<grid_for(n), kThreads, 0, c->stream>>>(y, n, c->slots, a);
  SW_LAUNCH_CHECK();
}
void blas_copy(sw_ctx* c, double2* y, const double2* x, long n) {
  if (n <= 0) return;
  SW_CUDA(cudaMemcpyAsync(y, x, n * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
}
void blas_zero(sw_ctx* c, double2* y, long n) {
  if (n <= 0) return;
  SW_CUDA(cudaMemsetAsync(y, 0, n * sizeof(double2), c->stream));
}
void blas_sub(sw_ctx* c, double2* out, const double2* a, const double2* b, long n) {
  if (n <= 0) return;
  k_sub<<<grid_for(n), kThreads, 0, c->stream>>>(out, a, b, n);
  SW_LAUNCH_CHECK();
}
void blas_add3(sw_ctx* c, double2* out, const double2* a, const double2* b, const double2* d,
               long n) {
  if (n <= 0) return;
  k_add3<<<grid_for(n), kThreads, 0, c->stream>>>(out, a, b, d, n);
  SW_LAUNCH_CHECK();
}
double2 slot_read(sw_ctx* c, int slot) {
  SW_CUDA(cudaMemcpyAsync(c->h_slots + slot, c->slots + slot, sizeof(double2),
                          cudaMemcpyDeviceToHost, c->stream));
  SW_CUDA(cudaStreamSynchronize(c->stream));
  if (!c->pending.empty()) timing_harvest(c);
  return c->h_slots[slot];
}

static cudaEvent_t take_event(sw_ctx* c) {
  if (!c->spare.empty()) {
    cudaEvent_t e = c->spare.back();
    c->spare.pop_back();
    return e;
  }
  cudaEvent_t e;
  SW_CUDA(cudaEventCreate(&e));
  return e;
}
int timing_begin(sw_ctx* c, int cat) {
  if (!c->timing) return -1;
  TimedPair t{cat, take_event(c), take_event(c)};
  SW_CUDA(cudaEventRecord(t.a, c->stream));
  c->pending.push_back(t);
  return (int)c->pending.size() - 1;
}
void timing_end(sw_ctx* c, int token) {
  if (token < 0) return;
  SW_CUDA(cudaEventRecord(c->pending[token].b, c->stream));
}
void timing_harvest(sw_ctx* c) {
  for (TimedPair& t : c->pending) {
    float ms = 0.f;
    SW_CUDA(cudaEventElapsedTime(&ms, t.a, t.b));
    c->t_ms[t.cat] += ms;
    c->t_count[t.cat] += 1;
    c->spare.push_back(t.a);
    c->spare.push_back(t.b);
  }
  c->pending.clear();
}
// Iteration control of a device-gated Krylov loop: ctl[0] = done, ctl[1] =
// iterations, ctl[2] = non-finite residual seen.  Loop body kernels return
// at once when ctl[0] is set, so the host can queue iterations without
// waiting for each stopping test.
__global__ void k_iter_init(int* ctl, const double2* __restrict__ S, int slot, double stop,
                            int maxit) {
  double rn = sqrt(S[slot].x);
  ctl[1] = 0;
  ctl[2] = isfinite(rn) ? 0 : 1;
  ctl[0] = (maxit <= 0 || !(rn > stop)) ? 1 : 0;
}
__global__ void k_iter_check(int* ctl, const double2* __restrict__ S, int slot, double stop,
                             int maxit) {
  if (ctl[0]) return;
  int k = ++ctl[1];
  double rn = sqrt(S[slot].x);
  if (!isfinite(rn)) ctl[2] = 1;
  if (k >= maxit || !(rn > stop)) ctl[0] = 1;
}
void iter_init(sw_ctx* c, int* ctl, int slot, double stop, int maxit) {
  k_iter_init<<<1, 1, 0, c->stream>>>(ctl, c->slots, slot, stop, maxit);
  SW_LAUNCH_CHECK();
}
void iter_check(sw_ctx* c, int* ctl, int slot, double stop, int maxit) {
  k_iter_check<<<1, 1, 0, c->stream>>>(ctl, c->slots, slot, stop, maxit);
  SW_LAUNCH_CHECK();
}
void iter_read(sw_ctx* c, const int* ctl, int* host3) {
  SW_CUDA(cudaMemcpyAsync(host3, ctl, 3 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  SW_CUDA(cudaStreamSynchronize(c->stream));
  if (!c->pending.empty()) timing_harvest(c);
}

void slot_set(sw_ctx* c, int slot, double2 v) {
  c->h_slots[slot] = v;
  SW_CUDA(cudaMemcpyAsync(c->slots + slot, c->h_slots + slot, sizeof(double2),
                          cudaMemcpyHostToDevice, c->stream));
  SW_CUDA(cudaStreamSynchronize(c->stream));
}
