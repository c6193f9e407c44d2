// Reduced-precision operators of the mixed-precision solve (Sec. IV's
// K-cycle is a preconditioner solved to 0.2, so its operators need not be
// FP64; the outer FGCR residual stays FP64):
//  - fine Schur operator S with FP32 links and B^-1 (FP64 vectors in and out),
//  - coarse stencil with FP16 storage, one FP32 scale per nc x nc block and
//    FP32 accumulation,
//  - conversion of a stencil to double-float (df64, used by the coarsest CGNE).
#include <cuda_fp16.h>

#include "sw_internal.h"

namespace {

__device__ __forceinline__ void cfmaf(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}
__device__ __forceinline__ void cfmacf(float2& acc, float2 a, float2 b) {  // conj(a) b
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(-a.y, b.x, acc.y);
}
__device__ __forceinline__ float2 f2(double2 v) { return make_float2((float)v.x, (float)v.y); }
__host__ __device__ __forceinline__ int nbr_site(int X, int d, int E0, int E1) {
  int X0 = X % E0, X1 = X / E0;
  if (d == 1) X0 = (X0 + 1 == E0) ? 0 : X0 + 1;
  if (d == 2) X0 = (X0 == 0) ? E0 - 1 : X0 - 1;
  if (d == 3) X1 = (X1 + 1 == E1) ? 0 : X1 + 1;
  if (d == 4) X1 = (X1 == 0) ? E1 - 1 : X1 - 1;
  return X0 + E0 * X1;
}
__host__ __device__ __forceinline__ int opp_dir(int d) {
  return d == 0 ? 0 : (d == 1 ? 2 : (d == 2 ? 1 : (d == 3 ? 4 : 3)));
}
inline int cdiv(long a, long b) { return (int)((a + b - 1) / b); }

// ------------------------------------------------------------------ fine FP32
__global__ void k_to_f32(const double2* __restrict__ in, float2* __restrict__ out, long n) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = f2(in[i]);
}

// out (float) = M in (double -> float), M per KD block of one parity half
__global__ void k_block_apply_df(const float2* __restrict__ M, const double2* __restrict__ in,
                                 float2* __restrict__ out, int nblk) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nblk) return;
  float2 v[4];
  for (int j = 0; j < 4; ++j) v[j] = f2(in[4 * b + j]);
  const float2* m = M + 16 * b;
  for (int i = 0; i < 4; ++i) {
    float2 acc = make_float2(0.f, 0.f);
    for (int j = 0; j < 4; ++j) cfmaf(acc, m[4 * i + j], v[j]);
    out[4 * b + i] = acc;
  }
}

// (C in)(s) for site f of its parity half; in = opposite half (float)
__device__ __forceinline__ float2 hop_out_f(const float2* __restrict__ W, const float2* __restrict__ in,
                                           int f, int L0, int L1, int N) {
  int x0, x1;
  ps_coords(f, L0, N, x0, x1);
  int half = N >> 1;
  float2 acc = make_float2(0.f, 0.f);
  if (x0 & 1) {
    int t = ps_index(x0 + 1 == L0 ? 0 : x0 + 1, x1, L0, N);
    cfmaf(acc, W[f], in[t % half]);
  } else {
    int t = ps_index(x0 == 0 ? L0 - 1 : x0 - 1, x1, L0, N);
    float2 w = W[t], v = in[t % half];
    acc.x -= w.x * v.x + w.y * v.y;
    acc.y -= w.x * v.y - w.y * v.x;
  }
  if (x1 & 1) {
    int t = ps_index(x0, x1 + 1 == L1 ? 0 : x1 + 1, L0, N);
    cfmaf(acc, W[N + f], in[t % half]);
  } else {
    int t = ps_index(x0, x1 == 0 ? L1 - 1 : x1 - 1, L0, N);
    float2 w = W[N + t], v = in[t % half];
    acc.x -= w.x * v.x + w.y * v.y;
    acc.y -= w.x * v.y - w.y * v.x;
  }
  return acc;
}

// out_o (float) = M_o (C_oe in_e), per odd KD block
__global__ void k_hop_block_ff(const float2* __restrict__ W, const float2* __restrict__ M, int par,
                               const float2* __restrict__ in, float2* __restrict__ out, int L0,
                               int L1) {
  int N = L0 * L1, half = N >> 1;
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= (half >> 2)) return;
  float2 u[4];
  for (int k = 0; k < 4; ++k) u[k] = hop_out_f(W, in, par * half + 4 * b + k, L0, L1, N);
  const float2* m = M + 16 * b;
  for (int i = 0; i < 4; ++i) {
    float2 acc = make_float2(0.f, 0.f);
    for (int j = 0; j < 4; ++j) cfmaf(acc, m[4 * i + j], u[j]);
    out[4 * b + i] = acc;
  }
}

// out_e (double) = src_e - C_eo in_o
__global__ void k_hop_sub_fd(const float2* __restrict__ W, int par,
                             const double2* __restrict__ src, const float2* __restrict__ in,
                             double2* __restrict__ out, int L0, int L1) {
  int N = L0 * L1, half = N >> 1;
  int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= half) return;
  float2 c = hop_out_f(W, in, par * half + h, L0, L1, N);
  double2 o = src[h];
  o.x -= (double)c.x;
  o.y -= (double)c.y;
  out[h] = o;
}

// ------------------------------------------------------------------ FP16 stencil
// One CTA per block (X, d): scale = largest |re| or |im| of the block; the
// block is stored as half2(entry / scale).
__global__ void k_to_half_scaled(const double2* __restrict__ Y, __half2* __restrict__ Yh,
                                 float* __restrict__ scale, int nc) {
  __shared__ double red[32];
  long base = (long)blockIdx.x * nc * nc;
  double m = 0.0;
  for (int e = threadIdx.x; e < nc * nc; e += blockDim.x) {
    double2 v = Y[base + e];
    m = fmax(m, fmax(fabs(v.x), fabs(v.y)));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double mm = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) mm = fmax(mm, red[q]);
    red[0] = mm > 0.0 ? mm : 1.0;
    scale[blockIdx.x] = (float)red[0];
  }
  __syncthreads();
  double inv = 1.0 / red[0];
  for (int e = threadIdx.x; e < nc * nc; e += blockDim.x) {
    double2 v = Y[base + e];
    Yh[base + e] = __floats2half2_rn((float)(v.x * inv), (float)(v.y * inv));
  }
}

// y_X = sum_d s[X][d] Yh[X][d] x_{X+d} (DAG: sum_d s[Z][opp] Yh[Z][opp]^dag x_Z, Z = X+d),
// FP32 products and sums, FP64 vectors in and out.  Thread layout as the FP64
// kernel: (direction d, row i), rs CTAs per site when there are few sites.
template <int NC, bool DAG>
__global__ void __launch_bounds__(5 * NC) k_coarse_apply_h(const __half2* __restrict__ Yh,
                                                           const float* __restrict__ scale,
                                                           const double2* __restrict__ in,
                                                           double2* __restrict__ out, int E0,
                                                           int E1, int rs) {
  __shared__ float2 xs[5][NC];
  __shared__ float2 part[5][NC];
  int rows = NC / rs;
  int X = blockIdx.x / rs;
  int r0 = (blockIdx.x - X * rs) * rows;
  int nthr = 5 * rows;
  for (int t = threadIdx.x; t < 5 * NC; t += nthr) {
    int d = t / NC, j = t - d * NC;
    xs[d][j] = f2(in[(long)nbr_site(X, d, E0, E1) * NC + j]);
  }
  __syncthreads();
  int d = threadIdx.x / rows;
  int i = r0 + threadIdx.x - d * rows;
  float2 acc = make_float2(0.f, 0.f);
  float sc;
  if (!DAG) {
    long blk = (long)X * 5 + d;
    sc = scale[blk];
    const __half2* y = Yh + blk * NC * NC + i;
#pragma unroll 16
    for (int j = 0; j < NC; ++j) cfmaf(acc, __half22float2(y[j * NC]), xs[d][j]);
  } else {
    long blk = (long)nbr_site(X, d, E0, E1) * 5 + opp_dir(d);
    sc = scale[blk];
    const __half2* y = Yh + (blk * NC + i) * NC;
#pragma unroll 16
    for (int j = 0; j < NC; ++j) cfmacf(acc, __half22float2(y[j]), xs[d][j]);
  }
  part[d][i] = make_float2(acc.x * sc, acc.y * sc);
  __syncthreads();
  if (d == 0) {
    float2 s = part[0][i];
#pragma unroll
    for (int q = 1; q < 5; ++q) {
      s.x += part[q][i].x;
      s.y += part[q][i].y;
    }
    out[(long)X * NC + i] = make_double2((double)s.x, (double)s.y);
  }
}

// Generic-nc fallback: one thread per (site, row), all five directions.
template <bool DAG>
__global__ void k_coarse_apply_h_any(const __half2* __restrict__ Yh, const float* __restrict__ scale,
                                     const double2* __restrict__ in, double2* __restrict__ out,
                                     int E0, int E1, int nc) {
  long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long)E0 * E1 * nc) return;
  int X = (int)(e / nc), i = (int)(e - (long)X * nc);
  float2 tot = make_float2(0.f, 0.f);
  for (int d = 0; d < 5; ++d) {
    int Z = nbr_site(X, d, E0, E1);
    float2 acc = make_float2(0.f, 0.f);
    long blk = DAG ? (long)Z * 5 + opp_dir(d) : (long)X * 5 + d;
    for (int j = 0; j < nc; ++j) {
      float2 xv = f2(in[(long)Z * nc + j]);
      if (!DAG)
        cfmaf(acc, __half22float2(Yh[(blk * nc + j) * nc + i]), xv);
      else
        cfmacf(acc, __half22float2(Yh[(blk * nc + i) * nc + j]), xv);
    }
    tot.x += acc.x * scale[blk];
    tot.y += acc.y * scale[blk];
  }
  out[e] = make_double2((double)tot.x, (double)tot.y);
}

__global__ void k_to_df64(const double2* __restrict__ Y, float4* __restrict__ Yd, long n) {
  long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  double2 v = Y[e];
  float rh = (float)v.x, ih = (float)v.y;
  Yd[e] = make_float4(rh, (float)(v.x - (double)rh), ih, (float)(v.y - (double)ih));
}

template <int NC>
void apply_h_nc(const CoarseGeom& g, const __half2* Yh, const float* sc, int dagger,
                const double2* in, double2* out, cudaStream_t s) {
  int nsites = g.E0 * g.E1;
  int rs = 1;
  while (rs < 8 && NC % (2 * rs) == 0 && (NC / (2 * rs)) % 8 == 0 && (long)nsites * rs < 4 * 152)
    rs *= 2;
  if (dagger)
    k_coarse_apply_h<NC, true><<<nsites * rs, 5 * (NC / rs), 0, s>>>(Yh, sc, in, out, g.E0, g.E1, rs);
  else
    k_coarse_apply_h<NC, false><<<nsites * rs, 5 * (NC / rs), 0, s>>>(Yh, sc, in, out, g.E0, g.E1,
                                                                      rs);
  SW_LAUNCH_CHECK();
}

}  // namespace

void launch_to_f32(const double2* in, float2* out, long n, cudaStream_t s) {
  k_to_f32<<<cdiv(n, 256), 256, 0, s>>>(in, out, n);
  SW_LAUNCH_CHECK();
}

// S x_e in FP32 arithmetic: t = B_e^-1 x_e, v = B_o^-1 C_oe t, y = x_e - C_eo v.
// tmp: N float2.  W32: FP32 links (parity-split), binv32: FP32 B^-1 table.
void fine_apply_S32(const sw_gauge* g, const float2* W32, const float2* binv32,
                    const double2* in_e, double2* out_e, float2* tmp, cudaStream_t s) {
  int N = g->N, half = N / 2, nblk = N / 8;
  k_block_apply_df<<<cdiv(nblk, 128), 128, 0, s>>>(binv32, in_e, tmp, nblk);
  SW_LAUNCH_CHECK();
  k_hop_block_ff<<<cdiv(nblk, 128), 128, 0, s>>>(W32, binv32 + (long)nblk * 16, 1, tmp, tmp + half,
                                                 g->L0, g->L1);
  SW_LAUNCH_CHECK();
  k_hop_sub_fd<<<cdiv(half, 256), 256, 0, s>>>(W32, 0, in_e, tmp + half, out_e, g->L0, g->L1);
  SW_LAUNCH_CHECK();
}

void launch_to_half_scaled(const CoarseGeom& g, const double2* Y, __half2* Yh, float* scale,
                           cudaStream_t s) {
  k_to_half_scaled<<<g.E0 * g.E1 * 5, 256, 0, s>>>(Y, Yh, scale, g.nc);
  SW_LAUNCH_CHECK();
}

void launch_coarse_apply_h(const CoarseGeom& g, const __half2* Yh, const float* scale, int dagger,
                           const double2* in, double2* out, cudaStream_t s) {
  switch (g.nc) {
    case 16: return apply_h_nc<16>(g, Yh, scale, dagger, in, out, s);
    case 24: return apply_h_nc<24>(g, Yh, scale, dagger, in, out, s);
    case 32: return apply_h_nc<32>(g, Yh, scale, dagger, in, out, s);
    case 48: return apply_h_nc<48>(g, Yh, scale, dagger, in, out, s);
    case 64: return apply_h_nc<64>(g, Yh, scale, dagger, in, out, s);
    default: break;
  }
  long n = (long)g.E0 * g.E1 * g.nc;
  if (dagger)
    k_coarse_apply_h_any<true><<<cdiv(n, 128), 128, 0, s>>>(Yh, scale, in, out, g.E0, g.E1, g.nc);
  else
    k_coarse_apply_h_any<false><<<cdiv(n, 128), 128, 0, s>>>(Yh, scale, in, out, g.E0, g.E1, g.nc);
  SW_LAUNCH_CHECK();
}

void launch_to_df64(const double2* Y, float4* Yd, long n, cudaStream_t s) {
  k_to_df64<<<cdiv(n, 256), 256, 0, s>>>(Y, Yd, n);
  SW_LAUNCH_CHECK();
}
