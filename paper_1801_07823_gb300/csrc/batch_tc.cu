// Host side of the tensor-core batched coarsest CGNE (kernel in batch_tc.cuh):
// tile preparation, the stage options of the autotuner and the dispatch; this
// unit also holds the instantiations for nc = 64.
#include "batch_tc.cuh"

using namespace swtc;

namespace {

// Stacked TF32 tiles of the forward (adj = 0) or adjoint (adj = 1) blocks of
// an FP64 stencil Y (column-major blocks): one CTA per (site, direction).
__global__ void k_stack_tiles(const double2* __restrict__ Y, float* __restrict__ T, int E0,
                              int E1, int nc, int adj) {
  const int X = blockIdx.x / 5, d = blockIdx.x - 5 * (blockIdx.x / 5);
  const size_t blk = adj ? ((size_t)nbr(X, d, E0, E1) * 5 + opp(d)) * nc * nc
                         : ((size_t)X * 5 + d) * nc * nc;
  float* out = T + (size_t)blockIdx.x * 128 * nc;
  for (int e = threadIdx.x; e < 128 * nc; e += blockDim.x) {
    const int row = e / nc, k = e - row * nc;  // stacked row, input dof
    float v = 0.f;
    if (row < 2 * nc) {
      const int i = row < nc ? row : row - nc;
      // forward: Z[i][k] = Y[X][d] (i, k) at k nc + i; adjoint: conj of (k, i)
      const double2 z = adj ? Y[blk + (size_t)i * nc + k] : Y[blk + (size_t)k * nc + i];
      const double part = row < nc ? z.x : (adj ? -z.y : z.y);
      v = to_tf32((float)part);
    }
    out[tile_off(row, k, 128) / 4] = v;
  }
}

}  // namespace

bool swtc::run_nc64(const TcArgs& a, int K, int S, bool f32, int device, cudaStream_t s,
                     int sms_use) {
  return run_nc<64>(a, K, S, f32, device, s, sms_use);
}

int tc_width(int nb) { return nb <= 8 ? 8 : (nb <= 16 ? 16 : (nb <= 32 ? 32 : 64)); }

bool tc_supported(int nc) { return nc == 16 || nc == 24 || nc == 64; }

long tc_tile_floats(int nc) { return 128L * nc; }

// Fraction of the stacked stencil tiles (forward and adjoint) that fits in
// three quarters of the L2 cache, for the evict-last variant.
float tc_l2_fraction(const CoarseGeom& g, int device) {
  int l2 = 0;
  if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, device) != cudaSuccess || l2 <= 0)
    return 0.5f;
  const double bytes = 2.0 * g.E0 * g.E1 * 5 * tc_tile_floats(g.nc) * 4;
  const double f = 0.75 * l2 / bytes;
  return (float)(f > 1.0 ? 1.0 : (f < 0.05 ? 0.05 : f));
}

void launch_stack_tiles(const CoarseGeom& g, const double2* Y, float* T, int adj, cudaStream_t s) {
  k_stack_tiles<<<g.E0 * g.E1 * 5, 256, 0, s>>>(Y, T, g.E0, g.E1, g.nc, adj);
  SW_LAUNCH_CHECK();
}

// Pipeline depths compiled for a width (2 or 4 stages up to 16 right-hand
// sides, 2 or 3 above) that fit the 227 KB of shared memory of a CTA with its
// static state; the autotuner picks among them.
int tc_stage_options(int nc, int K, int* out) {
  const long stage = 128L * nc * 4 + 2L * K * nc * 4;
  const long fixed = 128L * 32 * 4 + 1024 + 12 * 1024;
  const int cand[2] = {2, K <= 16 ? 4 : 3};
  int n = 0;
  for (int S : cand)
    if (S * stage + fixed <= 227L * 1024) out[n++] = S;
  return n;
}

bool launch_cgne_tc(const CoarseGeom& g, int stages, bool f32, const float* At, const float* Ad,
                    int nb, const double2* const* b, double2* const* x, double2* X, double2* R,
                    double2* P, float* Rt, float* Pt, double* partials, unsigned* bar,
                    int* status, int maxit, double tol, int device, cudaStream_t s, int stall,
                    int sms_use, float l2frac) {
  const int K = tc_width(nb);
  if (nb < 1 || nb > kMaxK || !tc_supported(g.nc)) return false;
  SW_CUDA(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s));
  SW_CUDA(cudaMemsetAsync(status, 0, (2 + kMaxK) * sizeof(int), s));
  TcArgs a{At, Ad, b, x, X, R, P, Rt, Pt, partials, bar, status, nb, g.E0, g.E1, maxit, tol,
           stall, l2frac < 0.f ? 0.f : (l2frac > 1.f ? 1.f : l2frac)};
  switch (g.nc) {
    case 16: return run_nc16(a, K, stages, f32, device, s, sms_use);
    case 24: return run_nc24(a, K, stages, f32, device, s, sms_use);
    case 64: return run_nc64(a, K, stages, f32, device, s, sms_use);
    default: return false;
  }
}
