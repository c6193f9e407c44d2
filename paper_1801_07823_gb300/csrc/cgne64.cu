// Coarsest-level CGNE in FP64 (CG on the normal error, Sec. IV and Table
// kcycle) as one persistent cooperative kernel, with the stencil products done
// by the three-multiplication complex product.
//
// GB300 runs FP64 at 4 flop per clock per SM, so the coarsest stencil (about
// 0.5 flop per byte) is bound by the FP64 pipe, not by memory.  A complex
// multiply-add a v (a = alpha + i beta, v = c + i d) costs four real FMAs done
// directly.  With the sum alpha + beta of every stencil entry stored beside the
// entry (one more double per entry, computed once per hierarchy) and the
// vector kept as (c, d, c + d, c - d), a row of the stencil needs three
// real FMAs per entry (Higham, "Stability of a method for multiplying complex
// matrices with three real matrix multiplications", SIAM J. Matrix Anal. Appl.
// 13 (1992)):
//   A v:     K1 += (alpha + beta) c,  K2 += beta (c + d),  K3 -= alpha (c - d)
//            Re = K1 - K2,  Im = K1 + K3
//   A^dag v: K1 += (alpha + beta) d,  K2 += alpha (c - d), K3 += beta (c + d)
//            Re = K1 + K2,  Im = K1 - K3
// The result differs from the four-FMA product only by rounding; its error
// bound is normwise (|alpha| + |beta|)(|c| + |d|) u per term instead of
// componentwise, which is immaterial for a solve stopped at 0.2.
//
// Iteration (same as cgne.cu): P1 w = A p, x += alpha p, r -= alpha w, |r|^2;
// grid barrier; P2 p = A^dag r + beta p, |p|^2; grid barrier.
//
// Work distribution.  One CTA of 16 warps per SM; the FP64 pipe belongs to
// an SM sub-partition (warp w runs on sub-partition w mod 4), so work is dealt
// to the 4 x gridDim sub-partitions first and to their four warps second.  A
// work unit is four rows of one site: eight lanes per row, lane q taking the
// columns j = q, q + 8, q + 16, ... of all five blocks, so that a warp's load
// covers whole 32-byte sectors for A (four consecutive rows of a column-major
// block column) and for A^dag (eight consecutive entries of a block column).
// At 16^2 sites x 64 rows this gives 4096 units over 608 sub-partitions
// (6.7 each, at most 7: 96 % balance).  The eight lanes of a row are added by
// a fixed shuffle butterfly; norms are summed per CTA in warp order and over
// CTAs in CTA order, so every CTA takes the same decision and every run gives
// the same bits.
//
// Four variants, chosen per hierarchy by timing (mg.cu).  Bit 0 of the
// variant selects the three-FMA product above, whose stencil plus its sum
// plane takes 1.5 times the bytes of the stencil (at 16^2 x 64 dof: 126 MB,
// more than the L2 holds), over the plain four-FMA product on the stencil
// alone (84 MB).  Bit 1 selects the reduce-scatter row sums and the
// per-component update (phase_rs), which spend fewer FP64 instructions
// outside the stencil products.  Stencil loads carry an L2
// eviction-priority policy: the fraction l2frac of the lines, sized on the host
// to what the L2 can keep, are marked evict-last and the rest evict-first, so
// that a cyclic sweep over a stencil larger than the L2 keeps hitting on most
// of it instead of missing on all of it.
//
// Grid barriers use one monotone arrival counter (no reset between phases);
// waits are bounded (SW_ERR_TIMEOUT on the host), and a CTA that gives up
// leaves at its next barrier.
#include "sw_internal.h"

namespace {

constexpr long kSpinLimit = 1L << 24;
constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int kRows = 4;   // rows per work unit
constexpr int kQ = 8;      // lanes per row

struct alignas(32) V4 {
  double c, d, cpd, cmd;  // c, d, c + d, c - d of v = c + i d
};

__device__ __forceinline__ V4 v4_of(double2 v) { return V4{v.x, v.y, v.x + v.y, v.x - v.y}; }
__device__ __forceinline__ V4 ld_v4(const V4* p) {
  const double2* q = reinterpret_cast<const double2*>(p);
  double2 lo = __ldcg(q), hi = __ldcg(q + 1);
  return V4{lo.x, lo.y, hi.x, hi.y};
}
__device__ __forceinline__ void st_v4(V4* p, V4 v) {
  double2* q = reinterpret_cast<double2*>(p);
  q[0] = make_double2(v.c, v.d);
  q[1] = make_double2(v.cpd, v.cmd);
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

struct Args {
  const double2* Y;   // stencil, column-major nc x nc blocks: ((X 5 + d) nc + j) nc + i
  const double* Ys;   // Re + Im of every entry of Y, same indexing
  const double2* b;
  double2* x;
  double2* r;
  double2* p;
  V4* r4;             // (c, d, c + d, c - d) forms of r and p read by the stencil
  V4* p4;
  double* partials;   // [2][gridDim.x]
  unsigned* bar;      // [0] monotone arrival counter
  int* status;        // [0] iterations, [1] barrier timeout, [2] non-finite residual
  int E0, E1, maxit;
  double tol;
  int stall_test;     // 1: CTA 0 never arrives at the first barrier
  float l2frac;       // fraction of stencil lines loaded with L2 evict-last priority
};

__device__ __forceinline__ unsigned long long l2_policy(float frac) {
  unsigned long long pol;
  asm volatile("createpolicy.fractional.L2::evict_last.L2::evict_first.b64 %0, %1;"
               : "=l"(pol)
               : "f"(frac));
  return pol;
}
__device__ __forceinline__ double2 ld_y(const double2* p, unsigned long long pol) {
  double2 v;
  asm volatile("ld.global.nc.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;"
               : "=d"(v.x), "=d"(v.y)
               : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ double ld_s(const double* p, unsigned long long pol) {
  double v;
  asm volatile("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ double2 ld_cd(const V4* p) {
  return __ldcg(reinterpret_cast<const double2*>(p));
}

// Grid barrier number `gen` (1, 2, ...): returns false if a wait gave up here
// or elsewhere.
__device__ bool grid_barrier(unsigned* bar, int* status, unsigned gen) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned target = gen * gridDim.x;
    __threadfence();
    atomicAdd(bar, 1u);
    volatile unsigned* cnt = bar;
    long spins = 0;
    while (*cnt < target) {
      if (++spins > kSpinLimit) {
        atomicExch(status + 1, 1);
        break;
      }
      __nanosleep(16);
    }
    __threadfence();
    ok = *((volatile int*)(status + 1)) == 0;
  }
  __syncthreads();
  return ok;
}

// One double per thread summed in a fixed order into partials[blockIdx.x].
__device__ void cta_partial(double v, double* red, double* partials) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < kWarps; ++q) s += red[q];
    partials[blockIdx.x] = s;
  }
}
// Sum of all partials in the same order in every CTA.
__device__ double grid_sum(const double* partials, double* bcast) {
  if (threadIdx.x < 32) {
    const int G = gridDim.x;
    double v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int q = threadIdx.x + 32 * k;
      v[k] = q < G ? __ldcg(partials + q) : 0.0;
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += v[k];
    for (int q = threadIdx.x + 256; q < G; q += 32) s += __ldcg(partials + q);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) *bcast = s;
  }
  __syncthreads();
  return *bcast;
}

// Row i of (A v)_X (DAG: (A^dag v)_X), the part of lane q; the caller adds the
// eight lanes.  M3: three-FMA partial sums (K1, K2, K3); otherwise K1, K2 are
// the real and imaginary parts of the four-FMA product and K3 stays 0.
template <int NC, bool DAG, bool M3>
__device__ __forceinline__ void row_part(const Args& a, const V4* __restrict__ v, int X, int i,
                                         int q, unsigned long long pol, double& K1, double& K2,
                                         double& K3) {
  K1 = K2 = K3 = 0.0;
#pragma unroll 1
  for (int d = 0; d < 5; ++d) {
    const int nb = nbr(X, d, a.E0, a.E1);
    // A: entry (i, j) of block (X, d) at j NC + i; A^dag: entry (j, i) of block
    // (nb, opp d) at i NC + j.
    const long base = DAG ? ((long)(nb * 5 + opp(d)) * NC + i) * NC + q
                          : ((long)(X * 5 + d) * NC + q) * NC + i;
    const long step = DAG ? kQ : (long)kQ * NC;
    const V4* vb = v + (long)nb * NC + q;
#pragma unroll 4
    for (int t = 0; t < NC / kQ; ++t) {
      const double2 y = ld_y(a.Y + base + t * step, pol);
      if (M3) {
        const double s = ld_s(a.Ys + base + t * step, pol);
        const V4 w = ld_v4(vb + t * kQ);
        if (!DAG) {
          K1 = fma(s, w.c, K1);
          K2 = fma(y.y, w.cpd, K2);
          K3 = fma(-y.x, w.cmd, K3);
        } else {
          K1 = fma(s, w.d, K1);
          K2 = fma(y.x, w.cmd, K2);
          K3 = fma(y.y, w.cpd, K3);
        }
      } else {
        const double2 w = ld_cd(vb + t * kQ);
        if (!DAG) {  // (a + i b)(c + i d)
          K1 = fma(y.x, w.x, K1);
          K1 = fma(-y.y, w.y, K1);
          K2 = fma(y.x, w.y, K2);
          K2 = fma(y.y, w.x, K2);
        } else {     // (a - i b)(c + i d)
          K1 = fma(y.x, w.x, K1);
          K1 = fma(y.y, w.y, K1);
          K2 = fma(y.x, w.y, K2);
          K2 = fma(-y.y, w.x, K2);
        }
      }
    }
  }
}

__device__ __forceinline__ double bfly8(double v) {
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  return v;
}

enum { kInit = 0, kP1 = 1, kP2 = 2 };

// Component c (0: real, 1: imaginary) of complex element e.
__device__ __forceinline__ double ld_comp(const double2* v, long e, int c) {
  return __ldcg(reinterpret_cast<const double*>(v + e) + c);
}
__device__ __forceinline__ void st_comp(double2* v, long e, int c, double x) {
  reinterpret_cast<double*>(v + e)[c] = x;
}

// Reduce-scatter form of the row sum and update (variants 2 and 3).  Each lane
// first combines its partial sums into its share of Re and Im (three-FMA form:
// Re = K1 -+ K2, Im = K1 +- K3); one exchange across lanes q and q ^ 4 leaves
// lanes 0-3 with Re and lanes 4-7 with Im, and two more levels complete the
// sums: five FP64 additions per lane instead of nine.  Lanes 0 and 4 then
// update one component each of the element (x, r and p are read and written
// per component), which halves the FP64 instructions of the update; the
// (c, d, c + d, c - d) form is completed with one more exchange.
template <int NC, bool M3, int MODE>
__device__ double phase_rs(const Args& a, double coef, unsigned long long pol) {
  constexpr int kUnitsPerSite = NC / kRows;
  const int G = gridDim.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int sub = warp & 3, wj = warp >> 2;
  const int rr = lane >> 3, q = lane & 7;
  const int comp = (q >> 2) & 1;  // 0: this lane ends with Re, 1: with Im
  const bool writer = (q & 3) == 0;
  const int nunits = a.E0 * a.E1 * kUnitsPerSite;
  const V4* v = MODE == kP1 ? a.p4 : a.r4;
  double acc = 0.0;
  for (int u = sub * G + blockIdx.x + 4 * G * wj; u < nunits; u += 16 * G) {  // warp-uniform
    const int X = u / kUnitsPerSite;
    const int i = (u - X * kUnitsPerSite) * kRows + rr;
    double K1, K2, K3;
    row_part<NC, MODE != kP1, M3>(a, v, X, i, q, pol, K1, K2, K3);
    double re, im;
    if (!M3) {
      re = K1;
      im = K2;
    } else if (MODE == kP1) {  // A v
      re = K1 - K2;
      im = K1 + K3;
    } else {  // A^dag v
      re = K1 + K2;
      im = K1 - K3;
    }
    double w = comp ? im : re;
    w += __shfl_xor_sync(0xffffffffu, comp ? re : im, 4);
    w += __shfl_xor_sync(0xffffffffu, w, 2);
    w += __shfl_xor_sync(0xffffffffu, w, 1);
    const long e = (long)X * NC + i;
    double out;  // this lane's component of the new r (P1) or p
    if (MODE == kP1) {
      const double pc = ld_comp(a.p, e, comp);
      const double xc = fma(coef, pc, ld_comp(a.x, e, comp));
      out = fma(-coef, w, ld_comp(a.r, e, comp));
      if (writer) {
        st_comp(a.x, e, comp, xc);
        st_comp(a.r, e, comp, out);
      }
    } else {
      out = MODE == kP2 ? fma(coef, ld_comp(a.p, e, comp), w) : w;
      if (writer) st_comp(a.p, e, comp, out);
    }
    // (c, d, c + d, c - d): the Re lane adds the Im lane's value, the Im lane
    // subtracts it from the Re lane's
    const double other = __shfl_xor_sync(0xffffffffu, out, 4);
    V4* f = (MODE == kP1 ? a.r4 : a.p4) + e;
    if (writer) {
      double* fd = reinterpret_cast<double*>(f);
      fd[comp] = out;                                // c or d
      fd[2 + comp] = comp ? other - out : out + other;  // c + d or c - d
    }
    if (writer) acc = fma(out, out, acc);
  }
  return acc;
}

// ---- staged variant (7): the stencil rows, their sum plane and the
// neighbour's vector forms reach shared memory by asynchronous copies
// (cp.async), two chunks ahead of the FMAs, so that the loads in flight do not
// take registers.  A chunk is four t-steps of one direction of one unit; each
// warp owns three stage buffers of kStageBytes.
constexpr int kCh = 4;  // t-steps per chunk
constexpr int kStageBytes = kCh * 32 * 16 + kCh * 32 * 8 + kCh * 8 * 32;  // Y, Ys, vector forms
constexpr int kStages = 3;
constexpr int kStagedSmem = kWarps * kStages * kStageBytes;  // 192 KB

__device__ __forceinline__ void cp16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                   (unsigned)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp16h(void* dst, const void* src, unsigned long long pol) {
  asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(
                   (unsigned)__cvta_generic_to_shared(dst)),
               "l"(src), "l"(pol)
               : "memory");
}
__device__ __forceinline__ void cp8h(void* dst, const void* src, unsigned long long pol) {
  asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1], 8, %2;" ::"r"(
                   (unsigned)__cvta_generic_to_shared(dst)),
               "l"(src), "l"(pol)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// This warp's chunks: chunk k is half h of direction d of unit m, the unit
// being u0 + m 16 G (units are dealt to sub-partitions first, as in phase).
template <int NC>
struct StMap {
  static constexpr int kUnitsPerSite = NC / kRows;
  static constexpr int kHalves = NC / (kQ * kCh);  // chunks per direction
  static constexpr int kItems = 5 * kHalves;       // chunks per unit
  int G, lane, rr, q, u0, nk;
  unsigned char* mine;  // this warp's three stages
  __device__ StMap(const Args& a, unsigned char* smem) {
    static_assert(NC % (kQ * kCh) == 0, "a direction must split into whole chunks");
    G = gridDim.x;
    const int warp = threadIdx.x >> 5;
    lane = threadIdx.x & 31;
    rr = lane >> 3;
    q = lane & 7;
    const int nunits = a.E0 * a.E1 * kUnitsPerSite;
    u0 = (warp & 3) * G + blockIdx.x + 4 * G * (warp >> 2);
    const int nmine = u0 < nunits ? (nunits - 1 - u0) / (16 * G) + 1 : 0;
    nk = nmine * kItems;
    mine = smem + (size_t)warp * kStages * kStageBytes;
  }
  __device__ void decode(int k, int& X, int& i, int& d, int& h) const {
    const int m = k / kItems, rem = k - m * kItems;
    d = rem / kHalves;
    h = rem - d * kHalves;
    const int u = u0 + m * 16 * G;
    X = u / kUnitsPerSite;
    i = (u - X * kUnitsPerSite) * kRows + rr;
  }
  __device__ unsigned char* stage(int k) const { return mine + (k % kStages) * kStageBytes; }
};

// Stencil rows and sum plane of chunk k (A: DAG = false; A^dag: true).
template <int NC, bool DAG>
__device__ __forceinline__ void st_stencil(const Args& a, const StMap<NC>& mp, int k,
                                           unsigned long long pol) {
  if (k >= mp.nk) return;
  int X, i, d, h;
  mp.decode(k, X, i, d, h);
  const int nb = nbr(X, d, a.E0, a.E1);
  const long base = DAG ? ((long)(nb * 5 + opp(d)) * NC + i) * NC + mp.q
                        : ((long)(X * 5 + d) * NC + mp.q) * NC + i;
  const long step = DAG ? kQ : (long)kQ * NC;
  unsigned char* st = mp.stage(k);
  double2* Yb = reinterpret_cast<double2*>(st);
  double* Sb = reinterpret_cast<double*>(st + kCh * 32 * 16);
#pragma unroll
  for (int tt = 0; tt < kCh; ++tt) {
    const long off = base + (long)(h * kCh + tt) * step;
    cp16h(Yb + tt * 32 + mp.lane, a.Y + off, pol);
    cp8h(Sb + tt * 32 + mp.lane, a.Ys + off, pol);
  }
}
// Vector forms of chunk k: the entries v[nb NC + (h kCh + tt) 8 + q] are 32
// consecutive V4s; lane copies entry `lane` (two 16-byte halves).
template <int NC>
__device__ __forceinline__ void st_vector(const Args& a, const StMap<NC>& mp, const V4* v,
                                          int k) {
  if (k >= mp.nk) return;
  int X, i, d, h;
  mp.decode(k, X, i, d, h);
  const int nb = nbr(X, d, a.E0, a.E1);
  V4* Wb = reinterpret_cast<V4*>(mp.stage(k) + kCh * 32 * 24);
  const V4* src = v + (long)nb * NC + h * kCh * kQ + mp.lane;
  cp16(Wb + mp.lane, src);
  cp16(reinterpret_cast<unsigned char*>(Wb + mp.lane) + 16,
       reinterpret_cast<const unsigned char*>(src) + 16);
}

// Issued before the grid barrier that precedes a phase: the stencil part of
// the phase's first two chunks (one copy group each), which depends on
// nothing the barrier waits for, so its latency overlaps the barrier.
template <int NC, int MODE>
__device__ void prefetch_st(const Args& a, unsigned long long pol, unsigned char* smem) {
  const StMap<NC> mp(a, smem);
  st_stencil<NC, MODE != kP1>(a, mp, 0, pol);
  cp_commit();
  st_stencil<NC, MODE != kP1>(a, mp, 1, pol);
  cp_commit();
}

// The phase itself, after prefetch_st<NC, MODE>: groups A, B (stencil of
// chunks 0, 1) are in flight; C, D bring their vector forms; then one group
// per chunk, two chunks ahead, so that waiting for all but the two newest
// groups always completes chunk k.
template <int NC, int MODE>
__device__ double phase_st(const Args& a, double coef, unsigned long long pol,
                           unsigned char* smem) {
  constexpr int kUnitsPerSite = StMap<NC>::kUnitsPerSite;
  constexpr int kItems = StMap<NC>::kItems;
  constexpr bool DAG = MODE != kP1;
  const StMap<NC> mp(a, smem);
  const int G = mp.G, lane = mp.lane, rr = mp.rr, q = mp.q, u0 = mp.u0, nk = mp.nk;
  const int comp = (q >> 2) & 1;
  const bool writer = (q & 3) == 0;
  const V4* v = MODE == kP1 ? a.p4 : a.r4;
  double acc = 0.0, K1 = 0.0, K2 = 0.0, K3 = 0.0;
  st_vector<NC>(a, mp, v, 0);
  cp_commit();
  st_vector<NC>(a, mp, v, 1);
  cp_commit();
  for (int k = 0; k < nk; ++k) {  // warp-uniform
    __syncwarp();  // every lane is done with chunk k - 1, whose stage chunk k + 2 reuses
    st_stencil<NC, DAG>(a, mp, k + 2, pol);
    st_vector<NC>(a, mp, v, k + 2);
    cp_commit();  // (an empty group past the end keeps the counting uniform)
    cp_wait<2>();  // this lane's copies of chunk k have landed
    __syncwarp();  // and so have the other lanes' (vector forms are shared)
    const unsigned char* st = mp.stage(k);
    const double2* Yb = reinterpret_cast<const double2*>(st);
    const double* Sb = reinterpret_cast<const double*>(st + kCh * 32 * 16);
    const V4* Wb = reinterpret_cast<const V4*>(st + kCh * 32 * 24);
#pragma unroll
    for (int tt = 0; tt < kCh; ++tt) {
      const double2 y = Yb[tt * 32 + lane];
      const double sv = Sb[tt * 32 + lane];
      const V4 w = Wb[tt * kQ + q];
      if (!DAG) {
        K1 = fma(sv, w.c, K1);
        K2 = fma(y.y, w.cpd, K2);
        K3 = fma(-y.x, w.cmd, K3);
      } else {
        K1 = fma(sv, w.d, K1);
        K2 = fma(y.x, w.cmd, K2);
        K3 = fma(y.y, w.cpd, K3);
      }
    }
    const int m = k / kItems;
    if (k - m * kItems != kItems - 1) continue;
    // unit complete: row sums and update, as in phase_rs
    const int u = u0 + m * 16 * G;
    const int X = u / kUnitsPerSite;
    const int i = (u - X * kUnitsPerSite) * kRows + rr;
    const double re = DAG ? K1 + K2 : K1 - K2;
    const double im = DAG ? K1 - K3 : K1 + K3;
    K1 = K2 = K3 = 0.0;
    double w = comp ? im : re;
    w += __shfl_xor_sync(0xffffffffu, comp ? re : im, 4);
    w += __shfl_xor_sync(0xffffffffu, w, 2);
    w += __shfl_xor_sync(0xffffffffu, w, 1);
    const long e = (long)X * NC + i;
    double out;
    if (MODE == kP1) {
      const double pc = ld_comp(a.p, e, comp);
      const double xc = fma(coef, pc, ld_comp(a.x, e, comp));
      out = fma(-coef, w, ld_comp(a.r, e, comp));
      if (writer) {
        st_comp(a.x, e, comp, xc);
        st_comp(a.r, e, comp, out);
      }
    } else {
      out = MODE == kP2 ? fma(coef, ld_comp(a.p, e, comp), w) : w;
      if (writer) st_comp(a.p, e, comp, out);
    }
    const double other = __shfl_xor_sync(0xffffffffu, out, 4);
    V4* f = (MODE == kP1 ? a.r4 : a.p4) + e;
    if (writer) {
      double* fd = reinterpret_cast<double*>(f);
      fd[comp] = out;
      fd[2 + comp] = comp ? other - out : out + other;
      acc = fma(out, out, acc);
    }
  }
  cp_wait<0>();
  return acc;
}

// One stencil application over this warp's units fused with its update;
// returns this thread's share of the new squared norm.
template <int NC, bool M3, int MODE>
__device__ double phase(const Args& a, double coef, unsigned long long pol) {
  constexpr int kUnitsPerSite = NC / kRows;
  const int G = gridDim.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int sub = warp & 3, wj = warp >> 2;  // sub-partition, warp within it
  const int rr = lane >> 3, q = lane & 7;
  const int nunits = a.E0 * a.E1 * kUnitsPerSite;
  const V4* v = MODE == kP1 ? a.p4 : a.r4;
  double acc = 0.0;
  for (int u = sub * G + blockIdx.x + 4 * G * wj; u < nunits; u += 16 * G) {  // warp-uniform
    const int X = u / kUnitsPerSite;
    const int i = (u - X * kUnitsPerSite) * kRows + rr;
    double K1, K2, K3;
    row_part<NC, MODE != kP1, M3>(a, v, X, i, q, pol, K1, K2, K3);
    K1 = bfly8(K1);
    K2 = bfly8(K2);
    if (M3) K3 = bfly8(K3);
    if (q == 0) {
      const long e = (long)X * NC + i;
      if (MODE == kP1) {
        const double2 w = M3 ? make_double2(K1 - K2, K1 + K3) : make_double2(K1, K2);
        const double2 pv = __ldcg(a.p + e);
        double2 xv = __ldcg(a.x + e), rv = __ldcg(a.r + e);
        xv.x = fma(coef, pv.x, xv.x);
        xv.y = fma(coef, pv.y, xv.y);
        rv.x = fma(-coef, w.x, rv.x);
        rv.y = fma(-coef, w.y, rv.y);
        a.x[e] = xv;
        a.r[e] = rv;
        st_v4(a.r4 + e, v4_of(rv));
        acc = fma(rv.x, rv.x, fma(rv.y, rv.y, acc));
      } else {
        const double2 w = M3 ? make_double2(K1 + K2, K1 - K3) : make_double2(K1, K2);
        double2 pv = w;
        if (MODE == kP2) {
          pv = __ldcg(a.p + e);
          pv.x = fma(coef, pv.x, w.x);
          pv.y = fma(coef, pv.y, w.y);
        }
        a.p[e] = pv;
        st_v4(a.p4 + e, v4_of(pv));
        acc = fma(pv.x, pv.x, fma(pv.y, pv.y, acc));
      }
    }
  }
  return acc;
}

template <int NC, bool M3, bool RS, bool ST, int MODE>
__device__ __forceinline__ double run_phase(const Args& a, double coef, unsigned long long pol,
                                           unsigned char* smem) {
  if constexpr (ST)
    return phase_st<NC, MODE>(a, coef, pol, smem);
  else if constexpr (RS)
    return phase_rs<NC, M3, MODE>(a, coef, pol);
  else
    return phase<NC, M3, MODE>(a, coef, pol);
}

// The staged variant's pre-barrier copies of the next phase (no-op otherwise).
template <int NC, bool ST, int MODE>
__device__ __forceinline__ void prefetch(const Args& a, unsigned long long pol,
                                         unsigned char* smem) {
  if constexpr (ST) prefetch_st<NC, MODE>(a, pol, smem);
}
// Every exit first waits for this thread's asynchronous copies still in flight
// (the staged variant prefetches ahead of barriers), so that none lands in
// shared memory after the CTA has left.
__device__ __forceinline__ void leave() { cp_wait<0>(); }

template <int NC, bool M3, bool RS, bool ST>
__global__ void __launch_bounds__(kThreads, 1) k_cgne64(Args a) {
  extern __shared__ __align__(128) unsigned char stage_smem[];  // staged variant only
  __shared__ double red[kWarps];
  __shared__ double bcast;
  __shared__ double sh_rr, sh_stop, sh_coef;
  __shared__ int sh_state;  // 0: continue, 1: converged / cap, 2: non-finite
  const long n = (long)a.E0 * a.E1 * NC;
  const long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long nthr = (long)gridDim.x * blockDim.x;
  unsigned gen = 0;
  const unsigned long long pol = l2_policy(a.l2frac);

  // x = 0, r = b, ||r||^2
  double acc = 0.0;
  for (long e = tid; e < n; e += nthr) {
    const double2 v = a.b[e];
    a.x[e] = make_double2(0.0, 0.0);
    a.r[e] = v;
    st_v4(a.r4 + e, v4_of(v));
    acc = fma(v.x, v.x, fma(v.y, v.y, acc));
  }
  int ph = 0;
  prefetch<NC, ST, kInit>(a, pol, stage_smem);
  cta_partial(acc, red, a.partials + ph * gridDim.x);
  if (a.stall_test && blockIdx.x == 0) return leave();  // the others' first wait must run out
  if (!grid_barrier(a.bar, a.status, ++gen)) return leave();
  {
    const double rr0 = grid_sum(a.partials + ph * gridDim.x, &bcast);
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
    return leave();
  }
  // p = A^dag r, ||p||^2
  acc = run_phase<NC, M3, RS, ST, kInit>(a, 0.0, pol, stage_smem);
  prefetch<NC, ST, kP1>(a, pol, stage_smem);
  cta_partial(acc, red, a.partials + ph * gridDim.x);
  if (!grid_barrier(a.bar, a.status, ++gen)) return leave();
  {
    const double pp = grid_sum(a.partials + ph * gridDim.x, &bcast);
    if (threadIdx.x == 0) sh_coef = sh_rr / pp;  // alpha
    __syncthreads();
  }
  ph ^= 1;
  int k = 0;
  for (;;) {
    acc = run_phase<NC, M3, RS, ST, kP1>(a, sh_coef, pol, stage_smem);  // w = A p; x += alpha p; r -= alpha w
    prefetch<NC, ST, kP2>(a, pol, stage_smem);  // unused if this was the last iteration
    cta_partial(acc, red, a.partials + ph * gridDim.x);
    if (!grid_barrier(a.bar, a.status, ++gen)) return leave();
    ++k;
    {
      const double rr_new = grid_sum(a.partials + ph * gridDim.x, &bcast);
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
    acc = run_phase<NC, M3, RS, ST, kP2>(a, sh_coef, pol, stage_smem);  // p = A^dag r + beta p
    prefetch<NC, ST, kP1>(a, pol, stage_smem);
    cta_partial(acc, red, a.partials + ph * gridDim.x);
    if (!grid_barrier(a.bar, a.status, ++gen)) return leave();
    {
      const double pp = grid_sum(a.partials + ph * gridDim.x, &bcast);
      if (threadIdx.x == 0) sh_coef = sh_rr / pp;  // alpha
      __syncthreads();
    }
    ph ^= 1;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.status[0] = k;
    if (sh_state == 2) a.status[2] = 1;
  }
  leave();
}

__global__ void k_sum_planes(const double2* __restrict__ Y, double* __restrict__ Ys, long n) {
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long)gridDim.x * blockDim.x) {
    const double2 y = Y[e];
    Ys[e] = y.x + y.y;
  }
}

template <int NC, bool M3, bool RS, bool ST>
bool launch_t(const Args& args, int device, cudaStream_t s, int sms_use) {
  static int cached_sms[64] = {0};
  int& sms = cached_sms[device & 63];
  const int smem = ST ? kStagedSmem : 0;
  if (sms == 0) {
    int occ = 0, coop = 0, n = 0;
    if (ST)
      SW_CUDA(cudaFuncSetAttribute(k_cgne64<NC, M3, RS, ST>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    SW_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cgne64<NC, M3, RS, ST>,
                                                          kThreads, smem));
    SW_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, device));
    SW_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device));
    if (!coop || occ < 1 || n > kReduceBlocks) return false;
    sms = n;
  }
  // one CTA of 16 warps per SM it may use (partials hold 2 x kReduceBlocks)
  const int grid = sms_use < sms ? (sms_use > 0 ? sms_use : 1) : sms;
  Args a = args;
  void* params[] = {&a};
  SW_CUDA(cudaLaunchCooperativeKernel((const void*)k_cgne64<NC, M3, RS, ST>, dim3(grid),
                                      dim3(kThreads), params, smem, s));
  sw_count_launch();
  return true;
}

// variant bit 0: three-FMA products; bit 1: reduce-scatter row sums and update;
// 7: both, with the operands staged in shared memory (nc a multiple of 32)
template <int NC>
bool launch_v(const Args& a, int variant, int device, cudaStream_t s, int sms_use) {
  switch (variant) {
    case 0: return launch_t<NC, false, false, false>(a, device, s, sms_use);
    case 1: return launch_t<NC, true, false, false>(a, device, s, sms_use);
    case 2: return launch_t<NC, false, true, false>(a, device, s, sms_use);
    case 3: return launch_t<NC, true, true, false>(a, device, s, sms_use);
    case 7:
      if constexpr (NC % (kQ * kCh) == 0) return launch_t<NC, true, true, true>(a, device, s, sms_use);
      return false;
    default: return false;
  }
}

}  // namespace

void launch_sum_planes(const double2* Y, double* Ys, long n, cudaStream_t s) {
  k_sum_planes<<<1216, 256, 0, s>>>(Y, Ys, n);
  SW_LAUNCH_CHECK();
}

bool cgne64_supported(int nc) {
  return nc == 16 || nc == 24 || nc == 32 || nc == 48 || nc == 64;
}
bool cgne64_staged_supported(int nc) { return nc % (kQ * kCh) == 0 && cgne64_supported(nc); }

// Fraction of a stencil of `bytes` that the L2 can keep resident across a
// sweep (three quarters of its capacity, the rest left to vectors and other
// traffic).
float cgne64_l2_fraction(long bytes, int device) {
  int l2 = 0;
  SW_CUDA(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, device));
  const double f = 0.75 * (double)l2 / (double)(bytes > 0 ? bytes : 1);
  return (float)(f < 1.0 ? f : 1.0);
}

bool launch_cgne64(const CoarseGeom& g, int variant, const double2* Y, const double* Ys,
                   const double2* b, double2* x, double2* r, double2* p, double* v4,
                   double* partials, unsigned* bar, int* status, int maxit, double tol,
                   int device, cudaStream_t s, int stall_test, int sms_use) {
  if (!cgne64_supported(g.nc)) return false;
  SW_REQUIRE(((size_t)v4 & 31) == 0, SW_ERR_ARG, "CGNE vector forms need 32-byte alignment");
  SW_REQUIRE((variant >= 0 && variant <= 3) || variant == 7, SW_ERR_ARG,
             "FP64 coarsest CGNE variant is 0..3 or 7");
  SW_REQUIRE(!(variant & 1) || Ys, SW_ERR_ARG, "three-FMA CGNE needs the sum plane");
  SW_CUDA(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s));
  SW_CUDA(cudaMemsetAsync(status, 0, 3 * sizeof(int), s));
  const long n = (long)g.E0 * g.E1 * g.nc;
  const long ybytes = (long)g.E0 * g.E1 * 5 * g.nc * g.nc * ((variant & 1) ? 24 : 16);
  Args a{Y, Ys, b, x, r, p, reinterpret_cast<V4*>(v4), reinterpret_cast<V4*>(v4) + n, partials,
         bar, status, g.E0, g.E1, maxit, tol, stall_test, cgne64_l2_fraction(ybytes, device)};
  switch (g.nc) {
    case 16: return launch_v<16>(a, variant, device, s, sms_use);
    case 24: return launch_v<24>(a, variant, device, s, sms_use);
    case 32: return launch_v<32>(a, variant, device, s, sms_use);
    case 48: return launch_v<48>(a, variant, device, s, sms_use);
    case 64: return launch_v<64>(a, variant, device, s, sms_use);
    default: return false;
  }
}
