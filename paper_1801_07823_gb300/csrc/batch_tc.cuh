// Batched coarsest-level CGNE with the stencil contraction on the tensor cores
// (tcgen05.mma, TF32 operands, FP32 accumulation in tensor memory), for
// batched solves of a mixed-precision hierarchy.
//
// The iteration is that of batch_cgne.cu (same steps, same stopping rules, one
// alpha, beta and stopping test per right-hand side); only the stencil
// products run differently.  For a coarse site X and direction d the product
// Z v (Z = Z_r + i Z_i the nc x nc block, v = v_r + i v_i the nc x K block of
// the neighbour's vectors) is one real matrix product
//     [Z_r; Z_i] (128 x nc)  x  [v_r | v_i] (nc x 2K)
// whose four quadrants are Z_r v_r, Z_r v_i, Z_i v_r and Z_i v_i; the
// complex result is formed afterwards:  Re = Z_r v_r - Z_i v_i,
// Im = Z_r v_i + Z_i v_r.  The five directions of a site accumulate into the
// same tensor-memory tile (the combination is linear), so a site costs
// 5 x nc / 8 MMAs of shape M = 128, N = 2K, K = 8 and one read of the tile.
// Rows 2 nc .. 127 of the stacked block are zero when nc < 64.
//
// Operands live in global memory already in the tensor cores' shared-memory
// layout (K-major, 8-row x 16-byte core matrices, no swizzle): the stacked
// blocks of A and of A^dag are built once per hierarchy, rounded to TF32, and
// the kernel writes the right-hand-side tiles of r and p in that layout when it
// updates them.  One bulk asynchronous copy moves a tile into a pipeline
// stage; stages complete on mbarrier transaction counts.
//
// Roles in a CTA of 256 threads: thread 0 issues the bulk copies, thread 32
// allocates tensor memory and issues the MMAs (one elected thread), warps 4-7
// read the accumulator tile (one TMEM lane per thread), combine real and
// imaginary parts through shared memory, and do the FP64 updates of x, r and
// p, the TF32 tiles of the next stencil input and the per-right-hand-side
// norms.  Two accumulator tiles alternate, so the MMAs of one site overlap the
// epilogue of the previous one.
//
// Determinism: every output element is one tensor-core dot product of its own
// row and column, and norms are summed per site over fixed row groups, per
// CTA over its sites in order and over the CTAs in order (one CTA per SM), so
// a right-hand side's scalars do not depend on its batch-mates.
//
// Every wait is bounded.  A wait that gives up records SW_ERR_TIMEOUT in the
// status word; the CTA then stops issuing work, waits (bounded) for the copies
// and MMAs it has in flight, frees its tensor memory and leaves at the next
// grid barrier, where every other CTA sees the status and leaves too.
#pragma once
#include <cstring>
#include <string>
#include <type_traits>

#include "sw_internal.h"

namespace swtc {

constexpr long kSpinLimit = 1L << 24;      // grid-barrier polls
constexpr long kWaitLimit = 1L << 22;      // mbarrier polls
constexpr int kThreads = 256;
constexpr int kEpiThreads = 128;           // warps 4..7
constexpr int kMaxK = 64;

// ------------------------------------------------------------ PTX helpers
__device__ __forceinline__ unsigned su32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect(unsigned long long* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
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
static __device__ bool mbar_wait(unsigned long long* b, unsigned parity) {
  for (long k = 0; k < kWaitLimit; ++k)
    if (mbar_test(b, parity)) return true;
  return false;
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes,
                                          unsigned long long* b) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(su32(dst)),
      "l"(src), "r"(bytes), "r"(su32(b))
      : "memory");
}
// The same bulk copy with an L2 eviction-priority policy (createpolicy).
__device__ __forceinline__ void bulk_load_hint(void* dst, const void* src, unsigned bytes,
                                               unsigned long long* b, unsigned long long pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint "
      "[%0], [%1], %2, [%3], %4;" ::"r"(su32(dst)),
      "l"(src), "r"(bytes), "r"(su32(b)), "l"(pol)
      : "memory");
}
__device__ __forceinline__ unsigned long long policy_evict_first() {
  unsigned long long pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
// evict-last priority for the fraction frac of the lines, evict-first for the rest
__device__ __forceinline__ unsigned long long policy_keep_fraction(float frac) {
  unsigned long long pol;
  asm volatile("createpolicy.fractional.L2::evict_last.L2::evict_first.b64 %0, %1;"
               : "=l"(pol)
               : "f"(frac));
  return pol;
}
__device__ __forceinline__ unsigned long long policy_evict_last() {
  unsigned long long pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ void fence_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}
__device__ __forceinline__ void fence_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void epi_sync() {  // named barrier of the epilogue warps
  asm volatile("bar.sync 1, %0;" ::"n"(kEpiThreads) : "memory");
}
// Rounds an FP32 value to TF32 (10 explicit mantissa bits), to nearest with
// ties away from zero, by integer arithmetic on its bits: add half a unit of
// the last kept place to the magnitude bits and clear the 13 dropped bits (a
// carry into the exponent is the correct rounding up).  The tensor cores then
// read exactly this value.
__host__ __device__ __forceinline__ float to_tf32(float x) {
#ifdef __CUDA_ARCH__
  unsigned u = __float_as_uint(x);
#else
  unsigned u;
  std::memcpy(&u, &x, 4);
#endif
  u = (u + 0x1000u) & 0xFFFFE000u;
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float y;
  std::memcpy(&y, &u, 4);
  return y;
#endif
}

// Shared-memory matrix descriptor, K-major without swizzle: start address,
// byte distance between core matrices adjacent along K (leading) and along
// M/N (stride), descriptor version 1 (sm_100 family).
__device__ __forceinline__ unsigned long long smem_desc(unsigned saddr, unsigned kstride,
                                                        unsigned mstride) {
  unsigned long long d = 0;
  d |= (unsigned long long)((saddr >> 4) & 0x3FFFu);
  d |= (unsigned long long)((kstride >> 4) & 0x3FFFu) << 16;
  d |= (unsigned long long)((mstride >> 4) & 0x3FFFu) << 32;
  d |= 1ull << 46;
  return d;
}
// Instruction descriptor of kind::tf32: D in FP32, A and B in TF32, both
// K-major, shape M x N.
__host__ __device__ constexpr unsigned idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned)(N >> 3) << 17) |
         ((unsigned)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_tf32(unsigned tmem, unsigned long long ad,
                                         unsigned long long bd, unsigned id, unsigned acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(id), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(unsigned long long* b) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          su32(b))
      : "memory");
}
// 32 consecutive accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(unsigned taddr, float* v) {
  unsigned r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int c = 0; c < 32; ++c) v[c] = __uint_as_float(r[c]);
}

// 16 consecutive accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(unsigned taddr, float* v) {
  unsigned r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int c = 0; c < 16; ++c) v[c] = __uint_as_float(r[c]);
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

// Byte offset of element (row, k) in a K-major no-swizzle tile with `rows`
// rows: core matrix (row / 8, k / 4) at (k / 4 * rows / 8 + row / 8) * 128.
__host__ __device__ __forceinline__ unsigned tile_off(int row, int k, int rows) {
  return (unsigned)(((k >> 2) * (rows >> 3) + (row >> 3)) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

// ------------------------------------------------------------ kernel
struct TcArgs {
  const float* At;         // [sites][5] stacked forward blocks, 128 x nc TF32 tiles
  const float* Ad;         // [sites][5] stacked adjoint blocks
  const double2* const* b; // [K] right-hand sides
  double2* const* xout;    // [K] solutions
  void* X;                 // [n][K] iterates: double2, or float2 with FP32 iterates
  void* R;
  void* P;
  float* Rt;               // [sites] 2K x nc TF32 tiles of r (stencil input of A^dag)
  float* Pt;               // [sites] tiles of p (stencil input of A)
  double* partials;        // [2][K][gridDim.x]
  unsigned* bar;           // [0] monotone arrival counter
  int* status;             // [0] timeout / setup failure, [1] non-finite, [2 + r] iterations
  int nb, E0, E1, maxit;
  double tol;
  int stall;               // 1: CTA 0 withholds its first grid-barrier arrival
  float l2frac;            // > 0: that fraction of the stencil-tile lines is loaded with
                           // L2 evict-last priority; 0: all of them evict-first
};

enum { kInit = 0, kXR = 1, kP = 2 };

template <int NC, int K, int S>
struct TcCfg {
  static constexpr int kN = 2 * K;                   // MMA N
  static constexpr int kATile = 128 * NC * 4;        // bytes of a stacked block
  static constexpr int kBTile = kN * NC * 4;         // bytes of a right-hand-side tile
  static constexpr int kStage = kATile + kBTile;
  static constexpr int kGroups = NC / 8;             // row groups of the norm tree
  static constexpr int kPairs = K * kGroups;         // (rhs, row group) pairs per site
  static constexpr int kCols = 2 * kN < 32 ? 32 : 2 * kN;  // TMEM columns (2 tiles)
  static constexpr int kExch = 128 * 32 * 4;         // exchange buffer, 32 columns
  static constexpr int kSmem = S * kStage + kExch + 1024;
  static_assert(NC % 8 == 0 && 2 * NC <= 128, "stacked block must fit M = 128");
  static_assert(K % 8 == 0 && K <= kMaxK && kN >= 16, "N = 2K in 16 .. 128");
  static_assert((kCols & (kCols - 1)) == 0 && kCols <= 512, "TMEM columns");
};

template <int NC, int K, int S>
struct TcSmem {
  unsigned long long full[S], empty[S], acc_full[2], acc_empty[2];
  unsigned tmem;
  int abort;        // a wait gave up: stop issuing work
  int epi_go;       // epilogue decision for the current site (uniform over its warps)
  unsigned issued;  // stages filled so far (producer)
  unsigned mmaed;   // stages whose MMAs were issued and committed so far
  double sq[TcCfg<NC, K, S>::kPairs];       // per (rhs, row group) squared norms of a site
  double cta_sum[K];
  double red[K][8];
  double sum[K], rr[K], stop[K], coef[K];
  float coef_f[K];                           // coef in FP32 (FP32 iterates)
  int state[K];                              // 0 active, 1 stopped, 2 non-finite
  int iters[K];
  int any;
};

static __device__ bool grid_barrier_tc(unsigned* bar, int* status, unsigned gen) {
  __shared__ int ok;
  fence_async_global();  // generic writes of this phase before other CTAs' bulk reads
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned target = gen * gridDim.x;
    __threadfence();
    atomicAdd(bar, 1u);
    volatile unsigned* cnt = bar;
    long spins = 0;
    while (*cnt < target) {
      if (++spins > kSpinLimit) {
        atomicExch(status, 1);
        break;
      }
      __nanosleep(16);
    }
    __threadfence();
    ok = *((volatile int*)status) == 0;
  }
  __syncthreads();
  return ok;
}

template <int K>
__device__ void grid_sums_tc(const double* part, double* out) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int G = gridDim.x;
  for (int r = w; r < K; r += kThreads / 32) {
    const double* pr = part + r * G;
    double v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = lane + 32 * k < G ? __ldcg(pr + lane + 32 * k) : 0.0;
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += v[k];
    for (int q = lane + 256; q < G; q += 32) s += __ldcg(pr + q);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[r] = s;
  }
  __syncthreads();
}

template <typename Sm>
__device__ __forceinline__ bool aborted(const Sm& sm) {
  return *((const volatile int*)&sm.abort) != 0;
}

// Counters of the pipeline that persist across phases.
struct Pipe {
  unsigned q;  // stages used so far (buffer q % S, parity (q / S) & 1)
  unsigned a;  // accumulator tiles used so far (tile a & 1, parity (a >> 1) & 1)
};

// One stencil application over this CTA's sites fused with the update of the
// phase; leaves this CTA's per-right-hand-side norm sums in sm.cta_sum.
template <int NC, int K, int S, bool F32, int MODE>
__device__ void tc_phase(const TcArgs& a, unsigned char* stages, float* exch,
                         TcSmem<NC, K, S>& sm, Pipe& pp) {
  using C = TcCfg<NC, K, S>;
  const int t = threadIdx.x, warp = t >> 5;
  const int G = gridDim.x, cta = blockIdx.x;
  const int nsites = a.E0 * a.E1;
  const int nmine = cta < nsites ? (nsites - 1 - cta) / G + 1 : 0;
  const int nitems = nmine * 5;
  const float* Ablk = MODE == kXR ? a.At : a.Ad;
  const float* Vt = MODE == kXR ? a.Pt : a.Rt;
  if (t < K) sm.cta_sum[t] = 0.0;

  if (t == 0) {
    // ---------------- producer: one (site, direction) pair per stage
    fence_async_global();
    // stencil tiles: read once per phase, so either streamed (evict first) or,
    // when the autotuner found it faster, a fraction of them kept in L2 across
    // iterations; right-hand-side tiles are read by the five sites around
    // their own: keep them
    const unsigned long long pol_stream =
        a.l2frac > 0.f ? policy_keep_fraction(a.l2frac) : policy_evict_first();
    const unsigned long long pol_keep = policy_evict_last();
    for (int it = 0; it < nitems && !aborted(sm); ++it) {
      const unsigned q = pp.q + it;
      const int s = q % S;
      if (q >= (unsigned)S && !mbar_wait(&sm.empty[s], ((q / S) - 1) & 1u)) {
        sm.abort = 1;
        atomicExch(a.status, 1);
        break;
      }
      const int m = it / 5, d = it - 5 * m;
      const int X = cta + G * m;
      const int nb = nbr(X, d, a.E0, a.E1);
      unsigned char* buf = stages + (size_t)s * C::kStage;
      mbar_expect(&sm.full[s], (unsigned)C::kStage);
      bulk_load_hint(buf, Ablk + ((size_t)X * 5 + d) * (C::kATile / 4), C::kATile, &sm.full[s],
                     pol_stream);
      bulk_load_hint(buf + C::kATile, Vt + (size_t)nb * (C::kBTile / 4), C::kBTile, &sm.full[s],
                     pol_keep);
      sm.issued = q + 1;
    }
  } else if (t == 32) {
    // ---------------- MMA issuer
    constexpr unsigned id = idesc_tf32(128, C::kN);
    for (int it = 0; it < nitems && !aborted(sm); ++it) {
      const unsigned q = pp.q + it;
      const int s = q % S;
      const int m = it / 5, d = it - 5 * m;
      const unsigned at = pp.a + m;
      const int tile = at & 1;
      if (d == 0 && at >= 2 && !mbar_wait(&sm.acc_empty[tile], ((at >> 1) - 1) & 1u)) {
        sm.abort = 1;
        atomicExch(a.status, 1);
        break;
      }
      if (!mbar_wait(&sm.full[s], (q / S) & 1u)) {
        sm.abort = 1;
        atomicExch(a.status, 1);
        break;
      }
      tc_fence_after();
      const unsigned base = su32(stages + (size_t)s * C::kStage);
      const unsigned tmem = sm.tmem + (unsigned)(tile * C::kN);
#pragma unroll
      for (int ks = 0; ks < NC / 8; ++ks) {
        const unsigned long long ad = smem_desc(base + ks * 2 * 2048, 2048, 128);
        const unsigned long long bd =
            smem_desc(base + C::kATile + ks * 2 * (C::kN / 8) * 128, (C::kN / 8) * 128, 128);
        mma_tf32(tmem, ad, bd, id, (d > 0 || ks > 0) ? 1u : 0u);
      }
      mma_commit(&sm.empty[s]);                     // stage free once these MMAs are done
      if (d == 4) mma_commit(&sm.acc_full[tile]);  // site's tile complete
      sm.mmaed = q + 1;
    }
  } else if (warp >= 4) {
    // ---------------- epilogue: one TMEM lane (stacked row) per thread
    const int e = t - 128;                 // 0 .. 127
    const int lrow = e;                    // TMEM lane = row of the stacked product
    constexpr int kg = K < 16 ? K : 16;    // right-hand sides per group
    constexpr int ngroups = K < 16 ? 1 : K / 16;
    constexpr int ioff = K < 16 ? K : 16;  // exchange column of the first imaginary-part product
    // this thread's work item in every group: right-hand side c0 + cr, rows
    // grp * 8 .. grp * 8 + 7 of the site
    const bool has_item = e < kg * C::kGroups;
    const int cr = e % kg, grp = e / kg;
    using V = typename std::conditional<F32, float2, double2>::type;
    V* Xv = reinterpret_cast<V*>(a.X);
    V* Rv = reinterpret_cast<V*>(a.R);
    V* Pv = reinterpret_cast<V*>(a.P);
    V xv[8], rv[8], pv[8];
    // The iterates of a group do not depend on the products, so their loads
    // are issued before the group's tensor-memory read (group 0's before the
    // wait for the site's accumulator tile) and their latency overlaps it.
    auto load_group = [&](int X, int g) {
      if (!has_item) return;
      const size_t el0 = ((size_t)X * NC + grp * 8) * K + (K < 16 ? 0 : 16 * g) + cr;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        if (MODE == kXR) {
          xv[k] = __ldcg(Xv + el0 + k * K);
          rv[k] = __ldcg(Rv + el0 + k * K);
          pv[k] = __ldcg(Pv + el0 + k * K);
        } else if (MODE == kP) {
          pv[k] = __ldcg(Pv + el0 + k * K);
        }
      }
    };
    for (int m = 0; m < nmine; ++m) {
      const unsigned at = pp.a + m;
      const int tile = at & 1;
      const int X = cta + G * m;
      load_group(X, 0);
      // one thread waits for the tile; the decision is shared so that every
      // epilogue thread takes the same branch at the named barriers below
      if (e == 0) {
        int go = !aborted(sm) && mbar_wait(&sm.acc_full[tile], (at >> 1) & 1u);
        if (!go && !aborted(sm)) {
          sm.abort = 1;
          atomicExch(a.status, 1);
        }
        sm.epi_go = go;
      }
      epi_sync();
      if (!sm.epi_go) break;
      tc_fence_after();
      // the combination of group g needs columns [16 g, 16 g + 16) and
      // [K + 16 g, K + 16 g + 16) of rows i and i + NC
      for (int g = 0; g < ngroups; ++g) {
        const int c0 = K < 16 ? 0 : 16 * g;       // K = 8: both halves in one 16-column load
        const unsigned lane_base = ((unsigned)(32 * (warp - 4))) << 16;
        if (g > 0) load_group(X, g);
        epi_sync();  // previous group's readers are done with exch
        {
          float w[32];
          if (K < 16) {
            tmem_ld16(sm.tmem + lane_base + tile * C::kN, w);
#pragma unroll
            for (int c = 0; c < 16; ++c) exch[lrow * 32 + ((c + lrow) & 31)] = w[c];
          } else {
            // (c0 & 31) and ((K + c0) & 31) are 0 or 16: select between two
            // static halves so that w stays in registers
            const bool h0 = (c0 & 31) != 0, h1 = ((K + c0) & 31) != 0;
            tmem_ld32(sm.tmem + lane_base + tile * C::kN + (c0 & ~31), w);
#pragma unroll
            for (int c = 0; c < 16; ++c)
              exch[lrow * 32 + ((c + lrow) & 31)] = h0 ? w[16 + c] : w[c];
            tmem_ld32(sm.tmem + lane_base + tile * C::kN + ((K + c0) & ~31), w);
#pragma unroll
            for (int c = 0; c < 16; ++c)
              exch[lrow * 32 + ((16 + c + lrow) & 31)] = h1 ? w[16 + c] : w[c];
          }
        }
        epi_sync();
        if (!has_item) continue;
        // combine: columns 0..15 hold Re-part products of rhs c0 + c (K = 8: 0..7),
        // columns 16..31 those of the imaginary parts (K = 8: columns 8..15)
        const int r = c0 + cr;
        float* vt = (MODE == kXR ? a.Rt : a.Pt) + (size_t)X * (C::kBTile / 4);
        const size_t el0 = ((size_t)X * NC + grp * 8) * K + r;  // row grp * 8, step K
        float re[8], im[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int i = grp * 8 + k;
          auto E = [&](int row, int col) { return exch[row * 32 + ((col + row) & 31)]; };
          re[k] = E(i, cr) - E(i + NC, ioff + cr);
          im[k] = E(i, ioff + cr) + E(i + NC, cr);
        }
        const bool live = MODE == kInit || sm.state[r] == 0;
        double q2 = 0.0;
        float tre[8], tim[8];  // TF32 copies of the new vector, stencil input of the next phase
        if constexpr (F32) {
          const float cf = sm.coef_f[r];
          float s8 = 0.f;
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            float2 o;
            if (MODE == kXR) {
              o = rv[k];
              if (live) {
                float2 xn = xv[k];
                xn.x = fmaf(cf, pv[k].x, xn.x);
                xn.y = fmaf(cf, pv[k].y, xn.y);
                o.x = fmaf(-cf, re[k], o.x);
                o.y = fmaf(-cf, im[k], o.y);
                Xv[el0 + k * K] = xn;
                Rv[el0 + k * K] = o;
              }
            } else {
              o = make_float2(re[k], im[k]);
              if (MODE == kP) {
                o = pv[k];
                if (live) {
                  o.x = fmaf(cf, o.x, re[k]);
                  o.y = fmaf(cf, o.y, im[k]);
                }
              }
              if (live) Pv[el0 + k * K] = o;
            }
            if (live) s8 = fmaf(o.x, o.x, fmaf(o.y, o.y, s8));
            tre[k] = to_tf32(o.x);
            tim[k] = to_tf32(o.y);
          }
          q2 = (double)s8;
        } else {
          const double cd = sm.coef[r];
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            double2 o;
            if (MODE == kXR) {
              o = rv[k];
              if (live) {
                double2 xn = xv[k];
                xn.x = fma(cd, pv[k].x, xn.x);
                xn.y = fma(cd, pv[k].y, xn.y);
                o.x = fma(-cd, (double)re[k], o.x);
                o.y = fma(-cd, (double)im[k], o.y);
                Xv[el0 + k * K] = xn;
                Rv[el0 + k * K] = o;
              }
            } else {
              o = make_double2((double)re[k], (double)im[k]);
              if (MODE == kP) {
                o = pv[k];
                if (live) {
                  o.x = fma(cd, o.x, (double)re[k]);
                  o.y = fma(cd, o.y, (double)im[k]);
                }
              }
              if (live) Pv[el0 + k * K] = o;
            }
            if (live) q2 += fma(o.x, o.x, o.y * o.y);
            tre[k] = to_tf32((float)o.x);
            tim[k] = to_tf32((float)o.y);
          }
        }
        // the eight rows of a tile column are two runs of four consecutive
        // K-major elements (rows grp * 8 .. + 3 and + 4 .. + 7): 16-byte stores
        {
          float4* d = reinterpret_cast<float4*>(vt + tile_off(r, grp * 8, C::kN) / 4);
          d[0] = make_float4(tre[0], tre[1], tre[2], tre[3]);
          d = reinterpret_cast<float4*>(vt + tile_off(r, grp * 8 + 4, C::kN) / 4);
          d[0] = make_float4(tre[4], tre[5], tre[6], tre[7]);
          d = reinterpret_cast<float4*>(vt + tile_off(K + r, grp * 8, C::kN) / 4);
          d[0] = make_float4(tim[0], tim[1], tim[2], tim[3]);
          d = reinterpret_cast<float4*>(vt + tile_off(K + r, grp * 8 + 4, C::kN) / 4);
          d[0] = make_float4(tim[4], tim[5], tim[6], tim[7]);
        }
        sm.sq[r * C::kGroups + grp] = q2;
      }
      // tile read: hand it back to the MMA issuer
      tc_fence_before();
      epi_sync();
      if (e == 0) mbar_arrive(&sm.acc_empty[tile]);
      // site sums over row groups in order, then the CTA's running sum
      if (e < K) {
        double sv = 0.0;
        for (int q = 0; q < C::kGroups; ++q) sv += sm.sq[e * C::kGroups + q];
        sm.cta_sum[e] += sv;
      }
    }
  }
  pp.q += (unsigned)nitems;
  pp.a += (unsigned)nmine;
  __syncthreads();
}

// After a wait gave up: wait (bounded) for every copy and MMA this CTA may
// still have in flight (the last fill of each stage and the MMAs issued on
// it), so that none is outstanding when the tensor memory is freed.
template <int NC, int K, int S>
__device__ void tc_drain(TcSmem<NC, K, S>& sm) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned is = sm.issued, mm = sm.mmaed;
    for (unsigned q = is >= (unsigned)S ? is - S : 0u; q < is; ++q)
      mbar_wait(&sm.full[q % S], (q / S) & 1u);
    for (unsigned q = mm >= (unsigned)S ? mm - S : 0u; q < mm; ++q)
      mbar_wait(&sm.empty[q % S], (q / S) & 1u);
  }
  __syncthreads();
}

template <int NC, int K, int S, bool F32>
__global__ void __launch_bounds__(kThreads, 1) k_cgne_tc(TcArgs a) {
  using C = TcCfg<NC, K, S>;
  extern __shared__ __align__(1024) unsigned char dyn[];
  __shared__ TcSmem<NC, K, S> sm;
  unsigned char* stages =
      reinterpret_cast<unsigned char*>((reinterpret_cast<size_t>(dyn) + 1023) & ~(size_t)1023);
  float* exch = reinterpret_cast<float*>(stages + (size_t)S * C::kStage);
  const int t = threadIdx.x;
  const long n = (long)a.E0 * a.E1 * NC;
  const long tid = (long)blockIdx.x * blockDim.x + t;
  const long nthr = (long)gridDim.x * blockDim.x;
  Pipe pp{0u, 0u};
  unsigned gen = 0;

  if (t == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&sm.full[s], 1);
      mbar_init(&sm.empty[s], 1);
    }
    for (int k = 0; k < 2; ++k) {
      mbar_init(&sm.acc_full[k], 1);
      mbar_init(&sm.acc_empty[k], 1);
    }
    sm.abort = 0;
    sm.issued = sm.mmaed = 0u;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fence_async_shared();
    const size_t gl = (size_t)a.At | (size_t)a.Ad | (size_t)a.Rt | (size_t)a.Pt;
    if (((su32(stages) & 1023u) | (unsigned)(gl & 127)) != 0) atomicExch(a.status, 1);
  }
  if ((t >> 5) == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(&sm.tmem)),
                 "r"(C::kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();

  // gather: X = 0, R = b, Rt = tf32(b); then ||r||^2 per right-hand side, each
  // summed over this thread's dofs in the same order for every width K
  for (long dof = tid; dof < n; dof += nthr) {
    const int X = (int)(dof / NC), i = (int)(dof - (long)X * NC);
    float* vt = a.Rt + (size_t)X * (C::kBTile / 4);
    for (int r = 0; r < K; ++r) {
      const double2 v = r < a.nb ? a.b[r][dof] : make_double2(0.0, 0.0);
      if (F32) {
        reinterpret_cast<float2*>(a.X)[dof * K + r] = make_float2(0.f, 0.f);
        reinterpret_cast<float2*>(a.R)[dof * K + r] = make_float2((float)v.x, (float)v.y);
      } else {
        reinterpret_cast<double2*>(a.X)[dof * K + r] = make_double2(0.0, 0.0);
        reinterpret_cast<double2*>(a.R)[dof * K + r] = v;
      }
      vt[tile_off(r, i, C::kN) / 4] = to_tf32((float)v.x);
      vt[tile_off(K + r, i, C::kN) / 4] = to_tf32((float)v.y);
    }
  }
  int ph = 0;
  {
    const int lane = t & 31, w = t >> 5;
    for (int r = 0; r < K; ++r) {
      double s = 0.0;
      if (r < a.nb)
        for (long dof = tid; dof < n; dof += nthr) {
          const double2 v = a.b[r][dof];
          s = fma(v.x, v.x, fma(v.y, v.y, s));
        }
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) sm.red[r][w] = s;
    }
    __syncthreads();
    if (t < K) {
      double s = 0.0;
      for (int q = 0; q < kThreads / 32; ++q) s += sm.red[t][q];
      a.partials[(ph * K + t) * gridDim.x + blockIdx.x] = s;
    }
  }
  bool go = true;
  if (a.stall && blockIdx.x == 0) go = false;  // withheld arrival: the others time out
  if (go) go = grid_barrier_tc(a.bar, a.status, ++gen);
  if (go) {
    grid_sums_tc<K>(a.partials + ph * K * gridDim.x, sm.sum);
    if (t < K) {
      const double rr0 = sm.sum[t];
      sm.rr[t] = rr0;
      sm.stop[t] = a.tol * sqrt(rr0);
      sm.iters[t] = 0;
      sm.state[t] = !isfinite(rr0) ? 2 : ((a.maxit <= 0 || !(sqrt(rr0) > sm.stop[t])) ? 1 : 0);
    }
    __syncthreads();
    ph ^= 1;
    // p = A^dag r, ||p||^2
    tc_phase<NC, K, S, F32, kInit>(a, stages, exch, sm, pp);
    if (t < K) a.partials[(ph * K + t) * gridDim.x + blockIdx.x] = sm.cta_sum[t];
    go = !aborted(sm) && grid_barrier_tc(a.bar, a.status, ++gen);
  }
  if (go) {
    grid_sums_tc<K>(a.partials + ph * K * gridDim.x, sm.sum);
    if (t < K) {
      sm.coef[t] = sm.rr[t] / sm.sum[t];  // alpha
      sm.coef_f[t] = (float)sm.coef[t];
    }
    if (t == 0) {
      int any = 0;
      for (int r = 0; r < K; ++r) any |= sm.state[r] == 0;
      sm.any = any;
    }
    __syncthreads();
    ph ^= 1;
    while (sm.any) {
      tc_phase<NC, K, S, F32, kXR>(a, stages, exch, sm, pp);  // w = A p; x += alpha p; r -= alpha w
      if (t < K) a.partials[(ph * K + t) * gridDim.x + blockIdx.x] = sm.cta_sum[t];
      if (aborted(sm) || !grid_barrier_tc(a.bar, a.status, ++gen)) {
        go = false;
        break;
      }
      grid_sums_tc<K>(a.partials + ph * K * gridDim.x, sm.sum);
      if (t < K && sm.state[t] == 0) {
        const double rr_new = sm.sum[t];
        const int k = ++sm.iters[t];
        if (!isfinite(rr_new))
          sm.state[t] = 2;
        else if (!(k < a.maxit && sqrt(rr_new) > sm.stop[t]))
          sm.state[t] = 1;
        sm.coef[t] = rr_new / sm.rr[t];  // beta
        sm.coef_f[t] = (float)sm.coef[t];
        sm.rr[t] = rr_new;
      }
      __syncthreads();
      if (t == 0) {
        int any = 0;
        for (int r = 0; r < K; ++r) any |= sm.state[r] == 0;
        sm.any = any;
      }
      __syncthreads();
      ph ^= 1;
      if (!sm.any) break;
      tc_phase<NC, K, S, F32, kP>(a, stages, exch, sm, pp);  // p = A^dag r + beta p
      if (t < K) a.partials[(ph * K + t) * gridDim.x + blockIdx.x] = sm.cta_sum[t];
      if (aborted(sm) || !grid_barrier_tc(a.bar, a.status, ++gen)) {
        go = false;
        break;
      }
      grid_sums_tc<K>(a.partials + ph * K * gridDim.x, sm.sum);
      if (t < K && sm.state[t] == 0) {
        sm.coef[t] = sm.rr[t] / sm.sum[t];  // alpha
        sm.coef_f[t] = (float)sm.coef[t];
      }
      __syncthreads();
      ph ^= 1;
    }
  }
  if (!go) {
    if (aborted(sm)) atomicExch(a.status, 1);
    tc_drain<NC, K, S>(sm);
  }
  // every MMA of this CTA has completed here (the epilogue waited for each
  // site's tile, or the drain above waited for the stages); free the columns
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if ((t >> 5) == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(sm.tmem),
                 "r"(C::kCols)
                 : "memory");
  if (!go) return;
  for (long dof = tid; dof < n; dof += nthr)
    for (int r = 0; r < a.nb; ++r) {
      if (F32) {
        const float2 v = __ldcg(reinterpret_cast<const float2*>(a.X) + dof * K + r);
        a.xout[r][dof] = make_double2((double)v.x, (double)v.y);
      } else {
        a.xout[r][dof] = __ldcg(reinterpret_cast<const double2*>(a.X) + dof * K + r);
      }
    }
  if (blockIdx.x == 0 && t < K) {
    if (sm.state[t] == 2) atomicExch(a.status + 1, 1);
    a.status[2 + t] = sm.iters[t];
  }
}

template <int NC, int K, int S, bool F32>
void launch_tc_t(const TcArgs& args, int grid, cudaStream_t s) {
  using C = TcCfg<NC, K, S>;
  TcArgs a = args;
  void* params[] = {&a};
  SW_CUDA(cudaLaunchCooperativeKernel((const void*)k_cgne_tc<NC, K, S, F32>, dim3(grid),
                                      dim3(kThreads), params, C::kSmem, s));
  sw_count_launch();
}

template <int NC, int K, int S, bool F32>
bool prepare_t(int device, int& grid) {
  using C = TcCfg<NC, K, S>;
  int occ = 0, sms = 0, coop = 0;
  SW_CUDA(cudaFuncSetAttribute((const void*)k_cgne_tc<NC, K, S, F32>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmem));
  SW_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cgne_tc<NC, K, S, F32>, kThreads,
                                                        C::kSmem));
  SW_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  SW_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device));
  if (!coop || occ < 1) return false;
  grid = sms;
  return true;
}

// Launches the kernel of one (NC, K, S) on the first call per device after
// checking that it fits; false if it cannot run cooperatively.
template <int NC, int K, int S, bool F32>
bool run_t(const TcArgs& a, int device, cudaStream_t s, int sms_use) {
  static int grids[64] = {0};
  int& sms = grids[device & 63];
  if (!sms && !prepare_t<NC, K, S, F32>(device, sms)) return false;
  launch_tc_t<NC, K, S, F32>(a, sms_use < sms ? (sms_use > 0 ? sms_use : 1) : sms, s);
  return true;
}

// Dispatch over the widths and depths compiled for one NC (one translation
// unit per NC, so that they compile in parallel).
template <int NC, bool F32>
bool run_ncf(const TcArgs& a, int K, int S, int device, cudaStream_t s, int sms_use) {
  if (K == 8 && S == 2) return run_t<NC, 8, 2, F32>(a, device, s, sms_use);
  if (K == 8 && S == 4) return run_t<NC, 8, 4, F32>(a, device, s, sms_use);
  if (K == 16 && S == 2) return run_t<NC, 16, 2, F32>(a, device, s, sms_use);
  if (K == 16 && S == 4) return run_t<NC, 16, 4, F32>(a, device, s, sms_use);
  if (K == 32 && S == 2) return run_t<NC, 32, 2, F32>(a, device, s, sms_use);
  if (K == 32 && S == 3) return run_t<NC, 32, 3, F32>(a, device, s, sms_use);
  if (K == 64 && S == 2) return run_t<NC, 64, 2, F32>(a, device, s, sms_use);
  if (K == 64 && S == 3) return run_t<NC, 64, 3, F32>(a, device, s, sms_use);
  return false;
}
template <int NC>
bool run_nc(const TcArgs& a, int K, int S, bool f32, int device, cudaStream_t s, int sms_use) {
  return f32 ? run_ncf<NC, true>(a, K, S, device, s, sms_use)
             : run_ncf<NC, false>(a, K, S, device, s, sms_use);
}

bool run_nc16(const TcArgs& a, int K, int S, bool f32, int device, cudaStream_t s,
              int sms_use);
bool run_nc24(const TcArgs& a, int K, int S, bool f32, int device, cudaStream_t s,
              int sms_use);
bool run_nc64(const TcArgs& a, int K, int S, bool f32, int device, cudaStream_t s,
              int sms_use);

}  // namespace swtc
