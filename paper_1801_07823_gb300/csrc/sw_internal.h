// Internal declarations shared by the translation units of libsw.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cstdint>
#include <exception>
#include <new>
#include <string>
#include <vector>

#include "../../include/sw.h"

// ---------------------------------------------------------------- errors
struct SwError {
  int code;
  std::string msg;
};
#define SW_CUDA(call)                                                                      \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      throw SwError{SW_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)};     \
  } while (0)
// Every kernel launch of the library goes through SW_LAUNCH_CHECK, which also
// counts it (sw_launch_count()).
void sw_count_launch();
#define SW_LAUNCH_CHECK()         \
  do {                            \
    sw_count_launch();            \
    SW_CUDA(cudaGetLastError());  \
  } while (0)
// Debug aid: with the environment variable SW_POISON=1 every device buffer the
// library allocates is filled with all-one bytes (NaN in every double and
// float), so that a kernel reading memory nothing has written produces NaN.
void sw_poison(void* p, size_t bytes);
// cudaFree that reports a failure on stderr (and clears it) instead of
// leaving it pending for the next launch check.
void dev_free(void* p, const char* what);
// Notes on stderr (first few times) that an entry point cleared a pending
// error of an earlier, unchecked runtime call of the process.
void report_stale_error(cudaError_t e);
// Body of every extern "C" entry point: makes the context's device current,
// clears (and reports) a non-sticky error left pending by an earlier unchecked
// runtime call of the process, runs f, and turns every C++ exception into an
// SW_ERR_* code with the message kept in the context.
inline int fail(sw_ctx* c, int code, const std::string& msg);
template <typename F>
int guarded(sw_ctx* c, F&& f);
#define SW_REQUIRE(cond, code, text)                 \
  do {                                               \
    if (!(cond)) throw SwError{(code), (text)};      \
  } while (0)

// ---------------------------------------------------------------- scalars
// Krylov coefficients live in a small device array of complex slots so that
// kernels can use them without a host round trip.  A Coef describes
//   value = scale * f(S[num]) / g(S[den].re)
// with f = identity or conjugate (num < 0: 1) and g = identity or sqrt
// (den < 0: 1).
enum { COEF_CONJ = 1, COEF_SQRT_DEN = 2 };
struct Coef {
  int num;
  int den;
  int mode;
  double scale;
};
static inline Coef coef_const(double s) { return Coef{-1, -1, 0, s}; }
static inline Coef coef_ratio(int num, int den, double s = 1.0, int mode = 0) {
  return Coef{num, den, mode, s};
}

__device__ __forceinline__ double2 coef_eval(const double2* S, Coef c) {
  double2 v = (c.num >= 0) ? S[c.num] : make_double2(1.0, 0.0);
  if (c.mode & COEF_CONJ) v.y = -v.y;
  if (c.den >= 0) {
    double d = S[c.den].x;
    if (c.mode & COEF_SQRT_DEN) d = sqrt(d);
    v.x /= d;
    v.y /= d;
  }
  v.x *= c.scale;
  v.y *= c.scale;
  return v;
}

constexpr int kSlotPage = 320;  // 64 per multigrid level (up to 4), 64 for other solvers
constexpr int kMaxBatch = 64;   // right-hand sides solved together by sw_mg_solve_batch
constexpr int kNumSlots = kSlotPage * (kMaxBatch + 1);  // page 0: single solves; 1..64: batch
constexpr int kReduceBlocks = 304;  // 2 x 152 SMs; fixed so every sum has one order

// Per-category kernel timing with CUDA events on the context stream.
constexpr int kTimeCats = 8;  // 0: fine Schur operator, l: coarse operator of level l + 1,
                              // kCatCgne: the persistent coarsest CGNE kernel
constexpr int kCatCgne = 5;
struct TimedPair {
  int cat;
  cudaEvent_t a, b;
};

struct sw_ctx {
  int device = 0;
  bool timing = false;
  std::vector<TimedPair> pending;
  std::vector<cudaEvent_t> spare;
  long long t_count[kTimeCats] = {0};
  double t_ms[kTimeCats] = {0};
  cudaStream_t stream = nullptr;
  std::string err;
  double2* slots = nullptr;      // device [kNumSlots]
  double* partials = nullptr;    // device [2 * kReduceBlocks]
  unsigned* counter = nullptr;   // device, last-block-done counter
  int* flag = nullptr;           // device error flag (breakdown etc.)
  int* ctl = nullptr;            // device iteration-control blocks, 4 ints per level
  unsigned long long* exec = nullptr;  // device count of executed (not skipped) timed kernels
  int* h_ctl = nullptr;          // pinned host mirror of one control block
  unsigned* bar = nullptr;       // grid-barrier state of persistent kernels (2 words)
  int* cgstat = nullptr;         // status words of the persistent CGNE (3 ints)
  double2* h_slots = nullptr;    // pinned host mirror
  int sm_num = 1, sm_den = 1;    // share of the SMs its persistent kernels may hold
};

struct sw_gauge {
  sw_ctx* ctx = nullptr;
  int L0 = 0, L1 = 0, N = 0;
  double2* W_lex = nullptr;   // [2][N]  W_mu(s) = eta_mu(s) U_mu(s) / 2, site order x0 + L0 x1
  float2* W_lex32 = nullptr;  // FP32 copy for the FP32 Dslash
  double2* W_ps = nullptr;    // [2][N]  same, parity-split block-major order
  float2* W_ps32 = nullptr;   // FP32 copy of W_ps (mixed-precision Schur operator)
  double binv_mass = -1.0;
  double2* binv = nullptr;    // [N/4][4][4] B^-1 per KD block for binv_mass
  double2* W3_lex = nullptr;  // [2][N] Naik long links (built on first use)
  double naik_mass = -1.0;
  double2* binv_naik = nullptr;  // B_Naik^-1 for naik_mass
  double2* tmp[4] = {nullptr, nullptr, nullptr, nullptr};  // [N] scratch for sw_dslash
};

// ------------------------------------------------------------- entry guard
inline int fail(sw_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}
template <typename F>
int guarded(sw_ctx* c, F&& f) {
  try {
    if (c) {
      c->err.clear();
      SW_CUDA(cudaSetDevice(c->device));
    }
    cudaError_t stale = cudaGetLastError();
    if (stale != cudaSuccess) report_stale_error(stale);
    return f();
  } catch (const SwError& e) {
    return fail(c, e.code, e.msg);
  } catch (const std::bad_alloc&) {
    return fail(c, SW_ERR_OOM, "host allocation failed");
  } catch (const std::exception& e) {
    return fail(c, SW_ERR_CUDA, std::string("unexpected host error: ") + e.what());
  }
}

// ------------------------------------------------------------- geometry
// Parity-split block-major order of a fine field: f = par * N/2 + 4 * hb + k,
// KD block (X0, X1) = (x0/2, x1/2), par = (X0 + X1) & 1,
// hb = X1 * (L0/4) + X0/2, k = (x0 & 1) + 2 (x1 & 1).
__host__ __device__ __forceinline__ int ps_index(int x0, int x1, int L0, int N) {
  int X0 = x0 >> 1, X1 = x1 >> 1;
  int par = (X0 + X1) & 1;
  int hb = X1 * (L0 >> 2) + (X0 >> 1);
  int k = (x0 & 1) | ((x1 & 1) << 1);
  return par * (N >> 1) + (hb << 2) + k;
}
__host__ __device__ __forceinline__ void ps_coords(int f, int L0, int N, int& x0, int& x1) {
  int half = N >> 1;
  int par = f >= half;
  int r = f - par * half;
  int hb = r >> 2, k = r & 3;
  int q = L0 >> 2;
  int X1 = hb / q;
  int X0 = 2 * (hb - X1 * q) + ((X1 + par) & 1);
  x0 = 2 * X0 + (k & 1);
  x1 = 2 * X1 + (k >> 1);
}

// ------------------------------------------------------------- fine.cu
void launch_dslash_lex(const sw_gauge* g, double mass, int dagger, const double2* in, double2* out,
                       cudaStream_t s);
void launch_dslash_lex32(const sw_gauge* g, float mass, int dagger, const float2* in, float2* out,
                         cudaStream_t s);
void launch_pack(const sw_gauge* g, const double2* lex, double2* ps, cudaStream_t s);
// D (or D^dag) on full parity-split vectors.
void launch_dslash_ps(const sw_gauge* g, double mass, int dagger, const double2* in, double2* out,
                      cudaStream_t s);
void launch_unpack(const sw_gauge* g, const double2* ps, double2* lex, cudaStream_t s);
// hop_scale multiplies the in-block hops (1 for D, 9/8 for the Naik operator).
void launch_binv_build(const sw_gauge* g, double mass, double2* binv, cudaStream_t s,
                       double hop_scale = 1.0);
// Naik-improved operator (three-link term with the product of the path's links).
void launch_long_links(const sw_gauge* g, double c3, double2* W3, cudaStream_t s);
void launch_dslash_naik_lex(const sw_gauge* g, const double2* W3, double mass, double c1,
                            const double2* in, double2* out, cudaStream_t s);
// Block-local 4x4 multiply on the KD blocks of one parity half: out = M in or M^dag in.
void launch_block_apply(const sw_gauge* g, const double2* binv, int par, int dagger,
                        const double2* in, double2* out, cudaStream_t s);
// out_p = src_p + sign * C_{p,1-p} in_{1-p} on the sites of parity half p.
void launch_hop(const sw_gauge* g, int par, double sign, const double2* src, const double2* in,
                double2* out, cudaStream_t s);
// out_p = src_p + sign * M_p (C_{p,1-p} in_{1-p}), M = B^-1 or B^-dag, per KD block.
void launch_hop_block(const sw_gauge* g, const double2* binv, int par, int dagger, double sign,
                      const double2* src, const double2* in, double2* out, cudaStream_t s);

// Fine operator compositions on parity-split vectors (full: N, half: N/2).
// tmp must hold N complex.
void fine_apply_A(const sw_gauge* g, const double2* binv, const double2* in, double2* out,
                  double2* tmp, cudaStream_t s);
void fine_apply_Adag(const sw_gauge* g, const double2* binv, const double2* in, double2* out,
                     cudaStream_t s);
void fine_apply_S(const sw_gauge* g, const double2* binv, const double2* in_e, double2* out_e,
                  double2* tmp, cudaStream_t s);

// ------------------------------------------------------------- blas.cu
// skip: optional device flag; when it holds a non-zero value the kernel does nothing.
void blas_dot(sw_ctx* c, const double2* a, const double2* b, long n, int slot,
              const int* skip = nullptr);
void blas_norm2(sw_ctx* c, const double2* a, long n, int slot, const int* skip = nullptr);
void blas_axpy(sw_ctx* c, double2* y, const double2* x, long n, Coef a,
               const int* skip = nullptr);                                    // y += a x
void blas_xpay(sw_ctx* c, double2* y, const double2* x, long n, Coef a,
               const int* skip = nullptr);                                    // y = x + a y
void blas_scale(sw_ctx* c, double2* y, long n, Coef a);                       // y *= a
void blas_copy(sw_ctx* c, double2* y, const double2* x, long n);
void blas_zero(sw_ctx* c, double2* y, long n);
void blas_sub(sw_ctx* c, double2* out, const double2* a, const double2* b, long n);  // a - b
void blas_add3(sw_ctx* c, double2* out, const double2* a, const double2* b, const double2* d,
               long n);                                                               // a + b + d
double2 slot_read(sw_ctx* c, int slot);  // synchronises the stream, harvests timings
// Device-gated iteration control (see blas.cu); ctl points to 3 device ints.
void iter_init(sw_ctx* c, int* ctl, int slot, double stop, int maxit);
void iter_check(sw_ctx* c, int* ctl, int slot, double stop, int maxit);
void iter_read(sw_ctx* c, const int* ctl, int* host3);  // synchronises
// Timing brackets (no-ops unless c->timing): timing_begin returns a token.
int timing_begin(sw_ctx* c, int cat);
void timing_end(sw_ctx* c, int token);
void timing_harvest(sw_ctx* c);  // stream must be synchronised
void slot_set(sw_ctx* c, int slot, double2 v);

// ------------------------------------------------------------- coarse.cu
struct CoarseGeom {
  int E0, E1;     // extents of this coarse level
  int nc;         // dof per site
};
// skip: optional device flag (see BLAS); exec: optional device counter, bumped
// once per launch that did run.
// dagger = 1 applies the adjoint stencil from the same storage.
void launch_coarse_apply(const CoarseGeom& g, const double2* Y, int dagger, const double2* in,
                         double2* out, cudaStream_t s, const int* skip = nullptr,
                         unsigned long long* exec = nullptr);
// Whole coarsest-level CGNE in one cooperative launch (cgne.cu); false when nc
// has no compiled variant.
// Y: complex128 stencil (df64 = 0) or double-float float4 stencil (df64 = 1,
// then rdf and pdf are n float4 of scratch).
bool launch_cgne_persistent(const CoarseGeom& g, const void* Y, int df64, const double2* b,
                            double2* x, double2* r, double2* p, float4* rdf, float4* pdf,
                            double* partials, unsigned* bar, int* status, int maxit, double tol,
                            int device, cudaStream_t s, int stall_test = 0,
                            int sms_use = 1 << 30);

// FP64 coarsest CGNE in one persistent kernel (cgne64.cu).  variant 1: three
// real FMAs per complex product, reading Ys = Re + Im of every entry of Y
// (launch_sum_planes); variant 0: four FMAs on Y alone (Ys may be NULL);
// variants 2 and 3: 0 and 1 with reduce-scatter row sums and a per-component
// update; variant 7: 3 with its operands staged in shared memory by
// asynchronous copies (nc a multiple of 32, cgne64_staged_supported).
// v4: 8 n doubles of 32-byte aligned scratch (forms of r and p).  False when
// nc has no compiled variant.
bool cgne64_supported(int nc);
bool cgne64_staged_supported(int nc);
void launch_sum_planes(const double2* Y, double* Ys, long n, cudaStream_t s);
bool launch_cgne64(const CoarseGeom& g, int variant, const double2* Y, const double* Ys,
                   const double2* b, double2* x, double2* r, double2* p, double* v4,
                   double* partials, unsigned* bar, int* status, int maxit, double tol,
                   int device, cudaStream_t s, int stall_test = 0, int sms_use = 1 << 30);

// Batched coarsest CGNE (batch_cgne.cu): nb <= 16 right-hand sides, FP32
// forward stencil Yf and adjoint stencil Yd (launch_adjoint_f32), FP64
// iterates.  X, R, P: [n][K] double2; Rf, Pf: n K float2 of scratch (the
// kernel keeps them planar per dof: K real parts, then K imaginary parts),
// K = cgne_batch_width(nb); partials: 2 K SMs doubles; status: 18 ints
// ([0] wait timeout or misaligned buffer, [1] non-finite, [2 + r] iterations).
int cgne_batch_width(int nb);
bool launch_cgne_batch(const CoarseGeom& g, const float2* Yf, const float2* Yd, int nb,
                       const double2* const* b, double2* const* x, double2* X, double2* R,
                       double2* P, float2* Rf, float2* Pf, double* partials, unsigned* bar,
                       int* status, int maxit, double tol, int device, cudaStream_t s,
                       int sms_use = 1 << 30);
// Batched coarsest CGNE on the tensor cores (batch_tc.cu): nb <= 64
// right-hand sides padded to the width tc_width(nb) in {8, 16, 32, 64}.
// At / Ad: stacked TF32 tiles (launch_stack_tiles, tc_tile_floats(nc) floats
// per (site, direction)); Rt / Pt: sites x 2 K x nc floats of scratch; X, R, P:
// [n][K] double2 (float2 with f32: FP32 iterates); partials: 2 K SMs doubles;
// status: 2 + 64 ints ([0] wait timeout or misaligned buffer, [1] non-finite,
// [2 + r] iterations).  stages: pipeline depth, one of tc_stage_options(nc, K).
// l2frac: 0 streams the stencil tiles through L2 (evict first); > 0 loads that
// fraction of their lines with evict-last priority (tc_l2_fraction sizes it).
int tc_width(int nb);
bool tc_supported(int nc);
long tc_tile_floats(int nc);
float tc_l2_fraction(const CoarseGeom& g, int device);
int tc_stage_options(int nc, int K, int* out);
void launch_stack_tiles(const CoarseGeom& g, const double2* Y, float* T, int adj, cudaStream_t s);
bool launch_cgne_tc(const CoarseGeom& g, int stages, bool f32, const float* At, const float* Ad,
                    int nb, const double2* const* b, double2* const* x, double2* X, double2* R,
                    double2* P, float* Rt, float* Pt, double* partials, unsigned* bar,
                    int* status, int maxit, double tol, int device, cudaStream_t s, int stall,
                    int sms_use = 1 << 30, float l2frac = 0.f);
// Yd[X][d] = Y[nb(X, d)][opp(d)]^dag in FP32, every block column-major like Y.
void launch_adjoint_f32(const CoarseGeom& g, const double2* Y, float2* Yd, cudaStream_t s);

// ------------------------------------------------------------- mixed.cu
void fine_apply_S32(const sw_gauge* g, const float2* W32, const float2* binv32,
                    const double2* in_e, double2* out_e, float2* tmp, cudaStream_t s);
void launch_to_f32(const double2* in, float2* out, long n, cudaStream_t s);
void launch_to_half_scaled(const CoarseGeom& g, const double2* Y, __half2* Yh, float* scale,
                           cudaStream_t s);
void launch_coarse_apply_h(const CoarseGeom& g, const __half2* Yh, const float* scale, int dagger,
                           const double2* in, double2* out, cudaStream_t s);
void launch_to_df64(const double2* Y, float4* Yd, long n, cudaStream_t s);
void launch_coarse_apply_df(const CoarseGeom& g, const float4* Y, int dagger, const double2* in,
                            double2* out, cudaStream_t s);
// Level-1 transfer on the even parity half.  P: [N][nv] parity-split rows.
// full = 1: full parity-split vectors (fine operator D) instead of the even half.
void launch_restrict_fine(const sw_gauge* g, int a0, int a1, int nv, const double2* P,
                          const double2* r_e, double2* out, cudaStream_t s, int full = 0);
void launch_prolong_fine(const sw_gauge* g, int a0, int a1, int nv, const double2* P,
                         const double2* ehat, double2* e_e, cudaStream_t s, int full = 0);
void launch_build_W_identity(const sw_gauge* g, int nv, const double2* P, double2* Wv,
                             cudaStream_t s);
// Level >= 2 transfer.  P: [sites][nc][nv].
void launch_restrict_coarse(const CoarseGeom& g, int b0, int b1, int nv, const double2* P,
                            const double2* r, double2* out, cudaStream_t s);
void launch_prolong_coarse(const CoarseGeom& g, int b0, int b1, int nv, const double2* P,
                           const double2* ehat, double2* e, cudaStream_t s);
// Aggregate / chirality maps of a level from the transfer kernels' index maps.
void launch_level_maps_fine(const sw_gauge* g, int a0, int a1, int* agg, int* chir,
                            cudaStream_t s);
void launch_level_maps_coarse(const CoarseGeom& g, int b0, int b1, int* agg, int* chir,
                              cudaStream_t s);
// Galerkin builds.
void launch_build_W(const sw_gauge* g, int nv, const double2* binv, const double2* P,
                    double2* Wv, cudaStream_t s);
void launch_build_Y_fine(const sw_gauge* g, double mass, int a0, int a1, int nv, const double2* P,
                         const double2* Wv, double2* Y, cudaStream_t s);
void launch_build_Y_coarse(const CoarseGeom& g, int b0, int b1, int nv, const double2* Y,
                           const double2* P, double2* T, double2* Ynext, cudaStream_t s);
// Block orthonormalisation of nv vector-major vectors V[nv][ndof] into P[ndof][nv].
// level 1: dof = parity-split site; coarse: dof = X * nc + k.
void launch_block_ortho_fine(const sw_gauge* g, int a0, int a1, int nv, const double2* V,
                             double2* P, int* flag, cudaStream_t s);
void launch_block_ortho_coarse(const CoarseGeom& g, int b0, int b1, int nv, const double2* V,
                               double2* P, int* flag, cudaStream_t s);
// Device-side SplitMix64 + Box-Muller Gaussian vector (same definition as the
// input module): element j uses outputs 2j and 2j+1 of stream seed.
void launch_gaussian(uint64_t seed, long n, double2* out, cudaStream_t s);
