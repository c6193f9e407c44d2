// Multigrid hierarchy: setup and K-cycle solve (Sec. IV, Table kcycle).
//
// Setup per level l (0 = fine): nv near-null vectors psi = psi0 + e, e from CG
// on A A^dag e = -A A^dag psi0 (tolerance setup_tol, setup_maxiter
// iterations); global modified Gram-Schmidt; chiral doubling and modified
// Gram-Schmidt per (aggregate, chirality) -> P; Galerkin stencil
// Y = P^dag A P and its adjoint stencil.
//
// Solve: flexible GCR(outer_restart) on S z_e = b_e - A_eo b_o with
// S = I - A_eo A_oe, preconditioned by the K-cycle: MR(smoother_iters, omega)
// on S; restrict (r_e, 0); GCR(inter_restart, max inter_maxiter, tol
// inter_tol) on A_hat preconditioned by the next K-cycle, or CGNE (tol
// coarsest_tol, max coarsest_maxiter) on the coarsest level; prolong and keep
// the even part; r2 = r1 - S e; MR post-smoother on r2; p = x1 + e + x3.
// Then z_o = b_o - A_oe z_e and x = B^-1 z.
//
// Krylov coefficients stay on the device (Coef slots); the host reads back
// only the residual norms its stopping tests branch on.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <condition_variable>
#include <map>
#include <mutex>
#include <tuple>

#include "sw_internal.h"
#include "sw_mg.h"

namespace {

double2* dalloc(long n) {
  void* p = nullptr;
  if (n <= 0) n = 1;
  cudaError_t e = cudaMalloc(&p, n * sizeof(double2));
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw SwError{SW_ERR_OOM, std::string("cudaMalloc of ") + std::to_string(n * 16) +
                                  " bytes failed: " + cudaGetErrorString(e)};
  }
  sw_poison(p, n * sizeof(double2));
  return (double2*)p;
}

}  // namespace

void sw_mg_release(sw_mg* mg) {
  for (double2* p : mg->allocs) dev_free(p, "hierarchy buffer");
  mg->allocs.clear();
}

double2* ScopedBuffers::get(long n) {
  double2* p = dalloc(n);
  list.push_back(p);
  return p;
}

ScopedBuffers::~ScopedBuffers() {
  for (double2* p : list) dev_free(p, "call scratch");
}

double2* mg_alloc(sw_mg* mg, long n) {
  double2* p = dalloc(n);
  mg->allocs.push_back(p);
  return p;
}

// ---------------------------------------------------------------- operators
long level_len(const sw_mg* mg, int l) {
  const MgLevel& L = mg->lev[l];
  if (l == 0) return mg->fine_D ? mg->g->N : mg->g->N / 2;
  return L.ndof;
}

// Operator of level l in the solve: S on level 0 (even half), A_hat below.
// skip: optional device flag that turns the (coarse) application into a no-op.
// lowp: inside the preconditioner of a mixed-precision hierarchy -- the fine
// Schur operator then runs in FP32 and intermediate stencils in scaled FP16.
void level_op(sw_mg* mg, int l, const double2* in, double2* out, const int* skip = nullptr,
              bool lowp = false) {
  sw_ctx* c = mg->ctx;
  int tk = timing_begin(c, l);
  if (l == 0) {
    if (mg->fine_D)
      launch_dslash_ps(mg->g, mg->mass, 0, in, out, c->stream);
    else if (lowp && mg->mixed)
      fine_apply_S32(mg->g, mg->g->W_ps32, mg->binv32, in, out, mg->s32tmp, c->stream);
    else
      fine_apply_S(mg->g, mg->binv, in, out, mg->lev[0].stmp, c->stream);
    mg->st_fine_applies++;
  } else if (lowp && mg->mixed && mg->lev[l].Yh) {
    const MgLevel& L = mg->lev[l];
    launch_coarse_apply_h(CoarseGeom{L.E0, L.E1, L.nc}, L.Yh, L.Ysc, 0, in, out, c->stream);
  } else {
    const MgLevel& L = mg->lev[l];
    launch_coarse_apply(CoarseGeom{L.E0, L.E1, L.nc}, L.Y, 0, in, out, c->stream, skip,
                        c->timing ? c->exec + l : nullptr);
  }
  timing_end(c, tk);
}
void level_opdag(sw_mg* mg, int l, const double2* in, double2* out, const int* skip = nullptr) {
  sw_ctx* c = mg->ctx;
  const MgLevel& L = mg->lev[l];
  int tk = timing_begin(c, l);
  launch_coarse_apply(CoarseGeom{L.E0, L.E1, L.nc}, L.Y, 1, in, out, c->stream, skip,
                      c->timing ? c->exec + l : nullptr);
  timing_end(c, tk);
}
// Normal operator used by the setup on level l: A A^dag (full fine vectors on
// level 0).
void level_normal(sw_mg* mg, int l, const double2* in, double2* out, double2* tmp) {
  cudaStream_t s = mg->ctx->stream;
  if (l == 0 && mg->fine_D) {
    launch_dslash_ps(mg->g, mg->mass, 1, in, tmp, s);
    launch_dslash_ps(mg->g, mg->mass, 0, tmp, out, s);
  } else if (l == 0) {
    fine_apply_Adag(mg->g, mg->binv, in, tmp, s);
    fine_apply_A(mg->g, mg->binv, tmp, out, mg->lev[0].stmp, s);
  } else {
    level_opdag(mg, l, in, tmp);
    level_op(mg, l, tmp, out);
  }
}

static void check_norm(double v, const char* where) {
  if (!std::isfinite(v)) throw SwError{SW_ERR_NAN, std::string("non-finite norm in ") + where};
}

// SW_VERBOSE >= 3: the 2-norm of a work vector on stderr (a trace of where a
// non-finite value first appears).  Costs a host round trip per call.
static void trace_norm(sw_mg* mg, int l, const char* what, const double2* v, long n) {
  if (mg->verbose < 3) return;
  blas_norm2(mg->ctx, v, n, slot_base(l) + 63);
  std::fprintf(stderr, "[sw]       level %d %s |v| %.6e\n", l + 1, what,
               std::sqrt(slot_read(mg->ctx, slot_base(l) + 63).x));
}

// ---------------------------------------------------------------- Krylov
// MR smoother with zero initial guess: x, r = b - op x.
static void mr(sw_mg* mg, int l, const double2* b, double2* x, double2* r, double2* q) {
  const bool lowp = true;  // the smoother always belongs to the preconditioner
  sw_ctx* c = mg->ctx;
  long n = level_len(mg, l);
  int sq = slot_base(l) + 8, sqq = slot_base(l) + 9;
  blas_zero(c, x, n);
  blas_copy(c, r, b, n);
  double om = mg->p.omega;
  for (int it = 0; it < mg->p.smoother_iters; ++it) {
    level_op(mg, l, r, q, nullptr, lowp);
    blas_dot(c, q, r, n, sq);
    blas_norm2(c, q, n, sqq);
    if (mg->verbose >= 3) {
      const double2 a = slot_read(c, sq), b = slot_read(c, sqq);
      std::fprintf(stderr, "[sw]       level %d MR %d (q, r) %.6e %+.6ei |q|^2 %.6e\n", l + 1,
                   it, a.x, a.y, b.x);
    }
    blas_axpy(c, x, r, n, coef_ratio(sq, sqq, om));
    blas_axpy(c, r, q, n, coef_ratio(sq, sqq, -om));
  }
}

static void solve_level(sw_mg* mg, int l, const double2* rhs, double2* sol);

// K-cycle preconditioner of level l: out = M(r).
static void kcycle(sw_mg* mg, int l, const double2* r, double2* out) {
  sw_ctx* c = mg->ctx;
  MgLevel& L = mg->lev[l];
  MgLevel& C = mg->lev[l + 1];
  long n = level_len(mg, l);
  cudaStream_t s = c->stream;
  trace_norm(mg, l, "K-cycle input", r, n);
  mr(mg, l, r, L.kx1, L.kr1, L.kq);
  trace_norm(mg, l, "pre-smoothed x", L.kx1, n);
  trace_norm(mg, l, "pre-smoothed r", L.kr1, n);
  if (l == 0)
    launch_restrict_fine(mg->g, L.b0, L.b1, L.nv, L.P, L.kr1, C.rhs, s, mg->fine_D ? 1 : 0);
  else
    launch_restrict_coarse(CoarseGeom{L.E0, L.E1, L.nc}, L.b0, L.b1, L.nv, L.P, L.kr1, C.rhs, s);
  trace_norm(mg, l + 1, "restricted r", C.rhs, level_len(mg, l + 1));
  solve_level(mg, l + 1, C.rhs, C.sol);
  if (l == 0)
    launch_prolong_fine(mg->g, L.b0, L.b1, L.nv, L.P, C.sol, L.ke, s, mg->fine_D ? 1 : 0);
  else
    launch_prolong_coarse(CoarseGeom{L.E0, L.E1, L.nc}, L.b0, L.b1, L.nv, L.P, C.sol, L.ke, s);
  level_op(mg, l, L.ke, L.kq, nullptr, true);
  blas_sub(c, L.kr2, L.kr1, L.kq, n);
  mr(mg, l, L.kr2, L.kx3, L.kr3, L.kq);
  blas_add3(c, out, L.kx1, L.ke, L.kx3, n);
}

struct GcrResult {
  int iters, restarts;
  bool converged;
};

// Flexible restarted GCR on level l (see the oracle's fgcr for the steps).
static GcrResult fgcr(sw_mg* mg, int l, const double2* b, double2* x, double tol_abs, int restart,
                      int maxiter, bool confirm) {
  sw_ctx* c = mg->ctx;
  MgLevel& L = mg->lev[l];
  long n = level_len(mg, l);
  int sb = slot_base(l);
  int s_rr = sb + 0, s_qq = sb + 2, s_a = sb + 3, s_b = sb + 4;
  blas_zero(c, x, n);
  blas_copy(c, L.gr, b, n);
  int k = 0, it = 0, restarts = 0;
  const bool lowp = l > 0;  // intermediate solves are part of the preconditioner
  for (;;) {
    blas_norm2(c, L.gr, n, s_rr);
    double rn = std::sqrt(slot_read(c, s_rr).x);
    check_norm(rn, "GCR residual");
    if (rn <= tol_abs) {
      if (!confirm) return GcrResult{it, restarts, true};
      level_op(mg, l, x, L.gtmp, nullptr, lowp);
      blas_sub(c, L.gtmp, b, L.gtmp, n);
      blas_norm2(c, L.gtmp, n, s_rr);
      double rt = std::sqrt(slot_read(c, s_rr).x);
      check_norm(rt, "GCR true residual");
      if (rt <= tol_abs) return GcrResult{it, restarts, true};
      blas_copy(c, L.gr, L.gtmp, n);
      k = 0;
      ++restarts;
      continue;
    }
    if (it >= maxiter) return GcrResult{it, restarts, false};
    double2* p = L.gp[k];
    double2* q = L.gq[k];
    if (l + 1 < mg->nlev)
      kcycle(mg, l, L.gr, p);
    else
      blas_copy(c, p, L.gr, n);
    level_op(mg, l, p, q, nullptr, lowp);
    for (int j = 0; j < k; ++j) {
      blas_dot(c, L.gq[j], q, n, s_b);
      blas_axpy(c, q, L.gq[j], n, coef_ratio(s_b, -1, -1.0));
      blas_axpy(c, p, L.gp[j], n, coef_ratio(s_b, -1, -1.0));
    }
    blas_norm2(c, q, n, s_qq);
    blas_scale(c, q, n, coef_ratio(-1, s_qq, 1.0, COEF_SQRT_DEN));
    blas_scale(c, p, n, coef_ratio(-1, s_qq, 1.0, COEF_SQRT_DEN));
    blas_dot(c, q, L.gr, n, s_a);
    blas_axpy(c, x, p, n, coef_ratio(s_a, -1, 1.0));
    blas_axpy(c, L.gr, q, n, coef_ratio(s_a, -1, -1.0));
    ++k;
    ++it;
    if (l == 1 && mg->verbose > 1) std::fprintf(stderr, "[sw]   level-2 GCR %d |r| %.3e (tol %.3e)\n", it, rn, tol_abs);
    if (l == 0 && mg->verbose)
      std::fprintf(stderr, "[sw] outer %d |r| %.3e  inter %lld/%lld coarsest %lld/%lld\n", it, rn,
                   mg->st_inter_iters, mg->st_inter_solves, mg->st_coarsest_iters,
                   mg->st_coarsest_solves);
    if (k == restart && it < maxiter) {
      level_op(mg, l, x, L.gtmp, nullptr, lowp);
      blas_sub(c, L.gr, b, L.gtmp, n);
      k = 0;
      ++restarts;
    }
  }
}

// CG on the normal error (Craig): x = op^dag y with op op^dag y = b.  The
// stopping test runs on the device (iter_check); the host queues kIterBatch
// iterations at a time and reads the control block between batches, so the
// iterations need no host round trip.  Iterates and counts are those of the
// sequential loop: every kernel after the stopping iteration is a no-op.
constexpr int kIterBatch = 8;

// SMs that persistent (cooperative) kernels of this process hold, per device.
// A persistent launch takes its context's share of the SMs (sw_context_set_
// sm_share; all of them by default) and waits while the kernels of other
// contexts hold too many for it to fit beside them.  Grids whose shares add
// up to at most the SM count run concurrently (one CTA per SM each); others
// run one after the other, so no cooperative grid waits at a barrier for CTAs
// that cannot become resident.
class SmLease {
 public:
  explicit SmLease(sw_ctx* c) : dev_(c->device & 63) {
    int total = 0;
    SW_CUDA(cudaDeviceGetAttribute(&total, cudaDevAttrMultiProcessorCount, c->device));
    n_ = (int)((long)total * c->sm_num / (c->sm_den > 0 ? c->sm_den : 1));
    n_ = n_ < 1 ? 1 : (n_ > total ? total : n_);
    std::unique_lock<std::mutex> lk(mu());
    cv().wait(lk, [&] { return used()[dev_] + n_ <= total; });
    used()[dev_] += n_;
  }
  ~SmLease() {
    {
      std::lock_guard<std::mutex> lk(mu());
      used()[dev_] -= n_;
    }
    cv().notify_all();
  }
  int sms() const { return n_; }

 private:
  static std::mutex& mu() {
    static std::mutex m;
    return m;
  }
  static std::condition_variable& cv() {
    static std::condition_variable v;
    return v;
  }
  static int* used() {
    static int u[64] = {0};
    return u;
  }
  int dev_, n_ = 0;
};

// Autotuner records, keyed by (device, nc, batch width, coarse sites, SMs used): for the
// batched tensor-core kernel the pipeline depth, for the single-right-hand-side
// FP64 kernel (width 1) its variant (0: four-FMA, 1: three-FMA products).
struct TuneRec {
  int stages;
  double us_per_iter;
};
static std::mutex g_tune_mutex;
static std::map<std::tuple<int, int, int, int, int>, TuneRec> g_tune;  // + SMs used

// Variant of the FP64 coarsest CGNE for this level, chosen on first use per
// (device, nc, sites) by timing each for a few iterations on the call's own
// data (the real solve then starts from scratch).
static int cgne64_variant(sw_mg* mg, MgLevel& L, const double2* b, double2* x, int sms) {
  sw_ctx* c = mg->ctx;
  // "0" .. "3" or "7": skip the timing, use this one
  const char* force = std::getenv("SW_CGNE64");
  if (force && ((force[0] >= '0' && force[0] <= '3') || force[0] == '7') && !force[1] &&
      (force[0] != '7' || cgne64_staged_supported(L.nc)))
    return force[0] - '0';
  const auto key = std::make_tuple(c->device, L.nc, 1, L.E0 * L.E1, sms);
  {
    std::lock_guard<std::mutex> lk(g_tune_mutex);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) return it->second.stages;
  }
  constexpr int kTuneIters = 8, kReps = 2;
  cudaEvent_t e0, e1;
  SW_CUDA(cudaEventCreate(&e0));
  SW_CUDA(cudaEventCreate(&e1));
  TuneRec best{0, 1e30};
  int cand[5] = {0, 1, 2, 3, 7};
  const int ncand = cgne64_staged_supported(L.nc) ? 5 : 4;
  for (int ci = 0; ci < ncand; ++ci) {
    const int v = cand[ci];
    float tot = 0.f;
    for (int rep = 0; rep <= kReps; ++rep) {  // rep 0 is a warm-up
      SW_CUDA(cudaEventRecord(e0, c->stream));
      bool ran = launch_cgne64(CoarseGeom{L.E0, L.E1, L.nc}, v, L.Y, L.Ys, b, x, L.gr, L.cp,
                               L.c4, c->partials, c->bar, c->cgstat, kTuneIters, 0.0, c->device,
                               c->stream, 0, sms);
      SW_CUDA(cudaEventRecord(e1, c->stream));
      SW_CUDA(cudaEventSynchronize(e1));
      SW_REQUIRE(ran, SW_ERR_ARG, "FP64 coarsest CGNE has no variant for this shape");
      int st[3];
      SW_CUDA(cudaMemcpy(st, c->cgstat, sizeof(st), cudaMemcpyDeviceToHost));
      SW_REQUIRE(st[1] == 0, SW_ERR_TIMEOUT, "coarsest CGNE: a grid barrier wait gave up");
      float ms = 0.f;
      SW_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (rep > 0) tot += ms;
    }
    const double us = 1e3 * tot / kReps / kTuneIters;
    if (us < best.us_per_iter) best = TuneRec{v, us};
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::lock_guard<std::mutex> lk(g_tune_mutex);
  g_tune[key] = best;
  return best.stages;
}

static int cgne(sw_mg* mg, int l, const double2* b, double2* x) {
  sw_ctx* c = mg->ctx;
  MgLevel& L = mg->lev[l];
  long n = level_len(mg, l);
  if (mg->persistent_cgne) {
    SmLease lease(c);  // held until the kernel has finished
    int tk = -1;
    const char* dfenv = std::getenv("SW_COARSEST_DF64");
    bool df = mg->mixed && L.Ydf && (!(L.Ys && L.c4) || (dfenv && dfenv[0] == '1'));
    bool ran;
    if (!df && L.Ys && L.c4) {
      const int v = cgne64_variant(mg, L, b, x, lease.sms());
      tk = timing_begin(c, kCatCgne);  // the bracket covers the solve, not the tuning
      ran = launch_cgne64(CoarseGeom{L.E0, L.E1, L.nc}, v, L.Y, L.Ys, b, x, L.gr, L.cp, L.c4,
                          c->partials, c->bar, c->cgstat, mg->p.coarsest_maxiter,
                          mg->p.coarsest_tol, c->device, c->stream, mg->stall_test,
                          lease.sms());
    }
    else {
      tk = timing_begin(c, kCatCgne);
      ran = launch_cgne_persistent(CoarseGeom{L.E0, L.E1, L.nc}, df ? (const void*)L.Ydf
                                                                   : (const void*)L.Y,
                                   df ? 1 : 0, b, x, L.gr, L.cp, L.cdf,
                                   L.cdf ? L.cdf + L.ndof : nullptr,
                                   c->partials, c->bar, c->cgstat, mg->p.coarsest_maxiter,
                                   mg->p.coarsest_tol, c->device, c->stream, mg->stall_test,
                                   lease.sms());
    }
    timing_end(c, tk);
    if (ran) {
      SW_CUDA(cudaMemcpyAsync(c->h_ctl, c->cgstat, 3 * sizeof(int), cudaMemcpyDeviceToHost,
                              c->stream));
      SW_CUDA(cudaStreamSynchronize(c->stream));
      if (!c->pending.empty()) timing_harvest(c);
      if (c->timing) c->t_count[kCatCgne + 1] += c->h_ctl[0];  // iterations, for flop counts
      if (c->h_ctl[1])
        throw SwError{SW_ERR_TIMEOUT, "coarsest CGNE: a grid barrier wait gave up"};
      if (c->h_ctl[2]) throw SwError{SW_ERR_NAN, "non-finite norm in CGNE residual"};
      if (mg->verbose > 1)
        std::fprintf(stderr, "[sw]     coarsest CGNE launch: %d iterations\n", c->h_ctl[0]);
      return c->h_ctl[0];
    }
  }
  int sb = slot_base(l);
  int s_rr[2] = {sb + 10, sb + 11}, s_pp = sb + 12;
  int* ctl = c->ctl + 4 * l;
  int maxit = mg->p.coarsest_maxiter;
  blas_zero(c, x, n);
  blas_copy(c, L.gr, b, n);
  blas_norm2(c, L.gr, n, s_rr[0]);
  double rr = slot_read(c, s_rr[0]).x;
  check_norm(rr, "CGNE residual");
  double stop = mg->p.coarsest_tol * std::sqrt(rr);
  level_opdag(mg, l, L.gr, L.cp);
  iter_init(c, ctl, s_rr[0], stop, maxit);
  int cur = 0;
  for (int issued = 0;;) {
    for (int q = 0; q < kIterBatch && issued < maxit; ++q, ++issued) {
      blas_norm2(c, L.cp, n, s_pp, ctl);
      blas_axpy(c, x, L.cp, n, coef_ratio(s_rr[cur], s_pp, 1.0), ctl);
      level_op(mg, l, L.cp, L.cw, ctl);
      blas_axpy(c, L.gr, L.cw, n, coef_ratio(s_rr[cur], s_pp, -1.0), ctl);
      blas_norm2(c, L.gr, n, s_rr[1 - cur], ctl);
      iter_check(c, ctl, s_rr[1 - cur], stop, maxit);
      level_opdag(mg, l, L.gr, L.cw, ctl);
      blas_xpay(c, L.cp, L.cw, n, coef_ratio(s_rr[1 - cur], s_rr[cur], 1.0), ctl);
      cur = 1 - cur;
    }
    iter_read(c, ctl, c->h_ctl);
    if (c->h_ctl[2]) throw SwError{SW_ERR_NAN, "non-finite norm in CGNE residual"};
    if (c->h_ctl[0] || issued >= maxit) break;
  }
  return c->h_ctl[1];
}

static void solve_level(sw_mg* mg, int l, const double2* rhs, double2* sol) {
  sw_ctx* c = mg->ctx;
  if (l == mg->nlev - 1) {
    mg->st_coarsest_iters += cgne(mg, l, rhs, sol);
    mg->st_coarsest_solves++;
    return;
  }
  long n = level_len(mg, l);
  int s = slot_base(l) + 1;
  blas_norm2(c, rhs, n, s);
  double bn = std::sqrt(slot_read(c, s).x);
  check_norm(bn, "intermediate right-hand side");
  GcrResult r = fgcr(mg, l, rhs, sol, mg->p.inter_tol * bn, mg->p.inter_restart,
                     mg->p.inter_maxiter, false);
  mg->st_inter_iters += r.iters;
  mg->st_inter_solves++;
}

// CG on a Hermitian positive semi-definite normal operator (setup).
static int cg_setup(sw_mg* mg, int l, const double2* b, double2* x) {
  sw_ctx* c = mg->ctx;
  MgLevel& L = mg->lev[l];
  long n = L.ndof;
  int sb = slot_base(l);
  int s_rr[2] = {sb + 20, sb + 21}, s_pq = sb + 22;
  blas_zero(c, x, n);
  blas_copy(c, L.sr, b, n);
  blas_copy(c, L.sp, L.sr, n);
  blas_norm2(c, L.sr, n, s_rr[0]);
  double rr = slot_read(c, s_rr[0]).x;
  check_norm(rr, "setup CG residual");
  double stop = mg->p.setup_tol * std::sqrt(rr);
  int k = 0, cur = 0;
  while (k < mg->p.setup_maxiter && std::sqrt(rr) > stop) {
    level_normal(mg, l, L.sp, L.sq, L.st);
    blas_dot(c, L.sp, L.sq, n, s_pq);
    blas_axpy(c, x, L.sp, n, coef_ratio(s_rr[cur], s_pq, 1.0));
    blas_axpy(c, L.sr, L.sq, n, coef_ratio(s_rr[cur], s_pq, -1.0));
    blas_norm2(c, L.sr, n, s_rr[1 - cur]);
    rr = slot_read(c, s_rr[1 - cur]).x;
    check_norm(rr, "setup CG residual");
    blas_xpay(c, L.sp, L.sr, n, coef_ratio(s_rr[1 - cur], s_rr[cur], 1.0));
    cur = 1 - cur;
    ++k;
  }
  return k;
}

int mg_coarsest_solve(sw_mg* mg, const double2* b, double2* x) {
  return cgne(mg, mg->nlev - 1, b, x);
}

// ---------------------------------------------------------------- setup
void mg_setup(sw_mg* mg, const double* const* psi0, uint64_t seed) {
  sw_ctx* c = mg->ctx;
  sw_gauge* g = mg->g;
  cudaStream_t s = c->stream;
  long N = g->N;
  mg->binv = mg_alloc(mg, N * 4);
  launch_binv_build(g, mg->mass, mg->binv, s);
  mg->lev[0].stmp = mg_alloc(mg, N);
  if (mg->mixed) {
    mg->binv32 = (float2*)mg_alloc(mg, N * 2);
    launch_to_f32(mg->binv, mg->binv32, N * 4, s);
    mg->s32tmp = (float2*)mg_alloc(mg, (N + 1) / 2);
  }
  ScopedBuffers tmp;
  for (int l = 0; l + 1 < mg->nlev; ++l) {
    MgLevel& L = mg->lev[l];
    MgLevel& C = mg->lev[l + 1];
    int nv = L.nv;
    long n = L.ndof;
    // work vectors of the setup
    L.sr = tmp.get(n); L.sp = tmp.get(n); L.sq = tmp.get(n);
    L.st = tmp.get(n);
    double2* V = tmp.get(n * nv);
    double2* e = tmp.get(n);
    double2* start = tmp.get(n);
    double2* lex = l == 0 ? tmp.get(n) : nullptr;
    int sb = slot_base(l);
    for (int i = 0; i < nv; ++i) {
      double2* target = l == 0 ? lex : start;
      if (psi0 && psi0[l]) {
        SW_CUDA(cudaMemcpyAsync(target, psi0[l] + 2 * (long)i * n, n * sizeof(double2),
                                cudaMemcpyHostToDevice, s));
      } else {
        launch_gaussian(sw_stream_seed(seed, l, i), n, target, s);
      }
      if (l == 0) launch_pack(g, lex, start, s);
      double2* psi = V + (long)i * n;
      for (int pass = 0; pass < mg->p.setup_passes; ++pass) {
        if (pass > 0) {
          blas_copy(c, start, psi, n);
          blas_norm2(c, start, n, sb + 30);
          blas_scale(c, start, n, coef_ratio(-1, sb + 30, 1.0, COEF_SQRT_DEN));
        }
        level_normal(mg, l, start, L.sq, L.st);
        blas_zero(c, L.sp, n);
        blas_sub(c, L.st, L.sp, L.sq, n);  // r = -A A^dag start
        int its = cg_setup(mg, l, L.st, e);  // L.st is read before CG reuses it
        mg->setup_iters.push_back(its);
        blas_copy(c, psi, start, n);  // psi = psi0 + e
        blas_axpy(c, psi, e, n, coef_const(1.0));
      }
    }
    // global modified Gram-Schmidt in index order
    for (int i = 0; i < nv; ++i) {
      double2* vi = V + (long)i * n;
      for (int j = 0; j < i; ++j) {
        blas_dot(c, V + (long)j * n, vi, n, sb + 31);
        blas_axpy(c, vi, V + (long)j * n, n, coef_ratio(sb + 31, -1, -1.0));
      }
      blas_norm2(c, vi, n, sb + 32);
      double nn = slot_read(c, sb + 32).x;
      if (!(nn > 0.0) || !std::isfinite(nn))
        throw SwError{SW_ERR_BREAKDOWN, "global Gram-Schmidt: vector " + std::to_string(i) +
                                            " on level " + std::to_string(l + 1) + " has norm 0"};
      blas_scale(c, vi, n, coef_ratio(-1, sb + 32, 1.0, COEF_SQRT_DEN));
    }
    // chiral doubling + block orthonormalisation
    L.P = mg_alloc(mg, n * nv);
    SW_CUDA(cudaMemsetAsync(c->flag, 0, sizeof(int), s));
    if (l == 0)
      launch_block_ortho_fine(g, L.b0, L.b1, nv, V, L.P, c->flag, s);
    else
      launch_block_ortho_coarse(CoarseGeom{L.E0, L.E1, L.nc}, L.b0, L.b1, nv, V, L.P, c->flag, s);
    int hflag = 0;
    SW_CUDA(cudaMemcpyAsync(&hflag, c->flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    SW_CUDA(cudaStreamSynchronize(s));
    if (hflag)
      throw SwError{SW_ERR_BREAKDOWN,
                    "block orthonormalisation met a zero vector on level " + std::to_string(l + 1)};
    // Galerkin coarse operator and its adjoint stencil
    long ysz = (long)C.E0 * C.E1 * 5 * C.nc * C.nc;
    C.Y = mg_alloc(mg, ysz);
    if (l == 0) {
      double2* Wv = tmp.get(N * 2 * nv);
      if (mg->fine_D)
        launch_build_W_identity(g, nv, L.P, Wv, s);  // Galerkin of D itself: P^dag D P
      else
        launch_build_W(g, nv, mg->binv, L.P, Wv, s);
      launch_build_Y_fine(g, mg->mass, L.b0, L.b1, nv, L.P, Wv, C.Y, s);
    } else {
      double2* T = tmp.get((long)L.E0 * L.E1 * 5 * L.nc * 2 * nv);
      launch_build_Y_coarse(CoarseGeom{L.E0, L.E1, L.nc}, L.b0, L.b1, nv, L.Y, L.P, T, C.Y, s);
    }
    if (l + 2 == mg->nlev && !mg->fine_D && cgne64_supported(C.nc)) {
      // coarsest level: the sum plane and vector forms of its FP64 CGNE
      C.Ys = (double*)mg_alloc(mg, (ysz + 1) / 2);
      launch_sum_planes(C.Y, C.Ys, ysz, s);
      C.c4 = (double*)mg_alloc(mg, 4 * C.ndof);
    }
    if (mg->mixed) {
      CoarseGeom cg{C.E0, C.E1, C.nc};
      if (l + 2 < mg->nlev) {  // intermediate level: scaled FP16 copy
        C.Yh = (__half2*)mg_alloc(mg, (ysz + 3) / 4);
        C.Ysc = (float*)mg_alloc(mg, ((long)C.E0 * C.E1 * 5 + 3) / 4);
        launch_to_half_scaled(cg, C.Y, C.Yh, C.Ysc, s);
      } else {  // coarsest level: double-float copy
        C.Ydf = (float4*)mg_alloc(mg, ysz);
        launch_to_df64(C.Y, C.Ydf, ysz, s);
        C.cdf = (float4*)mg_alloc(mg, 2 * C.ndof);
      }
    }
    SW_CUDA(cudaStreamSynchronize(s));
    L.sr = L.sp = L.sq = L.st = nullptr;
  }
  // solve workspace
  for (int l = 0; l < mg->nlev; ++l) {
    MgLevel& L = mg->lev[l];
    long n = level_len(mg, l);
    L.rhs = mg_alloc(mg, n);
    L.sol = mg_alloc(mg, n);
    L.gr = mg_alloc(mg, n);
    L.gtmp = mg_alloc(mg, n);
    int nb = l == 0 ? mg->p.outer_restart : mg->p.inter_restart;
    if (l == mg->nlev - 1) nb = 0;
    L.gp.assign(nb, nullptr);
    L.gq.assign(nb, nullptr);
    for (int k = 0; k < nb; ++k) { L.gp[k] = mg_alloc(mg, n); L.gq[k] = mg_alloc(mg, n); }
    L.cp = mg_alloc(mg, n);
    L.cw = mg_alloc(mg, n);
    if (l + 1 < mg->nlev) {
      L.kx1 = mg_alloc(mg, n); L.kr1 = mg_alloc(mg, n); L.kq = mg_alloc(mg, n);
      L.ke = mg_alloc(mg, n); L.kr2 = mg_alloc(mg, n); L.kx3 = mg_alloc(mg, n);
      L.kr3 = mg_alloc(mg, n);
    }
    if (l == 0) {
      mg->bps = mg_alloc(mg, N);
      mg->xps = mg_alloc(mg, N);
      mg->lexb = mg_alloc(mg, N);
      mg->lexx = mg_alloc(mg, N);
      mg->lext = mg_alloc(mg, N);
    }
  }
}

// ---------------------------------------------------------------- solve
int mg_solve_device(sw_mg* mg, const double2* b_lex, double2* x_lex, double tol,
                    sw_solve_stats* st) {
  sw_ctx* c = mg->ctx;
  sw_gauge* g = mg->g;
  cudaStream_t s = c->stream;
  long N = g->N, half = N / 2;
  auto t0 = std::chrono::steady_clock::now();
  mg->st_fine_applies = mg->st_inter_iters = mg->st_inter_solves = 0;
  mg->st_coarsest_iters = mg->st_coarsest_solves = 0;
  MgLevel& L = mg->lev[0];
  launch_pack(g, b_lex, mg->bps, s);
  int sb = slot_base(0);
  blas_norm2(c, mg->bps, N, sb + 40);
  double bn = std::sqrt(slot_read(c, sb + 40).x);
  check_norm(bn, "right-hand side");
  if (bn == 0.0) {
    blas_zero(c, x_lex, N);
    SW_CUDA(cudaStreamSynchronize(s));
    if (st) {
      std::memset(st, 0, sizeof(*st));
      st->converged = 1;
    }
    return SW_OK;
  }
  GcrResult r;
  if (mg->fine_D) {
    // Galerkin MG of D itself: flexible GCR on the full D, no KD preconditioning
    r = fgcr(mg, 0, mg->bps, L.sol, tol * bn, mg->p.outer_restart, mg->p.outer_maxiter, true);
    launch_unpack(g, L.sol, x_lex, s);
  } else {
    // b~_e = b_e - A_eo b_o = b_e - C_eo B_o^-1 b_o
    launch_block_apply(g, mg->binv, 1, 0, mg->bps + half, L.stmp + half, s);
    launch_hop(g, 0, -1.0, mg->bps, L.stmp + half, L.rhs, s);
    r = fgcr(mg, 0, L.rhs, L.sol, tol * bn, mg->p.outer_restart, mg->p.outer_maxiter, true);
    // z_o = b_o - C_oe B_e^-1 z_e ; x = B^-1 z
    launch_block_apply(g, mg->binv, 0, 0, L.sol, L.stmp, s);
    launch_hop(g, 1, -1.0, mg->bps + half, L.stmp, L.stmp + half, s);
    launch_block_apply(g, mg->binv, 0, 0, L.sol, mg->xps, s);
    launch_block_apply(g, mg->binv, 1, 0, L.stmp + half, mg->xps + half, s);
    launch_unpack(g, mg->xps, x_lex, s);
  }
  // true residual ||b - D x|| / ||b|| in FP64
  launch_dslash_lex(g, mg->mass, 0, x_lex, mg->lext, s);
  blas_sub(c, mg->lext, b_lex, mg->lext, N);
  blas_norm2(c, mg->lext, N, sb + 41);
  double tr = std::sqrt(slot_read(c, sb + 41).x) / bn;
  auto t1 = std::chrono::steady_clock::now();
  if (st) {
    st->converged = r.converged ? 1 : 0;
    st->outer_iters = r.iters;
    st->restarts = r.restarts;
    st->fine_applies = mg->st_fine_applies;
    st->inter_iters = mg->st_inter_iters;
    st->inter_solves = mg->st_inter_solves;
    st->coarsest_iters = mg->st_coarsest_iters;
    st->coarsest_solves = mg->st_coarsest_solves;
    st->true_resid = tr;
    st->seconds = std::chrono::duration<double>(t1 - t0).count();
  }
  return r.converged ? SW_OK : SW_ERR_NOCONV;
}

// ================================================================ batched solves
// Several right-hand sides of one mixed-precision hierarchy advance in
// lockstep through the same K-cycle: every step is issued for each of them
// in turn (own work vectors, own page of Krylov scalars, own stopping tests),
// so that all of them reach the coarsest level together and share one
// batched coarsest CGNE launch, which reads the coarsest stencil once for the
// whole batch.  A right-hand side that has met a stopping test drops out of
// the step while the others go on.  Operator scratch (fine S temporaries) is
// shared: all steps run in order on the one context stream.

namespace {

using Set = std::vector<int>;

inline int page(int r) { return (r + 1) * kSlotPage; }

// Reads the slot pages of the batch (page 0 and those of its nb right-hand
// sides) back once after the queued reductions.
const double2* slots_read_all(sw_ctx* c, int nb) {
  SW_CUDA(cudaMemcpyAsync(c->h_slots, c->slots, (size_t)kSlotPage * (nb + 1) * sizeof(double2),
                          cudaMemcpyDeviceToHost, c->stream));
  SW_CUDA(cudaStreamSynchronize(c->stream));
  if (!c->pending.empty()) timing_harvest(c);
  return c->h_slots;
}

struct BatchCounters {
  std::vector<long long> fine, inter_it, inter_solves, coarse_it, coarse_solves;
  explicit BatchCounters(int nb)
      : fine(nb, 0), inter_it(nb, 0), inter_solves(nb, 0), coarse_it(nb, 0),
        coarse_solves(nb, 0) {}
};

void op_b(sw_mg* mg, int l, int r, const double2* in, double2* out, bool lowp,
          BatchCounters& bc) {
  level_op(mg, l, in, out, nullptr, lowp);
  if (l == 0) bc.fine[r]++;
}

// MR smoother (zero guess) for each member: x in kx1, residual in kr1.
void mr_b(sw_mg* mg, int l, const Set& set, const std::vector<const double2*>& b,
          BatchCounters& bc) {
  sw_ctx* c = mg->ctx;
  long n = level_len(mg, l);
  double om = mg->p.omega;
  for (int r : set) {
    LevelWs& W = mg->batch.lv[l][r];
    blas_zero(c, W.kx1, n);
    blas_copy(c, W.kr1, b[r], n);
  }
  for (int it = 0; it < mg->p.smoother_iters; ++it)
    for (int r : set) {
      LevelWs& W = mg->batch.lv[l][r];
      int sq = slot_base(l) + page(r) + 8, sqq = sq + 1;
      op_b(mg, l, r, W.kr1, W.kq, true, bc);
      blas_dot(c, W.kq, W.kr1, n, sq);
      blas_norm2(c, W.kq, n, sqq);
      blas_axpy(c, W.kx1, W.kr1, n, coef_ratio(sq, sqq, om));
      blas_axpy(c, W.kr1, W.kq, n, coef_ratio(sq, sqq, -om));
    }
}

void solve_level_b(sw_mg* mg, int l, const Set& set, BatchCounters& bc);

// out_r = M(g_r) on level l for every member of the set.
void kcycle_b(sw_mg* mg, int l, const Set& set, const std::vector<const double2*>& g,
              const std::vector<double2*>& out, BatchCounters& bc) {
  sw_ctx* c = mg->ctx;
  cudaStream_t s = c->stream;
  MgLevel& L = mg->lev[l];
  long n = level_len(mg, l);
  mr_b(mg, l, set, g, bc);
  for (int r : set) {
    LevelWs& W = mg->batch.lv[l][r];
    LevelWs& CW = mg->batch.lv[l + 1][r];
    if (l == 0)
      launch_restrict_fine(mg->g, L.b0, L.b1, L.nv, L.P, W.kr1, CW.rhs, s);
    else
      launch_restrict_coarse(CoarseGeom{L.E0, L.E1, L.nc}, L.b0, L.b1, L.nv, L.P, W.kr1, CW.rhs, s);
  }
  solve_level_b(mg, l + 1, set, bc);
  std::vector<const double2*> r2(mg->batch.nb, nullptr);
  for (int r : set) {
    LevelWs& W = mg->batch.lv[l][r];
    LevelWs& CW = mg->batch.lv[l + 1][r];
    if (l == 0)
      launch_prolong_fine(mg->g, L.b0, L.b1, L.nv, L.P, CW.sol, W.ke, s);
    else
      launch_prolong_coarse(CoarseGeom{L.E0, L.E1, L.nc}, L.b0, L.b1, L.nv, L.P, CW.sol, W.ke, s);
    op_b(mg, l, r, W.ke, W.kq, true, bc);
    blas_sub(c, W.kr2, W.kr1, W.kq, n);
    blas_copy(c, W.kx3, W.kx1, n);  // keep x1 while the post-smoother reuses kx1 / kr1
    r2[r] = W.kr2;
  }
  mr_b(mg, l, set, r2, bc);
  for (int r : set) {
    LevelWs& W = mg->batch.lv[l][r];
    blas_add3(c, out[r], W.kx3, W.ke, W.kx1, n);  // (x1 + e) + x3
  }
}

struct SetResult {
  std::vector<int> it, restarts;
  std::vector<char> conv;
};

// Flexible GCR (the steps of fgcr above) for every member of the set.
SetResult fgcr_b(sw_mg* mg, int l, const Set& set, const std::vector<const double2*>& b,
                 const std::vector<double2*>& x, const std::vector<double>& tol_abs, int restart,
                 int maxiter, bool confirm, BatchCounters& bc) {
  sw_ctx* c = mg->ctx;
  long n = level_len(mg, l);
  int nb = mg->batch.nb;
  SetResult res{std::vector<int>(nb, 0), std::vector<int>(nb, 0), std::vector<char>(nb, 0)};
  std::vector<int> k(nb, 0);
  std::vector<char> done(nb, 1);
  for (int r : set) {
    LevelWs& W = mg->batch.lv[l][r];
    blas_zero(c, x[r], n);
    blas_copy(c, W.gr, b[r], n);
    done[r] = 0;
  }
  const bool lowp = l > 0;
  for (;;) {
    Set act;
    for (int r : set)
      if (!done[r]) act.push_back(r);
    if (act.empty()) break;
    for (int r : act) blas_norm2(c, mg->batch.lv[l][r].gr, n, slot_base(l) + page(r));
    const double2* hs = slots_read_all(c, nb);
    Set cand, go;
    for (int r : act) {
      double rn = std::sqrt(hs[slot_base(l) + page(r)].x);
      check_norm(rn, "batched GCR residual");
      if (rn <= tol_abs[r]) {
        if (confirm) {
          cand.push_back(r);
        } else {
          done[r] = 1;
          res.conv[r] = 1;
        }
      } else if (res.it[r] >= maxiter) {
        done[r] = 1;
      } else {
        go.push_back(r);
      }
    }
    if (!cand.empty()) {  // confirm on the true residual, then test everybody again
      for (int r : cand) {
        LevelWs& W = mg->batch.lv[l][r];
        op_b(mg, l, r, x[r], W.gtmp, lowp, bc);
        blas_sub(c, W.gtmp, b[r], W.gtmp, n);
        blas_norm2(c, W.gtmp, n, slot_base(l) + page(r) + 1);
      }
      const double2* hs2 = slots_read_all(c, nb);
      for (int r : cand) {
        double rt = std::sqrt(hs2[slot_base(l) + page(r) + 1].x);
        check_norm(rt, "batched GCR true residual");
        if (rt <= tol_abs[r]) {
          done[r] = 1;
          res.conv[r] = 1;
        } else {
          LevelWs& W = mg->batch.lv[l][r];
          blas_copy(c, W.gr, W.gtmp, n);
          k[r] = 0;
          res.restarts[r]++;
        }
      }
      continue;
    }
    if (go.empty()) continue;  // every active member has just stopped
    std::vector<const double2*> g(nb, nullptr);
    std::vector<double2*> p(nb, nullptr);
    for (int r : go) {
      LevelWs& W = mg->batch.lv[l][r];
      g[r] = W.gr;
      p[r] = W.gp[k[r]];
    }
    if (l + 1 < mg->nlev)
      kcycle_b(mg, l, go, g, p, bc);
    else
      for (int r : go) blas_copy(c, p[r], g[r], n);
    for (int r : go) {
      LevelWs& W = mg->batch.lv[l][r];
      int sb = slot_base(l) + page(r);
      int s_qq = sb + 2, s_a = sb + 3, s_b = sb + 4;
      double2* q = W.gq[k[r]];
      double2* pr = W.gp[k[r]];
      op_b(mg, l, r, pr, q, lowp, bc);
      for (int j = 0; j < k[r]; ++j) {
        blas_dot(c, W.gq[j], q, n, s_b);
        blas_axpy(c, q, W.gq[j], n, coef_ratio(s_b, -1, -1.0));
        blas_axpy(c, pr, W.gp[j], n, coef_ratio(s_b, -1, -1.0));
      }
      blas_norm2(c, q, n, s_qq);
      blas_scale(c, q, n, coef_ratio(-1, s_qq, 1.0, COEF_SQRT_DEN));
      blas_scale(c, pr, n, coef_ratio(-1, s_qq, 1.0, COEF_SQRT_DEN));
      blas_dot(c, q, W.gr, n, s_a);
      blas_axpy(c, x[r], pr, n, coef_ratio(s_a, -1, 1.0));
      blas_axpy(c, W.gr, q, n, coef_ratio(s_a, -1, -1.0));
      ++k[r];
      ++res.it[r];
      if (k[r] == restart && res.it[r] < maxiter) {
        op_b(mg, l, r, x[r], W.gtmp, lowp, bc);
        blas_sub(c, W.gr, b[r], W.gtmp, n);
        k[r] = 0;
        res.restarts[r]++;
      }
    }
  }
  return res;
}

// ---------------------------------------------------------------- autotuner
// Pipeline depth of the tensor-core batched CGNE, chosen on first use per
// (device, nc, width, coarse sites) by timing each candidate for a few
// iterations on the call's own data (the real solve then starts from scratch).

int tc_stages(sw_mg* mg, const MgLevel& L, int nb, double2* const* bptr, double2* const* xptr,
              int sms) {
  sw_ctx* c = mg->ctx;
  BatchWs& B = mg->batch;
  const int K = tc_width(nb);
  const bool f32 = mg->p.batch_iterates == SW_PREC_FP32;
  // batch widths of FP32-iterate runs are recorded as 100 + K
  const auto key = std::make_tuple(c->device, L.nc, f32 ? 100 + K : K, L.E0 * L.E1, sms);
  {
    std::lock_guard<std::mutex> lk(g_tune_mutex);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) return it->second.stages;
  }
  int opts[8];
  const int nopt = tc_stage_options(L.nc, K, opts);
  SW_REQUIRE(nopt > 0, SW_ERR_ARG, "no tensor-core tiling fits shared memory");
  // each candidate: a warm-up launch, then the fastest of kReps launches of
  // kTuneIters iterations (the minimum is robust against other streams' work)
  constexpr int kTuneIters = 16, kReps = 3;
  const CoarseGeom cg{L.E0, L.E1, L.nc};
  const float keep = tc_l2_fraction(cg, c->device);
  cudaEvent_t e0, e1;
  SW_CUDA(cudaEventCreate(&e0));
  SW_CUDA(cudaEventCreate(&e1));
  TuneRec best{opts[0], 1e30};
  // candidates: every pipeline depth, with the stencil tiles streamed through
  // L2 (choice S) or partly kept there (choice 10 + S)
  for (int k = 0; k < 2 * nopt; ++k) {
    const int choice = opts[k % nopt] + (k >= nopt ? 10 : 0);
    float fastest = 1e30f;
    for (int rep = 0; rep <= kReps; ++rep) {  // rep 0 is a warm-up
      SW_CUDA(cudaEventRecord(e0, c->stream));
      bool ran = launch_cgne_tc(cg, choice % 10, f32, B.At, B.Ad, nb, bptr, xptr, B.X, B.R, B.P,
                                B.Rt, B.Pt, B.partials, B.bar, B.status, kTuneIters, 0.0,
                                c->device, c->stream, 0, sms, choice >= 10 ? keep : 0.f);
      SW_CUDA(cudaEventRecord(e1, c->stream));
      SW_CUDA(cudaEventSynchronize(e1));
      SW_REQUIRE(ran, SW_ERR_ARG, "tensor-core batched CGNE has no variant for this shape");
      int st0 = 0;
      SW_CUDA(cudaMemcpy(&st0, B.status, sizeof(int), cudaMemcpyDeviceToHost));
      SW_REQUIRE(st0 == 0, SW_ERR_TIMEOUT, "batched coarsest CGNE: a wait gave up while tuning");
      float ms = 0.f;
      SW_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (rep > 0 && ms < fastest) fastest = ms;
    }
    const double us = 1e3 * fastest / kTuneIters;
    if (us < best.us_per_iter) best = TuneRec{choice, us};
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::lock_guard<std::mutex> lk(g_tune_mutex);
  g_tune[key] = best;
  return best.stages;
}

void cgne_b(sw_mg* mg, int l, const Set& set, BatchCounters& bc, int stall = 0) {
  if (set.empty()) return;
  sw_ctx* c = mg->ctx;
  MgLevel& L = mg->lev[l];
  BatchWs& B = mg->batch;
  const int nb = (int)set.size();
  const bool tc = tc_supported(L.nc) && !B.Yf;
  const bool f32 = mg->p.batch_iterates == SW_PREC_FP32;
  double2* hp[2 * kMaxBatch] = {nullptr};
  for (int i = 0; i < nb; ++i) {
    hp[i] = B.lv[l][set[i]].rhs;
    hp[kMaxBatch + i] = B.lv[l][set[i]].sol;
  }
  SW_CUDA(cudaMemcpyAsync(B.dptr, hp, sizeof(hp), cudaMemcpyHostToDevice, c->stream));
  SW_CUDA(cudaStreamSynchronize(c->stream));  // hp is a host stack array
  SmLease lease(c);
  std::vector<int> its(nb, 0);
  // the CUDA-core FP32 kernel (SW_BATCH_FP32=1) takes at most 16 at a time
  const int chunk = tc ? kMaxBatch : 16;
  for (int i0 = 0; i0 < nb; i0 += chunk) {
    const int m = std::min(chunk, nb - i0);
    bool ran;
    int tk;
    if (tc) {
      const int choice = tc_stages(mg, L, m, B.dptr + i0, B.dptr + kMaxBatch + i0, lease.sms());
      const CoarseGeom cg{L.E0, L.E1, L.nc};
      tk = timing_begin(c, kCatCgne);
      ran = launch_cgne_tc(cg, choice % 10, f32, B.At, B.Ad, m, B.dptr + i0,
                           B.dptr + kMaxBatch + i0, B.X, B.R, B.P, B.Rt, B.Pt, B.partials,
                           B.bar, B.status, mg->p.coarsest_maxiter, mg->p.coarsest_tol,
                           c->device, c->stream, stall, lease.sms(),
                           choice >= 10 ? tc_l2_fraction(cg, c->device) : 0.f);
    } else {
      tk = timing_begin(c, kCatCgne);
      ran = launch_cgne_batch(CoarseGeom{L.E0, L.E1, L.nc}, B.Yf, B.Yd, m, B.dptr + i0,
                              B.dptr + kMaxBatch + i0, B.X, B.R, B.P, B.Rf, B.Pf, B.partials,
                              B.bar, B.status, mg->p.coarsest_maxiter, mg->p.coarsest_tol,
                              c->device, c->stream, lease.sms());
    }
    timing_end(c, tk);
    if (!ran)
      throw SwError{SW_ERR_ARG, "no batched coarsest solver for nc = " + std::to_string(L.nc)};
    int hst[2 + kMaxBatch];
    SW_CUDA(cudaMemcpyAsync(hst, B.status, sizeof(hst), cudaMemcpyDeviceToHost, c->stream));
    SW_CUDA(cudaStreamSynchronize(c->stream));
    if (!c->pending.empty()) timing_harvest(c);
    if (hst[0])
      throw SwError{SW_ERR_TIMEOUT,
                    "batched coarsest CGNE: a wait gave up or a buffer was misaligned"};
    if (hst[1]) throw SwError{SW_ERR_NAN, "non-finite norm in batched CGNE"};
    int kernel_it = 0;  // the launch runs as many iterations as its slowest right-hand side
    for (int i = 0; i < m; ++i) {
      its[i0 + i] = hst[2 + i];
      kernel_it = std::max(kernel_it, hst[2 + i]);
    }
    if (c->timing) c->t_count[kCatCgne + 1] += kernel_it;
  }
  for (int i = 0; i < nb; ++i) {
    bc.coarse_it[set[i]] += its[i];
    bc.coarse_solves[set[i]]++;
  }
}

void solve_level_b(sw_mg* mg, int l, const Set& set, BatchCounters& bc) {
  sw_ctx* c = mg->ctx;
  if (l == mg->nlev - 1) {
    cgne_b(mg, l, set, bc);
    return;
  }
  long n = level_len(mg, l);
  int nb = mg->batch.nb;
  for (int r : set) blas_norm2(c, mg->batch.lv[l][r].rhs, n, slot_base(l) + page(r) + 5);
  const double2* hs = slots_read_all(c, nb);
  std::vector<double> tol(nb, 0.0);
  std::vector<const double2*> b(nb, nullptr);
  std::vector<double2*> x(nb, nullptr);
  for (int r : set) {
    double bn = std::sqrt(hs[slot_base(l) + page(r) + 5].x);
    check_norm(bn, "batched intermediate right-hand side");
    tol[r] = mg->p.inter_tol * bn;
    b[r] = mg->batch.lv[l][r].rhs;
    x[r] = mg->batch.lv[l][r].sol;
  }
  SetResult res =
      fgcr_b(mg, l, set, b, x, tol, mg->p.inter_restart, mg->p.inter_maxiter, false, bc);
  for (int r : set) {
    bc.inter_it[r] += res.it[r];
    bc.inter_solves[r]++;
  }
}

// Per-right-hand-side work vectors for nb right-hand sides (grown on demand)
// and, on the first call, the arrays all of them share.
void batch_alloc(sw_mg* mg, int nb) {
  BatchWs& B = mg->batch;
  sw_ctx* c = mg->ctx;
  long N = mg->g->N;
  if (B.lv.empty()) B.lv.assign(mg->nlev, std::vector<LevelWs>());
  if (nb > B.nb) {
    const int cap = std::min(kMaxBatch, std::max(nb, 2 * B.nb));
    for (int l = 0; l < mg->nlev; ++l) {
      long n = level_len(mg, l);
      bool last = l == mg->nlev - 1;
      int nbas = last ? 0 : (l == 0 ? mg->p.outer_restart : mg->p.inter_restart);
      B.lv[l].resize(cap);
      for (int r = B.nb; r < cap; ++r) {
        LevelWs& W = B.lv[l][r];
        W.rhs = mg_alloc(mg, n);
        W.sol = mg_alloc(mg, n);
        if (last) continue;
        W.gr = mg_alloc(mg, n);
        W.gtmp = mg_alloc(mg, n);
        W.gp.assign(nbas, nullptr);
        W.gq.assign(nbas, nullptr);
        for (int k = 0; k < nbas; ++k) {
          W.gp[k] = mg_alloc(mg, n);
          W.gq[k] = mg_alloc(mg, n);
        }
        W.kx1 = mg_alloc(mg, n); W.kr1 = mg_alloc(mg, n); W.kq = mg_alloc(mg, n);
        W.ke = mg_alloc(mg, n); W.kr2 = mg_alloc(mg, n); W.kx3 = mg_alloc(mg, n);
      }
    }
    B.nb = cap;
  }
  if (B.shared) return;
  MgLevel& C = mg->lev[mg->nlev - 1];
  const long nc = C.ndof;
  const long sites = (long)C.E0 * C.E1;
  const CoarseGeom cg{C.E0, C.E1, C.nc};
  B.X = mg_alloc(mg, nc * kMaxBatch);
  B.R = mg_alloc(mg, nc * kMaxBatch);
  B.P = mg_alloc(mg, nc * kMaxBatch);
  const char* fp32 = std::getenv("SW_BATCH_FP32");
  if (tc_supported(C.nc) && !(fp32 && fp32[0] == '1')) {
    // tensor-core kernel: stacked TF32 blocks of A and A^dag, right-hand-side tiles
    const long tiles = sites * 5 * tc_tile_floats(C.nc);
    B.At = (float*)mg_alloc(mg, (tiles + 3) / 4);
    B.Ad = (float*)mg_alloc(mg, (tiles + 3) / 4);
    launch_stack_tiles(cg, C.Y, B.At, 0, c->stream);
    launch_stack_tiles(cg, C.Y, B.Ad, 1, c->stream);
    const long vt = sites * 2L * kMaxBatch * C.nc;
    B.Rt = (float*)mg_alloc(mg, (vt + 3) / 4);
    B.Pt = (float*)mg_alloc(mg, (vt + 3) / 4);
  } else {
    // CUDA-core FP32 kernel: FP32 forward and adjoint blocks
    B.Rf = (float2*)mg_alloc(mg, (nc * 16 + 1) / 2);
    B.Pf = (float2*)mg_alloc(mg, (nc * 16 + 1) / 2);
    long ysz = sites * 5 * C.nc * C.nc;
    B.Yf = (float2*)mg_alloc(mg, (ysz + 1) / 2);
    launch_to_f32(C.Y, B.Yf, ysz, c->stream);
    B.Yd = (float2*)mg_alloc(mg, (ysz + 1) / 2);
    launch_adjoint_f32(cg, C.Y, B.Yd, c->stream);
  }
  int sms = 0;
  SW_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
  B.partials = (double*)mg_alloc(mg, (long)kMaxBatch * sms);  // 2 phases x 64 x SMs doubles
  B.bar = (unsigned*)mg_alloc(mg, 1);
  B.status = (int*)mg_alloc(mg, (2 + kMaxBatch + 3) / 4);
  B.dptr = (double2**)mg_alloc(mg, kMaxBatch);  // 2 x 64 pointers
  B.bps = mg_alloc(mg, N * kMaxBatch);
  B.xps = mg_alloc(mg, N * kMaxBatch);
  B.lex = mg_alloc(mg, N * kMaxBatch);
  B.shared = true;
}

}  // namespace

int mg_solve_batch_device(sw_mg* mg, int nb, const double2* Bl, double2* Xl, double tol,
                          sw_solve_stats* st) {
  sw_ctx* c = mg->ctx;
  sw_gauge* g = mg->g;
  cudaStream_t s = c->stream;
  SW_REQUIRE(nb >= 1 && nb <= kMaxBatch, SW_ERR_ARG, "batch of 1..64 right-hand sides");
  SW_REQUIRE(mg->mixed && !mg->fine_D, SW_ERR_ARG, "batched solves need a mixed hierarchy");
  auto t0 = std::chrono::steady_clock::now();
  batch_alloc(mg, nb);
  BatchWs& B = mg->batch;
  long N = g->N, half = N / 2;
  MgLevel& L = mg->lev[0];
  for (int r = 0; r < nb; ++r) {
    launch_pack(g, Bl + (long)r * N, B.bps + (long)r * N, s);
    blas_norm2(c, B.bps + (long)r * N, N, slot_base(0) + page(r) + 40);
  }
  const double2* hs = slots_read_all(c, nb);
  std::vector<double> bn(nb), tol_abs(nb);
  Set all;
  for (int r = 0; r < nb; ++r) {
    bn[r] = std::sqrt(hs[slot_base(0) + page(r) + 40].x);
    check_norm(bn[r], "right-hand side");
    tol_abs[r] = tol * bn[r];
    if (bn[r] > 0.0) all.push_back(r);
  }
  std::vector<const double2*> bt(kMaxBatch, nullptr);
  std::vector<double2*> z(kMaxBatch, nullptr);
  for (int r = 0; r < nb; ++r) {
    double2* bps = B.bps + (long)r * N;
    LevelWs& W = B.lv[0][r];
    // b~_e = b_e - C_eo B_o^-1 b_o
    launch_block_apply(g, mg->binv, 1, 0, bps + half, L.stmp + half, s);
    launch_hop(g, 0, -1.0, bps, L.stmp + half, W.rhs, s);
    bt[r] = W.rhs;
    z[r] = W.sol;
  }
  BatchCounters bc(kMaxBatch);
  SetResult res = fgcr_b(mg, 0, all, bt, z, tol_abs, mg->p.outer_restart, mg->p.outer_maxiter,
                         true, bc);
  for (int r = 0; r < nb; ++r) {
    double2* x = Xl + (long)r * N;
    if (bn[r] == 0.0) {
      blas_zero(c, x, N);
      continue;
    }
    double2* bps = B.bps + (long)r * N;
    double2* xps = B.xps + (long)r * N;
    LevelWs& W = B.lv[0][r];
    // z_o = b_o - C_oe B_e^-1 z_e ; x = B^-1 z
    launch_block_apply(g, mg->binv, 0, 0, W.sol, L.stmp, s);
    launch_hop(g, 1, -1.0, bps + half, L.stmp, L.stmp + half, s);
    launch_block_apply(g, mg->binv, 0, 0, W.sol, xps, s);
    launch_block_apply(g, mg->binv, 1, 0, L.stmp + half, xps + half, s);
    launch_unpack(g, xps, x, s);
    double2* t = B.lex + (long)r * N;
    launch_dslash_lex(g, mg->mass, 0, x, t, s);
    blas_sub(c, t, Bl + (long)r * N, t, N);
    blas_norm2(c, t, N, slot_base(0) + page(r) + 41);
  }
  const double2* hs2 = slots_read_all(c, nb);
  double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  bool ok = true;
  for (int r = 0; r < nb; ++r) {
    bool conv = bn[r] == 0.0 || res.conv[r];
    ok = ok && conv;
    if (!st) continue;
    sw_solve_stats& o = st[r];
    std::memset(&o, 0, sizeof(o));
    o.converged = conv ? 1 : 0;
    o.outer_iters = res.it[r];
    o.restarts = res.restarts[r];
    o.fine_applies = bc.fine[r];
    o.inter_iters = bc.inter_it[r];
    o.inter_solves = bc.inter_solves[r];
    o.coarsest_iters = bc.coarse_it[r];
    o.coarsest_solves = bc.coarse_solves[r];
    o.true_resid = bn[r] > 0.0 ? std::sqrt(hs2[slot_base(0) + page(r) + 41].x) / bn[r] : 0.0;
    o.seconds = secs;
  }
  return ok ? SW_OK : SW_ERR_NOCONV;
}

int mg_batch_stall(sw_mg* mg, int nb) {
  SW_REQUIRE(nb >= 1 && nb <= kMaxBatch, SW_ERR_ARG, "batch of 1..64 right-hand sides");
  SW_REQUIRE(mg->mixed && !mg->fine_D, SW_ERR_ARG, "batched solves need a mixed hierarchy");
  batch_alloc(mg, nb);
  const int l = mg->nlev - 1;
  for (int r = 0; r < nb; ++r) blas_zero(mg->ctx, mg->batch.lv[l][r].rhs, level_len(mg, l));
  Set set;
  for (int r = 0; r < nb; ++r) set.push_back(r);
  BatchCounters bc(kMaxBatch);
  cgne_b(mg, l, set, bc, 1);
  return SW_OK;
}

int mg_autotune_entries(int max, int* nc, int* K, int* sites, int* stages, double* us) {
  std::lock_guard<std::mutex> lk(g_tune_mutex);
  int n = 0;
  for (const auto& kv : g_tune) {
    if (n < max) {
      if (nc) nc[n] = std::get<1>(kv.first);
      if (K) K[n] = std::get<2>(kv.first);
      if (sites) sites[n] = std::get<3>(kv.first);
      if (stages) stages[n] = kv.second.stages;
      if (us) us[n] = kv.second.us_per_iter;
    }
    ++n;
  }
  return n;
}
