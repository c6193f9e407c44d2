/*
 * sw.h -- C ABI of libsw, a GB300 (sm_103a) implementation of the
 * Kaehler-Dirac preconditioned adaptive multigrid solver for the staggered
 * Dirac operator of the two-flavour 2D U(1) Schwinger model
 * (Brower, Clark, Strelchenko, Weinberg, "Multigrid for Staggered Lattice
 * Fermions", arXiv:1801.07823).
 *
 * Conventions shared by every call
 *  - Lattice L0 x L1, periodic, site index s = x0 + L0 * x1 (x0 fastest).
 *  - Complex numbers are interleaved (re, im): complex128 = two doubles,
 *    complex64 = two floats.  A fermion field is [L1][L0] complex.
 *  - Return value 0 is success; a negative SW_ERR_* code is failure, with a
 *    message from sw_last_error().  No C++ exception and no device trap ever
 *    crosses this interface.
 *  - "on_device" = 1: the pointer is device memory of the context's GPU;
 *    0: host memory (the call copies through the context stream and
 *    synchronises before returning).  Device-pointer calls are asynchronous
 *    on the context stream unless stated otherwise.
 *  - The library owns every object it returns; free it with the matching
 *    sw_*_free.  Buffers passed in stay owned by the caller.
 */
#ifndef SW_H
#define SW_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  SW_OK = 0,
  SW_ERR_ARG = -1,       /* bad argument value (NULL, mass <= 0, unknown op ...) */
  SW_ERR_SHAPE = -2,     /* lattice or aggregate extents not compatible */
  SW_ERR_OOM = -3,       /* device allocation failed */
  SW_ERR_NOCONV = -4,    /* solver hit its iteration cap (x holds the last iterate) */
  SW_ERR_BREAKDOWN = -5, /* zero norm in Gram-Schmidt or a Krylov recurrence */
  SW_ERR_NAN = -6,       /* NaN or Inf met in a residual norm */
  SW_ERR_CUDA = -7,      /* a CUDA runtime call failed */
  SW_ERR_TIMEOUT = -8    /* a bounded device-side wait gave up */
};

enum {
  SW_OP_D = 0,
  SW_OP_DDAG = 1,
  SW_OP_A = 2,
  SW_OP_ADAG = 3,
  SW_OP_S = 4,
  SW_OP_DNAIK = 5,
  SW_OP_ANAIK = 6
};
/* Arithmetic of an operator application: FP64; FP32; FP16S = FP16 storage with
 * one FP32 scale per stencil block and FP32 accumulation; DF64 = double-float
 * (pairs of FP32 numbers, 48-bit significand) on the FP32 pipes. */
enum { SW_PREC_FP64 = 0, SW_PREC_FP32 = 1, SW_PREC_FP16S = 2, SW_PREC_DF64 = 3 };
/* Precision of a multigrid hierarchy (sw_mg_params.precision). */
enum { SW_MG_FP64 = 0, SW_MG_MIXED = 1 };
/* Operator a hierarchy coarsens (sw_mg_params.fine_operator). */
enum { SW_MG_COARSEN_A = 0, SW_MG_COARSEN_D = 1 };

typedef struct sw_ctx sw_ctx;
typedef struct sw_gauge sw_gauge;
typedef struct sw_mg sw_mg;

/* Solver parameters.  sw_mg_params_default() fills the values of the paper's
 * Table kcycle (Sec. IV); the outer iteration cap (2000) is this library's. */
typedef struct {
  int setup_maxiter;     /* CG iterations per null vector (250) */
  double setup_tol;      /* CG relative residual per null vector (1e-4) */
  int setup_passes;      /* repetitions of the null-vector relaxation (1) */
  int outer_restart;     /* FGCR restart length on level 1 (32) */
  int outer_maxiter;     /* FGCR iteration cap on level 1 (2000) */
  int smoother_iters;    /* MR iterations pre and post, every level (2) */
  double omega;          /* MR relaxation parameter (0.85) */
  int inter_restart;     /* GCR restart on intermediate levels (8) */
  int inter_maxiter;     /* GCR iteration cap on intermediate levels (16) */
  double inter_tol;      /* GCR relative residual on intermediate levels (0.2) */
  int coarsest_maxiter;  /* CGNE iteration cap on the coarsest level (256) */
  double coarsest_tol;   /* CGNE relative residual on the coarsest level (0.2) */
  int precision;         /* SW_MG_FP64 (default): every operator in FP64.
                            SW_MG_MIXED: setup, Gram-Schmidt, coarse-operator build,
                            the outer FGCR (its S, residuals, restarts) and all
                            vectors and Krylov recurrences stay FP64; inside the
                            K-cycle the fine S runs in FP32 and intermediate-level
                            stencils in FP16S; the coarsest CGNE stays FP64
                            (environment SW_COARSEST_DF64=1: its stencil in DF64). */
  int fine_operator;     /* SW_MG_COARSEN_A (default): the paper's method, Galerkin
                            coarsening of A = D B^-1 with the Schur outer solve.
                            SW_MG_COARSEN_D: the same recipe applied to D itself
                            (P^dag D P, outer FGCR and MR on the full D), the
                            variant Sec. III.B shows to stall; FP64 only.  Level-1
                            transfers then act on all sites. */
  int batch_iterates;    /* Iterates of the batched coarsest CGNE of sw_mg_solve_batch
                            on a mixed hierarchy: SW_PREC_FP64 (default) or
                            SW_PREC_FP32 (x, r, p and their updates in FP32; norms
                            summed in FP64 from FP32 sums of eight rows; alpha and
                            beta computed in FP64).  On GB300 the FP64 updates of
                            wide batches cost more than their stencil products. */
} sw_mg_params;

/* Per-solve counters.  "fine applies" counts applications of the level-1
 * Schur operator I - A_eo A_oe (the paper's fine mat-vec, Sec. IV.A). */
typedef struct {
  int converged;              /* 1 if ||b - D x|| <= tol ||b|| */
  int outer_iters;            /* FGCR iterations on level 1 */
  int restarts;               /* FGCR restarts (incl. true-residual recomputes) */
  long long fine_applies;     /* Schur-operator applications */
  long long inter_iters;      /* GCR iterations summed over all intermediate solves */
  long long inter_solves;     /* number of intermediate-level solves */
  long long coarsest_iters;   /* CGNE iterations summed over all coarsest solves */
  long long coarsest_solves;  /* number of coarsest-level solves */
  double true_resid;          /* ||b - D x|| / ||b|| recomputed in FP64 at the end */
  double seconds;             /* wall time of the call */
} sw_solve_stats;

void sw_mg_params_default(sw_mg_params* p);

/* One GPU, one stream.  device: CUDA ordinal.  cuda_stream: a cudaStream_t
 * (e.g. torch.cuda.current_stream().cuda_stream) or NULL for the legacy
 * default stream.  Every later call on objects of this context runs on it. */
int sw_context_create(int device, void* cuda_stream, sw_ctx** out);
void sw_context_free(sw_ctx* ctx);
/* Share num/den (0 < num <= den) of the GPU's SMs that the persistent
 * (cooperative, grid-synchronised) coarsest-level kernels of this context may
 * hold: they run with one CTA on each of floor(SMs num / den) SMs (at least
 * one).  Default 1/1.  Persistent kernels of contexts of one process whose
 * shares fit the SM count together run concurrently; a launch that does not
 * fit beside the running ones waits for them (host side).  A result depends
 * on the share (the grid fixes the order of its sums), not on what else runs. */
int sw_context_set_sm_share(sw_ctx* ctx, int num, int den);
/* Last error message of the context (never NULL; "" after success). */
const char* sw_last_error(sw_ctx* ctx);

/* Gauge field: U_mu(x) = exp(i theta_mu(x)) (Sec. I: U(1) links), theta given
 * as FP64 [2][L1][L0].  L0 and L1 must be multiples of 4 and >= 4.  The
 * library copies theta; the caller keeps ownership. */
int sw_gauge_load(sw_ctx* ctx, int L0, int L1, const double* theta, int on_device,
                  sw_gauge** out);
void sw_gauge_free(sw_gauge* g);

/* One operator application out = op(in) on a [L1][L0] field.
 *  SW_OP_D    staggered operator, Eq. staggeredD:
 *             (Dx)(s) = m x(s) + 1/2 sum_mu eta_mu(s) [U_mu(s) x(s+mu) - U_mu(s-mu)^* x(s-mu)]
 *  SW_OP_DDAG its adjoint.
 *  SW_OP_A    Kaehler-Dirac preconditioned A = D B^-1 (Eq. defA), B = the
 *             2x2-block-diagonal part of D (Sec. II.A, Eq. localblock).
 *  SW_OP_ADAG its adjoint.
 *  SW_OP_S    Schur operator I - A_eo A_oe on the even KD blocks (Table kcycle):
 *             odd-block entries of in are ignored, of out are written as 0.
 *  SW_OP_DNAIK Naik-improved operator (Sec. II.A, Eq. freehisq) in Eq.
 *             staggeredD's sign and 1/2 normalisation: one-link hops x 9/8,
 *             three-link hops x (-1/24) carrying U_mu(x) U_mu(x+mu) U_mu(x+2mu)
 *             (the paper prints the free operator only).
 *  SW_OP_ANAIK D_Naik B_Naik^-1 with B_Naik its 2x2-block part (the three-link
 *             hops always leave the block, so B_Naik = B with hops x 9/8).
 * precision: SW_PREC_FP64 (complex128 buffers) or SW_PREC_FP32 (complex64
 * buffers; SW_OP_D and SW_OP_DDAG only).  mass must be > 0 for A, ADAG, S,
 * ANAIK.  The Naik ops build the long links (and B_Naik^-1) on first use. */
int sw_dslash(sw_gauge* g, double mass, int op, int precision, const void* in, void* out,
              int on_device);

/* Multigrid setup (Sec. IV): near-null vectors from CG on A A^dag, global
 * orthonormalisation, chiral doubling with (1 +- eps)/2 (level 1) or
 * (1 +- sigma3)/2 (coarser), block orthonormalisation, Galerkin coarse
 * operator P^dag A P, recursively.  The setup runs in FP64; with
 * params->precision = SW_MG_MIXED it also keeps the reduced-precision copies
 * of the operators that the mixed solve uses.
 *  levels    2, 3 or 4 (Sec. IV: the recursion applies to every coarser
 *            level).
 *  block     [levels-1][2] aggregate extents: block[0] in KD blocks (even
 *            values; 4,4 in the paper), block[l>0] in coarse sites (2,2).
 *  nvec      [levels-1] null vectors per level (8, 12 in the paper).
 *  params    NULL for the Table kcycle defaults.
 *  psi0      NULL, or [levels-1] host pointers; psi0[l] holds nvec[l] initial
 *            complex128 vectors of the level-(l+1) space, vector-major:
 *            level 1 [nvec][L1][L0]; level l+1 > 1 [nvec][sites][2 nvec[l-1]]
 *            with coarse site index X0 + E0 X1.  NULL: drawn from seed with
 *            SplitMix64 + Box-Muller (vector i of level l: stream
 *            sw_stream_seed(seed, l, i), element j from outputs 2j, 2j+1).
 * mass must be > 0: the 2x2 block B is singular at m = 0 for some links. */
int sw_mg_setup(sw_gauge* g, double mass, int levels, const int* block, const int* nvec,
                const sw_mg_params* params, uint64_t seed, const double* const* psi0,
                sw_mg** out);
void sw_mg_free(sw_mg* mg);

/* Solve D x = b to ||b - D x||_2 <= tol ||b||_2 (zero initial guess):
 * flexible GCR on the Schur system of A z = b with the K-cycle preconditioner,
 * then z_o = b_o - A_oe z_e, x = B^-1 z.  b, x: complex128 [L1][L0].
 * Synchronises the context stream.  Returns SW_ERR_NOCONV (x = last iterate,
 * st filled) when outer_maxiter is reached.  st may be NULL. */
int sw_mg_solve(sw_mg* mg, const void* b, void* x, double tol, int on_device,
                sw_solve_stats* st);

/* nrhs independent solves: B and X are [nrhs][L1][L0] complex128, st is
 * [nrhs] (or NULL).  Each right-hand side converges on its own (own Krylov
 * scalars and stopping tests, the same stopping rule as sw_mg_solve).  On an
 * SW_MG_FP64 hierarchy the solves run one after the other.  On an SW_MG_MIXED
 * hierarchy up to 64 right-hand sides advance together through the K-cycle
 * and the coarsest-level solves of all of them run in one batched kernel that
 * reads the coarsest stencil once per batch: its stencil products run on the
 * tensor cores (tcgen05, TF32 operands, FP32 accumulation) for coarse dof
 * counts 16, 24 and 64 (other counts run the same iteration on the CUDA
 * cores in FP32), with a pipeline depth and an L2 policy picked by timing on
 * first use (sw_autotune_entries); iterates and Krylov scalars stay FP64
 * unless params.batch_iterates is SW_PREC_FP32, and the outer FGCR is FP64.  Larger nrhs run in groups of 64.  A right-hand
 * side's scalars do not depend on the others in its batch.
 * Returns SW_ERR_NOCONV if any right-hand side did not converge. */
int sw_mg_solve_batch(sw_mg* mg, int nrhs, const void* B, void* X, double tol, int on_device,
                      sw_solve_stats* st);

/* The paper's comparison solver (Sec. II, Eq. normal; Sec. IV, Fig.
 * iterworst): CG on the even/odd normal system (m^2 - D_eo D_oe) x_e =
 * m b_e - D_eo b_o with even/odd = the site parity eps, then
 * x_o = (b_o - D_oe x_e) / m.  Stops when ||b - D x|| <= tol ||b|| (the CG
 * residual divided by m) or after maxiter iterations (SW_ERR_NOCONV).
 * b, x: complex128 [L1][L0].  st (may be NULL): outer_iters = CG iterations,
 * fine_applies = applications of m^2 - D_eo D_oe, true_resid recomputed.
 * Allocates its work buffers per call.  Synchronises the stream. */
int sw_cg_eo_solve(sw_gauge* g, double mass, const void* b, void* x, double tol, int maxiter,
                   int on_device, sw_solve_stats* st);

/* Integer maps of the lattice and hierarchy, for bit-exact comparison (host
 * buffers of N = L0 L1 int32 each; any may be NULL): eta [2][N] (eta_0, eta_1),
 * eps [N], kd_block [N], kd_parity [N], agg [N] (level-1 aggregate with
 * block a0 x a1 KD blocks).  Pure host computation. */
int sw_debug_maps(sw_gauge* g, int a0, int a1, int32_t* eta, int32_t* eps, int32_t* kd_block,
                  int32_t* kd_parity, int32_t* agg);

/* Shape of level l (1-based; 1 = fine) of a hierarchy: extents and dof per
 * site (1 on level 1, 2 nvec[l-2] below). */
int sw_mg_level_info(sw_mg* mg, int level, int* E0, int* E1, int* nc);

/* Integer maps of level l (1 = fine, up to levels - 1) of a hierarchy, as the
 * transfer kernels compute them, for bit-exact comparison (host buffers of
 * ndof_l int32 each; ndof_1 = L0 L1 in site order x0 + L0 x1, coarser levels
 * in dof order X nc + k): agg = the aggregate (site of level l + 1) each dof
 * belongs to; chir = its chirality, eps(x) on level 1 (Eq. epsilon) and sigma3
 * (+1 for k < nc/2, -1 above) on coarser levels (Sec. IV, chiral doubling). */
int sw_mg_level_maps(sw_mg* mg, int level, int32_t* agg, int32_t* chir);

/* Copies of level data, for tests (host buffers, complex128):
 *  P of level l (maps level l+1 to level l), [ndof_l][nvec_l]: row = dof of
 *  level l (fine: site s = x0 + L0 x1; coarser: X * nc + k), entry i = the
 *  column (aggregate of the row, chirality of the row, i).
 *  Y of level l >= 2 as [sites][5][nc][nc] row-major blocks (direction 0:
 *  self, 1: +0hat, 2: -0hat, 3: +1hat, 4: -1hat), so that
 *  (A_hat x)_X = sum_d Y[X][d] x_{X+d}. */
int sw_mg_export_P(sw_mg* mg, int level, double* P);
int sw_mg_export_Y(sw_mg* mg, int level, double* Y);

/* Test access to the level operators and transfers of a hierarchy.
 * sw_mg_apply_level: out = op_l(in).  Level 1: the Schur operator
 *   I - A_eo A_oe on [L1][L0] complex128 fields (odd-block entries of in
 *   ignored, of out written 0), precision SW_PREC_FP64, or SW_PREC_FP32 on a
 *   mixed hierarchy; on a SW_MG_COARSEN_D hierarchy, D on all sites; dagger
 *   must be 0.  Level >= 2: the coarse stencil A_hat
 *   (dagger = 1: A_hat^dag) on [sites][nc] complex128 (Sec. III: A_hat =
 *   P^dag A P as the nearest-neighbour stencil of the export above) in
 *   SW_PREC_FP64, or in the reduced copy a mixed hierarchy keeps for that
 *   level (SW_PREC_FP16S on intermediate levels, SW_PREC_DF64 on the
 *   coarsest).  Synchronises the stream.
 * sw_mg_transfer: dir = 0 restriction out = P^dag in from level l to l + 1;
 *   dir = 1 prolongation out = P in from level l + 1 to level l.  On level 1
 *   both act on the even KD-block sites only, as inside the solver (Sec. IV:
 *   odd contributions set to zero, odd part of the prolonged error dropped):
 *   odd entries of in are ignored, odd entries of out are written as 0; fine
 *   vectors are [L1][L0]. */
int sw_mg_apply_level(sw_mg* mg, int level, int precision, int dagger, const void* in, void* out,
                      int on_device);
int sw_mg_transfer(sw_mg* mg, int level, int dir, const void* in, void* out, int on_device);

/* Schur operator without any device allocation.  The paper has no
 * counterpart: this is a deployment variant of sw_dslash(..., SW_OP_S,
 * SW_PREC_FP64, ...) for callers that cannot call cudaMalloc -- applications
 * or frameworks that own every device allocation of the process, or loops
 * that must not enter the allocator.  Same result as sw_dslash with SW_OP_S
 * (odd-block entries of out written as 0).
 *  in, out  device pointers to complex128 [L1][L0] fields (no host path).
 *  Scratch  a fixed file-scope device array of 7 x 65536 complex128 (7.3 MB),
 *           held by every GPU that loads the library until the process exits;
 *           lattices with more than 65536 sites are rejected with
 *           SW_ERR_SHAPE.  The B^-1 table is rebuilt from the links on every
 *           call.
 *  The first call on a device looks up the scratch address on that device
 *  (cudaGetSymbolAddress); make that first call before any stream capture.
 *  All calls share the one array, which keeps the previous call's contents:
 *  calls that overlap on the GPU (other streams, other contexts of the same
 *  device) race.  Asynchronous on the context stream. */
int sw_dslash_schur_noalloc(sw_gauge* g, double mass, const void* in, void* out);

/* Measurement support.
 * sw_set_timing: enable (1) or disable (0) per-kernel timing on the context;
 *   resets the accumulators.  While enabled, CUDA events recorded on the
 *   context stream bracket every application of a level operator: category 0
 *   = fine Schur operator (3 kernels), category l = coarse stencil of level
 *   l + 1 (1 kernel, also its adjoint), category 5 = the coarsest-level CGNE
 *   when it runs as one persistent kernel (one launch per coarsest solve,
 *   or per batched coarsest solve of sw_mg_solve_batch); category 6 counts
 *   that kernel's CGNE iterations (a batched launch counts those of its
 *   slowest right-hand side; the ms stay 0).
 *   Synchronises the stream.
 * sw_kernel_times: for categories 0 .. n-1, the number of applications that
 *   ran and the summed event durations in ms (host arrays, either may be
 *   NULL).  The coarsest solver queues iterations ahead and skips those after
 *   its stopping test on the device; a skipped application is not counted but
 *   its (few-microsecond) event interval is included, so the average per
 *   application is an upper bound.  Synchronises the stream.
 * sw_launch_count: number of kernels this library has launched in the
 *   process so far (all contexts). */
int sw_set_timing(sw_ctx* ctx, int enable);
int sw_kernel_times(sw_ctx* ctx, int n, long long* launches, double* ms);
long long sw_launch_count(void);

/* Measured FP64 throughput of the context's device in TFLOP/s (*tflops): one
 * CTA of 16 warps per SM runs four independent chains of dependent FMAs per
 * thread, timed with CUDA events on the context stream after a warm-up
 * launch (two FLOPs per FMA).  It is the denominator of the FP64 kernels'
 * roofline, at the clock the device runs when it is called.  Allocates and
 * frees an SM-count x 512 array of doubles; synchronises the stream. */
int sw_fp64_peak(sw_ctx* ctx, double* tflops);

/* Failure-detection check of the persistent coarsest-level CGNE: runs it
 * once with one CTA withholding its arrival at the first grid barrier, so
 * every other CTA's bounded wait runs out (about a second).  Expected result:
 * SW_ERR_TIMEOUT, with the context still usable afterwards. */
int sw_debug_cgne_stall(sw_mg* mg);

/* Failure-detection check of the batched coarsest kernel: runs it once on
 * nrhs zero right-hand sides with one CTA withholding its first grid-barrier
 * arrival, so every other CTA's bounded wait runs out (about a second).
 * Expected result: SW_ERR_TIMEOUT, with the context still usable afterwards. */
int sw_debug_batch_stall(sw_mg* mg, int nrhs);

/* Choices of the autotuner in this process: entry k gives the coarse dof per
 * site nc[k], the batch width K[k], the number of coarse sites, the choice and
 * its measured microseconds per CGNE iteration.  For the batched tensor-core
 * coarsest kernel (K = 8, 16, 32 or 64; 100 + K with FP32 iterates) the
 * choice is its pipeline depth S, or 10 + S when part of its stencil tiles is
 * loaded with L2 evict-last priority (kept across iterations) instead of
 * streamed; for
 * the single-right-hand-side FP64 coarsest kernel (K = 1) it is the variant:
 * bit 0 the product form (0: four real FMAs per complex multiply-add, 1:
 * three, with a stored sum plane), bit 1 the row-sum form (0: every lane of a
 * row sums all partial sums, 1: reduce-scatter of the real and imaginary parts
 * and a per-component update), and 7 for variant 3 with its stencil, sum plane
 * and vector operands staged in shared memory by asynchronous copies.  Fills
 * at most max entries (any pointer may be NULL) and returns the number of
 * entries. */
int sw_autotune_entries(int max, int* nc, int* K, int* sites, int* stages, double* us);

/* SplitMix64 stream seed used when psi0 is NULL (level = index into psi0,
 * 0-based): s1 = mix(seed ^ level) + G, result = mix(s1 ^ index) + G, with
 * G = 0x9E3779B97F4A7C15 and mix the SplitMix64 finaliser (Steele, Lea and
 * Flood, OOPSLA 2014), arithmetic modulo 2^64. */
uint64_t sw_stream_seed(uint64_t seed, int level, int index);

#ifdef __cplusplus
}
#endif
#endif /* SW_H */
