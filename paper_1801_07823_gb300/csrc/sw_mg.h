// Multigrid hierarchy object shared by mg.cu and api.cu.
#pragma once
#include <vector>

#include "sw_internal.h"

// One level of the hierarchy.  Level 0 is the fine lattice (dof = site,
// parity-split order); level l > 0 is a coarse lattice E0 x E1 with nc dof per
// site (dof = X * nc + k).  b0, b1, nv and P describe the transfer from this
// level to level l + 1.
struct MgLevel {
  int E0 = 0, E1 = 0, nc = 1;
  long ndof = 0;
  int b0 = 0, b1 = 0, nv = 0;
  double2* P = nullptr;   // [ndof][nv]
  double2* Y = nullptr;   // stencil of this level (l > 0), see coarse.cu
  __half2* Yh = nullptr;  // mixed precision, intermediate levels: FP16 stencil ...
  float* Ysc = nullptr;   // ... with one scale per block
  float4* Ydf = nullptr;  // mixed precision, coarsest level: double-float stencil
  float4* cdf = nullptr;  // [2][ndof] double-float copies of r and p for its CGNE
  double* Ys = nullptr;   // coarsest level: Re + Im of every stencil entry (FP64 CGNE)
  double* c4 = nullptr;   // coarsest level: [2][ndof][4] vector forms of its FP64 CGNE
  // setup work vectors
  double2 *sr = nullptr, *sp = nullptr, *sq = nullptr, *st = nullptr;
  // solve work vectors
  double2 *rhs = nullptr, *sol = nullptr, *gr = nullptr, *gtmp = nullptr;
  double2 *cp = nullptr, *cw = nullptr;
  std::vector<double2*> gp, gq;
  double2 *kx1 = nullptr, *kr1 = nullptr, *kq = nullptr, *ke = nullptr, *kr2 = nullptr;
  double2 *kx3 = nullptr, *kr3 = nullptr;
  double2* stmp = nullptr;  // [N] scratch of the fine operators (level 0)
};

// Work vectors of one right-hand side on one level in a batched solve.
struct LevelWs {
  double2 *rhs = nullptr, *sol = nullptr, *gr = nullptr, *gtmp = nullptr;
  std::vector<double2*> gp, gq;
  double2 *kx1 = nullptr, *kr1 = nullptr, *kq = nullptr, *ke = nullptr, *kr2 = nullptr;
  double2 *kx3 = nullptr;
};

// Workspace of batched solves (allocated on the first one).
struct BatchWs {
  int nb = 0;                            // right-hand sides the workspace holds
  bool shared = false;                   // the arrays shared by all right-hand sides exist
  std::vector<std::vector<LevelWs>> lv;  // [level][rhs]
  double2 *X = nullptr, *R = nullptr, *P = nullptr;  // coarsest CGNE, [n][K]
  float2 *Rf = nullptr, *Pf = nullptr;
  float2* Yf = nullptr;                  // FP32 copy of the coarsest stencil
  float2* Yd = nullptr;                  // FP32 adjoint blocks of the coarsest stencil
  double* partials = nullptr;
  unsigned* bar = nullptr;
  int* status = nullptr;
  double2** dptr = nullptr;              // device arrays of b and x pointers, [2][64]
  float *At = nullptr, *Ad = nullptr;    // stacked TF32 tiles of the coarsest A and A^dag
  float *Rt = nullptr, *Pt = nullptr;    // TF32 right-hand-side tiles of r and p
  double2 *bps = nullptr, *xps = nullptr, *lex = nullptr;  // [16][N] fine buffers
};

struct sw_mg {
  sw_ctx* ctx = nullptr;
  sw_gauge* g = nullptr;
  double mass = 0.0;
  sw_mg_params p{};
  int nlev = 0;
  int stall_test = 0;  // sw_debug_cgne_stall: make the persistent CGNE's first barrier time out
  bool persistent_cgne = true;  // SW_CGNE_LOOP=1 selects the host-queued CGNE loop
  int verbose = 0;  // SW_VERBOSE=1: a stderr line per outer iteration; 2: also level 2
  double2* binv = nullptr;
  bool mixed = false;            // params.precision == SW_MG_MIXED
  bool fine_D = false;           // params.fine_operator == SW_MG_COARSEN_D
  float2* binv32 = nullptr;      // FP32 B^-1 (mixed)
  float2* s32tmp = nullptr;      // [N] FP32 scratch of the FP32 Schur operator
  std::vector<MgLevel> lev;
  std::vector<double2*> allocs;
  double2 *bps = nullptr, *xps = nullptr, *lexb = nullptr, *lexx = nullptr, *lext = nullptr;
  std::vector<int> setup_iters;
  BatchWs batch;
  long long st_fine_applies = 0, st_inter_iters = 0, st_inter_solves = 0;
  long long st_coarsest_iters = 0, st_coarsest_solves = 0;
};

// Device scalar slots owned by level l: [64 l, 64 l + 64).
inline int slot_base(int l) { return 64 * l; }

double2* mg_alloc(sw_mg* mg, long n);
// Device buffers owned by one library call, freed when it returns or throws.
struct ScopedBuffers {
  std::vector<double2*> list;
  double2* get(long n);
  ~ScopedBuffers();
};
void sw_mg_release(sw_mg* mg);
void mg_setup(sw_mg* mg, const double* const* psi0, uint64_t seed);
int mg_coarsest_solve(sw_mg* mg, const double2* b, double2* x);  // CGNE on the coarsest level
int mg_solve_device(sw_mg* mg, const double2* b_lex, double2* x_lex, double tol,
                    sw_solve_stats* st);
// nb (<= 64) right-hand sides of a mixed-precision hierarchy in lockstep, the
// coarsest solves of all of them in one batched kernel.  B, X: [nb][N]
// lexicographic device buffers; st: [nb] or NULL.
int mg_solve_batch_device(sw_mg* mg, int nb, const double2* B, double2* X, double tol,
                          sw_solve_stats* st);
// Failure-detection check of the batched coarsest kernel (sw_debug_batch_stall).
int mg_batch_stall(sw_mg* mg, int nb);
// Autotuner records: (nc, K, sites, stages, microseconds per iteration).
int mg_autotune_entries(int max, int* nc, int* K, int* sites, int* stages, double* us);
