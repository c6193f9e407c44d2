// C ABI of libsw (declared in include/sw.h): contexts, gauge fields, single
// operator applications, multigrid setup/solve and test exports.  Every entry
// point catches internal errors and returns an SW_ERR_* code.
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <new>

#include "sw_internal.h"
#include "sw_mg.h"

void report_stale_error(cudaError_t e) {
  static std::atomic<int> reported{0};
  if (reported.fetch_add(1) < 4)
    std::fprintf(stderr, "libsw: cleared a CUDA error pending from before this call: %s\n",
                 cudaGetErrorString(e));
}

void sw_poison(void* p, size_t bytes) {
  static const bool on = [] {
    const char* e = std::getenv("SW_POISON");
    return e && e[0] == '1';
  }();
  if (on && p && bytes) SW_CUDA(cudaMemset(p, 0xFF, bytes));  // all-ones: a NaN in every double
}

void dev_free(void* p, const char* what) {
  if (!p) return;
  cudaError_t e = cudaFree(p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    std::fprintf(stderr, "libsw: cudaFree(%s) failed: %s\n", what, cudaGetErrorString(e));
  }
}

namespace {

__global__ void k_links(const double* __restrict__ theta, double2* __restrict__ Wlex,
                        float2* __restrict__ Wlex32, double2* __restrict__ Wps,
                        float2* __restrict__ Wps32, int L0, int L1) {
  int N = L0 * L1;
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= N) return;
  int x0 = s % L0, x1 = s / L0;
  int f = ps_index(x0, x1, L0, N);
  for (int mu = 0; mu < 2; ++mu) {
    // W_mu(s) = eta_mu(s) U_mu(s) / 2, eta_0 = 1, eta_1 = (-1)^x0
    double eta = (mu == 1 && (x0 & 1)) ? -0.5 : 0.5;
    double sn, cs;
    sincos(theta[(long)mu * N + s], &sn, &cs);
    double2 w = make_double2(eta * cs, eta * sn);
    Wlex[(long)mu * N + s] = w;
    Wlex32[(long)mu * N + s] = make_float2((float)w.x, (float)w.y);
    Wps[(long)mu * N + f] = w;
    Wps32[(long)mu * N + f] = make_float2((float)w.x, (float)w.y);
  }
}

template <typename T>
T* dmalloc(size_t count) {
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, count * sizeof(T) > 0 ? count * sizeof(T) : 1);
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw SwError{SW_ERR_OOM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e)};
  }
  sw_poison(p, count * sizeof(T));
  return (T*)p;
}

void gauge_binv(sw_gauge* g, double mass) {
  if (!g->binv) g->binv = dmalloc<double2>((size_t)g->N * 4);
  if (g->binv_mass != mass) {
    launch_binv_build(g, mass, g->binv, g->ctx->stream);
    g->binv_mass = mass;
  }
}

}  // namespace

static std::atomic<long long> g_launches{0};
void sw_count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

extern "C" {

long long sw_launch_count(void) { return g_launches.load(); }

int sw_set_timing(sw_ctx* c, int enable) {
  if (!c) return SW_ERR_ARG;
  return guarded(c, [&] {
    SW_CUDA(cudaStreamSynchronize(c->stream));
    timing_harvest(c);
    c->timing = enable != 0;
    for (int k = 0; k < kTimeCats; ++k) {
      c->t_ms[k] = 0.0;
      c->t_count[k] = 0;
    }
    SW_CUDA(cudaMemsetAsync(c->exec, 0, kTimeCats * sizeof(unsigned long long), c->stream));
    SW_CUDA(cudaStreamSynchronize(c->stream));
    return SW_OK;
  });
}

int sw_kernel_times(sw_ctx* c, int n, long long* launches, double* ms) {
  if (!c || n < 0) return SW_ERR_ARG;
  return guarded(c, [&] {
    SW_CUDA(cudaStreamSynchronize(c->stream));
    timing_harvest(c);
    unsigned long long ex[kTimeCats];
    SW_CUDA(cudaMemcpy(ex, c->exec, sizeof(ex), cudaMemcpyDeviceToHost));
    for (int k = 0; k < n && k < kTimeCats; ++k) {
      // category 0 (fine S) is never skipped: count its event pairs; coarse
      // categories count the launches that ran (skipped ones are no-ops)
      bool host_counted = k == 0 || k >= kCatCgne;
      if (launches) launches[k] = host_counted ? c->t_count[k] : (long long)ex[k];
      if (ms) ms[k] = c->t_ms[k];
    }
    return SW_OK;
  });
}

void sw_mg_params_default(sw_mg_params* p) {
  if (!p) return;
  p->setup_maxiter = 250;
  p->setup_tol = 1e-4;
  p->setup_passes = 1;
  p->outer_restart = 32;
  p->outer_maxiter = 2000;
  p->smoother_iters = 2;
  p->omega = 0.85;
  p->inter_restart = 8;
  p->inter_maxiter = 16;
  p->inter_tol = 0.2;
  p->coarsest_maxiter = 256;
  p->coarsest_tol = 0.2;
  p->precision = SW_MG_FP64;
  p->fine_operator = SW_MG_COARSEN_A;
  p->batch_iterates = SW_PREC_FP64;
}

uint64_t sw_stream_seed(uint64_t seed, int level, int index) {
  auto mix = [](uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  const uint64_t G = 0x9E3779B97F4A7C15ull;
  uint64_t s = mix(seed ^ (uint64_t)(int64_t)level) + G;
  return mix(s ^ (uint64_t)(int64_t)index) + G;
}

int sw_context_create(int device, void* cuda_stream, sw_ctx** out) {
  if (!out) return SW_ERR_ARG;
  *out = nullptr;
  sw_ctx* c = new (std::nothrow) sw_ctx();
  if (!c) return SW_ERR_OOM;
  c->device = device;
  c->stream = (cudaStream_t)cuda_stream;
  int rc = guarded(c, [&] {
    int ndev = 0;
    SW_CUDA(cudaGetDeviceCount(&ndev));
    SW_REQUIRE(device >= 0 && device < ndev, SW_ERR_ARG, "no such CUDA device");
    c->slots = dmalloc<double2>(kNumSlots);
    c->partials = dmalloc<double>(2 * kReduceBlocks);
    c->counter = dmalloc<unsigned>(1);
    c->flag = dmalloc<int>(1);
    c->ctl = dmalloc<int>(4 * 8);
    c->bar = dmalloc<unsigned>(2);
    c->cgstat = dmalloc<int>(4);
    c->exec = dmalloc<unsigned long long>(kTimeCats);
    SW_CUDA(cudaMemset(c->ctl, 0, 4 * 8 * sizeof(int)));
    SW_CUDA(cudaMemset(c->exec, 0, kTimeCats * sizeof(unsigned long long)));
    SW_CUDA(cudaMallocHost(&c->h_ctl, 4 * sizeof(int)));
    SW_CUDA(cudaMemset(c->counter, 0, sizeof(unsigned)));
    SW_CUDA(cudaMemset(c->flag, 0, sizeof(int)));
    SW_CUDA(cudaMemset(c->slots, 0, kNumSlots * sizeof(double2)));
    SW_CUDA(cudaMallocHost(&c->h_slots, kNumSlots * sizeof(double2)));
    return SW_OK;
  });
  if (rc != SW_OK) {
    sw_context_free(c);
    return rc;
  }
  *out = c;
  return SW_OK;
}

void sw_context_free(sw_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (TimedPair& t : c->pending) {
    cudaEventDestroy(t.a);
    cudaEventDestroy(t.b);
  }
  for (cudaEvent_t e : c->spare) cudaEventDestroy(e);
  dev_free(c->slots, "slots");
  dev_free(c->partials, "partials");
  dev_free(c->counter, "counter");
  dev_free(c->flag, "flag");
  dev_free(c->ctl, "ctl");
  dev_free(c->exec, "exec");
  dev_free(c->bar, "bar");
  dev_free(c->cgstat, "cgstat");
  if (c->h_slots) cudaFreeHost(c->h_slots);
  if (c->h_ctl) cudaFreeHost(c->h_ctl);
  delete c;
}

const char* sw_last_error(sw_ctx* c) { return c ? c->err.c_str() : "null context"; }

int sw_gauge_load(sw_ctx* c, int L0, int L1, const double* theta, int on_device, sw_gauge** out) {
  if (!c || !out || !theta) return SW_ERR_ARG;
  *out = nullptr;
  sw_gauge* g = new (std::nothrow) sw_gauge();
  if (!g) return SW_ERR_OOM;
  int rc = guarded(c, [&] {
    SW_REQUIRE(L0 >= 4 && L1 >= 4 && L0 % 4 == 0 && L1 % 4 == 0, SW_ERR_SHAPE,
               "L0 and L1 must be multiples of 4");
    SW_REQUIRE((long)L0 * L1 < (1L << 30), SW_ERR_SHAPE, "lattice too large");
    g->ctx = c;
    g->L0 = L0;
    g->L1 = L1;
    g->N = L0 * L1;
    size_t N = g->N;
    g->W_lex = dmalloc<double2>(2 * N);
    g->W_lex32 = dmalloc<float2>(2 * N);
    g->W_ps = dmalloc<double2>(2 * N);
    g->W_ps32 = dmalloc<float2>(2 * N);
    const double* th = theta;
    double* tmp = nullptr;
    if (!on_device) {
      tmp = dmalloc<double>(2 * N);
      SW_CUDA(cudaMemcpyAsync(tmp, theta, 2 * N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
      th = tmp;
    }
    k_links<<<(unsigned)((N + 255) / 256), 256, 0, c->stream>>>(th, g->W_lex, g->W_lex32, g->W_ps,
                                                                g->W_ps32, L0, L1);
    SW_LAUNCH_CHECK();
    SW_CUDA(cudaStreamSynchronize(c->stream));
    dev_free(tmp, "theta staging");
    return SW_OK;
  });
  if (rc != SW_OK) {
    g->ctx = c;
    sw_gauge_free(g);
    return rc;
  }
  *out = g;
  return SW_OK;
}

void sw_gauge_free(sw_gauge* g) {
  if (!g) return;
  if (g->ctx) {
    cudaSetDevice(g->ctx->device);
    if (g->ctx->stream) cudaStreamSynchronize(g->ctx->stream);
  }
  dev_free(g->W_lex, "W_lex");
  dev_free(g->W_lex32, "W_lex32");
  dev_free(g->W_ps, "W_ps");
  dev_free(g->W_ps32, "W_ps32");
  dev_free(g->binv, "binv");
  dev_free(g->W3_lex, "W3_lex");
  dev_free(g->binv_naik, "binv_naik");
  for (auto& t : g->tmp) dev_free(t, "gauge scratch");
  delete g;
}

int sw_dslash(sw_gauge* g, double mass, int op, int precision, const void* in, void* out,
              int on_device) {
  if (!g || !in || !out) return SW_ERR_ARG;
  sw_ctx* c = g->ctx;
  return guarded(c, [&] {
    SW_REQUIRE(op >= SW_OP_D && op <= SW_OP_ANAIK, SW_ERR_ARG, "unknown op");
    SW_REQUIRE(precision == SW_PREC_FP64 || precision == SW_PREC_FP32, SW_ERR_ARG,
               "unknown precision");
    SW_REQUIRE(precision == SW_PREC_FP64 || op <= SW_OP_DDAG, SW_ERR_ARG,
               "FP32 is available for D and D^dag only");
    SW_REQUIRE(std::isfinite(mass), SW_ERR_ARG, "mass must be finite");
    SW_REQUIRE(op <= SW_OP_DDAG || op == SW_OP_DNAIK || mass > 0.0, SW_ERR_ARG,
               "A, A^dag, S and the Naik A need mass > 0");
    cudaStream_t s = c->stream;
    size_t N = g->N;
    size_t esz = precision == SW_PREC_FP64 ? sizeof(double2) : sizeof(float2);
    const void* din = in;
    void* dout = out;
    if (!on_device) {
      if (!g->tmp[0]) g->tmp[0] = dmalloc<double2>(N);
      if (!g->tmp[1]) g->tmp[1] = dmalloc<double2>(N);
      SW_CUDA(cudaMemcpyAsync(g->tmp[0], in, N * esz, cudaMemcpyHostToDevice, s));
      din = g->tmp[0];
      dout = g->tmp[1];
    }
    if (op == SW_OP_DNAIK || op == SW_OP_ANAIK) {
      const double c1 = 9.0 / 8.0, c3 = -1.0 / 24.0;
      if (!g->W3_lex) {
        g->W3_lex = dmalloc<double2>(2 * N);
        launch_long_links(g, c3, g->W3_lex, s);
      }
      if (op == SW_OP_DNAIK) {
        launch_dslash_naik_lex(g, g->W3_lex, mass, c1, (const double2*)din, (double2*)dout, s);
      } else {
        for (int t = 2; t < 4; ++t)
          if (!g->tmp[t]) g->tmp[t] = dmalloc<double2>(N);
        if (!g->binv_naik) g->binv_naik = dmalloc<double2>(N * 4);
        if (g->naik_mass != mass) {
          launch_binv_build(g, mass, g->binv_naik, s, c1);
          g->naik_mass = mass;
        }
        // A_Naik = D_Naik B_Naik^-1: t = B^-1 x per KD block, y = D_Naik t
        double2* a = g->tmp[2];
        double2* b = g->tmp[3];
        launch_pack(g, (const double2*)din, a, s);
        launch_block_apply(g, g->binv_naik, 0, 0, a, b, s);
        launch_block_apply(g, g->binv_naik, 1, 0, a + N / 2, b + N / 2, s);
        launch_unpack(g, b, a, s);
        launch_dslash_naik_lex(g, g->W3_lex, mass, c1, a, (double2*)dout, s);
      }
    } else if (op <= SW_OP_DDAG) {
      if (precision == SW_PREC_FP64)
        launch_dslash_lex(g, mass, op == SW_OP_DDAG, (const double2*)din, (double2*)dout, s);
      else
        launch_dslash_lex32(g, (float)mass, op == SW_OP_DDAG, (const float2*)din, (float2*)dout, s);
    } else {
      for (int t = 2; t < 4; ++t)
        if (!g->tmp[t]) g->tmp[t] = dmalloc<double2>(N);
      gauge_binv(g, mass);
      double2* a = g->tmp[2];
      double2* b = g->tmp[3];
      double2* w = (double2*)dout;  // scratch before the final unpack
      launch_pack(g, (const double2*)din, a, s);
      if (op == SW_OP_A) {
        fine_apply_A(g, g->binv, a, b, w, s);
      } else if (op == SW_OP_ADAG) {
        fine_apply_Adag(g, g->binv, a, b, s);
      } else {
        fine_apply_S(g, g->binv, a, b, w, s);
        SW_CUDA(cudaMemsetAsync(b + N / 2, 0, N / 2 * sizeof(double2), s));
      }
      launch_unpack(g, b, (double2*)dout, s);
    }
    if (!on_device) {
      SW_CUDA(cudaMemcpyAsync(out, dout, N * esz, cudaMemcpyDeviceToHost, s));
      SW_CUDA(cudaStreamSynchronize(s));
    }
    return SW_OK;
  });
}

int sw_mg_setup(sw_gauge* g, double mass, int levels, const int* block, const int* nvec,
                const sw_mg_params* params, uint64_t seed, const double* const* psi0,
                sw_mg** out) {
  if (!g || !out || !block || !nvec) return SW_ERR_ARG;
  *out = nullptr;
  sw_ctx* c = g->ctx;
  sw_mg* mg = new (std::nothrow) sw_mg();
  if (!mg) return SW_ERR_OOM;
  int rc = guarded(c, [&] {
    SW_REQUIRE(levels >= 2 && levels <= 4, SW_ERR_ARG, "levels must be 2, 3 or 4");
    SW_REQUIRE(std::isfinite(mass) && mass > 0.0, SW_ERR_ARG,
               "mass must be > 0 (B is singular at m = 0 for some links)");
    mg->ctx = c;
    mg->g = g;
    mg->mass = mass;
    mg->nlev = levels;
    const char* vb = std::getenv("SW_VERBOSE");
    mg->verbose = vb ? std::atoi(vb) : 0;
    const char* cl = std::getenv("SW_CGNE_LOOP");
    mg->persistent_cgne = !(cl && cl[0] == '1');
    if (params)
      mg->p = *params;
    else
      sw_mg_params_default(&mg->p);
    const sw_mg_params& p = mg->p;
    SW_REQUIRE(p.precision == SW_MG_FP64 || p.precision == SW_MG_MIXED, SW_ERR_ARG,
               "unknown precision");
    mg->mixed = p.precision == SW_MG_MIXED;
    SW_REQUIRE(p.fine_operator == SW_MG_COARSEN_A || p.fine_operator == SW_MG_COARSEN_D,
               SW_ERR_ARG, "unknown fine_operator");
    SW_REQUIRE(p.batch_iterates == SW_PREC_FP64 || p.batch_iterates == SW_PREC_FP32, SW_ERR_ARG,
               "batch_iterates must be SW_PREC_FP64 or SW_PREC_FP32");
    mg->fine_D = p.fine_operator == SW_MG_COARSEN_D;
    SW_REQUIRE(!(mg->fine_D && mg->mixed), SW_ERR_ARG,
               "the Galerkin MG of D is provided in FP64 only");
    SW_REQUIRE(p.setup_maxiter >= 0 && p.setup_passes >= 1 && p.outer_restart >= 1 &&
                   p.outer_maxiter >= 0 && p.smoother_iters >= 0 && p.inter_restart >= 1 &&
                   p.inter_maxiter >= 0 && p.coarsest_maxiter >= 0,
               SW_ERR_ARG, "invalid solver parameters");
    mg->lev.resize(levels);
    MgLevel& F = mg->lev[0];
    F.E0 = g->L0;
    F.E1 = g->L1;
    F.nc = 1;
    F.ndof = g->N;
    for (int l = 0; l + 1 < levels; ++l) {
      MgLevel& L = mg->lev[l];
      MgLevel& C = mg->lev[l + 1];
      int b0 = block[2 * l], b1 = block[2 * l + 1], nv = nvec[l];
      SW_REQUIRE(nv >= 1 && nv <= 64, SW_ERR_ARG, "nvec must be in [1, 64]");
      SW_REQUIRE(b0 >= 1 && b1 >= 1, SW_ERR_SHAPE, "aggregate extents must be >= 1");
      if (l == 0) {
        SW_REQUIRE(b0 % 2 == 0 && b1 % 2 == 0, SW_ERR_SHAPE,
                   "level-1 aggregates must span an even number of KD blocks");
        SW_REQUIRE(g->L0 % (2 * b0) == 0 && g->L1 % (2 * b1) == 0, SW_ERR_SHAPE,
                   "lattice not divisible by the level-1 aggregate");
        SW_REQUIRE(2 * b0 * b1 <= 1024, SW_ERR_SHAPE, "level-1 aggregate too large");
        C.E0 = g->L0 / (2 * b0);
        C.E1 = g->L1 / (2 * b1);
      } else {
        SW_REQUIRE(L.E0 % b0 == 0 && L.E1 % b1 == 0, SW_ERR_SHAPE,
                   "coarse lattice not divisible by the aggregate");
        SW_REQUIRE(b0 * b1 * L.nc / 2 <= 1024 && b0 * b1 * 5 <= 64, SW_ERR_SHAPE,
                   "coarse aggregate too large");
        C.E0 = L.E0 / b0;
        C.E1 = L.E1 / b1;
      }
      L.b0 = b0;
      L.b1 = b1;
      L.nv = nv;
      C.nc = 2 * nv;
      C.ndof = (long)C.E0 * C.E1 * C.nc;
    }
    mg_setup(mg, psi0, seed);
    return SW_OK;
  });
  if (rc != SW_OK) {
    sw_mg_release(mg);
    delete mg;
    return rc;
  }
  *out = mg;
  return SW_OK;
}

void sw_mg_free(sw_mg* mg) {
  if (!mg) return;
  cudaSetDevice(mg->ctx->device);
  if (mg->ctx->stream) cudaStreamSynchronize(mg->ctx->stream);
  sw_mg_release(mg);
  delete mg;
}

int sw_mg_solve(sw_mg* mg, const void* b, void* x, double tol, int on_device, sw_solve_stats* st) {
  if (!mg || !b || !x) return SW_ERR_ARG;
  sw_ctx* c = mg->ctx;
  return guarded(c, [&] {
    SW_REQUIRE(tol > 0.0 && std::isfinite(tol), SW_ERR_ARG, "tol must be > 0");
    auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = c->stream;
    size_t N = mg->g->N;
    const double2* db = (const double2*)b;
    double2* dx = (double2*)x;
    if (!on_device) {
      SW_CUDA(cudaMemcpyAsync(mg->lexb, b, N * sizeof(double2), cudaMemcpyHostToDevice, s));
      db = mg->lexb;
      dx = mg->lexx;
    }
    int rc = mg_solve_device(mg, db, dx, tol, st);
    if (!on_device)
      SW_CUDA(cudaMemcpyAsync(x, dx, N * sizeof(double2), cudaMemcpyDeviceToHost, s));
    SW_CUDA(cudaStreamSynchronize(s));
    if (st) st->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (rc == SW_ERR_NOCONV) c->err = "outer FGCR reached outer_maxiter";
    return rc;
  });
}

int sw_mg_solve_batch(sw_mg* mg, int nrhs, const void* B, void* X, double tol, int on_device,
                      sw_solve_stats* st) {
  if (!mg || !B || !X || nrhs < 0) return SW_ERR_ARG;
  size_t N = mg->g->N;
  if (!mg->mixed || mg->fine_D) {  // FP64 hierarchies: one solve after the other
    int worst = SW_OK;
    for (int k = 0; k < nrhs; ++k) {
      const double* b = (const double*)B + 2 * N * k;
      double* x = (double*)X + 2 * N * k;
      int rc = sw_mg_solve(mg, b, x, tol, on_device, st ? st + k : nullptr);
      if (rc != SW_OK && rc != SW_ERR_NOCONV) return rc;
      if (rc != SW_OK) worst = rc;
    }
    return worst;
  }
  sw_ctx* c = mg->ctx;
  return guarded(c, [&] {
    SW_REQUIRE(tol > 0.0 && std::isfinite(tol), SW_ERR_ARG, "tol must be > 0");
    cudaStream_t s = c->stream;
    int worst = SW_OK;
    ScopedBuffers scratch;  // host-side batches are staged through these
    double2 *db = nullptr, *dx = nullptr;
    if (!on_device) {
      db = scratch.get((long)N * kMaxBatch);
      dx = scratch.get((long)N * kMaxBatch);
    }
    for (int k0 = 0; k0 < nrhs; k0 += kMaxBatch) {
      int nb = std::min(kMaxBatch, nrhs - k0);
      const double2* bb = (const double2*)B + N * k0;
      double2* xx = (double2*)X + N * k0;
      if (!on_device) {
        SW_CUDA(cudaMemcpyAsync(db, bb, N * nb * sizeof(double2), cudaMemcpyHostToDevice, s));
        bb = db;
        xx = dx;
      }
      int rc = mg_solve_batch_device(mg, nb, bb, xx, tol, st ? st + k0 : nullptr);
      if (!on_device)
        SW_CUDA(cudaMemcpyAsync((double2*)X + N * k0, dx, N * nb * sizeof(double2),
                                cudaMemcpyDeviceToHost, s));
      SW_CUDA(cudaStreamSynchronize(s));
      if (rc != SW_OK) worst = rc;
    }
    if (worst == SW_ERR_NOCONV) c->err = "a right-hand side reached outer_maxiter";
    return worst;
  });
}

int sw_debug_maps(sw_gauge* g, int a0, int a1, int32_t* eta, int32_t* eps, int32_t* kd_block,
                  int32_t* kd_parity, int32_t* agg) {
  if (!g) return SW_ERR_ARG;
  int L0 = g->L0, L1 = g->L1, N = g->N;
  if (agg && (a0 < 1 || a1 < 1 || L0 % (2 * a0) || L1 % (2 * a1))) return SW_ERR_SHAPE;
  for (int s = 0; s < N; ++s) {
    int x0 = s % L0, x1 = s / L0;
    if (eta) {
      eta[s] = 1;
      eta[N + s] = (x0 & 1) ? -1 : 1;
    }
    if (eps) eps[s] = ((x0 + x1) & 1) ? -1 : 1;
    if (kd_block) kd_block[s] = (x0 >> 1) + (L0 >> 1) * (x1 >> 1);
    if (kd_parity) kd_parity[s] = ((x0 >> 1) + (x1 >> 1)) & 1;
    if (agg) agg[s] = x0 / (2 * a0) + (L0 / (2 * a0)) * (x1 / (2 * a1));
  }
  return SW_OK;
}

int sw_mg_level_info(sw_mg* mg, int level, int* E0, int* E1, int* nc) {
  if (!mg || level < 1 || level > mg->nlev) return SW_ERR_ARG;
  const MgLevel& L = mg->lev[level - 1];
  if (E0) *E0 = L.E0;
  if (E1) *E1 = L.E1;
  if (nc) *nc = L.nc;
  return SW_OK;
}

int sw_mg_level_maps(sw_mg* mg, int level, int32_t* agg, int32_t* chir) {
  if (!mg || !agg || !chir || level < 1 || level >= mg->nlev) return SW_ERR_ARG;
  return guarded(mg->ctx, [&] {
    const MgLevel& L = mg->lev[level - 1];
    const long n = level == 1 ? (long)mg->g->N : L.ndof;
    cudaStream_t s = mg->ctx->stream;
    ScopedBuffers scratch;
    int* d = (int*)scratch.get((2 * n + 3) / 4);
    if (level == 1)
      launch_level_maps_fine(mg->g, L.b0, L.b1, d, d + n, s);
    else
      launch_level_maps_coarse(CoarseGeom{L.E0, L.E1, L.nc}, L.b0, L.b1, d, d + n, s);
    SW_CUDA(cudaMemcpyAsync(agg, d, n * sizeof(int), cudaMemcpyDeviceToHost, s));
    SW_CUDA(cudaMemcpyAsync(chir, d + n, n * sizeof(int), cudaMemcpyDeviceToHost, s));
    SW_CUDA(cudaStreamSynchronize(s));
    return SW_OK;
  });
}

int sw_mg_export_P(sw_mg* mg, int level, double* P) {
  if (!mg || !P || level < 1 || level >= mg->nlev) return SW_ERR_ARG;
  return guarded(mg->ctx, [&] {
    const MgLevel& L = mg->lev[level - 1];
    std::vector<double2> h((size_t)L.ndof * L.nv);
    SW_CUDA(cudaStreamSynchronize(mg->ctx->stream));
    SW_CUDA(cudaMemcpy(h.data(), L.P, h.size() * sizeof(double2), cudaMemcpyDeviceToHost));
    double2* o = (double2*)P;
    if (level == 1) {
      int L0 = mg->g->L0, N = mg->g->N;
      for (int s = 0; s < N; ++s) {
        int f = ps_index(s % L0, s / L0, L0, N);
        std::memcpy(o + (size_t)s * L.nv, h.data() + (size_t)f * L.nv, L.nv * sizeof(double2));
      }
    } else {
      std::memcpy(o, h.data(), h.size() * sizeof(double2));
    }
    return SW_OK;
  });
}

int sw_mg_export_Y(sw_mg* mg, int level, double* Y) {
  if (!mg || !Y || level < 2 || level > mg->nlev) return SW_ERR_ARG;
  return guarded(mg->ctx, [&] {
    const MgLevel& L = mg->lev[level - 1];
    size_t nb = (size_t)L.E0 * L.E1 * 5;
    size_t nc = L.nc;
    std::vector<double2> h(nb * nc * nc);
    SW_CUDA(cudaStreamSynchronize(mg->ctx->stream));
    SW_CUDA(cudaMemcpy(h.data(), L.Y, h.size() * sizeof(double2), cudaMemcpyDeviceToHost));
    double2* o = (double2*)Y;
    for (size_t b = 0; b < nb; ++b)
      for (size_t i = 0; i < nc; ++i)
        for (size_t j = 0; j < nc; ++j) o[(b * nc + i) * nc + j] = h[(b * nc + j) * nc + i];
    return SW_OK;
  });
}

int sw_mg_apply_level(sw_mg* mg, int level, int precision, int dagger, const void* in, void* out,
                      int on_device) {
  if (!mg || !in || !out || level < 1 || level > mg->nlev) return SW_ERR_ARG;
  return guarded(mg->ctx, [&] {
    const MgLevel& L = mg->lev[level - 1];
    cudaStream_t s = mg->ctx->stream;
    sw_gauge* g = mg->g;
    size_t n = level == 1 ? (size_t)g->N : (size_t)L.ndof;
    ScopedBuffers scratch;
    double2* a = scratch.get(n);
    double2* b = scratch.get(n);
    double2* t = scratch.get(n);
    SW_CUDA(cudaMemcpyAsync(a, in, n * sizeof(double2),
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    if (level == 1) {
      SW_REQUIRE(!dagger, SW_ERR_ARG, "level 1 has no adjoint here");
      SW_REQUIRE(precision == SW_PREC_FP64 || (precision == SW_PREC_FP32 && mg->mixed), SW_ERR_ARG,
                 "level 1: FP64, or FP32 on a mixed-precision hierarchy");
      launch_pack(g, a, t, s);
      SW_CUDA(cudaMemsetAsync(a, 0, n * sizeof(double2), s));
      if (mg->fine_D)
        launch_dslash_ps(g, mg->mass, 0, t, a, s);
      else if (precision == SW_PREC_FP64)
        fine_apply_S(g, mg->binv, t, a, b, s);
      else
        fine_apply_S32(g, g->W_ps32, mg->binv32, t, a, mg->s32tmp, s);
      launch_unpack(g, a, b, s);
    } else {
      CoarseGeom cg{L.E0, L.E1, L.nc};
      // timed like the solver's applications (category level - 1), kernel only
      const int tk = timing_begin(mg->ctx, level - 1);
      if (precision == SW_PREC_FP64) {
        launch_coarse_apply(cg, L.Y, dagger ? 1 : 0, a, b, s);
      } else if (precision == SW_PREC_FP16S) {
        SW_REQUIRE(L.Yh, SW_ERR_ARG, "no scaled-FP16 stencil on this level");
        launch_coarse_apply_h(cg, L.Yh, L.Ysc, dagger ? 1 : 0, a, b, s);
      } else if (precision == SW_PREC_DF64) {
        SW_REQUIRE(L.Ydf, SW_ERR_ARG, "no double-float stencil on this level");
        launch_coarse_apply_df(cg, L.Ydf, dagger ? 1 : 0, a, b, s);
      } else {
        throw SwError{SW_ERR_ARG, "unknown precision"};
      }
      timing_end(mg->ctx, tk);
    }
    SW_CUDA(cudaMemcpyAsync(out, b, n * sizeof(double2),
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    SW_CUDA(cudaStreamSynchronize(s));
    return SW_OK;
  });
}

int sw_mg_transfer(sw_mg* mg, int level, int dir, const void* in, void* out, int on_device) {
  if (!mg || !in || !out || level < 1 || level >= mg->nlev || (dir != 0 && dir != 1))
    return SW_ERR_ARG;
  return guarded(mg->ctx, [&] {
    const MgLevel& L = mg->lev[level - 1];
    const MgLevel& C = mg->lev[level];
    cudaStream_t s = mg->ctx->stream;
    sw_gauge* g = mg->g;
    size_t nf = L.ndof, nc = C.ndof;
    size_t nin = dir == 0 ? nf : nc, nout = dir == 0 ? nc : nf;
    ScopedBuffers scratch;
    double2* a = scratch.get(nin);
    double2* b = scratch.get(nout);
    double2* t = scratch.get(nf);
    SW_CUDA(cudaMemcpyAsync(a, in, nin * sizeof(double2),
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    if (level == 1) {
      if (dir == 0) {
        launch_pack(g, a, t, s);
        launch_restrict_fine(g, L.b0, L.b1, L.nv, L.P, t, b, s, mg->fine_D ? 1 : 0);
      } else {
        SW_CUDA(cudaMemsetAsync(t, 0, nf * sizeof(double2), s));
        launch_prolong_fine(g, L.b0, L.b1, L.nv, L.P, a, t, s, mg->fine_D ? 1 : 0);
        launch_unpack(g, t, b, s);
      }
    } else {
      CoarseGeom cg{L.E0, L.E1, L.nc};
      if (dir == 0)
        launch_restrict_coarse(cg, L.b0, L.b1, L.nv, L.P, a, b, s);
      else
        launch_prolong_coarse(cg, L.b0, L.b1, L.nv, L.P, a, b, s);
    }
    SW_CUDA(cudaMemcpyAsync(out, b, nout * sizeof(double2),
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    SW_CUDA(cudaStreamSynchronize(s));
    return SW_OK;
  });
}

int sw_debug_cgne_stall(sw_mg* mg) {
  if (!mg) return SW_ERR_ARG;
  return guarded(mg->ctx, [&] {
    const MgLevel& L = mg->lev[mg->nlev - 1];
    SW_REQUIRE(mg->persistent_cgne, SW_ERR_ARG, "the persistent CGNE is disabled");
    SW_CUDA(cudaMemsetAsync(L.rhs, 0, L.ndof * sizeof(double2), mg->ctx->stream));
    mg->stall_test = 1;
    int rc = SW_OK;
    try {
      mg_coarsest_solve(mg, L.rhs, L.sol);
    } catch (const SwError& e) {
      mg->stall_test = 0;
      throw;
    }
    mg->stall_test = 0;
    return rc;
  });
}

int sw_context_set_sm_share(sw_ctx* ctx, int num, int den) {
  if (!ctx || num < 1 || den < 1 || num > den) return SW_ERR_ARG;
  ctx->sm_num = num;
  ctx->sm_den = den;
  return SW_OK;
}

int sw_debug_batch_stall(sw_mg* mg, int nrhs) {
  if (!mg) return SW_ERR_ARG;
  return guarded(mg->ctx, [&] { return mg_batch_stall(mg, nrhs); });
}

int sw_autotune_entries(int max, int* nc, int* K, int* sites, int* stages, double* us) {
  try {
    return mg_autotune_entries(max, nc, K, sites, stages, us);
  } catch (...) {
    return SW_ERR_ARG;
  }
}

}  // extern "C"
