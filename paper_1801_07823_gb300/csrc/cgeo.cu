// CG on the even/odd (checkerboard) normal system of the staggered operator,
// the paper's comparison solver (Sec. II, Eq. normal; Sec. IV, Fig. iterworst):
//   [m D_eo; D_oe m] [x_e; x_o] = [b_e; b_o]  ->
//   (m^2 - D_eo D_oe) x_e = m b_e - D_eo b_o,  x_o = (b_o - D_oe x_e) / m,
// with even/odd the site parity eps(x) = (-1)^(x0 + x1).  m^2 - D_eo D_oe is
// Hermitian positive definite (D_oe = -D_eo^dag).  The full residual is
// b - D x = ((m b_e - D_eo b_o) - (m^2 - D_eo D_oe) x_e) / m on even sites
// and 0 on odd ones, so CG stops when its residual is below m tol ||b||.
//
// Layout: half-lattice vectors, site (x0, x1) of parity p at (x1 L0 + x0) / 2.
#include <chrono>
#include <cmath>
#include <cstring>

#include "sw_internal.h"

namespace {

__device__ __forceinline__ void cfma(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}

// out_p(s) = a src_p(s) + c * sum_mu [W_mu(s) in(s+mu) - conj(W_mu(s-mu)) in(s-mu)]
// for the sites s of parity p; in is the opposite-parity half.  One thread per
// site, 2D grid over (x0 / 2, x1) so each row's threads read consecutive
// addresses.
__global__ void k_hop_eo(const double2* __restrict__ W, int par, double a, const double2* src,
                         double c, const double2* __restrict__ in, double2* __restrict__ out,
                         int L0, int L1) {
  int hx = blockIdx.x * blockDim.x + threadIdx.x;
  int x1 = blockIdx.y;
  if (hx >= L0 / 2) return;
  int x0 = 2 * hx + ((x1 + par) & 1);
  long N = (long)L0 * L1;
  long s = (long)x1 * L0 + x0;
  int xp0 = x0 + 1 == L0 ? 0 : x0 + 1, xm0 = x0 == 0 ? L0 - 1 : x0 - 1;
  int xp1 = x1 + 1 == L1 ? 0 : x1 + 1, xm1 = x1 == 0 ? L1 - 1 : x1 - 1;
  long sp0 = (long)x1 * L0 + xp0, sm0 = (long)x1 * L0 + xm0;
  long sp1 = (long)xp1 * L0 + x0, sm1 = (long)xm1 * L0 + x0;
  double2 h = make_double2(0.0, 0.0);
  cfma(h, W[s], in[sp0 >> 1]);
  cfma(h, W[N + s], in[sp1 >> 1]);
  double2 w = W[sm0], v = in[sm0 >> 1];
  h.x -= w.x * v.x + w.y * v.y;
  h.y -= w.x * v.y - w.y * v.x;
  w = W[N + sm1];
  v = in[sm1 >> 1];
  h.x -= w.x * v.x + w.y * v.y;
  h.y -= w.x * v.y - w.y * v.x;
  double2 o = src ? src[s >> 1] : make_double2(0.0, 0.0);
  o.x = fma(c, h.x, a * o.x);
  o.y = fma(c, h.y, a * o.y);
  out[s >> 1] = o;
}

// lexicographic <-> checkerboard halves
__global__ void k_split_eo(const double2* __restrict__ lex, double2* __restrict__ e,
                           double2* __restrict__ o, int L0, int L1) {
  long s = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= (long)L0 * L1) return;
  int x0 = (int)(s % L0), x1 = (int)(s / L0);
  (((x0 + x1) & 1) ? o : e)[s >> 1] = lex[s];
}
__global__ void k_join_eo(const double2* __restrict__ e, const double2* __restrict__ o,
                          double2* __restrict__ lex, int L0, int L1) {
  long s = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= (long)L0 * L1) return;
  int x0 = (int)(s % L0), x1 = (int)(s / L0);
  lex[s] = (((x0 + x1) & 1) ? o : e)[s >> 1];
}

void hop_eo(const sw_gauge* g, int par, double a, const double2* src, double c, const double2* in,
            double2* out, cudaStream_t s) {
  dim3 grid((g->L0 / 2 + 127) / 128, g->L1);
  k_hop_eo<<<grid, 128, 0, s>>>(g->W_lex, par, a, src, c, in, out, g->L0, g->L1);
  SW_LAUNCH_CHECK();
}

}  // namespace

// Solves D x = b by CG on the even normal system; b, x lexicographic device
// buffers.  work: 7 half vectors + 1 full.  Returns iterations (negative on
// non-convergence) and fills the true residual.
int cg_eo_device(sw_gauge* g, double m, const double2* b, double2* x, double tol, int maxit,
                 double2* work, int* iters, double* true_resid) {
  sw_ctx* c = g->ctx;
  cudaStream_t s = c->stream;
  long N = g->N, h = N / 2;
  double2 *be = work, *bo = work + h, *xe = work + 2 * h, *r = work + 3 * h, *p = work + 4 * h,
          *q = work + 5 * h, *t = work + 6 * h, *full = work + 7 * h;
  int blocks = (int)((N + 255) / 256);
  k_split_eo<<<blocks, 256, 0, s>>>(b, be, bo, g->L0, g->L1);
  SW_LAUNCH_CHECK();
  int sb = 256;  // slots of this solver (above the multigrid levels' 4 x 64)
  blas_norm2(c, b, N, sb + 0);
  double bn = std::sqrt(slot_read(c, sb + 0).x);
  if (!std::isfinite(bn)) throw SwError{SW_ERR_NAN, "non-finite right-hand side"};
  // rhs = m b_e - D_eo b_o (in place of b_e), x_e = 0
  hop_eo(g, 0, m, be, -1.0, bo, be, s);
  blas_zero(c, xe, h);
  double stop = bn > 0.0 ? tol * m * bn : 0.0;
  int* ctl = c->ctl + 4 * 7;
  int total = 0;
  // CG with reliable restarts: when the recurrence residual meets the target,
  // the true residual rhs - M x_e is recomputed; if it is still above the
  // target (recurrence drift at small m), CG restarts from it.
  for (int attempt = 0; attempt < 8 && bn > 0.0 && total < maxit; ++attempt) {
    hop_eo(g, 1, 0.0, nullptr, 1.0, xe, t, s);
    hop_eo(g, 0, m * m, xe, -1.0, t, q, s);
    blas_sub(c, r, be, q, h);
    blas_copy(c, p, r, h);
    blas_norm2(c, r, h, sb + 1);
    double rr0 = slot_read(c, sb + 1).x;
    if (!std::isfinite(rr0)) throw SwError{SW_ERR_NAN, "non-finite CG residual"};
    if (std::sqrt(rr0) <= stop) break;
    int budget = maxit - total;
    iter_init(c, ctl, sb + 1, stop, budget);
    int cur = 0, s_rr[2] = {sb + 1, sb + 2}, s_pq = sb + 3;
    for (int issued = 0;;) {
      for (int qq = 0; qq < 8 && issued < budget; ++qq, ++issued) {
        // q = (m^2 - D_eo D_oe) p
        hop_eo(g, 1, 0.0, nullptr, 1.0, p, t, s);      // t_o = D_oe p
        hop_eo(g, 0, m * m, p, -1.0, t, q, s);          // q = m^2 p - D_eo t
        blas_dot(c, p, q, h, s_pq, ctl);
        blas_axpy(c, xe, p, h, coef_ratio(s_rr[cur], s_pq, 1.0), ctl);
        blas_axpy(c, r, q, h, coef_ratio(s_rr[cur], s_pq, -1.0), ctl);
        blas_norm2(c, r, h, s_rr[1 - cur], ctl);
        iter_check(c, ctl, s_rr[1 - cur], stop, budget);
        blas_xpay(c, p, r, h, coef_ratio(s_rr[1 - cur], s_rr[cur], 1.0), ctl);
        cur = 1 - cur;
      }
      iter_read(c, ctl, c->h_ctl);
      if (c->h_ctl[2]) throw SwError{SW_ERR_NAN, "non-finite CG residual"};
      if (c->h_ctl[0] || issued >= budget) break;
    }
    total += c->h_ctl[1];
  }
  *iters = total;
  // x_o = (b_o - D_oe x_e) / m
  hop_eo(g, 1, 1.0 / m, bo, -1.0 / m, xe, t, s);
  k_join_eo<<<blocks, 256, 0, s>>>(xe, t, x, g->L0, g->L1);
  SW_LAUNCH_CHECK();
  launch_dslash_lex(g, m, 0, x, full, s);
  blas_sub(c, full, b, full, N);
  blas_norm2(c, full, N, sb + 4);
  double rn = std::sqrt(slot_read(c, sb + 4).x);
  *true_resid = bn > 0.0 ? rn / bn : 0.0;
  return (bn == 0.0 || *true_resid <= tol) ? SW_OK : SW_ERR_NOCONV;
}

extern "C" int sw_cg_eo_solve(sw_gauge* g, double mass, const void* b, void* x, double tol,
                              int maxiter, int on_device, sw_solve_stats* st) {
  if (!g || !b || !x) return SW_ERR_ARG;
  sw_ctx* c = g->ctx;
  try {
    c->err.clear();
    SW_CUDA(cudaSetDevice(c->device));
    cudaError_t stale = cudaGetLastError();
    if (stale != cudaSuccess) report_stale_error(stale);
    SW_REQUIRE(std::isfinite(mass) && mass > 0.0, SW_ERR_ARG, "mass must be > 0");
    SW_REQUIRE(tol > 0.0 && maxiter >= 0, SW_ERR_ARG, "tol must be > 0, maxiter >= 0");
    auto t0 = std::chrono::steady_clock::now();
    long N = g->N;
    double2* work = nullptr;
    cudaError_t e = cudaMalloc(&work, (size_t)(7 * (N / 2) + N + 2 * N) * sizeof(double2));
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw SwError{SW_ERR_OOM, "CG work buffers"};
    }
    double2* db = work + 7 * (N / 2) + N;
    double2* dx = db + N;
    int iters = 0, rc = SW_OK;
    double tr = 0.0;
    try {
      if (!on_device)
        SW_CUDA(cudaMemcpyAsync(db, b, N * sizeof(double2), cudaMemcpyHostToDevice, c->stream));
      rc = cg_eo_device(g, mass, on_device ? (const double2*)b : db,
                        on_device ? (double2*)x : dx, tol, maxiter, work, &iters, &tr);
      if (!on_device)
        SW_CUDA(cudaMemcpyAsync(x, dx, N * sizeof(double2), cudaMemcpyDeviceToHost, c->stream));
      SW_CUDA(cudaStreamSynchronize(c->stream));
    } catch (...) {
      dev_free(work, "CG work");
      throw;
    }
    dev_free(work, "CG work");
    if (st) {
      std::memset(st, 0, sizeof(*st));
      st->converged = rc == SW_OK;
      st->outer_iters = iters;
      st->fine_applies = iters + 1;
      st->true_resid = tr;
      st->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    if (rc != SW_OK) c->err = "CG reached maxiter";
    return rc;
  } catch (const SwError& err) {
    c->err = err.msg;
    return err.code;
  }
}
