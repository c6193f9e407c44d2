// Coarse-level kernels: the Galerkin coarse operator as a nearest-neighbour
// stencil of dense nc x nc blocks (Sec. III: A_hat = R A P with R = P^dag),
// restriction and prolongation through the block-orthonormal near-null
// vectors (Sec. III.A, III.C, Sec. IV), the Galerkin builds and the block
// orthonormalisation of the chirally doubled vectors.
//
// Stencil storage: Y[X][d] for directions d = 0 (self), 1 (+0hat), 2 (-0hat),
// 3 (+1hat), 4 (-1hat), each block column-major, element (row i, col j) at
// ((X * 5 + d) * nc + j) * nc + i.  (A_hat x)_X = sum_d Y[X][d] x_{X+d}, and
// the adjoint (A_hat^dag x)_X = sum_d Y[X+d][opp d]^dag x_{X+d} reads the same
// storage transposed.
// Direction d collects the couplings carried by fine hops that leave the
// aggregate in direction d, so the stencil is exact for any coarse extent,
// including 1 and 2 where X + 0hat and X - 0hat coincide.
#include "sw_internal.h"

namespace {

__device__ __forceinline__ void cfma(double2& acc, double2 a, double2 b) {  // acc += a b
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
__device__ __forceinline__ void cfmac(double2& acc, double2 a, double2 b) {  // acc += conj(a) b
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}
__host__ __device__ __forceinline__ int nbr_site(int X, int d, int E0, int E1) {
  int X0 = X % E0, X1 = X / E0;
  switch (d) {
    case 1: X0 = (X0 + 1 == E0) ? 0 : X0 + 1; break;
    case 2: X0 = (X0 == 0) ? E0 - 1 : X0 - 1; break;
    case 3: X1 = (X1 + 1 == E1) ? 0 : X1 + 1; break;
    case 4: X1 = (X1 == 0) ? E1 - 1 : X1 - 1; break;
    default: break;
  }
  return X0 + E0 * X1;
}
__host__ __device__ __forceinline__ int opp_dir(int d) {
  return d == 0 ? 0 : (d == 1 ? 2 : (d == 2 ? 1 : (d == 3 ? 4 : 3)));
}
inline int cdiv(long a, long b) { return (int)((a + b - 1) / b); }

// ---------------------------------------------------------------------------
// y_X = sum_d Y[X][d] x_{X+d}, generic nc.  A CTA holds spc sites x nc rows,
// one thread per output row; the five neighbour vectors of its sites are
// staged in shared memory and every Y load is a coalesced column segment.
__global__ void k_coarse_apply(const double2* __restrict__ Y, const double2* __restrict__ in,
                               double2* __restrict__ out, int E0, int E1, int nc, int spc,
                               int dagger, const int* __restrict__ skip,
                               unsigned long long* exec) {
  extern __shared__ double2 xs[];  // [spc][5][nc]
  if (skip && *skip) return;
  if (exec && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(exec, 1ull);
  int nsites = E0 * E1;
  int site0 = blockIdx.x * spc;
  int nstage = spc * 5 * nc;
  for (int t = threadIdx.x; t < nstage; t += blockDim.x) {
    int ls = t / (5 * nc);
    int r = t - ls * 5 * nc;
    int d = r / nc, j = r - d * nc;
    int X = site0 + ls;
    if (X < nsites) xs[t] = in[(long)nbr_site(X, d, E0, E1) * nc + j];
  }
  __syncthreads();
  int ls = threadIdx.x / nc, i = threadIdx.x - ls * nc;
  int X = site0 + ls;
  if (ls >= spc || X >= nsites) return;
  const double2* xv = xs + ls * 5 * nc;
  double2 acc = make_double2(0.0, 0.0);
  if (!dagger) {
    const double2* y = Y + (long)X * 5 * nc * nc + i;
    for (int dj = 0; dj < 5 * nc; ++dj) cfma(acc, __ldg(y + (long)dj * nc), xv[dj]);
  } else {
    for (int d = 0; d < 5; ++d) {
      const double2* y = Y + (((long)nbr_site(X, d, E0, E1) * 5 + opp_dir(d)) * nc + i) * nc;
      for (int j = 0; j < nc; ++j) cfmac(acc, __ldg(y + j), xv[d * nc + j]);
    }
  }
  out[(long)X * nc + i] = acc;
}

// Same product for a compile-time nc.  The work of one site is split over
// threads (d, i) -- direction d of the stencil, output row i -- and, when
// there are few sites, over rs CTAs that each take nc / rs rows, so that the
// grid fills all SMs.  Each thread streams one column-major block row of
// Y[X][d] (coalesced across i), unrolled so that many loads are in flight:
// in FP64 the kernel is bound by the FP64 pipe, which needs every SM busy.
// The five partial sums are added in direction order (deterministic).
template <int NC, bool DAG>
__global__ void __launch_bounds__(5 * NC) k_coarse_apply_nc(const double2* __restrict__ Y,
                                                            const double2* __restrict__ in,
                                                            double2* __restrict__ out, int E0,
                                                            int E1, int rs,
                                                            const int* __restrict__ skip,
                                                            unsigned long long* exec) {
  if (skip && *skip) return;
  if (exec && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(exec, 1ull);
  __shared__ double2 xs[5][NC];
  __shared__ double2 part[5][NC];
  int rows = NC / rs;
  int X = blockIdx.x / rs;
  int r0 = (blockIdx.x - X * rs) * rows;
  int nthr = 5 * rows;
  for (int t = threadIdx.x; t < 5 * NC; t += nthr) {
    int d = t / NC, j = t - d * NC;
    xs[d][j] = in[(long)nbr_site(X, d, E0, E1) * NC + j];
  }
  __syncthreads();
  int d = threadIdx.x / rows;
  int i = r0 + threadIdx.x - d * rows;
  double2 acc = make_double2(0.0, 0.0);
  if (!DAG) {
    const double2* y = Y + ((long)X * 5 + d) * NC * NC + i;
#pragma unroll 16
    for (int j = 0; j < NC; ++j) cfma(acc, __ldg(y + j * NC), xs[d][j]);
  } else {
    // (A^dag)(X, X+d) = Y[X+d][opp d]^dag: row i of it is column i of that
    // block, contiguous in memory (each thread streams its own column; the
    // warp's lines are reused from L1 over consecutive j)
    const double2* y = Y + (((long)nbr_site(X, d, E0, E1) * 5 + opp_dir(d)) * NC + i) * NC;
#pragma unroll 16
    for (int j = 0; j < NC; ++j) cfmac(acc, __ldg(y + j), xs[d][j]);
  }
  part[d][i] = acc;
  __syncthreads();
  if (d == 0) {
    double2 s = part[0][i];
#pragma unroll
    for (int q = 1; q < 5; ++q) {
      s.x += part[q][i].x;
      s.y += part[q][i].y;
    }
    out[(long)X * NC + i] = s;
  }
}

// ---------------------------------------------------------------------------
// Level-1 transfer, even parity half only (Sec. IV: coarsen with the odd
// contributions set to zero, keep the even part of the prolonged error).
// Chirality eps of site k of a KD block: + for k = 0, 3 and - for k = 1, 2.
// full = 1: r is a full parity-split vector and every KD block of the
// aggregate contributes (used when the fine operator is D itself).
__global__ void k_restrict_fine(const double2* __restrict__ P, const double2* __restrict__ r_e,
                                double2* __restrict__ out, int L0, int L1, int a0, int a1, int nv,
                                int full) {
  int A = blockIdx.x;
  int E0 = L0 / (2 * a0);
  int A0 = A % E0, A1 = A / E0;
  int t = threadIdx.x;
  if (t >= 2 * nv) return;
  int c = t / nv, i = t - c * nv;
  int ka = c ? 1 : 0, kb = c ? 2 : 3;
  double2 acc = make_double2(0.0, 0.0);
  const int N = L0 * L1;
  for (int by = 0; by < a1; ++by)
    for (int bx = 0; bx < a0; ++bx) {
      int X0 = A0 * a0 + bx, X1 = A1 * a1 + by;
      if (((X0 + X1) & 1) && !full) continue;
      // the two sites k = ka, kb of KD block (X0, X1), parity-split positions
      int ha = ps_index(2 * X0 + (ka & 1), 2 * X1 + (ka >> 1), L0, N);
      int hc = ps_index(2 * X0 + (kb & 1), 2 * X1 + (kb >> 1), L0, N);
      cfmac(acc, P[(long)ha * nv + i], r_e[ha]);
      cfmac(acc, P[(long)hc * nv + i], r_e[hc]);
    }
  out[(long)A * 2 * nv + t] = acc;
}

// Aggregate A and chirality half c (0: eps = +1, 1: eps = -1) of the fine dof
// at parity-split position h (level-1 aggregates of a0 x a1 KD blocks).
__device__ __forceinline__ void fine_dof_map(int h, int L0, int L1, int a0, int a1, int& A,
                                             int& c) {
  int x0, x1;
  ps_coords(h, L0, L0 * L1, x0, x1);
  const int E0 = L0 / (2 * a0);
  A = x0 / (2 * a0) + E0 * (x1 / (2 * a1));
  const int k = (x0 & 1) | ((x1 & 1) << 1);
  c = (k == 1 || k == 2);
}
// Aggregate A and chirality half c (0: sigma3 = +1, 1: sigma3 = -1) of dof
// X nc + k of a coarse level (aggregates of b0 x b1 coarse sites).
__device__ __forceinline__ void coarse_dof_map(long dof, int E0, int nc, int b0, int b1, int& A,
                                               int& c) {
  const int X = (int)(dof / nc), k = (int)(dof - (long)X * nc);
  const int X0 = X % E0, X1 = X / E0;
  A = X0 / b0 + (E0 / b0) * (X1 / b1);
  c = k >= nc / 2;
}

__global__ void k_prolong_fine(const double2* __restrict__ P, const double2* __restrict__ ehat,
                               double2* __restrict__ e_e, int L0, int L1, int a0, int a1, int nv,
                               int full) {
  int N = L0 * L1;
  int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= (full ? N : N / 2)) return;
  int A, c;
  fine_dof_map(h, L0, L1, a0, a1, A, c);
  const double2* p = P + (long)h * nv;
  const double2* eh = ehat + (long)A * 2 * nv + c * nv;
  double2 acc = make_double2(0.0, 0.0);
  for (int i = 0; i < nv; ++i) cfma(acc, p[i], eh[i]);
  e_e[h] = acc;
}

// Aggregate and chirality (+1 / -1) of every dof of a level, from the index
// maps of the prolongation kernels (test export): level 1 in lexicographic
// site order, coarser levels in dof order X nc + k.
__global__ void k_level_maps_fine(int* __restrict__ agg, int* __restrict__ chir, int L0, int L1,
                                  int a0, int a1) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= L0 * L1) return;
  int A, c;
  fine_dof_map(ps_index(s % L0, s / L0, L0, L0 * L1), L0, L1, a0, a1, A, c);
  agg[s] = A;
  chir[s] = c ? -1 : 1;
}
__global__ void k_level_maps_coarse(int* __restrict__ agg, int* __restrict__ chir, int E0, int E1,
                                    int nc, int b0, int b1) {
  long dof = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (dof >= (long)E0 * E1 * nc) return;
  int A, c;
  coarse_dof_map(dof, E0, nc, b0, b1, A, c);
  agg[dof] = A;
  chir[dof] = c ? -1 : 1;
}

// Level >= 2 transfer: chirality sigma3 = + for k < nc/2, - otherwise.
__global__ void k_restrict_coarse(const double2* __restrict__ P, const double2* __restrict__ r,
                                  double2* __restrict__ out, int E0, int b0, int b1, int nc,
                                  int nv) {
  int A = blockIdx.x;
  int F0 = E0 / b0;
  int A0 = A % F0, A1 = A / F0;
  int t = threadIdx.x;
  if (t >= 2 * nv) return;
  int c = t / nv, i = t - c * nv;
  int hn = nc / 2;
  double2 acc = make_double2(0.0, 0.0);
  for (int y = 0; y < b1; ++y)
    for (int x = 0; x < b0; ++x) {
      int X = (A0 * b0 + x) + E0 * (A1 * b1 + y);
      for (int k = c * hn; k < (c + 1) * hn; ++k) {
        long dof = (long)X * nc + k;
        cfmac(acc, P[dof * nv + i], r[dof]);
      }
    }
  out[(long)A * 2 * nv + t] = acc;
}

__global__ void k_prolong_coarse(const double2* __restrict__ P, const double2* __restrict__ ehat,
                                 double2* __restrict__ e, int E0, int E1, int b0, int b1, int nc,
                                 int nv) {
  long dof = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (dof >= (long)E0 * E1 * nc) return;
  int A, c;
  coarse_dof_map(dof, E0, nc, b0, b1, A, c);
  const double2* p = P + dof * nv;
  const double2* eh = ehat + (long)A * 2 * nv + c * nv;
  double2 acc = make_double2(0.0, 0.0);
  for (int i = 0; i < nv; ++i) cfma(acc, p[i], eh[i]);
  e[dof] = acc;
}

// ---------------------------------------------------------------------------
// Level-1 Galerkin build.  A P = D (B^-1 P); Wv = B^-1 P is local to the KD
// block:  Wv[f][c][i] = sum over the block sites t of chirality c of
// B^-1[f][t] P[t][i].
__global__ void k_build_W(const double2* __restrict__ binv, const double2* __restrict__ P,
                          double2* __restrict__ Wv, int N, int nv) {
  long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long)N * nv) return;
  int f = (int)(e / nv), i = (int)(e - (long)f * nv);
  int b = f >> 2, k = f & 3;
  const double2* m = binv + 16 * (long)b + 4 * k;
  double2 w0 = make_double2(0.0, 0.0), w1 = make_double2(0.0, 0.0);
  cfma(w0, m[0], P[(long)(4 * b + 0) * nv + i]);
  cfma(w0, m[3], P[(long)(4 * b + 3) * nv + i]);
  cfma(w1, m[1], P[(long)(4 * b + 1) * nv + i]);
  cfma(w1, m[2], P[(long)(4 * b + 2) * nv + i]);
  Wv[((long)f * 2 + 0) * nv + i] = w0;
  Wv[((long)f * 2 + 1) * nv + i] = w1;
}

// Wv from P alone (no B^-1): Wv[f][c][i] = P[f][i] if chirality(f) = c, else 0
// -- the Galerkin build of D itself.
__global__ void k_build_W_identity(const double2* __restrict__ P, double2* __restrict__ Wv, int N,
                                   int nv) {
  long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long)N * nv) return;
  int f = (int)(e / nv), i = (int)(e - (long)f * nv);
  int k = f & 3;
  int c = (k == 1 || k == 2);
  double2 z = make_double2(0.0, 0.0), v = P[e];
  Wv[((long)f * 2 + 0) * nv + i] = c == 0 ? v : z;
  Wv[((long)f * 2 + 1) * nv + i] = c == 1 ? v : z;
}

struct HopTerm {
  int fs, ft;    // parity-split indices of the row site s and column site t
  int cs;        // chirality of s (0: eps = +1, 1: eps = -1)
  int pad;
  double2 coef;  // D(s, t)
};

// Y[A][d](row (cr, i), col (c, j)) = sum over the terms (s, t, D(s,t)) of
// direction d with chirality(s) = cr of conj(P[s][i]) D(s,t) Wv[t][c][j].
// Terms: the mass at every site (d = 0) and the four hops of Eq. staggeredD;
// a hop's direction is the aggregate boundary it crosses (0 if none).
__global__ void k_build_Y_fine(const double2* __restrict__ Wg, const double2* __restrict__ P,
                               const double2* __restrict__ Wv, double2* __restrict__ Y, double mass,
                               int L0, int L1, int a0, int a1, int nv) {
  extern __shared__ HopTerm terms[];
  __shared__ int nterms;
  int N = L0 * L1;
  int E0 = L0 / (2 * a0);
  int A = blockIdx.x / 5, d = blockIdx.x % 5;
  int A0 = A % E0, A1 = A / E0;
  if (threadIdx.x == 0) {
    int n = 0;
    for (int y = 0; y < 2 * a1; ++y)
      for (int x = 0; x < 2 * a0; ++x) {
        int x0 = A0 * 2 * a0 + x, x1 = A1 * 2 * a1 + y;
        int fs = ps_index(x0, x1, L0, N);
        int cs = ((x0 + x1) & 1);
        if (d == 0) terms[n++] = HopTerm{fs, fs, cs, 0, make_double2(mass, 0.0)};
        for (int mu = 0; mu < 2; ++mu) {
          int xm = mu == 0 ? x : y;
          int am = mu == 0 ? a0 : a1;
          // forward hop s -> s + mu, coefficient W_mu(s)
          int tf0 = mu == 0 ? (x0 + 1 == L0 ? 0 : x0 + 1) : x0;
          int tf1 = mu == 0 ? x1 : (x1 + 1 == L1 ? 0 : x1 + 1);
          int typ = (xm == 2 * am - 1) ? (mu == 0 ? 1 : 3) : 0;
          if (typ == d) terms[n++] = HopTerm{fs, ps_index(tf0, tf1, L0, N), cs, 0, Wg[(long)mu * N + fs]};
          // backward hop s -> s - mu, coefficient -conj(W_mu(s - mu))
          int tb0 = mu == 0 ? (x0 == 0 ? L0 - 1 : x0 - 1) : x0;
          int tb1 = mu == 0 ? x1 : (x1 == 0 ? L1 - 1 : x1 - 1);
          typ = (xm == 0) ? (mu == 0 ? 2 : 4) : 0;
          if (typ == d) {
            int ft = ps_index(tb0, tb1, L0, N);
            double2 w = Wg[(long)mu * N + ft];
            terms[n++] = HopTerm{fs, ft, cs, 0, make_double2(-w.x, w.y)};
          }
        }
      }
    nterms = n;
  }
  __syncthreads();
  int nc = 2 * nv;
  int nt = nterms;
  for (int e = threadIdx.x; e < nc * nc; e += blockDim.x) {
    int row = e % nc, col = e / nc;
    int cr = row / nv, i = row - cr * nv;
    int c = col / nv, j = col - c * nv;
    double2 acc = make_double2(0.0, 0.0);
    for (int q = 0; q < nt; ++q) {
      HopTerm h = terms[q];
      if (h.cs != cr) continue;
      double2 z = make_double2(0.0, 0.0);
      cfma(z, h.coef, Wv[((long)h.ft * 2 + c) * nv + j]);
      cfmac(acc, P[(long)h.fs * nv + i], z);
    }
    Y[((long)blockIdx.x * nc + col) * nc + row] = acc;
  }
}

// Level >= 2 Galerkin build, step 1: T[x][d][k][(c, i)] = sum over l of
// chirality c of Y[x][d](k, l) P[x+d][l][i].
__global__ void k_build_T(const double2* __restrict__ Y, const double2* __restrict__ P,
                          double2* __restrict__ T, int E0, int E1, int nc, int nv) {
  int ncn = 2 * nv;
  long n = (long)E0 * E1 * 5 * nc * ncn;
  long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  int col = (int)(e % ncn);
  long t = e / ncn;
  int k = (int)(t % nc);
  t /= nc;
  int d = (int)(t % 5);
  int x = (int)(t / 5);
  int c = col / nv, i = col - c * nv;
  int xn = nbr_site(x, d, E0, E1);
  int hn = nc / 2;
  const double2* y = Y + ((long)x * 5 + d) * nc * nc;
  double2 acc = make_double2(0.0, 0.0);
  for (int l = c * hn; l < (c + 1) * hn; ++l)
    cfma(acc, y[(long)l * nc + k], P[((long)xn * nc + l) * nv + i]);
  T[e] = acc;
}

// Step 2: Ynext[A][d'](row (cr, i), col) = sum over (x in A, d of type d')
// sum over k of chirality cr of conj(P[x][k][i]) T[x][d][k][col].
__global__ void k_build_Y_coarse(const double2* __restrict__ T, const double2* __restrict__ P,
                                 double2* __restrict__ Yn, int E0, int E1, int b0, int b1, int nc,
                                 int nv) {
  __shared__ int tx[64], td[64];
  __shared__ int nterms;
  int ncn = 2 * nv;
  int F0 = E0 / b0;
  int A = blockIdx.x / 5, dn = blockIdx.x % 5;
  int A0 = A % F0, A1 = A / F0;
  if (threadIdx.x == 0) {
    int n = 0;
    for (int y = 0; y < b1; ++y)
      for (int x = 0; x < b0; ++x) {
        int X = (A0 * b0 + x) + E0 * (A1 * b1 + y);
        for (int d = 0; d < 5; ++d) {
          int typ = 0;
          if (d == 1 && x == b0 - 1) typ = 1;
          if (d == 2 && x == 0) typ = 2;
          if (d == 3 && y == b1 - 1) typ = 3;
          if (d == 4 && y == 0) typ = 4;
          if (typ == dn && n < 64) { tx[n] = X; td[n] = d; ++n; }
        }
      }
    nterms = n;
  }
  __syncthreads();
  int hn = nc / 2;
  for (int e = threadIdx.x; e < ncn * ncn; e += blockDim.x) {
    int row = e % ncn, col = e / ncn;
    int cr = row / nv, i = row - cr * nv;
    double2 acc = make_double2(0.0, 0.0);
    for (int q = 0; q < nterms; ++q) {
      int X = tx[q], d = td[q];
      const double2* tt = T + (((long)X * 5 + d) * nc) * ncn + col;
      for (int k = cr * hn; k < (cr + 1) * hn; ++k)
        cfmac(acc, P[((long)X * nc + k) * nv + i], tt[(long)k * ncn]);
    }
    Yn[((long)blockIdx.x * ncn + col) * ncn + row] = acc;
  }
}

// ---------------------------------------------------------------------------
// Modified Gram-Schmidt of the nv restricted vectors of one (aggregate,
// chirality) pair, in index order (block orthonormalisation, Sec. III.A and
// IV).  dofs[] lists the nd dofs of the pair; Q is [nd][nv] in shared memory.
__device__ void block_mgs(const int* dofs, int nd, int nv, const double2* __restrict__ V,
                          long ndof, double2* __restrict__ P, double2* Q, int* flag) {
  __shared__ double red[2][32];
  __shared__ double2 coef;
  for (int t = threadIdx.x; t < nd * nv; t += blockDim.x) {
    int dd = t / nv, i = t - dd * nv;
    Q[t] = V[(long)i * ndof + dofs[dd]];
  }
  __syncthreads();
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = 0; i < nv; ++i) {
    for (int j = 0; j <= i; ++j) {
      // j < i: projection coefficient <q_j, q_i>; j == i: squared norm.
      double re = 0.0, im = 0.0;
      for (int dd = threadIdx.x; dd < nd; dd += blockDim.x) {
        double2 a = Q[dd * nv + j], b = Q[dd * nv + i];
        re = fma(a.x, b.x, re); re = fma(a.y, b.y, re);
        im = fma(a.x, b.y, im); im = fma(-a.y, b.x, im);
      }
      for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
      }
      if (lane == 0) { red[0][w] = re; red[1][w] = im; }
      __syncthreads();
      if (threadIdx.x == 0) {
        double sr = 0.0, si = 0.0;
        for (int q = 0; q < nw; ++q) { sr += red[0][q]; si += red[1][q]; }
        coef = make_double2(sr, si);
      }
      __syncthreads();
      double2 cf = coef;
      if (j < i) {
        for (int dd = threadIdx.x; dd < nd; dd += blockDim.x) {
          double2 a = Q[dd * nv + j], b = Q[dd * nv + i];
          b.x -= cf.x * a.x - cf.y * a.y;
          b.y -= cf.x * a.y + cf.y * a.x;
          Q[dd * nv + i] = b;
        }
      } else {
        double nrm = sqrt(cf.x);
        if (!(nrm > 0.0) || !isfinite(nrm)) {
          if (threadIdx.x == 0) atomicExch(flag, 1);
          nrm = 1.0;
        }
        for (int dd = threadIdx.x; dd < nd; dd += blockDim.x) {
          double2 b = Q[dd * nv + i];
          Q[dd * nv + i] = make_double2(b.x / nrm, b.y / nrm);
        }
      }
      __syncthreads();
    }
  }
  for (int t = threadIdx.x; t < nd * nv; t += blockDim.x) {
    int dd = t / nv, i = t - dd * nv;
    P[(long)dofs[dd] * nv + i] = Q[t];
  }
}

__global__ void k_block_ortho_fine(const double2* __restrict__ V, double2* __restrict__ P, int L0,
                                   int L1, int a0, int a1, int nv, int* flag) {
  extern __shared__ double2 Q[];
  __shared__ int dofs[1024];
  __shared__ int nd;
  int N = L0 * L1;
  int E0 = L0 / (2 * a0);
  int A = blockIdx.x >> 1, c = blockIdx.x & 1;
  int A0 = A % E0, A1 = A / E0;
  if (threadIdx.x == 0) {
    int n = 0;
    for (int y = 0; y < 2 * a1; ++y)
      for (int x = 0; x < 2 * a0; ++x) {
        int x0 = A0 * 2 * a0 + x, x1 = A1 * 2 * a1 + y;
        if (((x0 + x1) & 1) == c && n < 1024) dofs[n++] = ps_index(x0, x1, L0, N);
      }
    nd = n;
  }
  __syncthreads();
  block_mgs(dofs, nd, nv, V, N, P, Q, flag);
}

__global__ void k_block_ortho_coarse(const double2* __restrict__ V, double2* __restrict__ P, int E0,
                                     int E1, int b0, int b1, int nc, int nv, int* flag) {
  extern __shared__ double2 Q[];
  __shared__ int dofs[1024];
  __shared__ int nd;
  int F0 = E0 / b0;
  int A = blockIdx.x >> 1, c = blockIdx.x & 1;
  int A0 = A % F0, A1 = A / F0;
  int hn = nc / 2;
  if (threadIdx.x == 0) {
    int n = 0;
    for (int y = 0; y < b1; ++y)
      for (int x = 0; x < b0; ++x) {
        int X = (A0 * b0 + x) + E0 * (A1 * b1 + y);
        for (int k = c * hn; k < (c + 1) * hn && n < 1024; ++k) dofs[n++] = X * nc + k;
      }
    nd = n;
  }
  __syncthreads();
  block_mgs(dofs, nd, nv, V, (long)E0 * E1 * nc, P, Q, flag);
}

// ---------------------------------------------------------------------------
// SplitMix64 (Steele, Lea, Flood 2014) output n of stream seed:
// mix(seed + (n + 1) G); uniform in (0, 1] from its top 53 bits; Box-Muller.
__device__ __forceinline__ uint64_t sm_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ double sm_uniform(uint64_t seed, uint64_t n) {
  uint64_t u = sm_mix(seed + (n + 1) * 0x9E3779B97F4A7C15ull);
  return ((double)(u >> 11) + 1.0) * 0x1.0p-53;
}
__global__ void k_gaussian(uint64_t seed, long n, double2* __restrict__ out) {
  long j = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double u1 = sm_uniform(seed, 2 * (uint64_t)j);
  double u2 = sm_uniform(seed, 2 * (uint64_t)j + 1);
  double r = sqrt(-2.0 * log(u1));
  double t = 2.0 * 3.141592653589793 * u2;
  out[j] = make_double2(r * cos(t), r * sin(t));
}

int pick_spc(int nc) {
  int spc = 256 / nc;
  return spc < 1 ? 1 : spc;
}

}  // namespace

template <int NC>
static void coarse_apply_nc(const CoarseGeom& g, const double2* Y, int dagger, const double2* in,
                            double2* out, cudaStream_t s, const int* skip,
                            unsigned long long* exec) {
  int nsites = g.E0 * g.E1;
  // split rows over CTAs until the grid covers the GPU about four times
  int rs = 1;
  while (rs < 8 && NC % (2 * rs) == 0 && (NC / (2 * rs)) % 8 == 0 && (long)nsites * rs < 4 * 152)
    rs *= 2;
  if (dagger)
    k_coarse_apply_nc<NC, true><<<nsites * rs, 5 * (NC / rs), 0, s>>>(Y, in, out, g.E0, g.E1, rs,
                                                                      skip, exec);
  else
    k_coarse_apply_nc<NC, false><<<nsites * rs, 5 * (NC / rs), 0, s>>>(Y, in, out, g.E0, g.E1, rs,
                                                                       skip, exec);
  SW_LAUNCH_CHECK();
}

void launch_coarse_apply(const CoarseGeom& g, const double2* Y, int dagger, const double2* in,
                         double2* out, cudaStream_t s, const int* skip,
                         unsigned long long* exec) {
  switch (g.nc) {
    case 8: return coarse_apply_nc<8>(g, Y, dagger, in, out, s, skip, exec);
    case 12: return coarse_apply_nc<12>(g, Y, dagger, in, out, s, skip, exec);
    case 16: return coarse_apply_nc<16>(g, Y, dagger, in, out, s, skip, exec);
    case 24: return coarse_apply_nc<24>(g, Y, dagger, in, out, s, skip, exec);
    case 32: return coarse_apply_nc<32>(g, Y, dagger, in, out, s, skip, exec);
    case 48: return coarse_apply_nc<48>(g, Y, dagger, in, out, s, skip, exec);
    case 64: return coarse_apply_nc<64>(g, Y, dagger, in, out, s, skip, exec);
    default: break;
  }
  int spc = pick_spc(g.nc);
  int nsites = g.E0 * g.E1;
  size_t smem = (size_t)spc * 5 * g.nc * sizeof(double2);
  k_coarse_apply<<<cdiv(nsites, spc), spc * g.nc, smem, s>>>(Y, in, out, g.E0, g.E1, g.nc, spc,
                                                              dagger, skip, exec);
  SW_LAUNCH_CHECK();
}
void launch_restrict_fine(const sw_gauge* g, int a0, int a1, int nv, const double2* P,
                          const double2* r_e, double2* out, cudaStream_t s, int full) {
  int nagg = (g->L0 / (2 * a0)) * (g->L1 / (2 * a1));
  int threads = cdiv(2 * nv, 32) * 32;
  k_restrict_fine<<<nagg, threads, 0, s>>>(P, r_e, out, g->L0, g->L1, a0, a1, nv, full);
  SW_LAUNCH_CHECK();
}
void launch_prolong_fine(const sw_gauge* g, int a0, int a1, int nv, const double2* P,
                         const double2* ehat, double2* e_e, cudaStream_t s, int full) {
  k_prolong_fine<<<cdiv(full ? g->N : g->N / 2, 128), 128, 0, s>>>(P, ehat, e_e, g->L0, g->L1, a0,
                                                                   a1, nv, full);
  SW_LAUNCH_CHECK();
}
void launch_restrict_coarse(const CoarseGeom& g, int b0, int b1, int nv, const double2* P,
                            const double2* r, double2* out, cudaStream_t s) {
  int nagg = (g.E0 / b0) * (g.E1 / b1);
  int threads = cdiv(2 * nv, 32) * 32;
  k_restrict_coarse<<<nagg, threads, 0, s>>>(P, r, out, g.E0, b0, b1, g.nc, nv);
  SW_LAUNCH_CHECK();
}
void launch_prolong_coarse(const CoarseGeom& g, int b0, int b1, int nv, const double2* P,
                           const double2* ehat, double2* e, cudaStream_t s) {
  long n = (long)g.E0 * g.E1 * g.nc;
  k_prolong_coarse<<<cdiv(n, 128), 128, 0, s>>>(P, ehat, e, g.E0, g.E1, b0, b1, g.nc, nv);
  SW_LAUNCH_CHECK();
}
void launch_build_W(const sw_gauge* g, int nv, const double2* binv, const double2* P,
                    double2* Wv, cudaStream_t s) {
  long n = (long)g->N * nv;
  k_build_W<<<cdiv(n, 256), 256, 0, s>>>(binv, P, Wv, g->N, nv);
  SW_LAUNCH_CHECK();
}
void launch_build_W_identity(const sw_gauge* g, int nv, const double2* P, double2* Wv,
                             cudaStream_t s) {
  long n = (long)g->N * nv;
  k_build_W_identity<<<cdiv(n, 256), 256, 0, s>>>(P, Wv, g->N, nv);
  SW_LAUNCH_CHECK();
}
void launch_build_Y_fine(const sw_gauge* g, double mass, int a0, int a1, int nv, const double2* P,
                         const double2* Wv, double2* Y, cudaStream_t s) {
  int nagg = (g->L0 / (2 * a0)) * (g->L1 / (2 * a1));
  size_t smem = (size_t)(4 * a0 * a1) * 5 * sizeof(HopTerm);
  if (smem > 48 * 1024)
    SW_CUDA(cudaFuncSetAttribute(k_build_Y_fine, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
  k_build_Y_fine<<<nagg * 5, 256, smem, s>>>(g->W_ps, P, Wv, Y, mass, g->L0, g->L1, a0, a1, nv);
  SW_LAUNCH_CHECK();
}
void launch_build_Y_coarse(const CoarseGeom& g, int b0, int b1, int nv, const double2* Y,
                           const double2* P, double2* T, double2* Ynext, cudaStream_t s) {
  long nT = (long)g.E0 * g.E1 * 5 * g.nc * 2 * nv;
  k_build_T<<<cdiv(nT, 256), 256, 0, s>>>(Y, P, T, g.E0, g.E1, g.nc, nv);
  SW_LAUNCH_CHECK();
  int nagg = (g.E0 / b0) * (g.E1 / b1);
  k_build_Y_coarse<<<nagg * 5, 256, 0, s>>>(T, P, Ynext, g.E0, g.E1, b0, b1, g.nc, nv);
  SW_LAUNCH_CHECK();
}
void launch_block_ortho_fine(const sw_gauge* g, int a0, int a1, int nv, const double2* V,
                             double2* P, int* flag, cudaStream_t s) {
  int nagg = (g->L0 / (2 * a0)) * (g->L1 / (2 * a1));
  int nd = 2 * a0 * a1;
  size_t smem = (size_t)nd * nv * sizeof(double2);
  SW_CUDA(cudaFuncSetAttribute(k_block_ortho_fine, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(smem > 1024 ? smem : 1024)));
  k_block_ortho_fine<<<nagg * 2, 128, smem, s>>>(V, P, g->L0, g->L1, a0, a1, nv, flag);
  SW_LAUNCH_CHECK();
}
void launch_block_ortho_coarse(const CoarseGeom& g, int b0, int b1, int nv, const double2* V,
                               double2* P, int* flag, cudaStream_t s) {
  int nagg = (g.E0 / b0) * (g.E1 / b1);
  int nd = b0 * b1 * g.nc / 2;
  size_t smem = (size_t)nd * nv * sizeof(double2);
  SW_CUDA(cudaFuncSetAttribute(k_block_ortho_coarse, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(smem > 1024 ? smem : 1024)));
  k_block_ortho_coarse<<<nagg * 2, 128, smem, s>>>(V, P, g.E0, g.E1, b0, b1, g.nc, nv, flag);
  SW_LAUNCH_CHECK();
}
void launch_gaussian(uint64_t seed, long n, double2* out, cudaStream_t s) {
  k_gaussian<<<cdiv(n, 256), 256, 0, s>>>(seed, n, out);
  SW_LAUNCH_CHECK();
}

void launch_level_maps_fine(const sw_gauge* g, int a0, int a1, int* agg, int* chir,
                            cudaStream_t s) {
  k_level_maps_fine<<<cdiv(g->N, 128), 128, 0, s>>>(agg, chir, g->L0, g->L1, a0, a1);
  SW_LAUNCH_CHECK();
}
void launch_level_maps_coarse(const CoarseGeom& g, int b0, int b1, int* agg, int* chir,
                              cudaStream_t s) {
  long n = (long)g.E0 * g.E1 * g.nc;
  k_level_maps_coarse<<<cdiv(n, 128), 128, 0, s>>>(agg, chir, g.E0, g.E1, g.nc, b0, b1);
  SW_LAUNCH_CHECK();
}
