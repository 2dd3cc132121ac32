// Geometric h-multigrid V-cycle in single precision, the preconditioner of the
// FP64 conjugate-gradient Poisson solver (Sec. 5.1).
//
// What Sec. 5.1 fixes: one V-cycle per CG iteration; Chebyshev smoothing of
// degree 5 before and after the coarse correction with smoothing range 20 on
// every level, needing only the level's diagonal and operator products; a
// Chebyshev coarse solver whose degree brings the Chebyshev error estimate to
// 1e-3; eigenvalue estimates from an initial CG run on every level; coarsening
// down to one cell where the mesh allows it; level transfer by tensorial
// embedding between mother and child cells; the whole cycle in single
// precision; no zero-mean projection inside the cycle.
//
// Levels.  Each level halves the cells of every direction whose count is even
// and > 1, keeps degree, penalty factor and boundary conditions, and
// re-discretises the SIPG Laplacian on its own geometry tables (a full Mesh).
// Coarse levels of the tanh channel keep the graded cell vertices and map each
// cell affinely (SIPG_MAP_CHANNEL_LINEAR).
//
// Transfer.  Prolongation evaluates the parent cell's polynomial at the child's
// nodes: x_child += (E_z (x) E_y (x) E_x) x_parent with E_c[a][b] = l_b((c + z_a)/2)
// for the child half c of a halved direction and the identity otherwise.
// Restriction is the transpose, gathered per parent cell over its children
// (one thread block owns a parent: no atomics, fixed order).  Both are
// sum-factorised contractions in shared memory, one thread per 1D line.
//
// Cycle on level l (vectors b, x, r, d, t of the level, D = diag(A_l)):
//   pre:  x = Chebyshev_deg(b) from x = 0          (deg - 1 operator products)
//   res:  r - A d  is the residual b - A x         (1 product), restricted
//         straight into the next level's b, r, d, x (the coarse smoother's start)
//   ...   coarse cycle, then x += P x_coarse
//   post: t = A x, r = b - t, deg Chebyshev steps from x (deg products)
// The coarsest level runs its Chebyshev iteration from zero.  On level 0 the
// last step also writes z = (double) x and the CG's partial sums (r.z, z.Ap).
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <vector>

#include "sipg_internal.h"

namespace sipg {

namespace {

constexpr int kVB = 152 * 8;  // vector-kernel grid (the CG reads kVB partial sums)
constexpr int kVT = 256;
constexpr int kMaxLevels = 32;
constexpr long long kDenseCoarseMax = 6144;  // coarsest unknowns for the precomputed coarse operator (151 MB)

// grid of a non-reducing vector kernel: no more blocks than the vector needs
inline unsigned vec_grid(long long n) {
  const long long b = (n + kVT - 1) / kVT;
  return (unsigned)(b < 1 ? 1 : (b > kVB ? kVB : b));
}

struct MgKey {
  int k = -1;
  double penalty = 0.0;
  int degree = 0, lanczos = 0, coarse_maxdeg = 0, zero_mean = 0;
  double range = 0.0, coarse_tol = 0.0;
  bool operator==(const MgKey& o) const {
    return k == o.k && penalty == o.penalty && degree == o.degree && lanczos == o.lanczos &&
           coarse_maxdeg == o.coarse_maxdeg && zero_mean == o.zero_mean && range == o.range &&
           coarse_tol == o.coarse_tol;
  }
};

struct MgLevel {
  Mesh* mesh = nullptr;  // level 0: the solver's mesh; others owned by the hierarchy
  long long n = 0;       // unknowns
  int fac[3] = {1, 1, 1};  // halving factor towards the next coarser level
  float *dinv = nullptr, *b = nullptr, *x = nullptr, *r = nullptr, *d = nullptr, *t = nullptr;
  float* d2 = nullptr;      // second direction buffer (the fused steps ping-pong d)
  float* dlast = nullptr;   // buffer holding the latest direction of the pre-smoother
  double lmin = 0.0, lmax = 0.0;  // Chebyshev interval of this level
  int degree = 0;                 // Chebyshev steps (smoother or coarse solve)
  float* Q = nullptr;             // coarsest level: the coarse Chebyshev operator as a dense matrix
  float inv_theta = 0.f;
  std::vector<float> c1, c2;      // recurrence coefficients per step
};

struct Hierarchy {
  MgKey key;
  std::vector<std::unique_ptr<Mesh>> owned;
  std::vector<MgLevel> lv;
  float* emb = nullptr;  // [3][P][P]: child 0, child 1, identity
  void* mem = nullptr;   // FP32 level vectors and two FP64 scratch vectors
  double *tmp_a = nullptr, *tmp_b = nullptr;
  float* Qmem = nullptr;
  ~Hierarchy() {
    if (mem) cudaFree(mem);
    if (emb) cudaFree(emb);
    if (Qmem) cudaFree(Qmem);
  }
};

// ------------------------------------------------------------ vector kernels
// Smoother start from zero: r = b, d = D^-1 b / theta, x = d.  With b_out the
// input is the CG residual (FP64) and is kept as the level's b.
template <typename Tin>
__global__ void k_mg_start(const int* __restrict__ skip, long long n, const Tin* __restrict__ bin,
                           float* __restrict__ b_out, const float* __restrict__ dinv, float* __restrict__ r,
                           float* __restrict__ d, float* __restrict__ x, float inv_theta) {
  if (skip && *skip) return;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float bi = (float)bin[i];
    if (b_out) b_out[i] = bi;
    const float di = bi * dinv[i] * inv_theta;
    r[i] = bi;
    d[i] = di;
    x[i] = di;
  }
}

// Partial sums (a, b) of one block to part[3 * block] (fixed order).
__device__ void mg_partial2(double a, double b, double* part) {
  __shared__ double sh[2][32];
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    sh[0][wid] = a;
    sh[1][wid] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) {
      s0 += sh[0][w];
      s1 += sh[1][w];
    }
    part[3 * blockIdx.x] = s0;
    part[3 * blockIdx.x + 1] = s1;
    part[3 * blockIdx.x + 2] = 0.0;
  }
}

// One Chebyshev step after t = A d:  r -= t;  d = c1 d + c2 D^-1 r;  x += d.
// POST_START instead begins the post-smoother after t = A x:  r = b - t;
// d = D^-1 r * c2 (c2 = 1/theta);  x += d.  FINAL also writes z = (double) x
// and the partials (r64.z, z.(ap - mean)) for the outer CG.
template <bool POST_START, bool FINAL>
__global__ void k_mg_step(const int* __restrict__ skip, long long n, const float* __restrict__ t,
                          const float* __restrict__ b, const float* __restrict__ dinv, float* __restrict__ r,
                          float* __restrict__ d, float* __restrict__ x, float c1, float c2, double* __restrict__ z,
                          const double* __restrict__ r64, const double* __restrict__ ap,
                          const double* __restrict__ mean, double* __restrict__ part) {
  if (skip && *skip) return;
  const double mu = (FINAL && mean) ? *mean : 0.0;
  double rz = 0.0, zq = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float ri, di;
    if (POST_START) {
      ri = b[i] - t[i];
      di = ri * dinv[i] * c2;
    } else {
      ri = r[i] - t[i];
      di = c1 * d[i] + c2 * ri * dinv[i];
    }
    const float xi = x[i] + di;
    r[i] = ri;
    d[i] = di;
    x[i] = xi;
    if (FINAL) {
      const double zi = (double)xi;
      z[i] = zi;
      rz += r64[i] * zi;
      if (ap) zq += zi * (ap[i] - mu);
    }
  }
  if (FINAL && part) mg_partial2(rz, zq, part);
}

// z = (double) x with the CG partials (a cycle whose last operation on level 0
// is not a Chebyshev step: single-level hierarchies of degree 1).
__global__ void k_mg_out(const int* __restrict__ skip, long long n, const float* __restrict__ x,
                         double* __restrict__ z, const double* __restrict__ r64, const double* __restrict__ ap,
                         const double* __restrict__ mean, double* __restrict__ part) {
  if (skip && *skip) return;
  const double mu = mean ? *mean : 0.0;
  double rz = 0.0, zq = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double zi = (double)x[i];
    z[i] = zi;
    rz += r64[i] * zi;
    if (ap) zq += zi * (ap[i] - mu);
  }
  if (part) mg_partial2(rz, zq, part);
}

__global__ void k_mg_inv32(long long n, const double* __restrict__ diag, float* __restrict__ dinv) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dinv[i] = (float)(1.0 / diag[i]);
}

// Start vector of the eigenvalue estimates: SplitMix64 of the index mapped to
// [-1/2, 1/2) (Steele, Lea, Flood, "Fast splittable pseudorandom number
// generators", 2014).
__global__ void k_mg_random(long long n, unsigned long long seed, double* __restrict__ v) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    unsigned long long zz = seed + (unsigned long long)(i + 1) * 0x9E3779B97F4A7C15ull;
    zz = (zz ^ (zz >> 30)) * 0xBF58476D1CE4E5B9ull;
    zz = (zz ^ (zz >> 27)) * 0x94D049BB133111EBull;
    zz ^= zz >> 31;
    v[i] = (double)(zz >> 11) * (1.0 / 9007199254740992.0) - 0.5;
  }
}

// ------------------------------------------------------------ dense coarse solve
// The coarse Chebyshev iteration from zero is a fixed polynomial in D^-1 A:
// x = Q b with Q = q(D^-1 A) D^-1.  For a small coarsest level Q is formed
// once, column by column, by running the same iteration in FP64 on the
// columns of the identity (one operator product on all columns at a time),
// and the cycle applies it as one dense product.
__global__ void k_q_start(long long n, const double* __restrict__ dinv, double* __restrict__ r,
                          double* __restrict__ d, double* __restrict__ x, double inv_theta) {
  const long long nn = n * n;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (long long)gridDim.x * blockDim.x) {
    const long long col = i / n, j = i - col * n;  // vector `col`, entry j
    const double bi = j == col ? 1.0 : 0.0;
    const double di = bi * dinv[j] * inv_theta;
    r[i] = bi;
    d[i] = di;
    x[i] = di;
  }
}

__global__ void k_q_step(long long n, const double* __restrict__ t, const double* __restrict__ dinv,
                         double* __restrict__ r, double* __restrict__ d, double* __restrict__ x, double c1,
                         double c2) {
  const long long nn = n * n;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (long long)gridDim.x * blockDim.x) {
    const long long j = i % n;
    const double ri = r[i] - t[i];
    const double di = c1 * d[i] + c2 * ri * dinv[j];
    r[i] = ri;
    d[i] = di;
    x[i] += di;
  }
}

// Q[i][j] = (result for b = e_j)[i]: row-major FP32 copy of the transpose
__global__ void k_q_store(long long n, const double* __restrict__ x, float* __restrict__ Q) {
  const long long nn = n * n;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < nn; k += (long long)gridDim.x * blockDim.x) {
    const long long i = k / n, j = k - i * n;
    Q[k] = (float)x[j * n + i];
  }
}

__global__ void k_inv64(long long n, const double* __restrict__ diag, double* __restrict__ dinv) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dinv[i] = 1.0 / diag[i];
}

// x = Q b, one warp per row (coalesced along the row), b staged in shared memory
__global__ void k_mg_dense(const int* __restrict__ skip, int n, const float* __restrict__ Q,
                           const float* __restrict__ b, float* __restrict__ x) {
  if (skip && *skip) return;
  extern __shared__ float sb[];
  for (int j = threadIdx.x; j < n; j += blockDim.x) sb[j] = b[j];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int row = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (row >= n) return;
  const float* q = Q + (long long)row * n;
  float acc = 0.f;
  for (int j = lane; j < n; j += 32) acc = fmaf(q[j], sb[j], acc);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) x[row] = acc;
}

// ------------------------------------------------------------ transfer kernels
constexpr int kTransferThreads = 512;

struct MgDims {
  int nf[3], nc[3], fac[3];
  long long ncc;  // coarse cells
  int nch;        // children per parent: fac[0] * fac[1] * fac[2]
  int cpb;        // coarse cells per block
};

__device__ __forceinline__ long long fine_cell(const MgDims& g, int cx, int cy, int cz, int hx, int hy, int hz) {
  const int fx = cx * g.fac[0] + hx, fy = cy * g.fac[1] + hy, fz = cz * g.fac[2] + hz;
  return ((long long)fz * g.nf[1] + fy) * g.nf[0] + fx;
}

// Thread layout of both transfer kernels: per coarse cell nch * P^2 threads,
// one 1D line of one child each, so that the children are processed at once.
struct TransferThread {
  int lc, h, l, rem;  // cell slot in the block, child, line, rank within the cell
  bool active;
  long long cell;
  int c[3], hh[3];    // coarse cell and child offsets
};

template <int P>
__device__ __forceinline__ TransferThread transfer_thread(const MgDims& g) {
  constexpr int P2 = P * P;
  TransferThread t;
  const int per = g.nch * P2;
  t.lc = threadIdx.x / per;
  t.rem = threadIdx.x - t.lc * per;
  t.h = t.rem / P2;
  t.l = t.rem - t.h * P2;
  t.cell = (long long)blockIdx.x * g.cpb + t.lc;
  t.active = t.lc < g.cpb && t.cell < g.ncc;
  t.c[0] = t.c[1] = t.c[2] = 0;
  if (t.active) {
    t.c[0] = (int)(t.cell % g.nc[0]);
    t.c[1] = (int)((t.cell / g.nc[0]) % g.nc[1]);
    t.c[2] = (int)(t.cell / ((long long)g.nc[0] * g.nc[1]));
  }
  t.hh[0] = t.h % g.fac[0];
  t.hh[1] = (t.h / g.fac[0]) % g.fac[1];
  t.hh[2] = t.h / (g.fac[0] * g.fac[1]);
  return t;
}

// Restriction of the residual r_f - t_f (t_f = A d, the last smoothing product)
// to the parent cells: b_c = sum over children of (E_z^T (x) E_y^T (x) E_x^T)
// (r_f - t_f)_child (children summed in a fixed order), written together with
// the coarse smoother's start r = b, d = x = D^-1 b / theta.
template <int P>
__global__ void __launch_bounds__(kTransferThreads) k_mg_restrict(const int* __restrict__ skip, MgDims g,
                                                                  const float* __restrict__ rf,
                                                                  const float* __restrict__ tf,
                                                                  const float* __restrict__ emb,
                                                                  float* __restrict__ b, float* __restrict__ r,
                                                                  float* __restrict__ d, float* __restrict__ x,
                                                                  const float* __restrict__ dinv, float inv_theta) {
  if (skip && *skip) return;
  constexpr int P2 = P * P, P3 = P * P * P;
  extern __shared__ float sm[];
  float* E = sm;                                      // [3][P][P]
  float* A = sm + 3 * P2;                             // [cpb][nch][P3]
  float* B = A + (size_t)g.cpb * g.nch * P3;          // [cpb][nch][P3]
  for (int i = threadIdx.x; i < 3 * P2; i += blockDim.x) E[i] = emb[i];
  const TransferThread t = transfer_thread<P>(g);
  const size_t slot = (size_t)(t.lc < g.cpb ? t.lc : 0) * g.nch;
  float* Ac = A + (slot + t.h) * P3;
  float* Bc = B + (slot + t.h) * P3;
  if (t.active) {
    const long long f = fine_cell(g, t.c[0], t.c[1], t.c[2], t.hh[0], t.hh[1], t.hh[2]) * P3;
    for (int i = t.l; i < P3; i += P2) Ac[i] = rf[f + i] - tf[f + i];
  }
  __syncthreads();
  const float* Ex = E + (g.fac[0] == 2 ? t.hh[0] : 2) * P2;
  const float* Ey = E + (g.fac[1] == 2 ? t.hh[1] : 2) * P2;
  const float* Ez = E + (g.fac[2] == 2 ? t.hh[2] : 2) * P2;
  if (t.active) {  // x lines (b, c): B[c][b][a'] = sum_a Ex[a][a'] A[c][b][a]
    const int bb = t.l % P, cc = t.l / P;
    float u[P];
#pragma unroll
    for (int a = 0; a < P; ++a) u[a] = Ac[(cc * P + bb) * P + a];
#pragma unroll
    for (int a2 = 0; a2 < P; ++a2) {
      float sacc = 0.f;
#pragma unroll
      for (int a = 0; a < P; ++a) sacc = fmaf(Ex[a * P + a2], u[a], sacc);
      Bc[(cc * P + bb) * P + a2] = sacc;
    }
  }
  __syncthreads();
  if (t.active) {  // y lines (a', c): A[c][b'][a'] = sum_b Ey[b][b'] B[c][b][a']
    const int aa = t.l % P, cc = t.l / P;
    float u[P];
#pragma unroll
    for (int bq = 0; bq < P; ++bq) u[bq] = Bc[(cc * P + bq) * P + aa];
#pragma unroll
    for (int b2 = 0; b2 < P; ++b2) {
      float sacc = 0.f;
#pragma unroll
      for (int bq = 0; bq < P; ++bq) sacc = fmaf(Ey[bq * P + b2], u[bq], sacc);
      Ac[(cc * P + b2) * P + aa] = sacc;
    }
  }
  __syncthreads();
  if (t.active) {  // z lines (a', b'): B[c'][b'][a'] = sum_c Ez[c][c'] A[c][b'][a']
    const int aa = t.l % P, bb = t.l / P;
    float u[P];
#pragma unroll
    for (int cq = 0; cq < P; ++cq) u[cq] = Ac[(cq * P + bb) * P + aa];
#pragma unroll
    for (int c2 = 0; c2 < P; ++c2) {
      float sacc = 0.f;
#pragma unroll
      for (int cq = 0; cq < P; ++cq) sacc = fmaf(Ez[cq * P + c2], u[cq], sacc);
      Bc[(c2 * P + bb) * P + aa] = sacc;
    }
  }
  __syncthreads();
  if (t.active) {  // sum over the children (fixed order), coalesced writes
    const float* Bs = B + slot * P3;
    const int per = g.nch * P2;
    for (int i = t.rem; i < P3; i += per) {
      float bi = 0.f;
      for (int hq = 0; hq < g.nch; ++hq) bi += Bs[(size_t)hq * P3 + i];
      const long long o = t.cell * P3 + i;
      const float di = bi * dinv[o] * inv_theta;
      b[o] = bi;
      r[o] = bi;
      d[o] = di;
      x[o] = di;
    }
  }
}

// Prolongation and correction: x_f(child) += (E_z (x) E_y (x) E_x) x_c(parent).
template <int P>
__global__ void __launch_bounds__(kTransferThreads) k_mg_prolong(const int* __restrict__ skip, MgDims g,
                                                                 const float* __restrict__ xc,
                                                                 const float* __restrict__ emb,
                                                                 float* __restrict__ xf) {
  if (skip && *skip) return;
  constexpr int P2 = P * P, P3 = P * P * P;
  extern __shared__ float sm[];
  float* E = sm;
  float* C = sm + 3 * P2;                           // parent values [cpb][P3]
  float* A = C + (size_t)g.cpb * P3;                // [cpb][nch][P3]
  float* B = A + (size_t)g.cpb * g.nch * P3;        // [cpb][nch][P3]
  for (int i = threadIdx.x; i < 3 * P2; i += blockDim.x) E[i] = emb[i];
  const TransferThread t = transfer_thread<P>(g);
  const int lcs = t.lc < g.cpb ? t.lc : 0;
  float* Cc = C + (size_t)lcs * P3;
  float* Ac = A + ((size_t)lcs * g.nch + t.h) * P3;
  float* Bc = B + ((size_t)lcs * g.nch + t.h) * P3;
  if (t.active) {
    const int per = g.nch * P2;
    for (int i = t.rem; i < P3; i += per) Cc[i] = xc[t.cell * P3 + i];
  }
  __syncthreads();
  const float* Ex = E + (g.fac[0] == 2 ? t.hh[0] : 2) * P2;
  const float* Ey = E + (g.fac[1] == 2 ? t.hh[1] : 2) * P2;
  const float* Ez = E + (g.fac[2] == 2 ? t.hh[2] : 2) * P2;
  if (t.active) {  // z lines (a, b): A[c][b][a] = sum_c' Ez[c][c'] C[c'][b][a]
    const int aa = t.l % P, bb = t.l / P;
    float u[P];
#pragma unroll
    for (int cq = 0; cq < P; ++cq) u[cq] = Cc[(cq * P + bb) * P + aa];
#pragma unroll
    for (int c = 0; c < P; ++c) {
      float sacc = 0.f;
#pragma unroll
      for (int cq = 0; cq < P; ++cq) sacc = fmaf(Ez[c * P + cq], u[cq], sacc);
      Ac[(c * P + bb) * P + aa] = sacc;
    }
  }
  __syncthreads();
  if (t.active) {  // y lines (a, c): B[c][b][a] = sum_b' Ey[b][b'] A[c][b'][a]
    const int aa = t.l % P, cc = t.l / P;
    float u[P];
#pragma unroll
    for (int bq = 0; bq < P; ++bq) u[bq] = Ac[(cc * P + bq) * P + aa];
#pragma unroll
    for (int b2 = 0; b2 < P; ++b2) {
      float sacc = 0.f;
#pragma unroll
      for (int bq = 0; bq < P; ++bq) sacc = fmaf(Ey[b2 * P + bq], u[bq], sacc);
      Bc[(cc * P + b2) * P + aa] = sacc;
    }
  }
  __syncthreads();
  if (t.active) {  // x lines (b, c): A[c][b][a] = sum_a' Ex[a][a'] B[c][b][a']
    const int bb = t.l % P, cc = t.l / P;
    float u[P];
#pragma unroll
    for (int a = 0; a < P; ++a) u[a] = Bc[(cc * P + bb) * P + a];
#pragma unroll
    for (int a2 = 0; a2 < P; ++a2) {
      float sacc = 0.f;
#pragma unroll
      for (int a = 0; a < P; ++a) sacc = fmaf(Ex[a2 * P + a], u[a], sacc);
      Ac[(cc * P + bb) * P + a2] = sacc;
    }
  }
  __syncthreads();
  if (t.active) {  // coalesced read-modify-write of the child
    const long long f = fine_cell(g, t.c[0], t.c[1], t.c[2], t.hh[0], t.hh[1], t.hh[2]) * P3;
    for (int i = t.l; i < P3; i += P2) xf[f + i] += Ac[i];
  }
}

template <int P>
int launch_restrict_p(const MgDims& g, const int* skip, const float* rf, const float* tf, const float* emb, float* b,
                      float* r, float* d, float* x, const float* dinv, float inv_theta, cudaStream_t s) {
  const int threads = (g.cpb * g.nch * P * P + 31) / 32 * 32;
  const size_t smem = (size_t)(3 * P * P + 2 * g.cpb * g.nch * P * P * P) * sizeof(float);
  const unsigned blocks = (unsigned)((g.ncc + g.cpb - 1) / g.cpb);
  k_mg_restrict<P><<<blocks, threads, smem, s>>>(skip, g, rf, tf, emb, b, r, d, x, dinv, inv_theta);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SIPG_OK : cuda_fail(e, "multigrid restriction launch");
}

template <int P>
int launch_prolong_p(const MgDims& g, const int* skip, const float* xc, const float* emb, float* xf, cudaStream_t s) {
  const int threads = (g.cpb * g.nch * P * P + 31) / 32 * 32;
  const size_t smem = (size_t)(3 * P * P + g.cpb * P * P * P + 2 * g.cpb * g.nch * P * P * P) * sizeof(float);
  const unsigned blocks = (unsigned)((g.ncc + g.cpb - 1) / g.cpb);
  k_mg_prolong<P><<<blocks, threads, smem, s>>>(skip, g, xc, emb, xf);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SIPG_OK : cuda_fail(e, "multigrid prolongation launch");
}

int launch_restrict(int p, const MgDims& g, const int* skip, const float* rf, const float* tf, const float* emb,
                    float* b, float* r, float* d, float* x, const float* dinv, float inv_theta, cudaStream_t s) {
#define CALL_R(P) launch_restrict_p<P>(g, skip, rf, tf, emb, b, r, d, x, dinv, inv_theta, s)
  switch (p) {
    case 2: return CALL_R(2);
    case 3: return CALL_R(3);
    case 4: return CALL_R(4);
    case 5: return CALL_R(5);
    case 6: return CALL_R(6);
    case 7: return CALL_R(7);
    case 8: return CALL_R(8);
    default: return fail(SIPG_EINVAL, "unsupported degree");
  }
#undef CALL_R
}

int launch_prolong(int p, const MgDims& g, const int* skip, const float* xc, const float* emb, float* xf,
                   cudaStream_t s) {
#define CALL_P(P) launch_prolong_p<P>(g, skip, xc, emb, xf, s)
  switch (p) {
    case 2: return CALL_P(2);
    case 3: return CALL_P(3);
    case 4: return CALL_P(4);
    case 5: return CALL_P(5);
    case 6: return CALL_P(6);
    case 7: return CALL_P(7);
    case 8: return CALL_P(8);
    default: return fail(SIPG_EINVAL, "unsupported degree");
  }
#undef CALL_P
}

MgDims dims_of(const MgLevel& fine, const MgLevel& coarse, int p) {
  MgDims g;
  for (int d = 0; d < 3; ++d) {
    g.nf[d] = fine.mesh->desc.n[d];
    g.nc[d] = coarse.mesh->desc.n[d];
    g.fac[d] = fine.fac[d];
  }
  g.ncc = coarse.mesh->ncell;
  g.nch = g.fac[0] * g.fac[1] * g.fac[2];
  const int per = g.nch * p * p;  // <= 8 * 64 = kTransferThreads
  g.cpb = kTransferThreads / per;
  return g;
}

// Chebyshev coefficients (the three-term recurrence of Chebyshev acceleration,
// Saad, "Iterative methods for sparse linear systems", Alg. 12.1) for the
// interval [lmin, lmax] of D^-1 A.
void set_chebyshev(MgLevel& L, double lmin, double lmax, int degree) {
  L.lmin = lmin;
  L.lmax = lmax;
  L.degree = degree;
  const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin), sigma = theta / delta;
  L.inv_theta = (float)(1.0 / theta);
  L.c1.assign(degree, 0.f);
  L.c2.assign(degree, 0.f);
  double rho = 1.0 / sigma;
  for (int step = 1; step < degree; ++step) {
    const double rn = 1.0 / (2.0 * sigma - rho);
    L.c1[step] = (float)(rn * rho);
    L.c2[step] = (float)(2.0 * rn / delta);
    rho = rn;
  }
}

// Smallest degree d with the Chebyshev error estimate 2 s^d / (1 + s^2d) <= tol
// (Varga, "Matrix iterative analysis"), s = (sqrt(kappa) - 1) / (sqrt(kappa) + 1).
int coarse_degree(double lmin, double lmax, double tol, int maxdeg) {
  const double sk = std::sqrt(lmax / lmin);
  const double sg = (sk - 1.0) / (sk + 1.0);
  double sd = 1.0;
  for (int d = 1; d <= maxdeg; ++d) {
    sd *= sg;
    if (2.0 * sd / (1.0 + sd * sd) <= tol) return d;
  }
  return maxdeg;
}

Hierarchy* H(const Mesh& m) { return static_cast<Hierarchy*>(m.mg); }

int vec_launched(Mesh& m) {
  m.launches++;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SIPG_OK : cuda_fail(e, "multigrid kernel launch");
}

// FP32 operator product on one level: t = A_l v (skipped when *skip != 0).
int level_apply(Mesh& m, const MgLevel& L, const float* v, float* t, const int* skip, cudaStream_t s) {
  DotSink ds;
  ds.skip = skip;
  ds.sums = 0;
  const long long before = L.mesh->launches;
  int st = launch_apply<float>(*L.mesh, v, t, 1, 0.f, 1.f, nullptr, true, &ds, nullptr, s);
  if (L.mesh != &m) m.launches += L.mesh->launches - before;
  return st;
}

// Q = q(D^-1 A) D^-1 of the coarse Chebyshev iteration (see k_q_start); the
// level's diagonal is in h.tmp_b.
int build_dense_coarse(Mesh& m, Hierarchy& h, MgLevel& L, cudaStream_t s) {
  const long long nc = L.n, nn = nc * nc;
  double* tmp = nullptr;
  cudaError_t e = cudaMalloc(&tmp, (size_t)(4 * nn + nc) * sizeof(double));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(SIPG_ENOMEM, "cudaMalloc for the dense coarse operator failed");
  }
  double *R = tmp, *D = tmp + nn, *X = tmp + 2 * nn, *T = tmp + 3 * nn, *dinv = tmp + 4 * nn;
  int st = SIPG_OK;
  k_inv64<<<vec_grid(nc), kVT, 0, s>>>(nc, h.tmp_b, dinv);
  st = vec_launched(m);
  const double theta = 0.5 * (L.lmax + L.lmin), delta = 0.5 * (L.lmax - L.lmin), sigma = theta / delta;
  if (!st) {
    k_q_start<<<kVB, kVT, 0, s>>>(nc, dinv, R, D, X, 1.0 / theta);
    st = vec_launched(m);
  }
  double rho = 1.0 / sigma;
  for (int step = 1; step < L.degree && !st; ++step) {
    const double rn = 1.0 / (2.0 * sigma - rho);
    const double c1 = rn * rho, c2 = 2.0 * rn / delta;
    rho = rn;
    st = launch_apply<double>(*L.mesh, D, T, (int)nc, 0.0, 1.0, nullptr, true, nullptr, nullptr, s);
    if (!st) {
      k_q_step<<<kVB, kVT, 0, s>>>(nc, T, dinv, R, D, X, c1, c2);
      st = vec_launched(m);
    }
  }
  if (!st) {
    e = cudaMalloc(&h.Qmem, (size_t)nn * sizeof(float));
    if (e != cudaSuccess) {
      cudaGetLastError();
      h.Qmem = nullptr;
      st = fail(SIPG_ENOMEM, "cudaMalloc for the dense coarse operator failed");
    }
  }
  if (!st) {
    k_q_store<<<kVB, kVT, 0, s>>>(nc, X, h.Qmem);
    st = vec_launched(m);
  }
  e = cudaStreamSynchronize(s);
  if (!st && e != cudaSuccess) st = cuda_fail(e, "dense coarse operator");
  cudaFree(tmp);
  if (!st) L.Q = h.Qmem;
  return st;
}

// One fused Chebyshev step on one level (operator product and update in the
// operator kernel's epilogue): reads d, writes dnext.
int level_cheb(Mesh& m, const MgLevel& L, const float* d, float* dnext, float c1, float c2, const int* skip,
               cudaStream_t s) {
  ChebEpi epi;
  epi.r = L.r;
  epi.dinv = L.dinv;
  epi.x = L.x;
  epi.dnew = dnext;
  epi.c1 = c1;
  epi.c2 = c2;
  const long long before = L.mesh->launches;
  int st = launch_cheb_step(*L.mesh, d, epi, skip, s);
  if (L.mesh != &m) m.launches += L.mesh->launches - before;
  return st;
}

}  // namespace

void mg_release(Mesh& m) {
  delete H(m);
  m.mg = nullptr;
}

int mg_setup(Mesh& m, const sipg_cg_opts& o, cudaStream_t s) {
  if (o.op != SIPG_OP_LAPLACE) return fail(SIPG_EINVAL, "the multigrid preconditioner supports the Laplace operator");
  if (o.mg_degree < 1 || o.mg_degree > 64) return fail(SIPG_EINVAL, "mg_degree must be in [1, 64]");
  if (!(o.mg_range > 1.0)) return fail(SIPG_EINVAL, "mg_range must be > 1");
  if (!(o.mg_coarse_tol > 0.0 && o.mg_coarse_tol < 1.0)) return fail(SIPG_EINVAL, "mg_coarse_tol must be in (0, 1)");
  if (o.mg_coarse_maxdeg < 1 || o.mg_coarse_maxdeg > 2000)
    return fail(SIPG_EINVAL, "mg_coarse_maxdeg must be in [1, 2000]");
  if (o.cheb_lanczos_steps < 2 || o.cheb_lanczos_steps > 120)
    return fail(SIPG_EINVAL, "cheb_lanczos_steps must be in [2, 120]");
  MgKey key;
  key.k = m.k;
  key.penalty = m.penalty;
  key.degree = o.mg_degree;
  key.lanczos = o.cheb_lanczos_steps;
  key.coarse_maxdeg = o.mg_coarse_maxdeg;
  key.zero_mean = o.zero_mean ? 1 : 0;
  key.range = o.mg_range;
  key.coarse_tol = o.mg_coarse_tol;
  if (H(m) && H(m)->key == key) return SIPG_OK;
  mg_release(m);
  std::unique_ptr<Hierarchy> h(new (std::nothrow) Hierarchy());
  if (!h) return fail(SIPG_ENOMEM, "host allocation failed");
  h->key = key;
  const int p = m.p, P3 = p * p * p;
  // level descriptions
  std::vector<sipg_mesh_desc> descs{m.desc};
  std::vector<std::array<int, 3>> facs;
  while ((int)descs.size() < kMaxLevels) {
    sipg_mesh_desc c = descs.back();
    std::array<int, 3> f{1, 1, 1};
    bool any = false;
    for (int d = 0; d < 3; ++d)
      if (c.n[d] > 1 && c.n[d] % 2 == 0) {
        f[d] = 2;
        c.n[d] /= 2;
        any = true;
      }
    if (!any) break;
    if (c.map == SIPG_MAP_CHANNEL_TANH) c.map = SIPG_MAP_CHANNEL_LINEAR;
    facs.push_back(f);
    descs.push_back(c);
  }
  const int nl = (int)descs.size();
  h->lv.resize(nl);
  for (int l = 0; l < nl; ++l) {
    MgLevel& L = h->lv[l];
    if (l == 0) {
      L.mesh = &m;
    } else {
      std::unique_ptr<Mesh> lm(new (std::nothrow) Mesh());
      if (!lm) return fail(SIPG_ENOMEM, "host allocation failed");
      lm->desc = descs[l];
      lm->ncell = (long long)descs[l].n[0] * descs[l].n[1] * descs[l].n[2];
      lm->device = m.device;
      lm->k = m.k;
      lm->p = m.p;
      lm->penalty = m.penalty;
      int st = build_tables(*lm);
      if (st) return st;
      L.mesh = lm.get();
      h->owned.push_back(std::move(lm));
    }
    L.n = L.mesh->ncell * P3;
    if (l + 1 < nl)
      for (int d = 0; d < 3; ++d) L.fac[d] = facs[l][d];
  }
  // device memory: 7 FP32 vectors per level, 2 FP64 scratch vectors of level 0
  size_t bytes = 0;
  auto take = [&](size_t b) {
    size_t off = bytes;
    bytes += (b + 255) & ~(size_t)255;
    return off;
  };
  std::vector<std::array<size_t, 7>> offs(nl);
  for (int l = 0; l < nl; ++l)
    for (int j = 0; j < 7; ++j) offs[l][j] = take((size_t)h->lv[l].n * 4);
  const size_t o_a = take((size_t)h->lv[0].n * 8), o_b = take((size_t)h->lv[0].n * 8);
  cudaError_t e = cudaMalloc(&h->mem, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    h->mem = nullptr;
    return fail(SIPG_ENOMEM, "cudaMalloc of the multigrid levels failed");
  }
  char* base = (char*)h->mem;
  for (int l = 0; l < nl; ++l) {
    MgLevel& L = h->lv[l];
    L.dinv = (float*)(base + offs[l][0]);
    L.b = (float*)(base + offs[l][1]);
    L.x = (float*)(base + offs[l][2]);
    L.r = (float*)(base + offs[l][3]);
    L.d = (float*)(base + offs[l][4]);
    L.t = (float*)(base + offs[l][5]);
    L.d2 = (float*)(base + offs[l][6]);
  }
  h->tmp_a = (double*)(base + o_a);
  h->tmp_b = (double*)(base + o_b);
  // child embeddings E_c[a][b] = l_b((c + z_a) / 2) and the identity
  {
    std::vector<double> zn, wn;
    gll_rule(p, zn, wn);
    std::vector<float> E(3 * p * p, 0.f);
    for (int c = 0; c < 2; ++c)
      for (int a = 0; a < p; ++a) {
        std::vector<double> val, der;
        lagrange_eval(zn, 0.5 * (c + zn[a]), val, der);
        for (int bq = 0; bq < p; ++bq) E[(c * p + a) * p + bq] = (float)val[bq];
      }
    for (int a = 0; a < p; ++a) E[(2 * p + a) * p + a] = 1.f;
    e = cudaMalloc(&h->emb, E.size() * sizeof(float));
    if (e != cudaSuccess) {
      cudaGetLastError();
      h->emb = nullptr;
      return fail(SIPG_ENOMEM, "cudaMalloc of the embedding tables failed");
    }
    e = cudaMemcpy(h->emb, E.data(), E.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "upload embedding tables");
  }
  // diagonals and eigenvalue estimates, level by level (Sec. 5.1: an initial
  // CG run on every level)
  for (int l = 0; l < nl; ++l) {
    MgLevel& L = h->lv[l];
    const bool coarsest = l == nl - 1;
    int st = launch_diagonal(*L.mesh, true, 0.0, 1.0, nullptr, h->tmp_b, s);
    if (st) return st;
    k_mg_inv32<<<kVB, kVT, 0, s>>>(L.n, h->tmp_b, L.dinv);
    if ((st = vec_launched(m))) return st;
    k_mg_random<<<kVB, kVT, 0, s>>>(L.n, 0x5eed0000ull + (unsigned long long)l, h->tmp_a);
    if ((st = vec_launched(m))) return st;
    int steps = o.cheb_lanczos_steps;
    if (coarsest) {
      const long long half = L.n / 2;
      steps = (int)(half > 120 ? 120 : half);
      if (steps < o.cheb_lanczos_steps) steps = o.cheb_lanczos_steps;
    }
    double rmin = 0.0, rmax = 0.0;
    if ((st = lanczos_extremes(*L.mesh, o, h->tmp_a, 1, steps, 1e-12, s, &rmin, &rmax))) return st;
    if (!(rmax > 0.0) || !std::isfinite(rmax)) return fail(SIPG_NONFINITE, "multigrid eigenvalue estimate failed");
    if (coarsest) {
      const double lmax = 1.1 * rmax;
      double lmin = 0.9 * rmin;
      if (!(lmin > 0.0) || lmin > lmax / 1.5) lmin = lmax / o.mg_range;  // guard against a poor estimate
      set_chebyshev(L, lmin, lmax, coarse_degree(lmin, lmax, o.mg_coarse_tol, o.mg_coarse_maxdeg));
      if (L.n <= kDenseCoarseMax && (st = build_dense_coarse(m, *h, L, s))) return st;
    } else {
      const double lmax = 1.1 * rmax;
      set_chebyshev(L, lmax / o.mg_range, lmax, o.mg_degree);
    }
  }
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "multigrid setup");
  m.mg = h.release();
  return SIPG_OK;
}

int mg_info(const Mesh& m, int max_levels, int* nlevels, int* n_cells, double* lmax, double* coarse_lmin,
            int* cdeg) {
  const Hierarchy* h = H(m);
  if (!h) return fail(SIPG_EINVAL, "no multigrid hierarchy set up on this mesh");
  const int nl = (int)h->lv.size();
  if (nlevels) *nlevels = nl;
  for (int l = 0; l < nl && l < max_levels; ++l) {
    if (n_cells)
      for (int d = 0; d < 3; ++d) n_cells[3 * l + d] = h->lv[l].mesh->desc.n[d];
    if (lmax) lmax[l] = h->lv[l].lmax;
  }
  if (coarse_lmin) *coarse_lmin = h->lv.back().lmin;
  if (cdeg) *cdeg = h->lv.back().degree;
  return SIPG_OK;
}

// z = V(r) on the hierarchy; skip/mean/ap/part as for the CG's preconditioner
// (may be null outside a CG iteration).
int mg_vcycle(Mesh& m, const double* r64, double* z, const double* ap, const int* skip, const double* mean,
              double* part, cudaStream_t s) {
  Hierarchy* h = H(m);
  if (!h) return fail(SIPG_EINVAL, "no multigrid hierarchy set up on this mesh");
  const int nl = (int)h->lv.size(), p = m.p;
  int st;
  MgLevel& L0 = h->lv[0];
  // level 0 start from the FP64 residual
  k_mg_start<double><<<kVB, kVT, 0, s>>>(skip, L0.n, r64, L0.b, L0.dinv, L0.r, L0.d, L0.x, L0.inv_theta);
  if ((st = vec_launched(m))) return st;
  // Chebyshev steps of one level (steps 1 .. degree-1) after its start;
  // `final_out` writes z on the last step
  auto steps = [&](int l, bool final_out) -> int {
    MgLevel& L = h->lv[l];
    float *dc = L.d, *dn = L.d2;
    for (int step = 1; step < L.degree; ++step) {
      int st2;
      if (final_out && step == L.degree - 1) {
        if ((st2 = level_apply(m, L, dc, L.t, skip, s))) return st2;
        k_mg_step<false, true><<<kVB, kVT, 0, s>>>(skip, L.n, L.t, L.b, L.dinv, L.r, dc, L.x, L.c1[step],
                                                    L.c2[step], z, r64, ap, mean, part);
        if ((st2 = vec_launched(m))) return st2;
      } else {
        if ((st2 = level_cheb(m, L, dc, dn, L.c1[step], L.c2[step], skip, s))) return st2;
        float* tmp = dc;
        dc = dn;
        dn = tmp;
      }
    }
    L.dlast = dc;
    return SIPG_OK;
  };
  // coarsest level: the dense operator, else the Chebyshev iteration from zero
  auto coarse_solve = [&](int l, bool final_out) -> int {
    MgLevel& C = h->lv[l];
    if (!C.Q) return steps(l, final_out);
    const int rows = kVT / 32;
    k_mg_dense<<<(unsigned)((C.n + rows - 1) / rows), kVT, (size_t)C.n * sizeof(float), s>>>(skip, (int)C.n, C.Q,
                                                                                            C.b, C.x);
    return vec_launched(m);
  };
  if (nl == 1) {
    if ((st = coarse_solve(0, true))) return st;
    if (L0.Q || L0.degree == 1) {
      k_mg_out<<<kVB, kVT, 0, s>>>(skip, L0.n, L0.x, z, r64, ap, mean, part);
      if ((st = vec_launched(m))) return st;
    }
    return SIPG_OK;
  }
  // down: pre-smooth, residual product, restrict (starts the next level)
  for (int l = 0; l + 1 < nl; ++l) {
    MgLevel& L = h->lv[l];
    MgLevel& C = h->lv[l + 1];
    if ((st = steps(l, false))) return st;
    if ((st = level_apply(m, L, L.dlast, L.t, skip, s))) return st;
    const MgDims g = dims_of(L, C, p);
    if ((st = launch_restrict(p, g, skip, L.r, L.t, h->emb, C.b, C.r, C.d, C.x, C.dinv, C.inv_theta, s))) return st;
    m.launches++;
  }
  if ((st = coarse_solve(nl - 1, false))) return st;
  // up: prolongate and correct, post-smooth
  for (int l = nl - 2; l >= 0; --l) {
    MgLevel& L = h->lv[l];
    MgLevel& C = h->lv[l + 1];
    const MgDims g = dims_of(L, C, p);
    if ((st = launch_prolong(p, g, skip, C.x, h->emb, L.x, s))) return st;
    m.launches++;
    if ((st = level_apply(m, L, L.x, L.t, skip, s))) return st;
    const bool fin = l == 0 && L.degree == 1;
    if (fin)
      k_mg_step<true, true><<<kVB, kVT, 0, s>>>(skip, L.n, L.t, L.b, L.dinv, L.r, L.d, L.x, 0.f, L.inv_theta, z, r64,
                                                 ap, mean, part);
    else
      k_mg_step<true, false><<<vec_grid(L.n), kVT, 0, s>>>(skip, L.n, L.t, L.b, L.dinv, L.r, L.d, L.x, 0.f,
                                                            L.inv_theta, nullptr, nullptr, nullptr, nullptr, nullptr);
    if ((st = vec_launched(m))) return st;
    if ((st = steps(l, l == 0))) return st;
  }
  return SIPG_OK;
}

}  // namespace sipg
