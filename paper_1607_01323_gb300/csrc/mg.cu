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
  double lmin = 0.0, lmax = 0.0;  // Chebyshev interval of this level
  int degree = 0;                 // Chebyshev steps (smoother or coarse solve)
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
  ~Hierarchy() {
    if (mem) cudaFree(mem);
    if (emb) cudaFree(emb);
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

// ------------------------------------------------------------ transfer kernels
struct MgDims {
  int nf[3], nc[3], fac[3];
  long long ncc;  // coarse cells
  int cpb;        // coarse cells per block
};

__device__ __forceinline__ long long fine_cell(const MgDims& g, int cx, int cy, int cz, int hx, int hy, int hz) {
  const int fx = cx * g.fac[0] + hx, fy = cy * g.fac[1] + hy, fz = cz * g.fac[2] + hz;
  return ((long long)fz * g.nf[1] + fy) * g.nf[0] + fx;
}

// Restriction of the residual r_f - t_f (t_f = A d, the last smoothing product)
// to the parent cells: b_c = sum over children of (E_z^T (x) E_y^T (x) E_x^T)
// (r_f - t_f)_child, written together with the coarse smoother's start
// r = b, d = x = D^-1 b / theta.
template <int P>
__global__ void __launch_bounds__(kMaxCellThreads) k_mg_restrict(const int* __restrict__ skip, MgDims g,
                                                                 const float* __restrict__ rf,
                                                                 const float* __restrict__ tf,
                                                                 const float* __restrict__ emb,
                                                                 float* __restrict__ b, float* __restrict__ r,
                                                                 float* __restrict__ d, float* __restrict__ x,
                                                                 const float* __restrict__ dinv, float inv_theta) {
  if (skip && *skip) return;
  constexpr int P2 = P * P, P3 = P * P * P;
  extern __shared__ float sm[];
  float* E = sm;                      // [3][P][P]
  float* A = sm + 3 * P2;             // [cpb][P3]
  float* B = A + (size_t)g.cpb * P3;  // [cpb][P3]
  for (int i = threadIdx.x; i < 3 * P2; i += blockDim.x) E[i] = emb[i];
  const int lc = threadIdx.x / P2, l = threadIdx.x % P2;
  const long long cell = (long long)blockIdx.x * g.cpb + lc;
  const bool active = lc < g.cpb && cell < g.ncc;
  int cx = 0, cy = 0, cz = 0;
  if (active) {
    cx = (int)(cell % g.nc[0]);
    cy = (int)((cell / g.nc[0]) % g.nc[1]);
    cz = (int)(cell / ((long long)g.nc[0] * g.nc[1]));
  }
  float* Ac = A + (size_t)(lc < g.cpb ? lc : 0) * P3;
  float* Bc = B + (size_t)(lc < g.cpb ? lc : 0) * P3;
  float acc[P];
#pragma unroll
  for (int c = 0; c < P; ++c) acc[c] = 0.f;
  for (int hz = 0; hz < g.fac[2]; ++hz)
    for (int hy = 0; hy < g.fac[1]; ++hy)
      for (int hx = 0; hx < g.fac[0]; ++hx) {
        __syncthreads();  // E loaded / previous child's z phase done with A
        if (active) {
          const long long f = fine_cell(g, cx, cy, cz, hx, hy, hz) * P3;
          for (int i = l; i < P3; i += P2) Ac[i] = rf[f + i] - tf[f + i];
        }
        __syncthreads();
        const float* Ex = E + (g.fac[0] == 2 ? hx : 2) * P2;
        const float* Ey = E + (g.fac[1] == 2 ? hy : 2) * P2;
        const float* Ez = E + (g.fac[2] == 2 ? hz : 2) * P2;
        if (active) {  // x lines (b, c): B[c][b][a'] = sum_a Ex[a][a'] A[c][b][a]
          const int bb = l % P, cc = l / P;
          float u[P];
#pragma unroll
          for (int a = 0; a < P; ++a) u[a] = Ac[(cc * P + bb) * P + a];
#pragma unroll
          for (int a2 = 0; a2 < P; ++a2) {
            float s = 0.f;
#pragma unroll
            for (int a = 0; a < P; ++a) s = fmaf(Ex[a * P + a2], u[a], s);
            Bc[(cc * P + bb) * P + a2] = s;
          }
        }
        __syncthreads();
        if (active) {  // y lines (a', c): A[c][b'][a'] = sum_b Ey[b][b'] B[c][b][a']
          const int aa = l % P, cc = l / P;
          float u[P];
#pragma unroll
          for (int bq = 0; bq < P; ++bq) u[bq] = Bc[(cc * P + bq) * P + aa];
#pragma unroll
          for (int b2 = 0; b2 < P; ++b2) {
            float s = 0.f;
#pragma unroll
            for (int bq = 0; bq < P; ++bq) s = fmaf(Ey[bq * P + b2], u[bq], s);
            Ac[(cc * P + b2) * P + aa] = s;
          }
        }
        __syncthreads();
        if (active) {  // z lines (a', b'): acc[c'] += sum_c Ez[c][c'] A[c][b'][a']
          const int aa = l % P, bb = l / P;
          float u[P];
#pragma unroll
          for (int cq = 0; cq < P; ++cq) u[cq] = Ac[(cq * P + bb) * P + aa];
#pragma unroll
          for (int c2 = 0; c2 < P; ++c2) {
            float s = acc[c2];
#pragma unroll
            for (int cq = 0; cq < P; ++cq) s = fmaf(Ez[cq * P + c2], u[cq], s);
            acc[c2] = s;
          }
        }
      }
  if (active) {
    const int aa = l % P, bb = l / P;
    const long long o = cell * P3 + bb * P + aa;
#pragma unroll
    for (int c = 0; c < P; ++c) {
      const long long i = o + (long long)c * P2;
      const float bi = acc[c];
      const float di = bi * dinv[i] * inv_theta;
      b[i] = bi;
      r[i] = bi;
      d[i] = di;
      x[i] = di;
    }
  }
}

// Prolongation and correction: x_f(child) += (E_z (x) E_y (x) E_x) x_c(parent).
template <int P>
__global__ void __launch_bounds__(kMaxCellThreads) k_mg_prolong(const int* __restrict__ skip, MgDims g,
                                                                const float* __restrict__ xc,
                                                                const float* __restrict__ emb,
                                                                float* __restrict__ xf) {
  if (skip && *skip) return;
  constexpr int P2 = P * P, P3 = P * P * P;
  extern __shared__ float sm[];
  float* E = sm;
  float* C = sm + 3 * P2;             // parent values [cpb][P3]
  float* A = C + (size_t)g.cpb * P3;  // [cpb][P3]
  float* B = A + (size_t)g.cpb * P3;  // [cpb][P3]
  for (int i = threadIdx.x; i < 3 * P2; i += blockDim.x) E[i] = emb[i];
  const int lc = threadIdx.x / P2, l = threadIdx.x % P2;
  const long long cell = (long long)blockIdx.x * g.cpb + lc;
  const bool active = lc < g.cpb && cell < g.ncc;
  int cx = 0, cy = 0, cz = 0;
  float* Cc = C + (size_t)(lc < g.cpb ? lc : 0) * P3;
  float* Ac = A + (size_t)(lc < g.cpb ? lc : 0) * P3;
  float* Bc = B + (size_t)(lc < g.cpb ? lc : 0) * P3;
  if (active) {
    cx = (int)(cell % g.nc[0]);
    cy = (int)((cell / g.nc[0]) % g.nc[1]);
    cz = (int)(cell / ((long long)g.nc[0] * g.nc[1]));
    for (int i = l; i < P3; i += P2) Cc[i] = xc[cell * P3 + i];
  }
  for (int hz = 0; hz < g.fac[2]; ++hz)
    for (int hy = 0; hy < g.fac[1]; ++hy)
      for (int hx = 0; hx < g.fac[0]; ++hx) {
        __syncthreads();  // C and E loaded / previous child's store done with A
        const float* Ex = E + (g.fac[0] == 2 ? hx : 2) * P2;
        const float* Ey = E + (g.fac[1] == 2 ? hy : 2) * P2;
        const float* Ez = E + (g.fac[2] == 2 ? hz : 2) * P2;
        if (active) {  // z lines (a, b): A[c][b][a] = sum_c' Ez[c][c'] C[c'][b][a]
          const int aa = l % P, bb = l / P;
          float u[P];
#pragma unroll
          for (int cq = 0; cq < P; ++cq) u[cq] = Cc[(cq * P + bb) * P + aa];
#pragma unroll
          for (int c = 0; c < P; ++c) {
            float s = 0.f;
#pragma unroll
            for (int cq = 0; cq < P; ++cq) s = fmaf(Ez[c * P + cq], u[cq], s);
            Ac[(c * P + bb) * P + aa] = s;
          }
        }
        __syncthreads();
        if (active) {  // y lines (a, c): B[c][b][a] = sum_b' Ey[b][b'] A[c][b'][a]
          const int aa = l % P, cc = l / P;
          float u[P];
#pragma unroll
          for (int bq = 0; bq < P; ++bq) u[bq] = Ac[(cc * P + bq) * P + aa];
#pragma unroll
          for (int b2 = 0; b2 < P; ++b2) {
            float s = 0.f;
#pragma unroll
            for (int bq = 0; bq < P; ++bq) s = fmaf(Ey[b2 * P + bq], u[bq], s);
            Bc[(cc * P + b2) * P + aa] = s;
          }
        }
        __syncthreads();
        if (active) {  // x lines (b, c): A[c][b][a] = sum_a' Ex[a][a'] B[c][b][a']
          const int bb = l % P, cc = l / P;
          float u[P];
#pragma unroll
          for (int a = 0; a < P; ++a) u[a] = Bc[(cc * P + bb) * P + a];
#pragma unroll
          for (int a2 = 0; a2 < P; ++a2) {
            float s = 0.f;
#pragma unroll
            for (int a = 0; a < P; ++a) s = fmaf(Ex[a2 * P + a], u[a], s);
            Ac[(cc * P + bb) * P + a2] = s;
          }
        }
        __syncthreads();
        if (active) {  // coalesced read-modify-write of the child
          const long long f = fine_cell(g, cx, cy, cz, hx, hy, hz) * P3;
          for (int i = l; i < P3; i += P2) xf[f + i] += Ac[i];
        }
      }
}

int transfer_cpb(int p) {
  int c = kMaxCellThreads / (p * p);
  return c < 1 ? 1 : c;
}

template <int P>
int launch_restrict_p(const MgDims& g, const int* skip, const float* rf, const float* tf, const float* emb, float* b,
                      float* r, float* d, float* x, const float* dinv, float inv_theta, cudaStream_t s) {
  const int threads = (g.cpb * P * P + 31) / 32 * 32;
  const size_t smem = (size_t)(3 * P * P + 2 * g.cpb * P * P * P) * sizeof(float);
  const unsigned blocks = (unsigned)((g.ncc + g.cpb - 1) / g.cpb);
  k_mg_restrict<P><<<blocks, threads, smem, s>>>(skip, g, rf, tf, emb, b, r, d, x, dinv, inv_theta);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SIPG_OK : cuda_fail(e, "multigrid restriction launch");
}

template <int P>
int launch_prolong_p(const MgDims& g, const int* skip, const float* xc, const float* emb, float* xf, cudaStream_t s) {
  const int threads = (g.cpb * P * P + 31) / 32 * 32;
  const size_t smem = (size_t)(3 * P * P + 3 * g.cpb * P * P * P) * sizeof(float);
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
  g.cpb = transfer_cpb(p);
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
  // device memory: 6 FP32 vectors per level, 2 FP64 scratch vectors of level 0
  size_t bytes = 0;
  auto take = [&](size_t b) {
    size_t off = bytes;
    bytes += (b + 255) & ~(size_t)255;
    return off;
  };
  std::vector<std::array<size_t, 6>> offs(nl);
  for (int l = 0; l < nl; ++l)
    for (int j = 0; j < 6; ++j) offs[l][j] = take((size_t)h->lv[l].n * 4);
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
    for (int step = 1; step < L.degree; ++step) {
      int st2;
      if ((st2 = level_apply(m, L, L.d, L.t, skip, s))) return st2;
      if (final_out && step == L.degree - 1)
        k_mg_step<false, true><<<kVB, kVT, 0, s>>>(skip, L.n, L.t, L.b, L.dinv, L.r, L.d, L.x, L.c1[step],
                                                    L.c2[step], z, r64, ap, mean, part);
      else
        k_mg_step<false, false><<<kVB, kVT, 0, s>>>(skip, L.n, L.t, L.b, L.dinv, L.r, L.d, L.x, L.c1[step],
                                                     L.c2[step], nullptr, nullptr, nullptr, nullptr, nullptr);
      if ((st2 = vec_launched(m))) return st2;
    }
    return SIPG_OK;
  };
  if (nl == 1) {
    if ((st = steps(0, true))) return st;
    if (L0.degree == 1) {
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
    if ((st = level_apply(m, L, L.d, L.t, skip, s))) return st;
    const MgDims g = dims_of(L, C, p);
    if ((st = launch_restrict(p, g, skip, L.r, L.t, h->emb, C.b, C.r, C.d, C.x, C.dinv, C.inv_theta, s))) return st;
    m.launches++;
  }
  // coarsest: Chebyshev from zero
  if ((st = steps(nl - 1, false))) return st;
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
      k_mg_step<true, false><<<kVB, kVT, 0, s>>>(skip, L.n, L.t, L.b, L.dinv, L.r, L.d, L.x, 0.f, L.inv_theta,
                                                  nullptr, nullptr, nullptr, nullptr, nullptr);
    if ((st = vec_launched(m))) return st;
    if ((st = steps(l, l == 0))) return st;
  }
  return SIPG_OK;
}

}  // namespace sipg
