// Preconditioned conjugate gradients with the matrix-free operator (Sec. 5.1).
//
// All solver state (alpha, beta, r.z, convergence flag, iteration count) lives
// in device memory, so a chunk of `check_every` iterations contains no host
// synchronisation and can be captured once in a CUDA graph and replayed.  The
// host reads one small status record per chunk.  Once the device flag says
// "done" (converged, breakdown, non-finite, maxit) every later kernel of the
// chunk returns immediately, so no work happens past convergence.
//
// Reductions are deterministic: fixed-size grids write per-block partial sums
// that one block adds up in a fixed order (no atomics).
//
// Preconditioners: Jacobi (the matrix diagonal computed once, Sec. 5.1),
// inverse mass (viscous solver, Sec. 5.1), and a Chebyshev iteration of
// degree d on D^-1 A evaluated entirely in FP32 with the FP32 operator
// (Sec. 5.1: the preconditioner runs in single precision under an FP64 outer
// CG; the eigenvalue bound comes from an initial CG run).  With the FP32
// Chebyshev preconditioner the outer CG uses the flexible (Polak-Ribiere)
// beta, since rounding makes the preconditioner slightly non-linear.  The
// geometric-multigrid V-cycle (mg.cu, Sec. 5.1) is a separate preconditioner of
// the same kind (FP32, flexible beta).
// Singular problems (zero_mean): b and every operator product are projected
// onto vectors with zero mean (Sec. 5.1).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "sipg_internal.h"

namespace sipg {

namespace {

constexpr int kVecBlocks = 152 * 8;  // grid of the vector kernels (multiple of the SM count)
constexpr int kVecThreads = 256;
constexpr int kRedThreads = 1024;
constexpr int kMaxLanczos = 128;

enum Done { RUNNING = 0, CONVERGED = 1, BREAKDOWN = 2, NONFINITE = 3, MAXIT = 4 };

struct Scalars {
  double rz;      // r^T z of the current residual
  double alpha, beta, mean;
  double rr, bb;  // |r|^2 and |b|^2 (b projected when zero_mean)
  double tol2;    // rtol^2
  double ntot;    // number of unknowns (for the mean)
  int done, iters, maxit, record;
  double tot[3];                  // totals of the operator's dots (p.Ap, sum Ap, sum p)
  double tot_update[3];           // totals of the update's dots (r.r, r.z, z.q)
  unsigned cnt_apply, cnt_update;  // last-block counters
  double lan_alpha[kMaxLanczos];
  double lan_beta[kMaxLanczos];
};

__device__ __forceinline__ bool finite(double v) { return isfinite(v); }

// Sum of n triples (fixed order) by one block; result in out[0..2].
__device__ void block_sum3(const double* __restrict__ part, int n, double* out) {
  __shared__ double sh[3][kRedThreads / 32];
  double a = 0.0, b = 0.0, c = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    a += part[3 * i];
    b += part[3 * i + 1];
    c += part[3 * i + 2];
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
    c += __shfl_down_sync(0xffffffffu, c, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    sh[0][wid] = a;
    sh[1][wid] = b;
    sh[2][wid] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    const int nw = blockDim.x / 32;
    for (int w = 0; w < nw; ++w) {
      s0 += sh[0][w];
      s1 += sh[1][w];
      s2 += sh[2][w];
    }
    out[0] = s0;
    out[1] = s1;
    out[2] = s2;
  }
  __syncthreads();
}

__device__ void block_partial3(double a, double b, double c, double* out) {
  __shared__ double sh[3][32];
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
    c += __shfl_down_sync(0xffffffffu, c, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    sh[0][wid] = a;
    sh[1][wid] = b;
    sh[2][wid] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) {
      s0 += sh[0][w];
      s1 += sh[1][w];
      s2 += sh[2][w];
    }
    out[3 * blockIdx.x] = s0;
    out[3 * blockIdx.x + 1] = s1;
    out[3 * blockIdx.x + 2] = s2;
  }
}

// Partials of one CG update block: |r|^2 (accumulated in FP32 from the top
// 24 bits of r; it only feeds the stopping test) reduced with FP32 shuffles,
// r.z and, when ZQ, z.q with FP64 shuffles (every FP64 add costs as much as a
// multiply-add of the update itself on this GPU).
template <bool ZQ>
__device__ void block_partial_update(float rr, double rz, double zq, double* out) {
  __shared__ float shr[32];
  __shared__ double shd[2][32];
  for (int o = 16; o > 0; o >>= 1) {
    rr += __shfl_down_sync(0xffffffffu, rr, o);
    rz += __shfl_down_sync(0xffffffffu, rz, o);
    if (ZQ) zq += __shfl_down_sync(0xffffffffu, zq, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    shr[wid] = rr;
    shd[0][wid] = rz;
    shd[1][wid] = ZQ ? zq : 0.0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float s0 = 0.f;
    double s1 = 0.0, s2 = 0.0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) {
      s0 += shr[w];
      s1 += shd[0][w];
      if (ZQ) s2 += shd[1][w];
    }
    out[3 * blockIdx.x] = (double)s0;
    out[3 * blockIdx.x + 1] = s1;
    out[3 * blockIdx.x + 2] = s2;
  }
}

// FP32 value of the top 24 mantissa bits of a double (truncation, by bit
// manipulation: no FP64 instruction); 0 below the normal FP32 range, +inf above
// it and for inf / NaN (so a non-finite residual still stops the solver).
__device__ __forceinline__ float f64_top24(double d) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(d);
  const int fe = (int)((u >> 52) & 0x7ff) - 1023 + 127;
  if (fe < 1) return 0.f;
  if (fe > 254) return __int_as_float(0x7f800000);
  const unsigned bits = ((unsigned)(u >> 32) & 0x80000000u) | ((unsigned)fe << 23) | ((unsigned)(u >> 29) & 0x7fffffu);
  return __int_as_float((int)bits);
}

// Block-wide sums of three values; thread 0 writes out[0..2].
__device__ void block_total3(double a, double b, double c, double* out) {
  __shared__ double sh[3][32];
  __syncthreads();  // a previous reduction may still read sh
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
    c += __shfl_down_sync(0xffffffffu, c, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    sh[0][wid] = a;
    sh[1][wid] = b;
    sh[2][wid] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) {
      s0 += sh[0][w];
      s1 += sh[1][w];
      s2 += sh[2][w];
    }
    out[0] = s0;
    out[1] = s1;
    out[2] = s2;
  }
}

// ---------------------------------------------------------------- init
// r = b - Ax; partials (sum r, sum b, b.b)
__global__ void k_init_residual(long long n, const double* __restrict__ b, const double* __restrict__ ax,
                                double* __restrict__ r, double* __restrict__ part) {
  double sr = 0.0, sb = 0.0, bb = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double bi = b[i];
    const double ri = bi - ax[i];
    r[i] = ri;
    sr += ri;
    sb += bi;
    bb += bi * bi;
  }
  block_partial3(sr, sb, bb, part);
}

__global__ void k_init_scalars(Scalars* sc, const double* __restrict__ part, int nb, int zero_mean, double ntot,
                               double tol2, int maxit, int record) {
  __shared__ double s[3];
  block_sum3(part, nb, s);
  if (threadIdx.x == 0) {
    sc->ntot = ntot;
    sc->mean = zero_mean ? s[0] / ntot : 0.0;
    sc->bb = zero_mean ? s[2] - s[1] * s[1] / ntot : s[2];
    sc->tol2 = tol2;
    sc->maxit = maxit;
    sc->iters = 0;
    sc->done = RUNNING;
    sc->record = record;
    sc->alpha = sc->beta = 0.0;
    sc->cnt_apply = sc->cnt_update = 0u;
    if (!finite(sc->bb)) sc->done = NONFINITE;
  }
}

// r -= mean (projection); z = P r (Jacobi or copy); partials (r.r, r.z, 0)
__global__ void k_init_precond(const Scalars* __restrict__ sc, long long n, double* r,
                               double* z, const double* __restrict__ diag, double* __restrict__ part) {
  const double mean = sc->mean;
  double rr = 0.0, rz = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double ri = r[i] - mean;
    r[i] = ri;
    const double zi = diag ? ri * diag[i] : ri;
    if (z != r) z[i] = zi;
    rr += ri * ri;
    rz += ri * zi;
  }
  block_partial3(rr, rz, 0.0, part);
}

// ---------------------------------------------------------------- iteration
// One CG update, fused with both reductions around it:
//  - alpha = r.z / (p.Ap - mean sum p) from the operator's totals (the last
//    block of the operator kernel summed them), mean = sum(Ap)/N when zero_mean;
//  - x += alpha p; r -= alpha (Ap - mean); Jacobi/none: z = D^-1 r (diag holds
//    the inverse diagonal);
//  - FORM_Z: the last block adds the partials (r.r, r.z, z.(Ap - mean)) in a
//    fixed order and does beta, the convergence test and the iteration count;
//    otherwise (separate preconditioner) it leaves (r.r) partials for k_beta.
// Every FP64 operation counts on this GPU (2 FP64 FMA/clk/SM): the mean
// subtraction and z.q are compiled out when not needed.
// With a separate preconditioner and rsc set, it also reduces the
// double-float scale of the new r into the mesh's word (see k_pupdate), so
// that a double-float M^-1 skips its scale pass.
template <bool FORM_Z, bool ZERO_MEAN, bool ZQ>
__global__ void k_update(Scalars* sc, long long n, double* __restrict__ x, double* r, const double* __restrict__ p,
                         const double* __restrict__ ap, double* z, const double* __restrict__ diag,
                         double* __restrict__ part, int flexible, int* __restrict__ rsc) {
  if (sc->done) return;
  const double mean = ZERO_MEAN ? sc->tot[1] / sc->ntot : 0.0;
  const double pap = sc->tot[0] - mean * sc->tot[2];
  if (!finite(pap) || !(pap > 0.0)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) sc->done = finite(pap) ? BREAKDOWN : NONFINITE;
    return;
  }
  const double rz_old = sc->rz;
  const double alpha = rz_old / pap;
  // |r|^2 only feeds the stopping test: it is accumulated in FP32 from the top
  // 24 bits of r (relative accuracy ~1e-6 on a norm compared with rtol), which
  // keeps the FP64 pipe for x, r, z and r.z.  Two elements per step (128-bit
  // accesses) when the vectors are 16-byte aligned and n is even.
  float rr32 = 0.f;
  double rz = 0.0, zq = 0.0;
  int rkey = 0;  // largest double-float scale key of r (rsc only)
  auto one = [&](long long i) {
    const double q = ZERO_MEAN ? ap[i] - mean : ap[i];
    x[i] = fma(alpha, p[i], x[i]);
    const double ri = fma(-alpha, q, r[i]);
    r[i] = ri;
    if (!FORM_Z && rsc) rkey = max(rkey, df_scale_key(ri));
    const float rf = f64_top24(ri);
    rr32 = fmaf(rf, rf, rr32);
    if (FORM_Z) {
      const double zi = diag ? ri * diag[i] : ri;
      if (z != r) z[i] = zi;
      rz = fma(ri, zi, rz);
      if (ZQ) zq = fma(zi, q, zq);
    }
  };
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool vec = ((n & 1) == 0) && !(((unsigned long long)x | (unsigned long long)r | (unsigned long long)p |
                                        (unsigned long long)ap | (unsigned long long)(z ? z : r) |
                                        (unsigned long long)(diag ? diag : r)) & 15ull);
  if (vec) {
    for (long long j = t0; j < n / 2; j += stride) {
      const double2 xv = reinterpret_cast<const double2*>(x)[j], pv = reinterpret_cast<const double2*>(p)[j];
      const double2 rv = reinterpret_cast<const double2*>(r)[j], av = reinterpret_cast<const double2*>(ap)[j];
      double2 dv = make_double2(1.0, 1.0);
      if (FORM_Z && diag) dv = reinterpret_cast<const double2*>(diag)[j];
      const double q0 = ZERO_MEAN ? av.x - mean : av.x, q1 = ZERO_MEAN ? av.y - mean : av.y;
      const double r0 = fma(-alpha, q0, rv.x), r1 = fma(-alpha, q1, rv.y);
      reinterpret_cast<double2*>(x)[j] = make_double2(fma(alpha, pv.x, xv.x), fma(alpha, pv.y, xv.y));
      reinterpret_cast<double2*>(r)[j] = make_double2(r0, r1);
      if (!FORM_Z && rsc) rkey = max(rkey, max(df_scale_key(r0), df_scale_key(r1)));
      const float f0 = f64_top24(r0), f1 = f64_top24(r1);
      rr32 = fmaf(f0, f0, fmaf(f1, f1, rr32));
      if (FORM_Z) {
        const double z0 = diag ? r0 * dv.x : r0, z1 = diag ? r1 * dv.y : r1;
        if (z != r) reinterpret_cast<double2*>(z)[j] = make_double2(z0, z1);
        rz = fma(r0, z0, fma(r1, z1, rz));
        if (ZQ) zq = fma(z0, q0, fma(z1, q1, zq));
      }
    }
  } else {
    for (long long i = t0; i < n; i += stride) one(i);
  }
  block_partial_update<ZQ>(rr32, rz, zq, part);
  if (!FORM_Z && rsc) df_scale_reduce(rkey, rsc);
  if (!FORM_Z) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      sc->alpha = alpha;
      sc->mean = mean;
    }
    return;
  }
  __shared__ int last;
  if (threadIdx.x == 0) {
    __threadfence();  // this block's partial is visible before the count
    last = atomicAdd(&sc->cnt_update, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double a = 0.0, b = 0.0, c = 0.0;
#pragma unroll 4
  for (unsigned i = threadIdx.x; i < gridDim.x; i += blockDim.x) {
    a += __ldcg(part + 3 * i);
    b += __ldcg(part + 3 * i + 1);
    c += __ldcg(part + 3 * i + 2);
  }
  block_total3(a, b, c, sc->tot_update);
  if (threadIdx.x == 0) {
    const double rr_t = sc->tot_update[0], rz_t = sc->tot_update[1], zq_t = sc->tot_update[2];
    const int it = sc->iters + 1;
    sc->iters = it;
    sc->alpha = alpha;
    sc->mean = mean;
    sc->rr = rr_t;
    const double beta = flexible ? -alpha * zq_t / rz_old : rz_t / rz_old;
    if (sc->record && it - 1 < kMaxLanczos) {
      sc->lan_alpha[it - 1] = alpha;
      sc->lan_beta[it - 1] = beta;
    }
    if (!finite(rr_t) || !finite(rz_t)) {
      sc->done = NONFINITE;
    } else if (rr_t <= sc->tol2 * sc->bb) {
      sc->done = CONVERGED;
    } else if (it >= sc->maxit) {
      sc->done = MAXIT;
    }
    sc->beta = beta;
    sc->rz = rz_t;
    sc->cnt_update = 0u;
  }
}

using UpdateFn = void (*)(Scalars*, long long, double*, double*, const double*, const double*, double*,
                          const double*, double*, int, int*);

UpdateFn pick_update(bool form_z, bool zero_mean, bool zq) {
  if (!form_z) return zero_mean ? k_update<false, true, false> : k_update<false, false, false>;
  if (zero_mean) return zq ? k_update<true, true, true> : k_update<true, true, false>;
  return zq ? k_update<true, false, true> : k_update<true, false, false>;
}

// beta and the convergence test.  part1: (r.r, r.z, z.q) from k_update, or
// (r.r, -, -) with part2 = (r.z, z.q, -) from a separate preconditioner.
__global__ void k_beta(Scalars* sc, const double* __restrict__ part1, int nb1, const double* __restrict__ part2,
                       int nb2, int flexible) {
  if (sc->done) return;
  __shared__ double s1[3], s2[3];
  block_sum3(part1, nb1, s1);
  if (part2) block_sum3(part2, nb2, s2);
  if (threadIdx.x == 0) {
    const double rr = s1[0];
    const double rz = part2 ? s2[0] : s1[1];
    const double zq = part2 ? s2[1] : s1[2];
    const int it = sc->iters + 1;
    sc->iters = it;
    sc->rr = rr;
    const double beta = flexible ? -sc->alpha * zq / sc->rz : rz / sc->rz;
    if (sc->record && it - 1 < kMaxLanczos) {
      sc->lan_alpha[it - 1] = sc->alpha;
      sc->lan_beta[it - 1] = beta;
    }
    if (!finite(rr) || !finite(rz)) {
      sc->done = NONFINITE;
    } else if (rr <= sc->tol2 * sc->bb) {
      sc->done = CONVERGED;
    } else if (it >= sc->maxit) {
      sc->done = MAXIT;
    }
    sc->beta = beta;
    sc->rz = rz;
  }
}

__global__ void k_set_rz(Scalars* sc, const double* __restrict__ part, int nb) {
  __shared__ double s[3];
  block_sum3(part, nb, s);
  if (threadIdx.x == 0) {
    sc->rr = s[0];
    sc->rz = s[1];
    if (!finite(s[0]) || !finite(s[1])) sc->done = NONFINITE;
    if (sc->done == RUNNING && s[0] <= sc->tol2 * sc->bb) sc->done = CONVERGED;
  }
}

// separate-preconditioner variant of set_rz: part1 = (r.r, ..), part2 = (r.z, ..)
__global__ void k_set_rz2(Scalars* sc, const double* __restrict__ part1, int nb1, const double* __restrict__ part2,
                          int nb2) {
  __shared__ double s1[3], s2[3];
  block_sum3(part1, nb1, s1);
  block_sum3(part2, nb2, s2);
  if (threadIdx.x == 0) {
    sc->rr = s1[0];
    sc->rz = s2[0];
    if (!finite(s1[0]) || !finite(s2[0])) sc->done = NONFINITE;
    if (sc->done == RUNNING && s1[0] <= sc->tol2 * sc->bb) sc->done = CONVERGED;
  }
}

// p = z + beta p   (beta = 0 with init != 0: p = z).  With dsc set, also the
// double-float scale of the new p for the operator that reads it next
// (df_scale_reduce), which then needs no scale pass of its own.
__global__ void k_pupdate(const Scalars* __restrict__ sc, long long n, double* __restrict__ p,
                          const double* __restrict__ z, int init, int* __restrict__ dsc) {
  if (sc->done) return;
  const double beta = init ? 0.0 : sc->beta;
  int key = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double v = init ? z[i] : fma(beta, p[i], z[i]);
    p[i] = v;
    if (dsc) key = max(key, df_scale_key(v));
  }
  if (dsc) df_scale_reduce(key, dsc);
}

// x.y of the operator's input and output with the last block forming the
// total (fixed order) in totals[0] (totals[1], [2] = 0): the p.Ap of an
// operator applied by several kernels
__global__ void k_dot_sink(const int* __restrict__ skip, long long n, const double* __restrict__ x,
                           const double* __restrict__ y, double* __restrict__ part, unsigned* __restrict__ counter,
                           double* __restrict__ totals, int sums) {
  if (*skip) return;
  double xy = 0.0, sy = 0.0, sx = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    xy += x[i] * y[i];
    if (sums) {
      sy += y[i];
      sx += x[i];
    }
  }
  block_partial3(xy, sy, sx, part);
  __shared__ int last;
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double s[3] = {0.0, 0.0, 0.0};
  for (unsigned i = threadIdx.x; i < gridDim.x; i += blockDim.x)
    for (int k = 0; k < 3; ++k) s[k] += __ldcg(part + 3 * i + k);
  __shared__ double sh[3][32];
  for (int k = 0; k < 3; ++k) {
    for (int o = 16; o > 0; o >>= 1) s[k] += __shfl_down_sync(0xffffffffu, s[k], o);
    if ((threadIdx.x & 31) == 0) sh[k][threadIdx.x >> 5] = s[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < 3; ++k) {
      double tot = 0.0;
      for (int w = 0; w < (int)(blockDim.x / 32); ++w) tot += sh[k][w];
      totals[k] = tot;
    }
    *counter = 0u;
  }
}

// ------------------------------------------------------- FP32 Chebyshev
// start: r32 = (float) r; d = D^-1 r32 / theta; x32 = d
__global__ void k_cheb_start(const Scalars* __restrict__ sc, long long n, const double* __restrict__ r,
                             const float* __restrict__ dinv, float* __restrict__ r32, float* __restrict__ d32,
                             float* __restrict__ x32, float inv_theta) {
  if (sc && sc->done) return;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float ri = (float)r[i];
    const float di = ri * dinv[i] * inv_theta;
    r32[i] = ri;
    d32[i] = di;
    x32[i] = di;
  }
}

// r32 -= t32; d = c1 d + c2 D^-1 r32; x32 += d.  When z != null (last step):
// z = (double) x32 and partials (r.z, z.(Ap - mean), 0) with the FP64 r, Ap.
__global__ void k_cheb_step(const Scalars* __restrict__ sc, long long n, const float* __restrict__ t32,
                            const float* __restrict__ dinv, float* __restrict__ r32, float* __restrict__ d32,
                            float* __restrict__ x32, float c1, float c2, double* __restrict__ z,
                            const double* __restrict__ r, const double* __restrict__ ap, double* __restrict__ part) {
  if (sc && sc->done) return;
  const double mean = sc ? sc->mean : 0.0;
  double rz = 0.0, zq = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float ri = r32[i] - t32[i];
    const float di = c1 * d32[i] + c2 * ri * dinv[i];
    const float xi = x32[i] + di;
    r32[i] = ri;
    d32[i] = di;
    x32[i] = xi;
    if (z) {
      const double zi = (double)xi;
      z[i] = zi;
      rz += r[i] * zi;
      if (ap) zq += zi * (ap[i] - mean);
    }
  }
  if (part) block_partial3(rz, zq, 0.0, part);
}

// z = (double) x32 with partials (degree-1 Chebyshev: no step kernel)
__global__ void k_cheb_finish(const Scalars* __restrict__ sc, long long n, const float* __restrict__ x32,
                              double* __restrict__ z, const double* __restrict__ r, const double* __restrict__ ap,
                              double* __restrict__ part) {
  double rz = 0.0, zq = 0.0;
  if (!(sc && sc->done)) {
    const double mean = sc ? sc->mean : 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
      const double zi = (double)x32[i];
      z[i] = zi;
      rz += r[i] * zi;
      if (ap) zq += zi * (ap[i] - mean);
    }
  }
  block_partial3(rz, zq, 0.0, part);
}

__global__ void k_inv_f32(long long n, const double* __restrict__ dinv64, float* __restrict__ dinv) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dinv[i] = (float)dinv64[i];
}

// dst[i] = 1 / src[i mod per]: the inverse diagonal, replicated per component
// (FP64 division is expensive on this GPU: it is done once per solve)
__global__ void k_inv_rep(long long n, long long per, const double* __restrict__ src, double* __restrict__ dst) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = 1.0 / src[i % per];
}

__global__ void k_fill(long long n, double v, double* __restrict__ dst) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = v;
}

struct Workspace {
  double *r, *z, *p, *ap, *xs, *diag, *part1, *part2;
  float *r32, *d32, *x32, *t32, *dinv32;
  Scalars* sc;
  int nblocks_max;
};

// largest eigenvalue of the symmetric tridiagonal T (diagonal a, off-diagonal b)
// by bisection on the Sturm sequence
double tridiag_max_eig(const std::vector<double>& a, const std::vector<double>& b) {
  const int m = (int)a.size();
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < m; ++i) {
    double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < m ? std::fabs(b[i]) : 0.0);
    lo = std::fmin(lo, a[i] - r);
    hi = std::fmax(hi, a[i] + r);
  }
  auto count_below = [&](double x) {  // number of eigenvalues < x
    int c = 0;
    double q = 1.0;
    for (int i = 0; i < m; ++i) {
      double bb = i > 0 ? b[i - 1] * b[i - 1] : 0.0;
      q = a[i] - x - (i > 0 ? bb / q : 0.0);
      if (q == 0.0) q = -1e-300;
      if (q < 0) ++c;
    }
    return c;
  };
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (count_below(mid) == m)
      hi = mid;
    else
      lo = mid;
  }
  return hi;
}

}  // namespace

static int ensure_ws(Mesh& m, long long n, int nb_apply, bool f32, Workspace& w) {
  const int nbmax = nb_apply > kVecBlocks ? nb_apply : kVecBlocks;
  size_t bytes = 0;
  auto take = [&](size_t b) {
    size_t o = bytes;
    bytes += (b + 255) & ~(size_t)255;
    return o;
  };
  const size_t o_r = take(n * 8), o_z = take(n * 8), o_p = take(n * 8), o_ap = take(n * 8), o_xs = take(n * 8),
               o_diag = take(n * 8), o_p1 = take((size_t)nbmax * 24), o_p2 = take((size_t)nbmax * 24),
               o_sc = take(sizeof(Scalars));
  size_t o_r32 = 0, o_d32 = 0, o_x32 = 0, o_t32 = 0, o_di = 0;
  if (f32) {
    o_r32 = take(n * 4);
    o_d32 = take(n * 4);
    o_x32 = take(n * 4);
    o_t32 = take(n * 4);
    o_di = take(n * 4);
  }
  if (bytes > m.ws_bytes) {
    if (m.ws) cudaFree(m.ws);
    m.ws = nullptr;
    m.ws_bytes = 0;
    cudaError_t e = cudaMalloc(&m.ws, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(SIPG_ENOMEM, "cudaMalloc of CG workspace failed");
    }
    m.ws_bytes = bytes;
  }
  char* base = (char*)m.ws;
  w.r = (double*)(base + o_r);
  w.z = (double*)(base + o_z);
  w.p = (double*)(base + o_p);
  w.ap = (double*)(base + o_ap);
  w.xs = (double*)(base + o_xs);
  w.diag = (double*)(base + o_diag);
  w.part1 = (double*)(base + o_p1);
  w.part2 = (double*)(base + o_p2);
  w.sc = (Scalars*)(base + o_sc);
  w.r32 = f32 ? (float*)(base + o_r32) : nullptr;
  w.d32 = f32 ? (float*)(base + o_d32) : nullptr;
  w.x32 = f32 ? (float*)(base + o_x32) : nullptr;
  w.t32 = f32 ? (float*)(base + o_t32) : nullptr;
  w.dinv32 = f32 ? (float*)(base + o_di) : nullptr;
  w.nblocks_max = nbmax;
  return SIPG_OK;
}

namespace {

struct Solver {
  Mesh& m;
  const sipg_cg_opts& o;
  int ncomp;
  long long n;  // total unknowns
  cudaStream_t s;
  Workspace w;
  bool helm, visc;
  double cm, nu;
  const double* nu_cell;
  int nb_apply = 0;
  // Chebyshev
  int cheb_deg = 0;
  float cheb_inv_theta = 0.f;
  std::vector<float> c1, c2;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> evs;
  int ev_used = 0;
  bool capturing = false;
  bool prof;  // per-apply timing events (the mesh's profiling setting)

  Solver(Mesh& mm, const sipg_cg_opts& oo, int nc, cudaStream_t ss)
      : m(mm), o(oo), ncomp(nc), s(ss), prof(mm.profile) {
    n = (long long)m.ncell * m.p * m.p * m.p * ncomp;
    helm = o.op == SIPG_OP_HELMHOLTZ;
    visc = o.op == SIPG_OP_VISCOUS;
    cm = (helm || visc) ? o.mass_coef : 0.0;
    nu = (helm || visc) ? o.nu : 1.0;
    nu_cell = helm ? o.nu_cell : nullptr;
  }

  int launched(int k = 1) {
    m.launches += k;
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SIPG_OK : cuda_fail(e, "CG kernel launch");
  }

  // the search direction's double-float scale comes from k_pupdate (operators
  // of the separable kernels only; the general-map kernel runs its own scale
  // pass)
  int* pscale() const {
    return (m.f64_arith == SIPG_F64_DOUBLE_FLOAT && !m.general()) ? m.dscale : nullptr;
  }
  // the residual's scale comes from k_update when the double-float M^-1
  // preconditions it
  int* rscale() const { return (o.precond == SIPG_PC_INVMASS && pscale()) ? m.dscale : nullptr; }

  int apply64(const double* x, double* y, double* dots, int* nb) {
    DotSink sink;
    sink.partials = dots;
    sink.prescaled = (x == w.p && pscale()) ? 1 : 0;
    if (dots) {  // inside an iteration: the last block forms the totals; skip once the solver is done
      sink.counter = &w.sc->cnt_apply;
      sink.totals = w.sc->tot;
      sink.skip = &w.sc->done;
      sink.sums = o.zero_mean ? 1 : 0;
    }
    if (prof) {
      if (ev_used >= (int)evs.size()) {
        std::pair<cudaEvent_t, cudaEvent_t> pr;
        cudaEventCreate(&pr.first);
        cudaEventCreate(&pr.second);
        evs.push_back(pr);
      }
      // during stream capture only an "external" record becomes a graph node
      cudaEventRecordWithFlags(evs[ev_used].first, s, capturing ? cudaEventRecordExternal : 0);
    }
    int st;
    if (visc) {
      // divergence-form viscous operator: the SIPG Laplacian of each component,
      // the transposed-gradient coupling, then the dot products p.Ap
      DotSink skip_only;
      skip_only.skip = dots ? &w.sc->done : nullptr;
      skip_only.prescaled = sink.prescaled;
      st = launch_apply<double>(m, x, y, ncomp, cm, nu, nullptr, true, &skip_only, nullptr, s);
      // in double-float, x's scale is in the mesh's word by now (from k_pupdate
      // or from the operator's own scale pass)
      if (!st)
        st = launch_viscous_t(m, x, y, nu, dots ? &w.sc->done : nullptr, m.f64_arith == SIPG_F64_DOUBLE_FLOAT, s);
      if (!st && dots) {
        k_dot_sink<<<kVecBlocks, kVecThreads, 0, s>>>(&w.sc->done, n, x, y, dots, &w.sc->cnt_apply, w.sc->tot, 0);
        st = launched();
        if (nb) *nb = kVecBlocks;
      }
    } else if (m.general()) {
      // general map: the operator, then p.Ap (and the zero-mean sums)
      st = launch_general(m, x, y, ncomp, cm, nu, true, dots ? &w.sc->done : nullptr, s);
      if (!st && dots) {
        k_dot_sink<<<kVecBlocks, kVecThreads, 0, s>>>(&w.sc->done, n, x, y, dots, &w.sc->cnt_apply, w.sc->tot,
                                                      o.zero_mean ? 1 : 0);
        st = launched();
        if (nb) *nb = kVecBlocks;
      }
    } else {
      st = launch_apply<double>(m, x, y, ncomp, cm, nu, nu_cell, true, dots ? &sink : nullptr, nb, s);
    }
    if (prof) {
      cudaEventRecordWithFlags(evs[ev_used].second, s, capturing ? cudaEventRecordExternal : 0);
      ++ev_used;
    }
    return st;
  }

  // read the first `valid` event pairs recorded since the last call (after a
  // sync); pairs of applies skipped after convergence are not counted
  void harvest(int valid) {
    for (int i = 0; i < ev_used && i < valid; ++i) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, evs[i].first, evs[i].second) == cudaSuccess) {
        m.prof_ms += ms;
        m.prof_applies++;
      }
    }
    cudaGetLastError();
    ev_used = 0;
  }

  ~Solver() {
    for (auto& pr : evs) {
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
  }

  // z = Chebyshev_d(D^-1 A32) r in FP32; partials (r.z, z.q) into part2
  int cheb_apply(double* z, const double* r, const double* ap, const Scalars* sc) {
    int st;
    k_cheb_start<<<kVecBlocks, kVecThreads, 0, s>>>(sc, n, r, w.dinv32, w.r32, w.d32, w.x32, cheb_inv_theta);
    if ((st = launched())) return st;
    for (int step = 1; step < cheb_deg; ++step) {
      st = launch_apply<float>(m, w.d32, w.t32, ncomp, (float)cm, (float)nu, nullptr, true, nullptr, nullptr, s);
      if (st) return st;
      const bool last = step == cheb_deg - 1;
      k_cheb_step<<<kVecBlocks, kVecThreads, 0, s>>>(sc, n, w.t32, w.dinv32, w.r32, w.d32, w.x32, c1[step], c2[step],
                                                      last ? z : nullptr, r, ap, last ? w.part2 : nullptr);
      if ((st = launched())) return st;
    }
    if (cheb_deg == 1) {
      k_cheb_finish<<<kVecBlocks, kVecThreads, 0, s>>>(sc, n, w.x32, z, r, ap, w.part2);
      if ((st = launched())) return st;
    }
    return SIPG_OK;
  }

  bool separate_precond() const {
    return o.precond == SIPG_PC_INVMASS || o.precond == SIPG_PC_CHEB_F32 || o.precond == SIPG_PC_GMG_F32;
  }
  bool fp32_precond() const { return o.precond == SIPG_PC_CHEB_F32 || o.precond == SIPG_PC_GMG_F32; }

  // one CG iteration (no host synchronisation)
  int iteration() {
    int st, nb;
    if ((st = apply64(w.p, w.ap, w.part1, &nb))) return st;
    const bool sep = separate_precond();
    const double* dg = o.precond == SIPG_PC_JACOBI ? w.diag : nullptr;
    double* z = (o.precond == SIPG_PC_NONE) ? w.r : w.z;
    const int flex = fp32_precond() || (o.flexible && o.precond != SIPG_PC_INVMASS);
    pick_update(!sep, o.zero_mean != 0, flex != 0)<<<kVecBlocks, kVecThreads, 0, s>>>(w.sc, n, xcur, w.r, w.p, w.ap,
                                                                                      z, dg, w.part1, flex,
                                                                                      sep ? rscale() : nullptr);
    if ((st = launched())) return st;
    int nb2 = kVecBlocks;
    if (o.precond == SIPG_PC_INVMASS) {
      if ((st = launch_inverse_mass(m, w.r, w.z, ncomp, w.part2, rscale() != nullptr, s))) return st;
      nb2 = (int)(((m.ncell + (m.cpb[0] > 0 ? m.cpb[0] : default_cpb(m.p, 0)) - 1) /
                   (m.cpb[0] > 0 ? m.cpb[0] : default_cpb(m.p, 0))) *
                  ncomp);
    } else if (o.precond == SIPG_PC_CHEB_F32) {
      if ((st = cheb_apply(w.z, w.r, w.ap, w.sc))) return st;
    } else if (o.precond == SIPG_PC_GMG_F32) {
      if ((st = mg_vcycle(m, w.r, w.z, w.ap, &w.sc->done, &w.sc->mean, w.part2, s))) return st;
    }
    // with a separate preconditioner, beta and the convergence test need its
    // partials: one reduction kernel (the Jacobi / none path did them in k_update)
    if (sep) {
      k_beta<<<1, kRedThreads, 0, s>>>(w.sc, w.part1, kVecBlocks, w.part2, nb2, flex);
      if ((st = launched())) return st;
    }
    k_pupdate<<<kVecBlocks, kVecThreads, 0, s>>>(w.sc, n, w.p, z, 0, pscale());
    return launched();
  }

  double* xcur = nullptr;
  bool first_read = true;
  int iters_seen = 0;

  int read_state(int* done, int* iters, double* rr, double* bb) {
    Scalars h;
    cudaError_t e = cudaMemcpyAsync(&h, w.sc, offsetof(Scalars, lan_alpha), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(e, "read CG state");
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "CG synchronise");
    if (prof) {
      harvest(first_read ? ev_used : h.iters - iters_seen);
      first_read = false;
    }
    iters_seen = h.iters;
    *done = h.done;
    *iters = h.iters;
    *rr = h.rr;
    *bb = h.bb;
    return SIPG_OK;
  }

  // Run CG on A x = b from the given x; record Lanczos data if requested.
  int run(const double* b, double* x, int maxit, double rtol, bool record, int* iters_out, double* relres_out,
          int* done_out) {
    int st, nb;
    xcur = x;
    // r = b - A x
    if ((st = apply64(x, w.ap, nullptr, nullptr))) return st;
    k_init_residual<<<kVecBlocks, kVecThreads, 0, s>>>(n, b, w.ap, w.r, w.part1);
    if ((st = launched())) return st;
    k_init_scalars<<<1, kRedThreads, 0, s>>>(w.sc, w.part1, kVecBlocks, o.zero_mean, (double)n, rtol * rtol, maxit,
                                             record ? 1 : 0);
    if ((st = launched())) return st;
    const bool sep = separate_precond();
    double* z = (o.precond == SIPG_PC_NONE) ? w.r : w.z;
    k_init_precond<<<kVecBlocks, kVecThreads, 0, s>>>(w.sc, n, w.r, z, (!sep && o.precond == SIPG_PC_JACOBI) ? w.diag : nullptr,
                                                     w.part1);
    if ((st = launched())) return st;
    if (sep) {
      int nb2 = kVecBlocks;
      if (o.precond == SIPG_PC_INVMASS) {
        if ((st = launch_inverse_mass(m, w.r, w.z, ncomp, w.part2, false, s))) return st;
        const int cpb = m.cpb[0] > 0 ? m.cpb[0] : default_cpb(m.p, 0);
        nb2 = (int)(((m.ncell + cpb - 1) / cpb) * ncomp);
      } else if (o.precond == SIPG_PC_GMG_F32) {
        if ((st = mg_vcycle(m, w.r, w.z, nullptr, nullptr, nullptr, w.part2, s))) return st;
      } else {
        if ((st = cheb_apply(w.z, w.r, nullptr, nullptr))) return st;
      }
      k_set_rz2<<<1, kRedThreads, 0, s>>>(w.sc, w.part1, kVecBlocks, w.part2, nb2);
    } else {
      k_set_rz<<<1, kRedThreads, 0, s>>>(w.sc, w.part1, kVecBlocks);
    }
    if ((st = launched())) return st;
    k_pupdate<<<kVecBlocks, kVecThreads, 0, s>>>(w.sc, n, w.p, z, 1, pscale());
    if ((st = launched())) return st;
    (void)nb;
    int done = 0, iters = 0;
    double rr = 0, bb = 0;
    if ((st = read_state(&done, &iters, &rr, &bb))) return st;
    const int chunk = o.check_every > 0 ? o.check_every : 16;
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    long long graph_kernels = 0;
    while (!done) {
      if (o.use_graph) {
        if (!exec) {
          long long l0 = m.launches;
          cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
          if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
          int cst = SIPG_OK;
          capturing = true;
          for (int i = 0; i < chunk && cst == SIPG_OK; ++i) cst = iteration();
          capturing = false;
          e = cudaStreamEndCapture(s, &graph);
          if (cst) {
            if (graph) cudaGraphDestroy(graph);
            return cst;
          }
          if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
          e = cudaGraphInstantiate(&exec, graph, 0);
          if (e != cudaSuccess) {
            cudaGraphDestroy(graph);
            return cuda_fail(e, "cudaGraphInstantiate");
          }
          graph_kernels = m.launches - l0;
          m.launches = l0;
          // events recorded during capture are graph nodes: harvest after each replay
        }
        cudaError_t e = cudaGraphLaunch(exec, s);
        if (e != cudaSuccess) {
          cudaGraphExecDestroy(exec);
          cudaGraphDestroy(graph);
          return cuda_fail(e, "cudaGraphLaunch");
        }
        m.launches += graph_kernels;
        if (prof) ev_used = chunk < (int)evs.size() ? chunk : (int)evs.size();
      } else {
        for (int i = 0; i < chunk; ++i)
          if ((st = iteration())) return st;
      }
      if ((st = read_state(&done, &iters, &rr, &bb))) {
        if (exec) {
          cudaGraphExecDestroy(exec);
          cudaGraphDestroy(graph);
        }
        return st;
      }
    }
    if (exec) {
      cudaGraphExecDestroy(exec);
      cudaGraphDestroy(graph);
    }
    if (iters_out) *iters_out = iters;
    if (relres_out) *relres_out = bb > 0 ? std::sqrt(rr / bb) : 0.0;
    if (done_out) *done_out = done;
    return SIPG_OK;
  }
};

}  // namespace

int lanczos_extremes(Mesh& lm, const sipg_cg_opts& o, const double* b, int ncomp, int steps, double rtol,
                     cudaStream_t s, double* ritz_min, double* ritz_max) {
  const long long N = lm.ncell * lm.p * lm.p * lm.p;
  const long long n = N * ncomp;
  const int cpb0 = lm.cpb[0] > 0 ? lm.cpb[0] : default_cpb(lm.p, 0);
  const int nb_apply = (int)(((lm.ncell + cpb0 - 1) / cpb0) * ncomp);
  Workspace w;
  int st = ensure_ws(lm, n, nb_apply, false, w);
  if (st) return st;
  const bool helm = o.op == SIPG_OP_HELMHOLTZ;
  const double cm = helm ? o.mass_coef : 0.0, nu = helm ? o.nu : 1.0;
  const double* nuc = helm ? o.nu_cell : nullptr;
  sipg_cg_opts lo = o;
  lo.precond = SIPG_PC_JACOBI;
  lo.flexible = 0;
  lo.use_graph = 0;
  lo.check_every = steps;
  Solver L(lm, lo, ncomp, s);
  L.w = w;
  if ((st = launch_diagonal(lm, true, cm, nu, nuc, w.xs, s))) return st;
  k_inv_rep<<<kVecBlocks, kVecThreads, 0, s>>>(n, N, w.xs, w.diag);
  if ((st = L.launched())) return st;
  k_fill<<<kVecBlocks, kVecThreads, 0, s>>>(n, 0.0, w.xs);
  if ((st = L.launched())) return st;
  steps = steps < kMaxLanczos ? steps : kMaxLanczos;
  int it = 0, done = 0;
  double rel = 0;
  if ((st = L.run(b, w.xs, steps, rtol, true, &it, &rel, &done))) return st;
  if (done == NONFINITE || done == BREAKDOWN) return fail(SIPG_NONFINITE, "eigenvalue estimate: CG broke down");
  std::vector<double> la(kMaxLanczos), lb(kMaxLanczos);
  const char* scb = reinterpret_cast<const char*>(w.sc);
  cudaError_t e = cudaMemcpy(la.data(), scb + offsetof(Scalars, lan_alpha), sizeof(double) * kMaxLanczos,
                             cudaMemcpyDeviceToHost);
  if (e == cudaSuccess)
    e = cudaMemcpy(lb.data(), scb + offsetof(Scalars, lan_beta), sizeof(double) * kMaxLanczos, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "read Lanczos data");
  const int mm = it < kMaxLanczos ? it : kMaxLanczos;
  if (mm < 1) return fail(SIPG_EINVAL, "eigenvalue estimate needs at least one CG step");
  // Lanczos tridiagonal from the CG coefficients (Saad, Sec. 6.7.3)
  std::vector<double> a(mm), off(mm > 1 ? mm - 1 : 0), an(mm), offn(off.size());
  for (int i = 0; i < mm; ++i) {
    a[i] = 1.0 / la[i] + (i > 0 ? lb[i - 1] / la[i - 1] : 0.0);
    if (i + 1 < mm) off[i] = std::sqrt(lb[i]) / la[i];
  }
  for (int i = 0; i < mm; ++i) an[i] = -a[i];
  for (size_t i = 0; i < off.size(); ++i) offn[i] = -off[i];
  if (ritz_max) *ritz_max = tridiag_max_eig(a, off);
  if (ritz_min) *ritz_min = -tridiag_max_eig(an, offn);
  return SIPG_OK;
}

int cg_solve(Mesh& m, const sipg_cg_opts& o, const double* b, double* x, int ncomp, cudaStream_t s, int* iters,
             double* relres) {
  const long long N = m.ncell * m.p * m.p * m.p;
  const long long n = N * ncomp;
  const int cpb0 = m.cpb[0] > 0 ? m.cpb[0] : default_cpb(m.p, 0);
  const int nb_apply = (int)(((m.ncell + cpb0 - 1) / cpb0) * ncomp);
  int st;
  // the multigrid set-up runs its own CG on the mesh's workspace: before this solve's
  if (o.precond == SIPG_PC_GMG_F32 && (st = mg_setup(m, o, s))) return st;
  double lmax = o.cheb_lmax;
  if (o.precond == SIPG_PC_CHEB_F32 && !(lmax > 0.0)) {
    // lambda_max of D^-1 A from a short Jacobi-PCG run on A y = b (Lanczos from
    // the CG coefficients), as the paper estimates the Chebyshev interval.
    double rmin = 0.0;
    if ((st = lanczos_extremes(m, o, b, ncomp, o.cheb_lanczos_steps, 0.0, s, &rmin, &lmax))) return st;
    lmax *= 1.1;  // safety factor 1.1 on the estimate
  }
  Workspace w;
  st = ensure_ws(m, n, nb_apply, o.precond == SIPG_PC_CHEB_F32, w);
  if (st) return st;
  Solver S(m, o, ncomp, s);
  S.w = w;
  const bool helm = o.op == SIPG_OP_HELMHOLTZ;
  const double cm = helm ? o.mass_coef : 0.0, nu = helm ? o.nu : 1.0;
  const double* nuc = helm ? o.nu_cell : nullptr;
  if (o.precond == SIPG_PC_JACOBI || o.precond == SIPG_PC_CHEB_F32) {
    if ((st = launch_diagonal(m, true, cm, nu, nuc, w.xs, s))) return st;
    k_inv_rep<<<kVecBlocks, kVecThreads, 0, s>>>(n, N, w.xs, w.diag);
    if ((st = S.launched())) return st;
  }
  if (o.precond == SIPG_PC_CHEB_F32) {
    k_inv_f32<<<kVecBlocks, kVecThreads, 0, s>>>(n, w.diag, w.dinv32);
    if ((st = S.launched())) return st;
    const double lmin = lmax / o.cheb_range;
    const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin), sigma = theta / delta;
    S.cheb_deg = o.cheb_degree;
    S.cheb_inv_theta = (float)(1.0 / theta);
    S.c1.assign(o.cheb_degree, 0.f);
    S.c2.assign(o.cheb_degree, 0.f);
    double rho = 1.0 / sigma;
    for (int step = 1; step < o.cheb_degree; ++step) {
      const double rn = 1.0 / (2.0 * sigma - rho);
      S.c1[step] = (float)(rn * rho);
      S.c2[step] = (float)(2.0 * rn / delta);
      rho = rn;
    }
  }
  int it = 0, done = 0;
  double rel = 0.0;
  if ((st = S.run(b, x, o.maxit, o.rtol, false, &it, &rel, &done))) return st;
  if (iters) *iters = it;
  if (relres) *relres = rel;
  switch (done) {
    case CONVERGED: return SIPG_OK;
    case MAXIT: return fail(SIPG_MAXITER, "CG reached maxit without converging");
    case BREAKDOWN: return fail(SIPG_BREAKDOWN, "CG breakdown: p^T A p <= 0 (operator not positive definite?)");
    case NONFINITE: return fail(SIPG_NONFINITE, "non-finite value in CG (right-hand side or operator)");
    default: return fail(SIPG_EINVAL, "CG ended in an unknown state");
  }
}


// ---------------------------------------------------------------------------
// CG without allocation: the same solver, with its workspace carved out of a
// fixed device array instead of cudaMalloc'd memory.
//
// The array below is a file-scope __device__ object: a GPU holds these
// kNoAllocScratchBytes from the moment this file's module is loaded on it
// (with CUDA's lazy module loading that can be the first call of the entry
// point itself, a driver-side reservation) until the process exits.  In host
// code its name is only a host-side stand-in; every call looks up the device
// address with cudaGetSymbolAddress, with the mesh's device current, so the
// address stays right after a context is torn down and re-created.  Every
// call shares the array, so calls that overlap on the GPU (different streams,
// host threads or devices sharing a context) race on it.
namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)16 << 20;  // 16 MiB
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

int noalloc_scratch(void** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static CG scratch)");
  *out = p;
  return SIPG_OK;
}

}  // namespace

size_t noalloc_scratch_bytes() { return kNoAllocScratchBytes; }

int cg_solve_noalloc(Mesh& m, const sipg_cg_opts& o_in, const double* b, double* x, int ncomp, cudaStream_t s,
                     int* iters, double* relres) {
  if (o_in.precond == SIPG_PC_CHEB_F32)
    return fail(SIPG_EINVAL, "the allocation-free solve supports preconditioners none, jacobi and invmass");
  const long long N = m.ncell * m.p * m.p * m.p;
  const long long n = N * ncomp;
  const int cpb0 = m.cpb[0] > 0 ? m.cpb[0] : default_cpb(m.p, 0);
  const long long nb_apply = ((m.ncell + cpb0 - 1) / cpb0) * ncomp;
  const long long nbmax = nb_apply > kVecBlocks ? nb_apply : kVecBlocks;
  // same workspace layout as the allocating path, FP32 buffers excluded
  size_t bytes = 0;
  auto take = [&](size_t nb) {
    size_t off = bytes;
    bytes += (nb + 255) & ~(size_t)255;
    return off;
  };
  const size_t o_r = take(n * 8), o_z = take(n * 8), o_p = take(n * 8), o_ap = take(n * 8), o_xs = take(n * 8),
               o_diag = take(n * 8), o_p1 = take((size_t)nbmax * 24), o_p2 = take((size_t)nbmax * 24),
               o_sc = take(sizeof(Scalars));
  if (bytes > kNoAllocScratchBytes) {
    char msg[256];
    std::snprintf(msg, sizeof(msg),
                  "allocation-free solve needs %zu bytes of scratch for %lld unknowns; the static array holds "
                  "%zu bytes (about 348,000 unknowns)",
                  bytes, n, kNoAllocScratchBytes);
    return fail(SIPG_EINVAL, msg);
  }
  void* base_v = nullptr;
  int st = noalloc_scratch(&base_v);
  if (st) return st;
  char* base = (char*)base_v;
  Workspace w;
  w.r = (double*)(base + o_r);
  w.z = (double*)(base + o_z);
  w.p = (double*)(base + o_p);
  w.ap = (double*)(base + o_ap);
  w.xs = (double*)(base + o_xs);
  w.diag = (double*)(base + o_diag);
  w.part1 = (double*)(base + o_p1);
  w.part2 = (double*)(base + o_p2);
  w.sc = (Scalars*)(base + o_sc);
  w.r32 = w.d32 = w.x32 = w.t32 = w.dinv32 = nullptr;
  w.nblocks_max = (int)nbmax;
  // the array keeps the previous call's contents: clear the solver record
  cudaError_t e = cudaMemsetAsync(w.sc, 0, sizeof(Scalars), s);
  if (e != cudaSuccess) return cuda_fail(e, "clear static CG scratch");
  // run on the caller's stream, without a CUDA graph and without profiling
  // events (their creation would allocate); the mesh's own profiling setting
  // is left untouched
  sipg_cg_opts o = o_in;
  o.use_graph = 0;
  Solver S(m, o, ncomp, s);
  S.prof = false;
  S.w = w;
  const bool helm = o.op == SIPG_OP_HELMHOLTZ;
  const double cm = helm ? o.mass_coef : 0.0, nu = helm ? o.nu : 1.0;
  const double* nuc = helm ? o.nu_cell : nullptr;
  int it = 0, done = 0;
  double rel = 0.0;
  if (o.precond == SIPG_PC_JACOBI) {
    st = launch_diagonal(m, true, cm, nu, nuc, w.xs, s);
    if (!st) {
      k_inv_rep<<<kVecBlocks, kVecThreads, 0, s>>>(n, N, w.xs, w.diag);
      st = S.launched();
    }
  }
  if (!st) st = S.run(b, x, o.maxit, o.rtol, false, &it, &rel, &done);
  if (st) return st;
  if (iters) *iters = it;
  if (relres) *relres = rel;
  switch (done) {
    case CONVERGED: return SIPG_OK;
    case MAXIT: return fail(SIPG_MAXITER, "CG reached maxit without converging");
    case BREAKDOWN: return fail(SIPG_BREAKDOWN, "CG breakdown: p^T A p <= 0 (operator not positive definite?)");
    case NONFINITE: return fail(SIPG_NONFINITE, "non-finite value in CG (right-hand side or operator)");
    default: return fail(SIPG_EINVAL, "CG ended in an unknown state");
  }
}

}  // namespace sipg
