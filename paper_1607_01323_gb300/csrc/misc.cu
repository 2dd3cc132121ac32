// Inverse mass, diagonal and adjoint-gradient launchers (FP64), and the scale
// pass of the double-float calls.
#include <cmath>

#include "adjoint.cuh"

namespace sipg {

namespace {

constexpr int kScaleThreads = 256, kScaleBlocks = 152 * 4;

// Largest df_scale_key over v[0..n) and v2[0..n2) into the scale word
// (df_scale_reduce).
__global__ void __launch_bounds__(kScaleThreads) df_scale_kernel(const double* __restrict__ v, long long n,
                                                                 const double* __restrict__ v2, long long n2,
                                                                 int* __restrict__ dsc, const int* __restrict__ skip) {
  if (skip && *skip) return;
  int key = 0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (long long i = t0; i < n; i += stride) key = max(key, df_scale_key(__ldg(v + i)));
  if (v2)
    for (long long i = t0; i < n2; i += stride) key = max(key, df_scale_key(__ldg(v2 + i)));
  df_scale_reduce(key, dsc);
}

template <int P>
int launch_inverse_mass_p(const Mesh& m, const double* x, double* y, int ncomp, double* dots, bool prescaled,
                          cudaStream_t s) {
  const int cpb = m.cpb[0] > 0 ? m.cpb[0] : default_cpb(P, 0);
  const dim3 grid((unsigned)((m.ncell + cpb - 1) / cpb), (unsigned)ncomp);
  const size_t smem = (size_t)cpb * P * P * P * sizeof(double);
  const int threads = (cpb * P * P + 31) / 32 * 32;  // whole warps
  if (threads > kMaxCellThreads) return fail(SIPG_EINVAL, "cells per block too large for this degree");
  // same arithmetic choice as the operator (double-float keeps FP64 data)
  if (m.f64_arith == SIPG_F64_DOUBLE_FLOAT) {
    if (!prescaled) {
      const int st = launch_df_scale(m, x, m.ncell * P * P * P * ncomp, nullptr, 0, nullptr, s);
      if (st) return st;
    }
    if (smem + 2048 > 48 * 1024) {  // dynamic + static shared memory above the default limit
      cudaError_t e = cudaFuncSetAttribute(inverse_mass_kernel<dfl, double, P>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(inverse mass)");
    }
    inverse_mass_kernel<dfl, double, P><<<grid, threads, smem, s>>>(make_geo<dfl>(m), x, y, cpb, dots);
  } else {
    if (smem + 2048 > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(inverse_mass_kernel<double, double, P>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(inverse mass)");
    }
    inverse_mass_kernel<double, double, P><<<grid, threads, smem, s>>>(make_geo<double>(m), x, y, cpb, dots);
  }
  const_cast<Mesh&>(m).launches++;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SIPG_OK : cuda_fail(e, "inverse mass kernel launch");
}

template <int P>
int launch_diagonal_p(const Mesh& m, bool stiffness, double cm, double nu, const double* nu_cell, double* diag,
                      cudaStream_t s) {
  const Geo<double> g = make_geo<double>(m);
  const long long n = m.ncell * P * P * P;
  const int threads = 256;
  diagonal_kernel<P><<<(unsigned)((n + threads - 1) / threads), threads, 0, s>>>(g, stiffness ? 1 : 0, cm, nu,
                                                                                nu_cell, diag);
  const_cast<Mesh&>(m).launches++;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SIPG_OK : cuda_fail(e, "diagonal kernel launch");
}

}  // namespace

int launch_df_scale(const Mesh& m, const double* v, long long n, const double* v2, long long n2, const int* skip,
                    cudaStream_t s) {
  if (!m.dscale) return fail(SIPG_EINVAL, "mesh has no scale word");
  const long long work = (n > n2 ? n : n2) / 4;  // a few elements per thread
  long long blocks = (work + kScaleThreads - 1) / kScaleThreads;
  blocks = blocks < 1 ? 1 : (blocks > kScaleBlocks ? kScaleBlocks : blocks);
  df_scale_kernel<<<(unsigned)blocks, kScaleThreads, 0, s>>>(v, n, v2, v2 ? n2 : 0, m.dscale, skip);
  const_cast<Mesh&>(m).launches++;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SIPG_OK : cuda_fail(e, "double-float scale pass launch");
}

bool df_coef_ok(double v) {
  const double a = std::fabs(v);
  return a == 0.0 || (a >= 0x1p-100 && a <= 0x1p100);
}

#define SIPG_DISPATCH_P(FN, ...)                       \
  switch (m.p) {                                       \
    case 2: return FN<2>(__VA_ARGS__);                 \
    case 3: return FN<3>(__VA_ARGS__);                 \
    case 4: return FN<4>(__VA_ARGS__);                 \
    case 5: return FN<5>(__VA_ARGS__);                 \
    case 6: return FN<6>(__VA_ARGS__);                 \
    case 7: return FN<7>(__VA_ARGS__);                 \
    case 8: return FN<8>(__VA_ARGS__);                 \
    default: return fail(SIPG_EINVAL, "unsupported degree"); \
  }

int launch_inverse_mass(const Mesh& m, const double* x, double* y, int ncomp, double* dots, bool prescaled,
                        cudaStream_t s) {
  SIPG_DISPATCH_P(launch_inverse_mass_p, m, x, y, ncomp, dots, prescaled, s)
}

int launch_diagonal(const Mesh& m, bool stiffness, double cm, double nu, const double* nu_cell, double* diag,
                    cudaStream_t s) {
  if (m.general()) {
    if (nu_cell) return fail(SIPG_EINVAL, "a perturbed mesh supports a constant viscosity only");
    return launch_general_diagonal(m, stiffness, cm, nu, diag, s);
  }
  SIPG_DISPATCH_P(launch_diagonal_p, m, stiffness, cm, nu, nu_cell, diag, s)
}

namespace {
template <int P>
int launch_adjoint_p(const Mesh& m, const double* nu_cell, const double* u, const double* lam, double* grad,
                     cudaStream_t s) {
  const int cpb = m.cpb[0] > 0 ? m.cpb[0] : default_cpb(P, 0);
  const Geo<double> g = make_geo<double>(m);
  const int threads = (cpb * P * P + 31) / 32 * 32;
  if (threads > kMaxCellThreads) return fail(SIPG_EINVAL, "cells per block too large for this degree");
  const size_t smem = sizeof(double) * ((size_t)3 * cpb * P * P * P + (size_t)8 * cpb * P * P + threads);
  if (smem + 2048 > 48 * 1024) {  // dynamic + static shared memory above the default limit
    cudaError_t e = cudaFuncSetAttribute(adjoint_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(adjoint)");
  }
  adjoint_kernel<P><<<(unsigned)((m.ncell + cpb - 1) / cpb), threads, smem, s>>>(g, nu_cell, u, lam, grad, cpb);
  const_cast<Mesh&>(m).launches++;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SIPG_OK : cuda_fail(e, "adjoint kernel launch");
}
}  // namespace

int launch_adjoint(const Mesh& m, const double* nu_cell, const double* u, const double* lam, double* grad,
                   cudaStream_t s) {
  SIPG_DISPATCH_P(launch_adjoint_p, m, nu_cell, u, lam, grad, s)
}

}  // namespace sipg
