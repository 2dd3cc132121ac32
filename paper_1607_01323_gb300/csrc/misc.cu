// Inverse mass, diagonal and adjoint-gradient launchers (FP64).
#include "adjoint.cuh"

namespace sipg {

namespace {

template <int P>
int launch_inverse_mass_p(const Mesh& m, const double* x, double* y, int ncomp, double* dots, cudaStream_t s) {
  const int cpb = m.cpb[0] > 0 ? m.cpb[0] : default_cpb(P, 0);
  const dim3 grid((unsigned)((m.ncell + cpb - 1) / cpb), (unsigned)ncomp);
  const size_t smem = (size_t)cpb * P * P * P * sizeof(double);
  const int threads = (cpb * P * P + 31) / 32 * 32;  // whole warps
  if (threads > kMaxCellThreads) return fail(SIPG_EINVAL, "cells per block too large for this degree");
  // same arithmetic choice as the operator (double-float keeps FP64 data)
  if (m.f64_arith == SIPG_F64_DOUBLE_FLOAT) {
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

int launch_inverse_mass(const Mesh& m, const double* x, double* y, int ncomp, double* dots, const double*,
                        cudaStream_t s) {
  SIPG_DISPATCH_P(launch_inverse_mass_p, m, x, y, ncomp, dots, s)
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
