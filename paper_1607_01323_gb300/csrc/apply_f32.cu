// FP32 instantiation of the operator kernels (the preconditioner precision of
// Sec. 5.1).
#include "apply_launch.cuh"

namespace sipg {

template <>
int launch_apply<float>(const Mesh& m, const float* x, float* y, int ncomp, float cm, float nu, const float* nu_cell,
                        bool stiff, const DotSink* sink, int* nblocks, cudaStream_t s) {
  return launch_apply_dispatch<float>(m, x, y, ncomp, cm, nu, nu_cell, stiff, sink, nblocks, s);
}

template <int P>
static int launch_cheb_step_p(const Mesh& m, const float* d, const ChebEpi& epi, const int* skip, cudaStream_t s) {
  // line mapping with its default cells per block (the plane variant has no epilogue)
  const int cpb = m.f32_mapping == 1 ? default_cpb(P, 1) : cells_per_block(m, 1);
  const dim3 grid((unsigned)((m.ncell + cpb - 1) / cpb), 1);
  const int threads = (cpb * P * P + 31) / 32 * 32;
  const size_t smem = uniform_smem_bytes<float, P>(cpb);
  if (threads > kMaxCellThreads) return fail(SIPG_EINVAL, "cells per block too large for this degree");
  DotSink ds;
  ds.skip = skip;
  ds.sums = 0;
  const cudaError_t e = launch_uniform<float, float, P, true>(m, grid, threads, smem, s, make_geo<float>(m), d,
                                                              (float*)nullptr, cpb, 0.f, 1.f, 0, 0, ds, epi);
  const_cast<Mesh&>(m).launches++;
  return e == cudaSuccess ? SIPG_OK : cuda_fail(e, "apply kernel launch (Chebyshev step)");
}

int launch_cheb_step(const Mesh& m, const float* d, const ChebEpi& epi, const int* skip, cudaStream_t s) {
  switch (m.p) {
    case 2: return launch_cheb_step_p<2>(m, d, epi, skip, s);
    case 3: return launch_cheb_step_p<3>(m, d, epi, skip, s);
    case 4: return launch_cheb_step_p<4>(m, d, epi, skip, s);
    case 5: return launch_cheb_step_p<5>(m, d, epi, skip, s);
    case 6: return launch_cheb_step_p<6>(m, d, epi, skip, s);
    case 7: return launch_cheb_step_p<7>(m, d, epi, skip, s);
    case 8: return launch_cheb_step_p<8>(m, d, epi, skip, s);
    default: return fail(SIPG_EINVAL, "unsupported degree");
  }
}

}  // namespace sipg
