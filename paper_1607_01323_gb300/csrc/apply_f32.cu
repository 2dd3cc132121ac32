// FP32 instantiation of the operator kernels (the preconditioner precision of
// Sec. 5.1).
#include "apply_launch.cuh"

namespace sipg {

template <>
int launch_apply<float>(const Mesh& m, const float* x, float* y, int ncomp, float cm, float nu, const float* nu_cell,
                        bool stiff, const DotSink* sink, int* nblocks, cudaStream_t s) {
  return launch_apply_dispatch<float>(m, x, y, ncomp, cm, nu, nu_cell, stiff, sink, nblocks, s);
}

}  // namespace sipg
