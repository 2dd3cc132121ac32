// FP64 instantiation of the operator kernels.
#include "apply_launch.cuh"

namespace sipg {

template <>
int launch_apply<double>(const Mesh& m, const double* x, double* y, int ncomp, double cm, double nu,
                         const double* nu_cell, bool stiff, const DotSink* sink, int* nblocks, cudaStream_t s) {
  return launch_apply_dispatch<double>(m, x, y, ncomp, cm, nu, nu_cell, stiff, sink, nblocks, s);
}

}  // namespace sipg
