// Launchers of the operator kernel for one scalar type (included by
// apply_f64.cu and apply_f32.cu so that the two compile in parallel).
#pragma once

#include <type_traits>

#include "apply.cuh"

namespace sipg {

// Launch of apply_uniform_kernel, with the even-odd x/z contractions when the
// mesh allows them (p >= 5, Mesh::eo_xz) and, in FP32 and double-float, the x
// and z tables as kernel parameters when each of the two directions has one
// table for all its layers (the FP64 kernel is bound by its FP64 pipe, not
// by its loads).
template <typename T, typename S, int P, bool CHEB>
static cudaError_t launch_uniform(const Mesh& m, dim3 grid, int threads, size_t smem, cudaStream_t s, const Geo<T>& g,
                                  const S* x, S* y, int cpb, T mass_rel, T scale, int do_scale, int do_mass,
                                  const DotSink& ds, const ChebEpi& epi) {
  const bool big = smem + 2048 > 48 * 1024;  // dynamic + static shared memory above the default limit
  if constexpr (!std::is_same<T, double>::value) {
    if (m.lay_same[0] && m.lay_same[2]) {
      XZTab<T, P> xz;
      for (int j = 0; j < LayerOff<P>::stride; ++j) {
        xz.x[j] = T(m.htab[0][j]);  // the same conversion as the device tables'
        xz.z[j] = T(m.htab[2][j]);
      }
      auto k = apply_uniform_kernel<T, S, P, CHEB, false, true>;
      if constexpr (P >= 5) {
        if (m.eo_xz) k = apply_uniform_kernel<T, S, P, CHEB, true, true>;
      }
      if (big) {
        const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
      }
      k<<<grid, threads, smem, s>>>(g, x, y, cpb, mass_rel, scale, do_scale, do_mass, ds, epi, xz);
      return cudaGetLastError();
    }
  }
  auto k = apply_uniform_kernel<T, S, P, CHEB, false, false>;
  if constexpr (P >= 5) {
    if (m.eo_xz) k = apply_uniform_kernel<T, S, P, CHEB, true, false>;
  }
  if (big) {
    const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k<<<grid, threads, smem, s>>>(g, x, y, cpb, mass_rel, scale, do_scale, do_mass, ds, epi, NoXZTab());
  return cudaGetLastError();
}

template <typename T, int P>
static int launch_apply_p(const Mesh& m, const T* x, T* y, int ncomp, T cm, T nu, const T* nu_cell, bool stiff,
                          const DotSink* sink, int* nblocks, cudaStream_t s) {
  const int prec = sizeof(T) == 8 ? 0 : 1;
  const bool uniform_ = stiff && nu_cell == nullptr;
  if constexpr (std::is_same<T, float>::value) {
    if (uniform_ && m.f32_mapping == 1 && (!sink || !sink->partials)) {
      // FP32 plane mapping: P threads per cell
      const int cpbp = cells_per_block(m, 1);
      const int thr = (cpbp * P + 31) / 32 * 32;
      const size_t smp = (size_t)3 * cpbp * P * P * P * sizeof(float);
      if (thr > kMaxCellThreads) return fail(SIPG_EINVAL, "cells per block too large for this degree");
      if (smp + 2048 > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(apply_plane_kernel<float, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smp);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(apply plane)");
      }
      const dim3 gridp((unsigned)((m.ncell + cpbp - 1) / cpbp), (unsigned)ncomp);
      apply_plane_kernel<float, P><<<gridp, thr, smp, s>>>(make_geo<float>(m), x, y, cpbp, cm / nu, nu,
                                                           nu != 1.f ? 1 : 0, cm != 0.f ? 1 : 0);
      if (nblocks) *nblocks = (int)(gridp.x * gridp.y);
      const_cast<Mesh&>(m).launches++;
      cudaError_t e = cudaGetLastError();
      return e == cudaSuccess ? SIPG_OK : cuda_fail(e, "apply kernel launch");
    }
  }
  const int cpb = m.f32_mapping == 1 && prec == 1 ? default_cpb(P, prec) : cells_per_block(m, prec);
  const Geo<T> g = make_geo<T>(m);
  const dim3 grid((unsigned)((m.ncell + cpb - 1) / cpb), (unsigned)ncomp);
  const int threads = (cpb * P * P + 31) / 32 * 32;  // whole warps (the block reduction shuffles full warps)
  const bool uniform = stiff && nu_cell == nullptr;
  const size_t smem = uniform ? uniform_smem_bytes<T, P>(cpb) : (size_t)3 * cpb * P * P * P * sizeof(T);
  if (threads > kMaxCellThreads) return fail(SIPG_EINVAL, "cells per block too large for this degree");
  const DotSink ds = sink ? *sink : DotSink();
  if (!uniform && smem + 2048 > 48 * 1024) {  // dynamic + static shared memory above the default limit
    cudaError_t e = cudaFuncSetAttribute(apply_kernel<T, T, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(apply)");
  }
  if (uniform) {
    // y = nu (L x + (mass_coef / nu) M x)
    const int do_scale = nu != T(1) ? 1 : 0, do_mass = cm != T(0) ? 1 : 0;
    if constexpr (std::is_same<T, double>::value) {
      if (m.f64_arith == SIPG_F64_DOUBLE_FLOAT) {
        if (!df_coef_ok(cm / nu) || !df_coef_ok(nu))
          return fail(SIPG_EINVAL, "double-float arithmetic needs mass_coef / nu and nu in [2^-100, 2^100]");
        if (!ds.prescaled) {
          const int st = launch_df_scale(m, x, m.ncell * P * P * P * ncomp, nullptr, 0, ds.skip, s);
          if (st) return st;
        }
        const Geo<dfl> gd = make_geo<dfl>(m);
        const cudaError_t e = launch_uniform<dfl, double, P, false>(m, grid, threads, smem, s, gd, x, y, cpb,
                                                                    dfl(cm / nu), dfl(nu), do_scale, do_mass, ds,
                                                                    ChebEpi());
        if (nblocks) *nblocks = (int)(grid.x * grid.y);
        const_cast<Mesh&>(m).launches++;
        return e == cudaSuccess ? SIPG_OK : cuda_fail(e, "apply kernel launch");
      }
    }
    const cudaError_t e = launch_uniform<T, T, P, false>(m, grid, threads, smem, s, g, x, y, cpb, cm / nu, nu,
                                                         do_scale, do_mass, ds, ChebEpi());
    if (nblocks) *nblocks = (int)(grid.x * grid.y);
    const_cast<Mesh&>(m).launches++;
    return e == cudaSuccess ? SIPG_OK : cuda_fail(e, "apply kernel launch");
  } else {
    if constexpr (std::is_same<T, double>::value) {
      if (m.f64_arith == SIPG_F64_DOUBLE_FLOAT) {
        if (!df_coef_ok(cm) || !df_coef_ok(nu))
          return fail(SIPG_EINVAL, "double-float arithmetic needs mass_coef and nu in [2^-100, 2^100]");
        if (!ds.prescaled) {
          const int st = launch_df_scale(m, x, m.ncell * P * P * P * ncomp, nullptr, 0, ds.skip, s);
          if (st) return st;
        }
        if (smem + 2048 > 48 * 1024) {
          cudaError_t e = cudaFuncSetAttribute(apply_kernel<dfl, double, P>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
          if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(apply)");
        }
        apply_kernel<dfl, double, P><<<grid, threads, smem, s>>>(make_geo<dfl>(m), x, y, cpb, dfl(cm), dfl(nu),
                                                                 nu_cell, stiff ? 1 : 0, ds);
        if (nblocks) *nblocks = (int)(grid.x * grid.y);
        const_cast<Mesh&>(m).launches++;
        cudaError_t e = cudaGetLastError();
        return e == cudaSuccess ? SIPG_OK : cuda_fail(e, "apply kernel launch");
      }
    }
    apply_kernel<T, T, P><<<grid, threads, smem, s>>>(g, x, y, cpb, cm, nu, nu_cell, stiff ? 1 : 0, ds);
  }
  if (nblocks) *nblocks = (int)(grid.x * grid.y);
  const_cast<Mesh&>(m).launches++;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SIPG_OK : cuda_fail(e, "apply kernel launch");
}

template <typename T>
static int launch_apply_dispatch(const Mesh& m, const T* x, T* y, int ncomp, T cm, T nu, const T* nu_cell, bool stiff,
                                 const DotSink* sink, int* nblocks, cudaStream_t s) {
  switch (m.p) {
    case 2: return launch_apply_p<T, 2>(m, x, y, ncomp, cm, nu, nu_cell, stiff, sink, nblocks, s);
    case 3: return launch_apply_p<T, 3>(m, x, y, ncomp, cm, nu, nu_cell, stiff, sink, nblocks, s);
    case 4: return launch_apply_p<T, 4>(m, x, y, ncomp, cm, nu, nu_cell, stiff, sink, nblocks, s);
    case 5: return launch_apply_p<T, 5>(m, x, y, ncomp, cm, nu, nu_cell, stiff, sink, nblocks, s);
    case 6: return launch_apply_p<T, 6>(m, x, y, ncomp, cm, nu, nu_cell, stiff, sink, nblocks, s);
    case 7: return launch_apply_p<T, 7>(m, x, y, ncomp, cm, nu, nu_cell, stiff, sink, nblocks, s);
    case 8: return launch_apply_p<T, 8>(m, x, y, ncomp, cm, nu, nu_cell, stiff, sink, nblocks, s);
    default: return fail(SIPG_EINVAL, "unsupported degree");
  }
}

}  // namespace sipg
