// Adjoint gradient with respect to a per-cell viscosity (FP64).
//
// For A(nu) = c M + L(nu) (Sec. 3.2 (iii) in Laplace form, per-cell nu):
//   grad_e = - lambda^T (dA/dnu_e) u
//          = - [ lambda_e^T K_e u_e                              (cell, unit nu)
//                + sum over the faces F of e of
//                  int_F -1/2 d_n u_e [lambda] - 1/2 d_n lambda_e [u]
//                        + tau_F w_e [u][lambda]                  (interior)
//                  int_F -d_n u_e lambda_e - d_n lambda_e u_e
//                        + 2 tau_e u_e lambda_e                   (Dirichlet) ]
// with n the outward normal of e, [w] = w_e - w_neighbour, and w_e = 1 when
// nu_e > nu_neighbour (nu_e is the max of Eq. (tau)'s nu_F), 1/2 on a tie, 0
// otherwise.  Face integrals of face-nodal fields f, g are f^T (M_t1 x M_t2) g
// with the cell's transverse 1D mass matrices, so each face costs two
// transverse contractions; the cell term reuses the sum-factorised stiffness
// evaluation of the operator kernel.  Per-cell sums are reduced in a fixed
// order (deterministic).
#pragma once

#include "apply.cuh"

namespace sipg {

template <int P>
__global__ void __launch_bounds__(kMaxCellThreads) adjoint_kernel(Geo<double> g, const double* __restrict__ nu_cell,
                                                                  const double* __restrict__ u,
                                                                  const double* __restrict__ lam,
                                                                  double* __restrict__ grad, int cpb) {
  constexpr int P2 = P * P, P3 = P * P * P;
  using O = LayerOff<P>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* su = reinterpret_cast<double*>(smem_raw);
  double* s1 = su + cpb * P3;
  double* s2 = s1 + cpb * P3;
  double* fa = s2 + cpb * P3;    // [cpb][8][P2] face arrays
  double* part = fa + cpb * 8 * P2;  // [blockDim] per-thread partial sums
  const int cs = threadIdx.x / P2;
  const int t = threadIdx.x - cs * P2;
  const int ti = t % P, tj = t / P;
  const long long cell0 = (long long)blockIdx.x * cpb;
  const int e = (int)(cell0 + cs);
  const bool active = cs < cpb && e < g.ncell;
  {
    const int nc = (int)min((long long)cpb, (long long)g.ncell - cell0);
    const double* xb = u + cell0 * P3;
    for (int idx = threadIdx.x; idx < nc * P3; idx += blockDim.x) su[idx] = xb[idx];
  }
  __syncthreads();
  double* us = su + cs * P3;
  double* w1 = s1 + cs * P3;
  double* w2 = s2 + cs * P3;
  double* f = fa + cs * 8 * P2;
  int id[3] = {0, 0, 0};
  double nue = 1.0, tau_e = 0.0;
  if (active) {
    id[0] = e % g.n[0];
    id[1] = (e / g.n[0]) % g.n[1];
    id[2] = e / (g.n[0] * g.n[1]);
    nue = nu_cell[e];
    tau_e = g.tau_scale * (g.tab[0][id[0] * O::stride + O::t] + g.tab[1][id[1] * O::stride + O::t] +
                           g.tab[2][id[2] * O::stride + O::t]);
  }
  const double* __restrict__ lc = lam + (long long)e * P3;
  double acc = 0.0;
  // ------------------------------------------------------------ face terms
  for (int dir = 0; dir < 3; ++dir) {
    double cA[2] = {0.0, 0.0}, cP[2] = {0.0, 0.0};
    if (active) {
      int start, step;
      line_geom<P>(dir, ti, tj, start, step);
      DirCtx<double, P> c = dir_ctx<double, P>(g, dir, id, e, nue, tau_e, nu_cell, 0.0);
      double uu[P], ll[P], un[P], ln[P];
      load_line<double, P>(uu, us, start, step);
      load_line_global<double, P>(ll, lc, start, step);
      // face 0: high side (outward normal +dir), face 1: low side (outward -dir)
      for (int side = 0; side < 2; ++side) {
        const int kind = side == 0 ? c.kindR : c.kindL;
        const double* dv = c.L + (side == 0 ? O::dR : O::dL);
        const double sgn = side == 0 ? 1.0 : -1.0;
        const int own = side == 0 ? P - 1 : 0, oth = side == 0 ? 0 : P - 1;
        double Du = 0.0, Dl = 0.0, Ju = 0.0, Jl = 0.0;
        if (kind == 0 || kind == SIPG_BC_DIRICHLET) {
#pragma unroll
          for (int a = 0; a < P; ++a) {
            Du = fma(dv[a], uu[a], Du);
            Dl = fma(dv[a], ll[a], Dl);
          }
          Du *= sgn;
          Dl *= sgn;
          Ju = uu[own];
          Jl = ll[own];
        }
        if (kind == 0) {
          const int nb = side == 0 ? c.nbR : c.nbL;
          load_line_global<double, P>(un, u + (long long)nb * P3, start, step);
          load_line_global<double, P>(ln, lam + (long long)nb * P3, start, step);
          Ju -= un[oth];
          Jl -= ln[oth];
          const double nun = side == 0 ? c.nuR : c.nuL;
          const double wgt = nue > nun ? 1.0 : (nue == nun ? 0.5 : 0.0);
          cA[side] = -0.5;
          cP[side] = (side == 0 ? c.tauFR : c.tauFL) * wgt;
        } else if (kind == SIPG_BC_DIRICHLET) {
          cA[side] = -1.0;
          cP[side] = 2.0 * tau_e;
        }
        double* fs = f + side * 4 * P2;
        fs[0 * P2 + t] = Du;
        fs[1 * P2 + t] = Dl;
        fs[2 * P2 + t] = Ju;
        fs[3 * P2 + t] = Jl;
      }
    }
    __syncthreads();
    if (active) {
      const int d1 = dir == 0 ? 1 : 0, d2 = dir == 2 ? 1 : 2;
      const double* M1 = g.tab[d1] + id[d1] * O::stride + O::M;
      const double* M2 = g.tab[d2] + id[d2] * O::stride + O::M;
      for (int side = 0; side < 2; ++side) {
        if (cA[side] == 0.0 && cP[side] == 0.0) continue;
        const double* fs = f + side * 4 * P2;
        double TJu = 0.0, TJl = 0.0;
        for (int t2 = 0; t2 < P; ++t2) {
          double su_ = 0.0, sl_ = 0.0;
#pragma unroll
          for (int t1 = 0; t1 < P; ++t1) {
            su_ = fma(M1[ti * P + t1], fs[2 * P2 + t2 * P + t1], su_);
            sl_ = fma(M1[ti * P + t1], fs[3 * P2 + t2 * P + t1], sl_);
          }
          TJu = fma(M2[tj * P + t2], su_, TJu);
          TJl = fma(M2[tj * P + t2], sl_, TJl);
        }
        acc += cA[side] * (fs[0 * P2 + t] * TJl + fs[1 * P2 + t] * TJu) + cP[side] * fs[2 * P2 + t] * TJl;
      }
    }
    __syncthreads();
  }
  // ---------------------------------------------- cell term lambda^T K_e u
  double zero[P];
#pragma unroll
  for (int a = 0; a < P; ++a) zero[a] = 0.0;
  if (active) {
    for (int dir = 0; dir < 2; ++dir) {
      int start, step;
      line_geom<P>(dir, ti, tj, start, step);
      const double* L = g.tab[dir] + id[dir] * O::stride;
      double uu[P], w[P];
      load_line<double, P>(uu, us, start, step);
      line_op<double, P>(w, uu, L, 1.0, true, 0.0, false, SIPG_BC_NEUMANN, zero, L, 0.0, 0.0, SIPG_BC_NEUMANN, zero,
                         L, 0.0, 0.0, 0.0);
      store_line<double, P>(dir == 0 ? w1 : w2, w, start, step);
    }
  }
  __syncthreads();
  if (active) {
    int start, step;
    line_geom<P>(2, ti, tj, start, step);
    const double* L = g.tab[2] + id[2] * O::stride;
    double uu[P], w[P], v1[P], v2[P], a1[P], a2[P];
    load_line<double, P>(uu, us, start, step);
    line_op<double, P>(w, uu, L, 1.0, true, 0.0, false, SIPG_BC_NEUMANN, zero, L, 0.0, 0.0, SIPG_BC_NEUMANN, zero, L,
                       0.0, 0.0, 0.0);
    load_line<double, P>(v1, w1, start, step);
    load_line<double, P>(v2, w2, start, step);
    matvec(a1, L + O::M, v1);
    matvec(a2, L + O::M, v2);
    store_line<double, P>(us, w, start, step);
    store_line<double, P>(w1, a1, start, step);
    store_line<double, P>(w2, a2, start, step);
  }
  __syncthreads();
  if (active) {
    int start, step;
    line_geom<P>(1, ti, tj, start, step);
    const double* My = g.tab[1] + id[1] * O::stride + O::M;
    double v[P], r1[P], r2[P], a2[P];
    load_line<double, P>(v, w1, start, step);
    matvec(r1, My, v);
    load_line<double, P>(v, us, start, step);
    matvec(r2, My, v);
    load_line<double, P>(a2, w2, start, step);
#pragma unroll
    for (int a = 0; a < P; ++a) r2[a] += a2[a];
    store_line<double, P>(w1, r1, start, step);
    store_line<double, P>(w2, r2, start, step);
  }
  __syncthreads();
  if (active) {
    int start, step;
    line_geom<P>(0, ti, tj, start, step);
    const double* Mx = g.tab[0] + id[0] * O::stride + O::M;
    double v[P], out[P], r1[P], ll[P];
    load_line<double, P>(v, w2, start, step);
    matvec(out, Mx, v);
    load_line<double, P>(r1, w1, start, step);
    load_line_global<double, P>(ll, lc, start, step);
#pragma unroll
    for (int a = 0; a < P; ++a) acc = fma(out[a] + r1[a], ll[a], acc);
  }
  part[threadIdx.x] = acc;
  __syncthreads();
  if (active && t == 0) {
    double s = 0.0;
    for (int i = 0; i < P2; ++i) s += part[cs * P2 + i];
    grad[e] = -s;
  }
}

}  // namespace sipg
