// Matrix-free SIPG kernels for sm_103a (templated on the scalar type and on
// p = k+1).
//
// Operator (Sec. 3.2 (ii)/(iii), Sec. 5).  For a separable iso-parametric map
// the Jacobian is diagonal and depends on one reference coordinate per
// direction, so every cell and face integral of the SIPG form factorises into
// 1D matrices (M: mass, K: stiffness, per direction and layer).  Sum
// factorisation then applies the operator of one cell e as
//
//   y_e = (I x My x Mz) w_x + (Mx x I x Mz) w_y + (Mx x My x I) w_z
//
// where w_d is a 1D operator along direction d acting on every line of the
// cell: nu_e K_d u plus the two face terms of Sec. 3.2 (ii) in that direction
// (jump and average with the neighbour's line, penalty tau_F nu_F with tau of
// Eq. (taue)/(tau)), and for the Helmholtz operator w_z also carries the mass
// term mass_coef Mz u.  The transverse mass matrices of a face are the cell's
// own 1D mass matrices (the face quadrature is the cell quadrature restricted
// to the face), which is why the face terms enter w_d before the transverse
// contractions.  Evaluation order per cell (lines owned by one thread each):
//   X: w_x (x-lines)              Y: w_y (y-lines)
//   Z: w_z, A1 = Mz w_x, A2 = Mz w_y (z-lines)
//   Y2: R1 = My A1, R2 = My w_z + A2 (y-lines)
//   X2: y = Mx R2 + R1 (x-lines) -> global
// 8 contractions of p FMAs per DoF plus the face terms.  Faces are handled
// cell-centrically: every cell reads its six neighbours' lines and writes only
// its own outputs, so there are no atomics and the result is deterministic.
#pragma once

#include <type_traits>

#include "dfloat.cuh"
#include "sipg_internal.h"

namespace sipg {

// storage <-> compute conversions (identity unless FP64 data is computed in
// double-float).  sc is the call's scale exponent: data enter as v 2^-sc and
// leave as v 2^sc (a product of two scaled data leaves with 2 sc);
// coefficients and geometry convert unscaled (sc = 0).
template <typename T, typename S>
__device__ __forceinline__ T cvt_in(S v, int sc = 0) {
  return (T)v;
}
template <>
__device__ __forceinline__ dfl cvt_in<dfl, double>(double v, int sc) {
  return df_from_double(v, sc);
}
template <typename S, typename T>
__device__ __forceinline__ S cvt_out(T v, int sc = 0) {
  return (S)v;
}
template <>
__device__ __forceinline__ double cvt_out<double, dfl>(dfl v, int sc) {
  return df_to_double(v, sc);
}

// the call's scale exponent (double-float kernels only)
template <typename T>
__device__ __forceinline__ int call_scale(const Geo<T>& g) {
  if constexpr (std::is_same<T, dfl>::value)
    return g.dsc ? *g.dsc : 0;
  else
    return 0;
}

template <int P>
struct LayerOff {
  static constexpr int RM = (P * P + 3) / 4 * 4, RV = (P + 3) / 4 * 4;  // padded block sizes (lmat, lvec)
  static constexpr int M = 0, K = RM, Mi = 2 * RM, Kc = 3 * RM, dL = 4 * RM, dR = 4 * RM + RV, dLh = 4 * RM + 2 * RV,
                       dRh = 4 * RM + 3 * RV, h = 4 * RM + 4 * RV, t = 4 * RM + 4 * RV + 1, ts = 4 * RM + 4 * RV + 2,
                       dTL = 4 * RM + 4 * RV + 3, dTR = 4 * RM + 4 * RV + 4, Qc = 4 * RM + 4 * RV + 8,
                       mL = 5 * RM + 4 * RV + 8, mR = 5 * RM + 5 * RV + 8, qL = 5 * RM + 6 * RV + 8,
                       qR = 5 * RM + 7 * RV + 8, cs = 4 * RM + 4 * RV + 5, EQc = 5 * RM + 8 * RV + 8,
                       EKc = 6 * RM + 8 * RV + 8, EM = 7 * RM + 8 * RV + 8, stride = 8 * RM + 8 * RV + 8;
};

// Neighbour across side (0 = low, 1 = high) of direction dir.  kind: 0 interior
// (or periodic), SIPG_BC_DIRICHLET, SIPG_BC_NEUMANN.
template <typename T>
__device__ __forceinline__ void face_neighbor(const Geo<T>& g, int dir, int side, int id, int e, int& nb, int& kind,
                                              int& jlayer) {
  const int n = g.n[dir];
  int j = id + (side ? 1 : -1);
  const int bc = side ? g.bc_hi[dir] : g.bc_lo[dir];
  kind = 0;
  if (j < 0 || j >= n) {
    if (bc == SIPG_BC_PERIODIC) {
      j = (j + n) % n;
    } else {
      kind = bc;
      nb = -1;
      jlayer = -1;
      return;
    }
  }
  const int stride = dir == 0 ? 1 : (dir == 1 ? g.n[0] : g.n[0] * g.n[1]);
  nb = e + (j - id) * stride;
  jlayer = j;
}

// The 1D operator of one line along one direction: nu_e K u + face terms
// (+ cm Mm u when mass is true).  uL / uR are the neighbours' lines at the same
// transverse position, LL / LR their layer tables.
template <typename T, int P>
__device__ __forceinline__ void line_op(T (&w)[P], const T (&u)[P], const T* __restrict__ L, T nue, bool stiffness,
                                        T cm, bool mass, int kindL, const T (&uL)[P], const T* __restrict__ LL,
                                        T nuL, T tauFL, int kindR, const T (&uR)[P], const T* __restrict__ LR, T nuR,
                                        T tauFR, T tau_e) {
  using O = LayerOff<P>;
#pragma unroll
  for (int a = 0; a < P; ++a) w[a] = T(0);
  if (stiffness) {
#pragma unroll
    for (int a = 0; a < P; ++a) {
      T s = T(0);
#pragma unroll
      for (int b = 0; b < P; ++b) s = fma(L[O::K + a * P + b], u[b], s);
      w[a] = nue * s;
    }
    // high face: this cell is the "-" side, n points out of it
    if (kindR == 0) {
      T gO = T(0), gN = T(0);
#pragma unroll
      for (int a = 0; a < P; ++a) {
        gO = fma(L[O::dR + a], u[a], gO);
        gN = fma(LR[O::dL + a], uR[a], gN);
      }
      const T J = u[P - 1] - uR[0];
      const T avg = T(0.5) * (nue * gO + nuR * gN);
      const T tn = tauFR * (nue > nuR ? nue : nuR);
      w[P - 1] += tn * J - avg;
      const T c = T(-0.5) * nue * J;
#pragma unroll
      for (int a = 0; a < P; ++a) w[a] = fma(c, L[O::dR + a], w[a]);
    } else if (kindR == SIPG_BC_DIRICHLET) {
      T gO = T(0);
#pragma unroll
      for (int a = 0; a < P; ++a) gO = fma(L[O::dR + a], u[a], gO);
      w[P - 1] += T(2) * tau_e * nue * u[P - 1] - nue * gO;
      const T c = -nue * u[P - 1];
#pragma unroll
      for (int a = 0; a < P; ++a) w[a] = fma(c, L[O::dR + a], w[a]);
    }
    // low face: this cell is the "+" side, n points into it
    if (kindL == 0) {
      T gO = T(0), gN = T(0);
#pragma unroll
      for (int a = 0; a < P; ++a) {
        gO = fma(L[O::dL + a], u[a], gO);
        gN = fma(LL[O::dR + a], uL[a], gN);
      }
      const T J = uL[P - 1] - u[0];
      const T avg = T(0.5) * (nuL * gN + nue * gO);
      const T tn = tauFL * (nue > nuL ? nue : nuL);
      w[0] += avg - tn * J;
      const T c = T(-0.5) * nue * J;
#pragma unroll
      for (int a = 0; a < P; ++a) w[a] = fma(c, L[O::dL + a], w[a]);
    } else if (kindL == SIPG_BC_DIRICHLET) {
      T gO = T(0);
#pragma unroll
      for (int a = 0; a < P; ++a) gO = fma(L[O::dL + a], u[a], gO);
      w[0] += nue * gO + T(2) * tau_e * nue * u[0];
      const T c = nue * u[0];
#pragma unroll
      for (int a = 0; a < P; ++a) w[a] = fma(c, L[O::dL + a], w[a]);
    }
  }
  if (mass) {
#pragma unroll
    for (int a = 0; a < P; ++a) {
      T s = T(0);
#pragma unroll
      for (int b = 0; b < P; ++b) s = fma(L[O::M + a * P + b], u[b], s);
      w[a] = fma(cm, s, w[a]);
    }
  }
}

// y[a] = sum_b A[a][b] v[b]
template <typename T, int P>
__device__ __forceinline__ void matvec(T (&out)[P], const T* __restrict__ A, const T (&v)[P]) {
#pragma unroll
  for (int a = 0; a < P; ++a) {
    T s = T(0);
#pragma unroll
    for (int b = 0; b < P; ++b) s = fma(A[a * P + b], v[b], s);
    out[a] = s;
  }
}

// sum_b a[b] v[b]
template <typename T, int P>
__device__ __forceinline__ T dotp(const T* __restrict__ a, const T (&v)[P]) {
  T s = T(0);
#pragma unroll
  for (int b = 0; b < P; ++b) s = fma(a[b], v[b], s);
  return s;
}
template <int P>
__device__ __forceinline__ dfl dotp(const dfl* __restrict__ a, const dfl (&v)[P]) {
  return df_dot<P>(a, v);
}

// double-float contraction: one lazily renormalised dot product per output
template <int P>
__device__ __forceinline__ void matvec(dfl (&out)[P], const dfl* __restrict__ A, const dfl (&v)[P]) {
#pragma unroll
  for (int a = 0; a < P; ++a) out[a] = df_dot<P>(A + a * P, v);
}

// FP32 versions reading the 16-byte aligned table blocks with 128-bit loads
// (four entries per load instruction); the FMAs run in the same order as the
// generic versions, so the results are identical.
template <int P>
__device__ __forceinline__ void matvec(float (&out)[P], const float* __restrict__ A, const float (&v)[P]) {
  constexpr int N4 = (P * P + 3) / 4;
  const float4* __restrict__ A4 = reinterpret_cast<const float4*>(A);
#pragma unroll
  for (int a = 0; a < P; ++a) out[a] = 0.f;
#pragma unroll
  for (int q = 0; q < N4; ++q) {
    const float4 f = A4[q];
    const float e[4] = {f.x, f.y, f.z, f.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int k = 4 * q + j;
      if (k < P * P) out[k / P] = fmaf(e[j], v[k % P], out[k / P]);
    }
  }
}

template <int P>
__device__ __forceinline__ float dotp(const float* __restrict__ a, const float (&v)[P]) {
  constexpr int N4 = (P + 3) / 4;
  const float4* __restrict__ a4 = reinterpret_cast<const float4*>(a);
  float s = 0.f;
#pragma unroll
  for (int q = 0; q < N4; ++q) {
    const float4 f = a4[q];
    const float e[4] = {f.x, f.y, f.z, f.w};
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (4 * q + j < P) s = fmaf(e[j], v[4 * q + j], s);
  }
  return s;
}

// sum_b a[b] v[b] with scalar loads of a (no alignment assumed)
template <typename T, int N>
__device__ __forceinline__ T dot_s(const T* __restrict__ a, const T (&v)[N]) {
  if constexpr (std::is_same<T, dfl>::value) {
    return df_dot<N>(a, v);
  } else {
    T s = T(0);
#pragma unroll
    for (int b = 0; b < N; ++b) s = fma(a[b], v[b], s);
    return s;
  }
}

// out = A v for a centrosymmetric A in the even-odd form packed by the table
// builder (E: h x (h + odd), O: h x h, Z: h + 1 for odd p; h = p / 2): with
// e_b = v_b + v_(p-1-b), o_b = v_b - v_(p-1-b), s_a = E_a . (e, v_h) and
// d_a = O_a . o, out_a = s_a + d_a, out_(p-1-a) = s_a - d_a, out_h = Z . (e, v_h).
template <typename T, int P>
__device__ __forceinline__ void matvec_eo(T (&out)[P], const T* __restrict__ E, const T (&v)[P]) {
  constexpr int H = P / 2, OD = P & 1, EW = H + OD;
  const T* __restrict__ Oo = E + H * EW;
  T ev[EW], o[H];
#pragma unroll
  for (int b = 0; b < H; ++b) {
    ev[b] = v[b] + v[P - 1 - b];
    o[b] = v[b] - v[P - 1 - b];
  }
  if constexpr (OD) ev[H] = v[H];
#pragma unroll
  for (int a = 0; a < H; ++a) {
    const T s = dot_s<T, EW>(E + a * EW, ev), d = dot_s<T, H>(Oo + a * H, o);
    out[a] = s + d;
    out[P - 1 - a] = s - d;
  }
  if constexpr (OD) out[H] = dot_s<T, EW>(Oo + H * H, ev);
}

// out = A v with the layer's matrix at offset `plain`, or its even-odd form at
// offset `eo_off` when the layer is centrosymmetric (p >= 5)
template <typename T, int P>
__device__ __forceinline__ void matvec_l(T (&out)[P], const T* __restrict__ L, int plain, int eo_off, bool eo,
                                         const T (&v)[P]) {
  if constexpr (P >= 5) {
    if (eo) {
      matvec_eo<T, P>(out, L + eo_off, v);
      return;
    }
  }
  matvec(out, L + plain, v);
}

// w += c * (table vector block d): FP32 reads the block with 128-bit loads,
// the other types stream it entry by entry (fewer live registers)
template <typename T, int P>
__device__ __forceinline__ void axpy_vec(T (&w)[P], const T* __restrict__ d, T c) {
#pragma unroll
  for (int a = 0; a < P; ++a) w[a] = fma(d[a], c, w[a]);
}
template <int P>
__device__ __forceinline__ void load_vec(float (&out)[P], const float* __restrict__ src) {
  constexpr int N4 = (P + 3) / 4;
  const float4* __restrict__ s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
  for (int q = 0; q < N4; ++q) {
    const float4 f = s4[q];
    const float e[4] = {f.x, f.y, f.z, f.w};
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (4 * q + j < P) out[4 * q + j] = e[j];
  }
}
template <int P>
__device__ __forceinline__ void axpy_vec(float (&w)[P], const float* __restrict__ d, float c) {
  float dv[P];
  load_vec(dv, d);
#pragma unroll
  for (int a = 0; a < P; ++a) w[a] = fmaf(dv[a], c, w[a]);
}

// Index of element (a, b, c) inside one cell.
template <int P>
__device__ __forceinline__ int nidx(int a, int b, int c) {
  return (c * P + b) * P + a;
}

// Stride between consecutive line entries and line start for direction dir and
// transverse thread coordinates (ti, tj): x-line (b=ti, c=tj), y-line (a=ti,
// c=tj), z-line (a=ti, b=tj).
template <int P>
__device__ __forceinline__ void line_geom(int dir, int ti, int tj, int& start, int& step) {
  if (dir == 0) {
    start = nidx<P>(0, ti, tj);
    step = 1;
  } else if (dir == 1) {
    start = nidx<P>(ti, 0, tj);
    step = P;
  } else {
    start = nidx<P>(ti, tj, 0);
    step = P * P;
  }
}

template <typename T, int P>
__device__ __forceinline__ void load_line(T (&v)[P], const T* __restrict__ base, int start, int step) {
#pragma unroll
  for (int a = 0; a < P; ++a) v[a] = base[start + a * step];
}

template <typename T, int P>
__device__ __forceinline__ void load_line_global(T (&v)[P], const T* __restrict__ base, int start, int step) {
#pragma unroll
  for (int a = 0; a < P; ++a) v[a] = __ldg(base + start + a * step);
}

template <typename T, typename S, int P>
__device__ __forceinline__ void load_line_global_cvt(T (&v)[P], const S* __restrict__ base, int start, int step,
                                                     int sc) {
  S r[P];  // all loads issued before the conversions
#pragma unroll
  for (int a = 0; a < P; ++a) r[a] = __ldg(base + start + a * step);
#pragma unroll
  for (int a = 0; a < P; ++a) v[a] = cvt_in<T, S>(r[a], sc);
}

// dst[0..n) = src[0..n) converted to T, the whole block cooperating
// (consecutive threads take consecutive entries), each thread issuing four
// loads before it converts them
template <typename T, typename S>
__device__ __forceinline__ void stage_cvt(T* __restrict__ dst, const S* __restrict__ src, int n, int sc) {
  const int bd = blockDim.x;
  for (int i = threadIdx.x; i < n; i += 4 * bd) {
    S r[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) r[j] = i + j * bd < n ? __ldg(src + i + j * bd) : S(0);
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (i + j * bd < n) dst[i + j * bd] = cvt_in<T, S>(r[j], sc);
  }
}

template <typename T, int P>
__device__ __forceinline__ void store_line(T* base, const T (&v)[P], int start, int step) {
#pragma unroll
  for (int a = 0; a < P; ++a) base[start + a * step] = v[a];
}

// Block reduction of NV doubles (the others of the three written as 0);
// thread 0 writes out[0..2].  Every add is an FP64 instruction, which costs
// as much as a multiply-add of the operator on this GPU, so only the values
// in use are reduced, and the second level covers only the block's warps.
template <int NV>
__device__ __forceinline__ void block_reduce_n(double a, double b, double c, double* out) {
  __shared__ double red[3][32];
  double v[3] = {a, b, c};
  __syncthreads();  // a previous call may still read red
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) red[k][wid] = v[k];
  __syncthreads();
  if (wid == 0) {
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = lane < nw ? red[k][lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      if (o < nw) {  // uniform across the warp
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
      }
    }
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < 3; ++k) out[k] = k < NV ? v[k] : 0.0;
    }
  }
}
__device__ __forceinline__ void block_reduce3(double a, double b, double c, double* out) {
  block_reduce_n<3>(a, b, c, out);
}

// Partial sums of one block to the sink; the last block of the grid adds all
// partials (fixed order, deterministic) into sink.totals.  Called by every
// thread of the block.
__device__ __forceinline__ void sink_dots(const DotSink& s, double a, double b, double c) {
  const unsigned nb = gridDim.x * gridDim.y;
  const unsigned bid = blockIdx.y * gridDim.x + blockIdx.x;
  if (s.sums)
    block_reduce_n<3>(a, b, c, s.partials + 3 * (long long)bid);
  else
    block_reduce_n<1>(a, b, c, s.partials + 3 * (long long)bid);
  if (!s.counter) return;
  __shared__ int last;
  if (threadIdx.x == 0) {
    __threadfence();  // this block's partial is visible before the count
    last = atomicAdd(s.counter, 1u) == nb - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // several loads in flight per thread (this tail runs on one block only);
  // without the zero-mean sums only x.y is read
  double x = 0.0, y = 0.0, z = 0.0;
  if (s.sums) {
#pragma unroll 4
    for (unsigned i = threadIdx.x; i < nb; i += blockDim.x) {
      x += __ldcg(s.partials + 3 * i);
      y += __ldcg(s.partials + 3 * i + 1);
      z += __ldcg(s.partials + 3 * i + 2);
    }
  } else {
#pragma unroll 8
    for (unsigned i = threadIdx.x; i < nb; i += blockDim.x) x += __ldcg(s.partials + 3 * i);
  }
  double t[3];
  if (s.sums)  // thread 0 holds the totals
    block_reduce_n<3>(x, y, z, t);
  else
    block_reduce_n<1>(x, y, z, t);
  if (threadIdx.x == 0) {
    s.totals[0] = t[0];
    s.totals[1] = t[1];
    s.totals[2] = t[2];
    *s.counter = 0u;
  }
}

// Per-direction data of one line operator for cell e.
template <typename T, int P>
struct DirCtx {
  const T* L;
  const T* LL;
  const T* LR;
  int kindL, kindR, nbL, nbR;
  T nuL, nuR, tauFL, tauFR;
};

template <typename T, int P, typename S>
__device__ __forceinline__ DirCtx<T, P> dir_ctx(const Geo<T>& g, int dir, const int (&id)[3], int e, T nue, T tau_e,
                                                const S* __restrict__ nu_cell, T nu) {
  using O = LayerOff<P>;
  DirCtx<T, P> c;
  c.L = g.tab[dir] + id[dir] * O::stride;
  const T t_own = c.L[O::t];
  int jl, jr;
  face_neighbor(g, dir, 0, id[dir], e, c.nbL, c.kindL, jl);
  face_neighbor(g, dir, 1, id[dir], e, c.nbR, c.kindR, jr);
  c.LL = c.L;
  c.LR = c.L;
  c.nuL = c.nuR = nue;
  c.tauFL = c.tauFR = tau_e;
  if (c.kindL == 0) {
    c.LL = g.tab[dir] + jl * O::stride;
    c.nuL = nu_cell ? cvt_in<T, S>(__ldg(nu_cell + c.nbL)) : nu;
    const T tn = tau_e + g.tau_scale * (c.LL[O::t] - t_own);
    c.tauFL = tn > tau_e ? tn : tau_e;
  }
  if (c.kindR == 0) {
    c.LR = g.tab[dir] + jr * O::stride;
    c.nuR = nu_cell ? cvt_in<T, S>(__ldg(nu_cell + c.nbR)) : nu;
    const T tn = tau_e + g.tau_scale * (c.LR[O::t] - t_own);
    c.tauFR = tn > tau_e ? tn : tau_e;
  }
  return c;
}

// y = mass_coef M x + nu L x for CPB cells per block, p^2 threads per cell
// (per-cell viscosity or mass only).  T is the arithmetic, S the storage type
// of x, y and nu_cell.
template <typename T, typename S, int P>
__global__ void __launch_bounds__(kMaxCellThreads) apply_kernel(Geo<T> g, const S* __restrict__ x, S* __restrict__ y,
                                                                int cpb, T mass_coef, T nu,
                                                                const S* __restrict__ nu_cell, int stiffness,
                                                                DotSink sink) {
  if (sink.skip && *sink.skip) return;
  double* dots = sink.partials;
  constexpr int P2 = P * P, P3 = P * P * P;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* su = reinterpret_cast<T*>(smem_raw);
  T* s1 = su + cpb * P3;
  T* s2 = s1 + cpb * P3;
  const int cs = threadIdx.x / P2;
  const int t = threadIdx.x - cs * P2;
  const int ti = t % P, tj = t / P;
  const long long cell0 = (long long)blockIdx.x * cpb;
  const int e = (int)(cell0 + cs);
  const bool active = cs < cpb && e < g.ncell;  // blocks are rounded up to whole warps
  const long long cbase = (long long)blockIdx.y * g.ncell * P3;
  const S* __restrict__ xc = x + cbase;
  const int sc = call_scale(g);
  {
    const int nc = (int)min((long long)cpb, (long long)g.ncell - cell0);
    const S* xb = xc + cell0 * P3;
    stage_cvt<T, S>(su, xb, nc * P3, sc);
  }
  __syncthreads();
  T* us = su + cs * P3;
  T* w1 = s1 + cs * P3;
  T* w2 = s2 + cs * P3;
  int id[3] = {0, 0, 0};
  T nue = nu, tau_e = T(0);
  const bool stiff = stiffness != 0;
  if (active) {
    id[0] = e % g.n[0];
    id[1] = (e / g.n[0]) % g.n[1];
    id[2] = e / (g.n[0] * g.n[1]);
    if (nu_cell) nue = cvt_in<T, S>(__ldg(nu_cell + e));
    using O = LayerOff<P>;
    tau_e = g.tau_scale * (g.tab[0][id[0] * O::stride + O::t] + g.tab[1][id[1] * O::stride + O::t] +
                           g.tab[2][id[2] * O::stride + O::t]);
  }
  T ux[P];  // this thread's x-line of x, kept for the dot products
  if (active) {
#pragma unroll
    for (int dir = 0; dir < 2; ++dir) {
      int start, step;
      line_geom<P>(dir, ti, tj, start, step);
      T u[P], uL[P], uR[P], w[P];
      load_line<T, P>(u, us, start, step);
      if (dir == 0) {
#pragma unroll
        for (int a = 0; a < P; ++a) ux[a] = u[a];
      }
      if (stiff) {
        DirCtx<T, P> c = dir_ctx<T, P, S>(g, dir, id, e, nue, tau_e, nu_cell, nu);
        if (c.kindL == 0) load_line_global_cvt<T, S, P>(uL, xc + (long long)c.nbL * P3, start, step, sc);
        if (c.kindR == 0) load_line_global_cvt<T, S, P>(uR, xc + (long long)c.nbR * P3, start, step, sc);
        line_op<T, P>(w, u, c.L, nue, true, T(0), false, c.kindL, uL, c.LL, c.nuL, c.tauFL, c.kindR, uR, c.LR, c.nuR,
                      c.tauFR, tau_e);
      } else {
#pragma unroll
        for (int a = 0; a < P; ++a) w[a] = T(0);
      }
      store_line<T, P>(dir == 0 ? w1 : w2, w, start, step);
    }
  }
  __syncthreads();
  if (active) {
    int start, step;
    line_geom<P>(2, ti, tj, start, step);
    T u[P], uL[P], uR[P], w[P], v1[P], v2[P], a1[P], a2[P];
    load_line<T, P>(u, us, start, step);
    DirCtx<T, P> c = dir_ctx<T, P, S>(g, 2, id, e, nue, tau_e, nu_cell, nu);
    if (stiff) {
      if (c.kindL == 0) load_line_global_cvt<T, S, P>(uL, xc + (long long)c.nbL * P3, start, step, sc);
      if (c.kindR == 0) load_line_global_cvt<T, S, P>(uR, xc + (long long)c.nbR * P3, start, step, sc);
    }
    line_op<T, P>(w, u, c.L, nue, stiff, mass_coef, mass_coef != T(0), c.kindL, uL, c.LL, c.nuL, c.tauFL, c.kindR, uR,
                  c.LR, c.nuR, c.tauFR, tau_e);
    load_line<T, P>(v1, w1, start, step);
    load_line<T, P>(v2, w2, start, step);
    matvec(a1, c.L + LayerOff<P>::M, v1);
    matvec(a2, c.L + LayerOff<P>::M, v2);
    store_line<T, P>(us, w, start, step);
    store_line<T, P>(w1, a1, start, step);
    store_line<T, P>(w2, a2, start, step);
  }
  __syncthreads();
  if (active) {
    int start, step;
    line_geom<P>(1, ti, tj, start, step);
    const T* My = g.tab[1] + id[1] * LayerOff<P>::stride + LayerOff<P>::M;
    T v[P], r1[P], r2[P], a2[P];
    load_line<T, P>(v, w1, start, step);
    matvec(r1, My, v);
    load_line<T, P>(v, us, start, step);
    matvec(r2, My, v);
    load_line<T, P>(a2, w2, start, step);
#pragma unroll
    for (int a = 0; a < P; ++a) r2[a] += a2[a];
    store_line<T, P>(w1, r1, start, step);
    store_line<T, P>(w2, r2, start, step);
  }
  __syncthreads();
  double d_xy = 0.0, d_y = 0.0, d_x = 0.0;
  if (active) {
    int start, step;
    line_geom<P>(0, ti, tj, start, step);
    const T* Mx = g.tab[0] + id[0] * LayerOff<P>::stride + LayerOff<P>::M;
    T v[P], out[P], r1[P];
    load_line<T, P>(v, w2, start, step);
    matvec(out, Mx, v);
    load_line<T, P>(r1, w1, start, step);
    S* yo = y + cbase + (long long)e * P3 + start;
#pragma unroll
    for (int a = 0; a < P; ++a) {
      out[a] += r1[a];
      yo[a] = cvt_out<S, T>(out[a], sc);
    }
    if (dots) {
      T sxy(0), sy(0), sx(0);
#pragma unroll
      for (int a = 0; a < P; ++a) sxy = fma(out[a], ux[a], sxy);
      if (sink.sums) {
#pragma unroll
        for (int a = 0; a < P; ++a) {
          sy += out[a];
          sx += ux[a];
        }
      }
      d_xy = cvt_out<double, T>(sxy, 2 * sc);
      d_y = cvt_out<double, T>(sy, sc);
      d_x = cvt_out<double, T>(sx, sc);
    }
  }
  if (dots) sink_dots(sink, d_xy, d_y, d_x);
}

// Uniform-viscosity line operator (unit viscosity; the caller scales): the own
// cell's part of the 1D stiffness and of both faces' consistency terms is the
// precombined matrix Kc; what remains per interior face is the neighbour's
// half normal derivative, the jump penalty tau_F [u] and the scatter of the
// neighbour's trace; a Dirichlet face adds 2 tau_e u.
template <typename T, int P>
__device__ __forceinline__ void line_op_u(T (&w)[P], const T (&u)[P], const T* __restrict__ L, int kindL,
                                          const T (&uL)[P], const T* __restrict__ LL, T tauFL, int kindR,
                                          const T (&uR)[P], const T* __restrict__ LR, T tauFR, T tau2e,
                                          bool eo = false) {
  using O = LayerOff<P>;
  matvec_l<T, P>(w, L, O::Kc, O::EKc, eo, u);
  if (kindR == 0) {
    const T gn = dotp(LR + O::dLh, uR);
    const T J = u[P - 1] - uR[0];
    w[P - 1] += fma(tauFR, J, -gn);
    axpy_vec(w, L + O::dRh, uR[0]);
  } else if (kindR == SIPG_BC_DIRICHLET) {
    w[P - 1] = fma(tau2e, u[P - 1], w[P - 1]);
  }
  if (kindL == 0) {
    const T gn = dotp(LL + O::dRh, uL);
    const T J = uL[P - 1] - u[0];
    w[0] += fma(-tauFL, J, gn);
    axpy_vec(w, L + O::dLh, -uL[P - 1]);
  } else if (kindL == SIPG_BC_DIRICHLET) {
    w[0] = fma(tau2e, u[0], w[0]);
  }
}

// The uniform-viscosity line operator premultiplied by the layer's inverse 1D
// mass: Mi (Kc u + face terms) = Qc u + sR mR + uR[0] qR + sL mL - uL[p-1] qL
// with the precomputed Qc = Mi Kc, mL, mR = Mi e_0, Mi e_(p-1) (the columns
// through which the end-value terms enter) and qL, qR = Mi dLh, Mi dRh (the
// scatter of the neighbour's trace); sR, sL are the end-value terms of
// line_op_u (penalty of the jump minus / plus the neighbour's half normal
// derivative; 2 tau_e u on a Dirichlet face).
template <typename T, int P>
__device__ __forceinline__ void line_op_q(T (&w)[P], const T (&u)[P], const T* __restrict__ L, int kindL,
                                          const T (&uL)[P], const T* __restrict__ LL, T tauFL, int kindR,
                                          const T (&uR)[P], const T* __restrict__ LR, T tauFR, T tau2e,
                                          bool eo) {
  using O = LayerOff<P>;
  matvec_l<T, P>(w, L, O::Qc, O::EQc, eo, u);
  if (kindR == 0) {
    const T gn = dotp(LR + O::dLh, uR);
    axpy_vec(w, L + O::mR, fma(tauFR, u[P - 1] - uR[0], -gn));
    axpy_vec(w, L + O::qR, uR[0]);
  } else if (kindR == SIPG_BC_DIRICHLET) {
    axpy_vec(w, L + O::mR, tau2e * u[P - 1]);
  }
  if (kindL == 0) {
    const T gn = dotp(LL + O::dRh, uL);
    axpy_vec(w, L + O::mL, fma(-tauFL, uL[P - 1] - u[0], gn));
    axpy_vec(w, L + O::qL, -uL[P - 1]);
  } else if (kindL == SIPG_BC_DIRICHLET) {
    axpy_vec(w, L + O::mL, tau2e * u[0]);
  }
}

// y = scale * (L x + mass_rel M x) for a uniform viscosity: scale = nu,
// mass_rel = mass_coef / nu (Laplace: scale 1, mass_rel 0).  With the 1D
// masses of the cell's layers, (I x My x Mz) = (Mx x My x I)(Mx^-1 x I x Mz)
// and (Mx x I x Mz) = (Mx x My x I)(I x My^-1 x Mz), so
//   y_e = (Mx x My x I) [ Mz ((Mx^-1 w_x) + (My^-1 w_y) + mass_rel u) + w_z ]
// (each Md^-1, Md along its own direction): the x and y line operators
// premultiplied by the inverse mass (line_op_q), the z line operator plain
// (line_op_u), and three mass contractions instead of five.  Phases per cell
// (one line per thread): X (x-lines) -> V1, Y (y-lines) -> V2, Z (z-lines):
// Mz (V1 + V2 + mass_rel u) + w_z -> V1, Y2: My -> V1, X2: Mx -> global.  The
// factorisation is exact; its rounding grows by the row sums of
// |M||M^-1 Kc| against |Kc| (2.3x at p = 5).  On centrosymmetric layers
// (p >= 5) the contractions with Qc, Kc and M take the even-odd form.
// Blocks per SM requested from the register allocator: the double-float
// kernel fits 80 registers up to p = 5, which allows three 256-thread blocks
// (24 warps) per SM, and 128 (two blocks) up to p = 7; the FP32 kernel fits 64
// registers (four blocks) up to p = 6; native FP64 keeps two blocks (128
// registers) up to p = 6 so that enough warps feed the FP64 pipe.
template <typename T, int P>
struct UniformMinBlocks {
  static constexpr int value = std::is_same<T, dfl>::value ? (P <= 5 ? 3 : (P <= 7 ? 2 : 1))
                               : (std::is_same<T, float>::value ? (P <= 6 ? 4 : (P == 7 ? 3 : 2)) : (P <= 5 ? 3 : (P <= 6 ? 2 : 1)));
};

// Shared memory of apply_uniform_kernel: own cells (kept to the end for the
// dot products and the Chebyshev epilogue) and two line-result buffers.
template <typename T, int P>
__host__ __device__ constexpr size_t uniform_smem_bytes(int cpb) {
  return (size_t)3 * cpb * P * P * P * sizeof(T);
}

// The layer tables of the x and z directions passed by value in the kernel's
// parameter space, for a mesh whose x-layers all share one table and whose
// z-layers do too (uniform spacing; Mesh::lay_same): the contractions then
// read their entries as constant-bank operands instead of issuing loads.
template <typename T, int P>
struct __align__(16) XZTab {
  T x[LayerOff<P>::stride];
  T z[LayerOff<P>::stride];
};
struct NoXZTab {};

// CHEB (FP32 only): instead of storing y = A x, apply one Chebyshev step of the
// multigrid smoother to the block's own unknowns with x = d (see ChebEpi).
// EOXZ: every x- and z-layer of the mesh is centrosymmetric (Mesh::eo_xz):
// their contractions take the even-odd form (p >= 5).
// PXZ: the x and z tables come in xz (XZTab) instead of g.tab[0], g.tab[2].
template <typename T, typename S, int P, bool CHEB = false, bool EOXZ = false, bool PXZ = false>
__global__ void __launch_bounds__(kMaxCellThreads, UniformMinBlocks<T, P>::value)
    apply_uniform_kernel(Geo<T> g, const S* __restrict__ x, S* __restrict__ y, int cpb, T mass_rel, T scale,
                         int do_scale, int do_mass, DotSink sink, ChebEpi epi,
                         const __grid_constant__ std::conditional_t<PXZ, XZTab<T, P>, NoXZTab> xz) {
  if (sink.skip && *sink.skip) return;
  double* dots = sink.partials;
  using O = LayerOff<P>;
  constexpr int P2 = P * P, P3 = P * P * P;
  constexpr bool EOX = EOXZ && P >= 5;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* su = reinterpret_cast<T*>(smem_raw);
  T* s1 = su + cpb * P3;
  T* s2 = s1 + cpb * P3;
  const int cs = threadIdx.x / P2;
  const int t = threadIdx.x - cs * P2;
  const int ti = t % P, tj = t / P;
  const long long cell0 = (long long)blockIdx.x * cpb;
  const int e = (int)(cell0 + cs);
  const bool active = cs < cpb && e < g.ncell;  // blocks are rounded up to whole warps
  const long long cbase = (long long)blockIdx.y * g.ncell * P3;
  const S* __restrict__ xc = x + cbase;
  const int nc = (int)min((long long)cpb, (long long)g.ncell - cell0);  // cells staged in this block
  const int sc = call_scale(g);
  {
    const S* xb = xc + cell0 * P3;
    stage_cvt<T, S>(su, xb, nc * P3, sc);
  }
  __syncthreads();
  // the table of `layer` along direction dir
  auto tab = [&](int dir, int layer) -> const T* {
    if constexpr (PXZ) {
      if (dir == 0) return xz.x;
      if (dir == 2) return xz.z;
    }
    return g.tab[dir] + (layer & g.lm[dir]) * O::stride;
  };
  T* us = su + cs * P3;
  T* v1 = s1 + cs * P3;
  T* v2 = s2 + cs * P3;
  int id[3] = {0, 0, 0};
  T tau_e = T(0);
  if (active) {
    id[0] = e % g.n[0];
    id[1] = (e / g.n[0]) % g.n[1];
    id[2] = e / (g.n[0] * g.n[1]);
    tau_e = tab(0, id[0])[O::ts] + tab(1, id[1])[O::ts] + tab(2, id[2])[O::ts];
  }
  const T tau2e = tau_e + tau_e;
  if (active) {
    // phases X and Y: Mx^-1 w_x on the x-lines -> V1, My^-1 w_y on the y-lines -> V2
#pragma unroll
    for (int dir = 0; dir < 2; ++dir) {
      int start, step;
      line_geom<P>(dir, ti, tj, start, step);
      const T* L = tab(dir, id[dir]);
      int nbL, nbR, kL, kR, jl, jr;
      face_neighbor(g, dir, 0, id[dir], e, nbL, kL, jl);
      face_neighbor(g, dir, 1, id[dir], e, nbR, kR, jr);
      T u[P], uL[P], uR[P], w[P];
      load_line<T, P>(u, us, start, step);
      // a neighbour staged in this block is read from shared memory (read-only
      // from here on), otherwise from global memory
      if (kL == 0) {
        const long long sl = (long long)nbL - cell0;
        if (sl >= 0 && sl < nc)
          load_line<T, P>(uL, su + sl * P3, start, step);
        else
          load_line_global_cvt<T, S, P>(uL, xc + (long long)nbL * P3, start, step, sc);
      }
      if (kR == 0) {
        const long long sr = (long long)nbR - cell0;
        if (sr >= 0 && sr < nc)
          load_line<T, P>(uR, su + sr * P3, start, step);
        else
          load_line_global_cvt<T, S, P>(uR, xc + (long long)nbR * P3, start, step, sc);
      }
      line_op_q<T, P>(w, u, L, kL, uL, kL == 0 ? tab(dir, jl) : L, tau_e + L[O::dTL], kR, uR,
                      kR == 0 ? tab(dir, jr) : L, tau_e + L[O::dTR], tau2e, dir == 0 && EOX);
      store_line<T, P>(dir == 0 ? v1 : v2, w, start, step);
    }
  }
  __syncthreads();
  if (active) {
    // phase Z on the z-lines: Mz (V1 + V2 + mass_rel u) + w_z -> V1
    int start, step;
    line_geom<P>(2, ti, tj, start, step);
    const T* L = tab(2, id[2]);
    constexpr bool eoz = EOX;
    int nbL, nbR, kL, kR, jl, jr;
    face_neighbor(g, 2, 0, id[2], e, nbL, kL, jl);
    face_neighbor(g, 2, 1, id[2], e, nbR, kR, jr);
    T u[P], uL[P], uR[P], w[P];
    load_line<T, P>(u, us, start, step);
    if (kL == 0) load_line_global_cvt<T, S, P>(uL, xc + (long long)nbL * P3, start, step, sc);
    if (kR == 0) load_line_global_cvt<T, S, P>(uR, xc + (long long)nbR * P3, start, step, sc);
    line_op_u<T, P>(w, u, L, kL, uL, kL == 0 ? tab(2, jl) : L, tau_e + L[O::dTL], kR, uR,
                    kR == 0 ? tab(2, jr) : L, tau_e + L[O::dTR], tau2e, eoz);
    T v[P], r[P];
    load_line<T, P>(v, v1, start, step);
    {
      T v2l[P];
      load_line<T, P>(v2l, v2, start, step);
#pragma unroll
      for (int a = 0; a < P; ++a) v[a] += v2l[a];
    }
    if (do_mass) {
#pragma unroll
      for (int a = 0; a < P; ++a) v[a] = fma(mass_rel, u[a], v[a]);
    }
    matvec_l<T, P>(r, L, O::M, O::EM, eoz, v);
#pragma unroll
    for (int a = 0; a < P; ++a) r[a] += w[a];
    store_line<T, P>(v1, r, start, step);
  }
  __syncthreads();
  if (active) {
    // phase Y2 on the y-lines: My -> V1
    int start, step;
    line_geom<P>(1, ti, tj, start, step);
    T v[P], r[P];
    load_line<T, P>(v, v1, start, step);
    const T* Ly = tab(1, id[1]);
    matvec_l<T, P>(r, Ly, O::M, O::EM, false, v);
    store_line<T, P>(v1, r, start, step);
  }
  __syncthreads();
  double d_xy = 0.0, d_y = 0.0, d_x = 0.0;
  if (active) {
    // phase X2 on the x-lines: Mx -> V2 (the block's result, written to
    // global memory below in one coalesced sweep)
    int start, step;
    line_geom<P>(0, ti, tj, start, step);
    T v[P], out[P];
    load_line<T, P>(v, v1, start, step);
    const T* Lx = tab(0, id[0]);
    matvec_l<T, P>(out, Lx, O::M, O::EM, EOX, v);
#pragma unroll
    for (int a = 0; a < P; ++a)
      if (do_scale) out[a] *= scale;
    store_line<T, P>(v2, out, start, step);  // V2 is free since phase Z
    if (!CHEB && dots) {
      // line sums in the compute type, one conversion per line; the x-line of
      // the input from the staged cell
      T ux[P];
      load_line<T, P>(ux, us, start, step);
      T sxy(0), sy(0), sx(0);
#pragma unroll
      for (int a = 0; a < P; ++a) sxy = fma(out[a], ux[a], sxy);
      if (sink.sums) {  // sums of y and x only for the zero-mean projection
#pragma unroll
        for (int a = 0; a < P; ++a) {
          sy += out[a];
          sx += ux[a];
        }
      }
      d_xy = cvt_out<double, T>(sxy, 2 * sc);
      d_y = cvt_out<double, T>(sy, sc);
      d_x = cvt_out<double, T>(sx, sc);
    }
  }
  // the block's partial sums go out (and are fenced) before the block writes
  // y, so that the fence waits for the partials only; y is read by later
  // kernels, after this one has finished
  if (dots) sink_dots(sink, d_xy, d_y, d_x);
  __syncthreads();
  // the block's cells are contiguous in memory: consecutive threads write
  // (or, for the Chebyshev step, update) consecutive entries
  const long long o0 = cbase + cell0 * P3;
  if constexpr (CHEB) {
    static_assert(std::is_same<T, float>::value && std::is_same<S, float>::value, "FP32 only");
    // r -= A d, dnew = c1 d + c2 D^-1 r, x += dnew with d the staged input;
    // each thread loads r, D^-1 and x of four entries before it updates them
    // (the stores of one entry could otherwise hold back the next one's loads)
    const int n = nc * P3, bd = blockDim.x;
    for (int i0 = threadIdx.x; i0 < n; i0 += 4 * bd) {
      float rv[4], dv[4], xv[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int i = i0 + j * bd;
        rv[j] = i < n ? epi.r[o0 + i] : 0.f;
        dv[j] = i < n ? epi.dinv[o0 + i] : 0.f;
        xv[j] = i < n ? epi.x[o0 + i] : 0.f;
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int i = i0 + j * bd;
        if (i < n) {
          const float ri = rv[j] - s2[i];
          const float di = epi.c1 * su[i] + epi.c2 * ri * dv[j];
          epi.r[o0 + i] = ri;
          epi.dnew[o0 + i] = di;
          epi.x[o0 + i] = xv[j] + di;
        }
      }
    }
  } else {
    for (int idx = threadIdx.x; idx < nc * P3; idx += blockDim.x) y[o0 + idx] = cvt_out<S, T>(s2[idx], sc);
  }
}

// Plane variant of the uniform-viscosity operator for FP32 (the line variant
// issues one load of a 1D-matrix entry per FMA; measured slower on GB300 at
// k = 4, 5 -- less parallelism per cell -- and kept as an autotuner candidate).
// P threads per cell; thread t owns the plane c = t in the phases along x and
// y (X, Y, Y2, X2) and the plane b = t in the phase along z, and loads each
// phase's 1D matrices once into registers for its P lines: P times fewer
// table loads.  Same arithmetic and results as apply_uniform_kernel.
template <typename T, int P>
__device__ __forceinline__ void load_mat(T (&A)[P * P], const T* __restrict__ src) {
#pragma unroll
  for (int i = 0; i < P * P; ++i) A[i] = src[i];
}

template <typename T, int P>
__device__ __forceinline__ void matvec_reg(T (&out)[P], const T (&A)[P * P], const T (&v)[P]) {
#pragma unroll
  for (int a = 0; a < P; ++a) {
    T s = T(0);
#pragma unroll
    for (int b = 0; b < P; ++b) s = fma(A[a * P + b], v[b], s);
    out[a] = s;
  }
}

template <typename T, int P>
__global__ void __launch_bounds__(kMaxCellThreads) apply_plane_kernel(Geo<T> g, const T* __restrict__ x,
                                                                      T* __restrict__ y, int cpb, T mass_rel,
                                                                      T scale, int do_scale, int do_mass) {
  using O = LayerOff<P>;
  constexpr int P3 = P * P * P;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* su = reinterpret_cast<T*>(smem_raw);
  T* s1 = su + cpb * P3;
  T* s2 = s1 + cpb * P3;
  const int cs = threadIdx.x / P;
  const int t = threadIdx.x - cs * P;
  const long long cell0 = (long long)blockIdx.x * cpb;
  const int e = (int)(cell0 + cs);
  const bool active = cs < cpb && e < g.ncell;
  const long long cbase = (long long)blockIdx.y * g.ncell * P3;
  const T* __restrict__ xc = x + cbase;
  const int nc = (int)min((long long)cpb, (long long)g.ncell - cell0);
  for (int idx = threadIdx.x; idx < nc * P3; idx += blockDim.x) su[idx] = xc[cell0 * P3 + idx];
  __syncthreads();
  T* us = su + cs * P3;
  T* w1 = s1 + cs * P3;
  T* w2 = s2 + cs * P3;
  int id[3] = {0, 0, 0};
  T tau_e = T(0);
  if (active) {
    id[0] = e % g.n[0];
    id[1] = (e / g.n[0]) % g.n[1];
    id[2] = e / (g.n[0] * g.n[1]);
    tau_e = g.tab[0][id[0] * O::stride + O::ts] + g.tab[1][id[1] * O::stride + O::ts] +
            g.tab[2][id[2] * O::stride + O::ts];
  }
  const T tau2e = tau_e + tau_e;
  // neighbour line: from shared memory when staged in this block (phases X, Y
  // only: the input stays unchanged there), else from global memory
  auto nb_line = [&](T (&v)[P], int nb, int start, int step, bool smem_ok) {
    const long long sl = (long long)nb - cell0;
    if (smem_ok && sl >= 0 && sl < nc)
      load_line<T, P>(v, su + sl * P3, start, step);
    else
      load_line_global<T, P>(v, xc + (long long)nb * P3, start, step);
  };
  if (active) {
    // phases X and Y on the plane c = t
#pragma unroll 1
    for (int dir = 0; dir < 2; ++dir) {
      const T* L = g.tab[dir] + id[dir] * O::stride;
      int nbL, nbR, kL, kR, jl, jr;
      face_neighbor(g, dir, 0, id[dir], e, nbL, kL, jl);
      face_neighbor(g, dir, 1, id[dir], e, nbR, kR, jr);
      const T* LL = kL == 0 ? g.tab[dir] + jl * O::stride : L;
      const T* LR = kR == 0 ? g.tab[dir] + jr * O::stride : L;
      T Kc[P * P], dRh[P], dLh[P], nLh[P], nRh[P];
      load_mat<T, P>(Kc, L + O::Kc);
#pragma unroll
      for (int a = 0; a < P; ++a) {
        dRh[a] = L[O::dRh + a];
        dLh[a] = L[O::dLh + a];
        nLh[a] = LR[O::dLh + a];  // right neighbour's low-end half derivative
        nRh[a] = LL[O::dRh + a];  // left neighbour's high-end half derivative
      }
      const T tFL = tau_e + L[O::dTL], tFR = tau_e + L[O::dTR];
#pragma unroll 1
      for (int q = 0; q < P; ++q) {
        int start, step;
        line_geom<P>(dir, q, t, start, step);  // x-line (b=q, c=t) or y-line (a=q, c=t)
        T u[P], uL[P], uR[P], w[P];
        load_line<T, P>(u, us, start, step);
        if (kL == 0) nb_line(uL, nbL, start, step, true);
        if (kR == 0) nb_line(uR, nbR, start, step, true);
        matvec_reg<T, P>(w, Kc, u);
        if (kR == 0) {
          T gn = T(0);
#pragma unroll
          for (int a = 0; a < P; ++a) gn = fma(nLh[a], uR[a], gn);
          w[P - 1] += fma(tFR, u[P - 1] - uR[0], -gn);
#pragma unroll
          for (int a = 0; a < P; ++a) w[a] = fma(dRh[a], uR[0], w[a]);
        } else if (kR == SIPG_BC_DIRICHLET) {
          w[P - 1] = fma(tau2e, u[P - 1], w[P - 1]);
        }
        if (kL == 0) {
          T gn = T(0);
#pragma unroll
          for (int a = 0; a < P; ++a) gn = fma(nRh[a], uL[a], gn);
          w[0] += fma(-tFL, uL[P - 1] - u[0], gn);
#pragma unroll
          for (int a = 0; a < P; ++a) w[a] = fma(dLh[a], -uL[P - 1], w[a]);
        } else if (kL == SIPG_BC_DIRICHLET) {
          w[0] = fma(tau2e, u[0], w[0]);
        }
        store_line<T, P>(dir == 0 ? w1 : w2, w, start, step);
      }
    }
  }
  __syncthreads();
  if (active) {
    // phase Z on the plane b = t: w_z, Mz w_x, Mz w_y (each thread only touches
    // its own z-lines)
    const T* L = g.tab[2] + id[2] * O::stride;
    int nbL, nbR, kL, kR, jl, jr;
    face_neighbor(g, 2, 0, id[2], e, nbL, kL, jl);
    face_neighbor(g, 2, 1, id[2], e, nbR, kR, jr);
    const T* LL = kL == 0 ? g.tab[2] + jl * O::stride : L;
    const T* LR = kR == 0 ? g.tab[2] + jr * O::stride : L;
    T Mz[P * P];
    load_mat<T, P>(Mz, L + O::M);
#pragma unroll 1
    for (int q = 0; q < P; ++q) {
      int start, step;
      line_geom<P>(2, q, t, start, step);  // z-line (a=q, b=t)
      T v[P], r[P];
      load_line<T, P>(v, w1, start, step);
      matvec_reg<T, P>(r, Mz, v);
      store_line<T, P>(w1, r, start, step);
      load_line<T, P>(v, w2, start, step);
      matvec_reg<T, P>(r, Mz, v);
      store_line<T, P>(w2, r, start, step);
      T u[P], uL[P], uR[P], w[P];
      load_line<T, P>(u, us, start, step);
      if (kL == 0) nb_line(uL, nbL, start, step, false);
      if (kR == 0) nb_line(uR, nbR, start, step, false);
      line_op_u<T, P>(w, u, L, kL, uL, LL, tau_e + L[O::dTL], kR, uR, LR, tau_e + L[O::dTR], tau2e);
      if (do_mass) {
        T mu[P];
        matvec_reg<T, P>(mu, Mz, u);
#pragma unroll
        for (int a = 0; a < P; ++a) w[a] = fma(mass_rel, mu[a], w[a]);
      }
      store_line<T, P>(us, w, start, step);
    }
  }
  __syncthreads();
  if (active) {
    // phase Y2 on the plane c = t
    T My[P * P];
    load_mat<T, P>(My, g.tab[1] + id[1] * O::stride + O::M);
#pragma unroll 1
    for (int q = 0; q < P; ++q) {
      int start, step;
      line_geom<P>(1, q, t, start, step);
      T v[P], r[P];
      load_line<T, P>(v, w1, start, step);
      matvec_reg<T, P>(r, My, v);
      store_line<T, P>(w1, r, start, step);
      load_line<T, P>(v, us, start, step);
      matvec_reg<T, P>(r, My, v);
      load_line<T, P>(v, w2, start, step);
#pragma unroll
      for (int a = 0; a < P; ++a) r[a] += v[a];
      store_line<T, P>(w2, r, start, step);
    }
  }
  __syncthreads();
  if (active) {
    // phase X2 on the plane c = t: y = Mx R2 + R1 -> global
    T Mx[P * P];
    load_mat<T, P>(Mx, g.tab[0] + id[0] * O::stride + O::M);
#pragma unroll 1
    for (int q = 0; q < P; ++q) {
      int start, step;
      line_geom<P>(0, q, t, start, step);
      T v[P], out[P], r1[P];
      load_line<T, P>(v, w2, start, step);
      matvec_reg<T, P>(out, Mx, v);
      load_line<T, P>(r1, w1, start, step);
      T* yo = y + cbase + (long long)e * P3 + start;
#pragma unroll
      for (int a = 0; a < P; ++a) {
        out[a] += r1[a];
        if (do_scale) out[a] *= scale;
        yo[a] = out[a];
      }
    }
  }
}

// y = M^-1 x = (Mx^-1 x My^-1 x Mz^-1) x cell by cell (Sec. 5: tensorial inverse
// mass with square 1D transforms).  T is the arithmetic (double or
// double-float), S the storage type.  Optional per-block partials (x.y, sum y,
// sum x) for the CG.
template <typename T, typename S, int P>
__global__ void __launch_bounds__(kMaxCellThreads) inverse_mass_kernel(Geo<T> g, const S* __restrict__ x,
                                                                       S* __restrict__ y, int cpb,
                                                                       double* __restrict__ dots) {
  constexpr int P2 = P * P, P3 = P * P * P;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* su = reinterpret_cast<T*>(smem_raw);
  const int cs = threadIdx.x / P2;
  const int t = threadIdx.x - cs * P2;
  const int ti = t % P, tj = t / P;
  const long long cell0 = (long long)blockIdx.x * cpb;
  const int e = (int)(cell0 + cs);
  const bool active = cs < cpb && e < g.ncell;  // blocks are rounded up to whole warps
  const long long cbase = (long long)blockIdx.y * g.ncell * P3;
  const int sc = call_scale(g);
  {
    const int nc = (int)min((long long)cpb, (long long)g.ncell - cell0);
    const S* xb = x + cbase + cell0 * P3;
    stage_cvt<T, S>(su, xb, nc * P3, sc);
  }
  __syncthreads();
  T* us = su + cs * P3;
  int id[3] = {0, 0, 0};
  if (active) {
    id[0] = e % g.n[0];
    id[1] = (e / g.n[0]) % g.n[1];
    id[2] = e / (g.n[0] * g.n[1]);
  }
  using O = LayerOff<P>;
  for (int dir = 2; dir >= 1; --dir) {
    if (active) {
      int start, step;
      line_geom<P>(dir, ti, tj, start, step);
      T v[P], o[P];
      load_line<T, P>(v, us, start, step);
      matvec(o, g.tab[dir] + id[dir] * O::stride + O::Mi, v);
      store_line<T, P>(us, o, start, step);
    }
    __syncthreads();
  }
  double d_xy = 0.0, d_y = 0.0, d_x = 0.0;
  if (active) {
    int start, step;
    line_geom<P>(0, ti, tj, start, step);
    T v[P], o[P];
    load_line<T, P>(v, us, start, step);
    matvec(o, g.tab[0] + id[0] * O::stride + O::Mi, v);
    const long long off = cbase + (long long)e * P3 + start;
    for (int a = 0; a < P; ++a) y[off + a] = cvt_out<S, T>(o[a], sc);
    if (dots) {
      T xv[P];
      load_line_global_cvt<T, S, P>(xv, x + cbase + (long long)e * P3, start, step, sc);
      T sxy(0), sy(0), sx(0);
      for (int a = 0; a < P; ++a) {
        sxy = fma(o[a], xv[a], sxy);
        sy += o[a];
        sx += xv[a];
      }
      d_xy = cvt_out<double, T>(sxy, 2 * sc);
      d_y = cvt_out<double, T>(sy, sc);
      d_x = cvt_out<double, T>(sx, sc);
    }
  }
  if (dots) block_reduce3(d_xy, d_y, d_x, dots + 3 * ((long long)blockIdx.y * gridDim.x + blockIdx.x));
}

// diag(A) in closed form: the self-coupling of the 1D line operators on the
// diagonal, times the diagonals of the transverse 1D mass matrices.
template <int P>
__global__ void diagonal_kernel(Geo<double> g, int stiffness, double mass_coef, double nu,
                                const double* __restrict__ nu_cell, double* __restrict__ diag) {
  constexpr int P3 = P * P * P;
  using O = LayerOff<P>;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)g.ncell * P3) return;
  const int e = (int)(i / P3);
  const int r = (int)(i - (long long)e * P3);
  const int idx[3] = {r % P, (r / P) % P, r / (P * P)};
  int id[3];
  id[0] = e % g.n[0];
  id[1] = (e / g.n[0]) % g.n[1];
  id[2] = e / (g.n[0] * g.n[1]);
  const double nue = nu_cell ? nu_cell[e] : nu;
  const double tau_e = g.tau_scale * (g.tab[0][id[0] * O::stride + O::t] + g.tab[1][id[1] * O::stride + O::t] +
                                      g.tab[2][id[2] * O::stride + O::t]);
  double md[3], kd[3];
  for (int dir = 0; dir < 3; ++dir) {
    DirCtx<double, P> c = dir_ctx<double, P>(g, dir, id, e, nue, tau_e, nu_cell, nu);
    const int a = idx[dir];
    md[dir] = c.L[O::M + a * P + a];
    double k = nue * c.L[O::K + a * P + a];
    if (a == P - 1) {
      if (c.kindR == 0) {
        k += -nue * c.L[O::dR + P - 1] + c.tauFR * (nue > c.nuR ? nue : c.nuR);
        // one cell across a periodic direction: the "neighbour" trace is this
        // node's own left-end derivative (self-coupling on the diagonal)
        if (c.nbR == e) k += -nue * c.L[O::dL + P - 1];
      } else if (c.kindR == SIPG_BC_DIRICHLET) {
        k += -2.0 * nue * c.L[O::dR + P - 1] + 2.0 * tau_e * nue;
      }
    }
    if (a == 0) {
      if (c.kindL == 0) {
        k += nue * c.L[O::dL] + c.tauFL * (nue > c.nuL ? nue : c.nuL);
        if (c.nbL == e) k += nue * c.L[O::dR];
      } else if (c.kindL == SIPG_BC_DIRICHLET) {
        k += 2.0 * nue * c.L[O::dL] + 2.0 * tau_e * nue;
      }
    }
    kd[dir] = k;
  }
  double v = mass_coef * md[0] * md[1] * md[2];
  if (stiffness) v += kd[0] * md[1] * md[2] + md[0] * kd[1] * md[2] + md[0] * md[1] * kd[2];
  diag[i] = v;
}

}  // namespace sipg
