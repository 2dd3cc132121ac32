// Convective term of the explicit convective step, Eq. (convstepspat), with
// the local Lax-Friedrichs flux (Sec. 3.2 (i)):
//   y_i = (grad phi, u_i u)_e - (phi, (F^c* n)_i)_de
//   F^c* n = {{u (x) u}} n + Lambda/2 (u^- - u^+)     interior / periodic faces,
//          = u^- (u^- . n) + Lambda u^-             no-slip (Dirichlet, g = 0) faces,
//          = u^- (u^- . n)                          Neumann faces,
//   Lambda = max(2 |u^- . n|, 2 |u^+ . n|) at every face quadrature point.
// Cell and face integrals use Gauss quadrature with Q = floor(3k/2)+1 points
// per direction (Sec. 5: exact on affine cells, no aliasing).
//
// On the separable map the Jacobian is diagonal, J = diag(J_x, J_y, J_z), one
// 1D factor per direction and layer.  With S[q][a] = l_a(z_q), D[a][q] =
// w_q l_a'(z_q) and wj_d(q) = w_q J_d(z_q):
//   (d_k phi_a, f)_e = D along k and S^T along the other two directions,
//                      applied to f times the product of wj_m over m != k
// (J_k cancels), and a d-face integral is S^T along its two tangential
// directions applied to the flux times wj_t1 wj_t2 (the normal is +-e_d).
//
// One thread block holds `cpb` cells.  Every stage is one pass over all lines
// of all cells of the block followed by one barrier:
//   interpolation of the three components to the Q^3 points (3 stages);
//   the cell term, the nine products u_i u_k folded into three chains per
//   component (x: D F_i0, S^T F_i1, S^T F_i2; y: S^T A0 + D A1, S^T A2;
//   z: S^T B01 + D B2) (3 stages);
//   the six faces at once: own and neighbour face values (1), interpolation
//   to the Q^2 face points (2), flux (1), test (2), and a conflict-free
//   gather of the face results onto the cell's boundary nodes (1).
// The arithmetic is FP64 or double-float (the mesh's FP64 arithmetic).
#include "apply.cuh"

namespace sipg {

namespace {

constexpr int kConvThreads = 128;

template <int P>
struct ConvDims {
  static constexpr int Q = (3 * (P - 1)) / 2 + 1;
  static constexpr int P2 = P * P, P3 = P * P * P, Q2 = Q * Q, Q3 = Q * Q * Q;
  static constexpr int XI = 3 * Q * P2 + 3 * Q2 * P;  // interpolation temporaries
  static constexpr int XC = 9 * P * Q2 + 6 * P2 * Q;  // cell-term temporaries
  static constexpr int XF = 36 * Q2 + 36 * P * Q;     // face temporaries (two regions)
  static constexpr int X = XI > XC ? (XI > XF ? XI : XF) : (XC > XF ? XC : XF);
  static constexpr int per_cell = 6 * P3 + 3 * Q3 + 3 * Q + X;  // su, so, uq, wj, X
  static constexpr int shared = 2 * P * Q;                       // S, D
};

template <int P>
__host__ __device__ constexpr int nstride(int dir) {
  return dir == 0 ? 1 : (dir == 1 ? P : P * P);
}

template <typename T, int P>
__global__ void __launch_bounds__(kConvThreads) convective_kernel(Geo<T> g, const T* __restrict__ tabs, int off_D,
                                                                  int off_W0, int off_W1, int off_W2,
                                                                  const double* __restrict__ u,
                                                                  double* __restrict__ y, int cpb) {
  using Dm = ConvDims<P>;
  constexpr int Q = Dm::Q, P2 = Dm::P2, P3 = Dm::P3, Q2 = Dm::Q2, Q3 = Dm::Q3, PC = Dm::per_cell;
  const int sc = call_scale(g);  // data enter as u 2^-sc; the result leaves with 2^(2 sc)
  extern __shared__ __align__(16) unsigned char smraw[];
  T* Sq = reinterpret_cast<T*>(smraw);  // Sq[q * P + a] = l_a(z_q)
  T* Dq = Sq + Q * P;                    // Dq[a * Q + q] = w_q l_a'(z_q)
  T* base = Dq + P * Q;                  // cpb cells of PC values
  int* fnb = reinterpret_cast<int*>(base + (size_t)cpb * PC);  // [cpb][6] face neighbours
  int* fkind = fnb + 6 * cpb;                                    // [cpb][6] 0 interior, else bc
#define SU(lc) (base + (lc) * PC)
#define SO(lc) (base + (lc) * PC + 3 * P3)
#define UQ(lc) (base + (lc) * PC + 6 * P3)
#define WJ(lc) (base + (lc) * PC + 6 * P3 + 3 * Q3)
#define XB(lc) (base + (lc) * PC + 6 * P3 + 3 * Q3 + 3 * Q)
  const int NT = blockDim.x;
  const int e0 = blockIdx.x * cpb;
  const long long N = (long long)g.ncell * P3;
  const int nx = g.n[0], nxy = g.n[0] * g.n[1];

  // stage 0: tables, face neighbours, layer weights, nodal input
  for (int i = threadIdx.x; i < Q * P; i += NT) {
    Sq[i] = tabs[i];
    Dq[i] = tabs[off_D + i];
  }
  for (int i = threadIdx.x; i < 6 * cpb; i += NT) {
    const int lc = i / 6, f = i % 6, e = e0 + lc;
    int nb = -1, kind = SIPG_BC_NEUMANN, jl;
    if (e < g.ncell) {
      const int d = f >> 1;
      const int id = d == 0 ? e % nx : (d == 1 ? (e / nx) % g.n[1] : e / nxy);
      face_neighbor(g, d, f & 1, id, e, nb, kind, jl);
    }
    fnb[i] = nb;
    fkind[i] = kind;
  }
  for (int i = threadIdx.x; i < cpb * 3 * Q; i += NT) {
    const int lc = i / (3 * Q), r = i % (3 * Q), d = r / Q, q = r % Q, e = e0 + lc;
    const int id = e < g.ncell ? (d == 0 ? e % nx : (d == 1 ? (e / nx) % g.n[1] : e / nxy)) : 0;
    const int off = d == 0 ? off_W0 : (d == 1 ? off_W1 : off_W2);
    WJ(lc)[r] = tabs[off + id * Q + q];
  }
  for (int i0 = threadIdx.x; i0 < cpb * 3 * P3; i0 += 4 * NT) {
    double v[4];  // all loads issued before the conversions
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int i = i0 + j * NT, lc = i / (3 * P3), r = i % (3 * P3), e = e0 + lc;
      v[j] = i < cpb * 3 * P3 && e < g.ncell ? __ldg(u + (r / P3) * N + (long long)e * P3 + r % P3) : 0.0;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int i = i0 + j * NT, lc = i / (3 * P3), r = i % (3 * P3);
      if (i < cpb * 3 * P3) SU(lc)[r] = cvt_in<T, double>(v[j], sc);
    }
  }
  __syncthreads();

  // stages 1-3: u at the Q^3 points (x, then y, then z)
  for (int l = threadIdx.x; l < cpb * 3 * P2; l += NT) {
    const int lc = l / (3 * P2), r = l % (3 * P2), c = r / P2, yz = r % P2;
    const T* s = SU(lc) + c * P3 + yz * P;
    T v[P];
#pragma unroll
    for (int a = 0; a < P; ++a) v[a] = s[a];
    T* d = XB(lc) + c * Q * P2 + yz * Q;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      T acc = T(0);
#pragma unroll
      for (int a = 0; a < P; ++a) acc = fma(Sq[q * P + a], v[a], acc);
      d[q] = acc;
    }
  }
  __syncthreads();
  for (int l = threadIdx.x; l < cpb * 3 * Q * P; l += NT) {
    const int lc = l / (3 * Q * P), r = l % (3 * Q * P), c = r / (Q * P), rem = r % (Q * P), qx = rem % Q,
              z = rem / Q;
    const T* s = XB(lc) + c * Q * P2 + z * P * Q + qx;
    T v[P];
#pragma unroll
    for (int b = 0; b < P; ++b) v[b] = s[b * Q];
    T* d = XB(lc) + 3 * Q * P2 + c * Q2 * P + z * Q2 + qx;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      T acc = T(0);
#pragma unroll
      for (int b = 0; b < P; ++b) acc = fma(Sq[q * P + b], v[b], acc);
      d[q * Q] = acc;
    }
  }
  __syncthreads();
  for (int l = threadIdx.x; l < cpb * 3 * Q2; l += NT) {
    const int lc = l / (3 * Q2), r = l % (3 * Q2), c = r / Q2, qxy = r % Q2;
    const T* s = XB(lc) + 3 * Q * P2 + c * Q2 * P + qxy;
    T v[P];
#pragma unroll
    for (int b = 0; b < P; ++b) v[b] = s[b * Q2];
    T* d = UQ(lc) + c * Q3 + qxy;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      T acc = T(0);
#pragma unroll
      for (int b = 0; b < P; ++b) acc = fma(Sq[q * P + b], v[b], acc);
      d[q * Q2] = acc;
    }
  }
  __syncthreads();

  // stage 4: cell term along x, A_m[i] = (D | S^T | S^T) of wj-weighted u_i u_m
  for (int l = threadIdx.x; l < cpb * 3 * Q2; l += NT) {
    const int lc = l / (3 * Q2), r = l % (3 * Q2), i = r / Q2, qyz = r % Q2, qy = qyz % Q, qz = qyz / Q;
    const T* uq = UQ(lc);
    const T* wj = WJ(lc);
    const T wyz = wj[Q + qy] * wj[2 * Q + qz];
    T g0[Q], g1[Q], g2[Q];
#pragma unroll
    for (int qx = 0; qx < Q; ++qx) {
      const int pt = qyz * Q + qx;
      const T ui = uq[i * Q3 + pt];
      const T wx = wj[qx];
      g0[qx] = ui * uq[pt] * wyz;
      g1[qx] = ui * uq[Q3 + pt] * (wx * wj[2 * Q + qz]);
      g2[qx] = ui * uq[2 * Q3 + pt] * (wx * wj[Q + qy]);
    }
    T* A = XB(lc) + i * 3 * P * Q2 + qyz * P;
#pragma unroll
    for (int a = 0; a < P; ++a) {
      T a0 = T(0), a1 = T(0), a2 = T(0);
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        a0 = fma(Dq[a * Q + q], g0[q], a0);
        a1 = fma(Sq[q * P + a], g1[q], a1);
        a2 = fma(Sq[q * P + a], g2[q], a2);
      }
      A[a] = a0;
      A[P * Q2 + a] = a1;
      A[2 * P * Q2 + a] = a2;
    }
  }
  __syncthreads();
  // stage 5: along y, B01 = S^T A0 + D A1, B2 = S^T A2
  for (int l = threadIdx.x; l < cpb * 3 * P * Q; l += NT) {
    const int lc = l / (3 * P * Q), r = l % (3 * P * Q), i = r / (P * Q), rem = r % (P * Q), ax = rem % P,
              qz = rem / P;
    const T* A = XB(lc) + i * 3 * P * Q2 + qz * Q * P + ax;
    T v0[Q], v1[Q], v2[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      v0[q] = A[q * P];
      v1[q] = A[P * Q2 + q * P];
      v2[q] = A[2 * P * Q2 + q * P];
    }
    T* B = XB(lc) + 9 * P * Q2 + i * 2 * P2 * Q + qz * P2 + ax;
#pragma unroll
    for (int a = 0; a < P; ++a) {
      T b01 = T(0), b2 = T(0);
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        b01 = fma(Sq[q * P + a], v0[q], b01);
        b01 = fma(Dq[a * Q + q], v1[q], b01);
        b2 = fma(Sq[q * P + a], v2[q], b2);
      }
      B[a * P] = b01;
      B[P2 * Q + a * P] = b2;
    }
  }
  __syncthreads();
  // stage 6: along z, so[i] = S^T B01 + D B2
  for (int l = threadIdx.x; l < cpb * 3 * P2; l += NT) {
    const int lc = l / (3 * P2), r = l % (3 * P2), i = r / P2, axy = r % P2;
    const T* B = XB(lc) + 9 * P * Q2 + i * 2 * P2 * Q + axy;
    T v0[Q], v1[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      v0[q] = B[q * P2];
      v1[q] = B[P2 * Q + q * P2];
    }
    T* o = SO(lc) + i * P3 + axy;
#pragma unroll
    for (int a = 0; a < P; ++a) {
      T acc = T(0);
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        acc = fma(Sq[q * P + a], v0[q], acc);
        acc = fma(Dq[a * Q + q], v1[q], acc);
      }
      o[a * P2] = acc;
    }
  }
  __syncthreads();

  // faces, all six at once.  Region a = XB[0, 36 Q^2), region b after it.
  // stage 7: own (s = 0) and neighbour (s = 1) nodal face values,
  // fa[(f*2+s)*3+c][cc*P+b] with b along t1 and cc along t2
  for (int l = threadIdx.x; l < cpb * 36 * P2; l += NT) {
    const int lc = l / (36 * P2), r = l % (36 * P2), fsc = r / P2, bc = r % P2, b = bc % P, cc = bc / P;
    const int c = fsc % 3, s = (fsc / 3) & 1, f = fsc / 6, d = f >> 1, side = f & 1;
    const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
    const int tr = b * nstride<P>(t1) + cc * nstride<P>(t2);
    const int aend = side ? P - 1 : 0;
    T v = T(0);
    if (s == 0) {
      v = SU(lc)[c * P3 + aend * nstride<P>(d) + tr];
    } else if (fkind[lc * 6 + f] == 0) {
      const int nend = P - 1 - aend;
      v = cvt_in<T, double>(u[c * N + (long long)fnb[lc * 6 + f] * P3 + nend * nstride<P>(d) + tr], sc);
    }
    XB(lc)[r] = v;
  }
  __syncthreads();
  // stages 8-9: to the Q^2 face points (t1, then t2)
  for (int l = threadIdx.x; l < cpb * 36 * P; l += NT) {
    const int lc = l / (36 * P), r = l % (36 * P), fsc = r / P, cc = r % P;
    const T* s = XB(lc) + fsc * P2 + cc * P;
    T v[P];
#pragma unroll
    for (int b = 0; b < P; ++b) v[b] = s[b];
    T* d = XB(lc) + 36 * Q2 + fsc * Q * P + cc * Q;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      T acc = T(0);
#pragma unroll
      for (int b = 0; b < P; ++b) acc = fma(Sq[q * P + b], v[b], acc);
      d[q] = acc;
    }
  }
  __syncthreads();
  for (int l = threadIdx.x; l < cpb * 36 * Q; l += NT) {
    const int lc = l / (36 * Q), r = l % (36 * Q), fsc = r / Q, q1 = r % Q;
    const T* s = XB(lc) + 36 * Q2 + fsc * Q * P + q1;
    T v[P];
#pragma unroll
    for (int b = 0; b < P; ++b) v[b] = s[b * Q];
    T* d = XB(lc) + fsc * Q2 + q1;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      T acc = T(0);
#pragma unroll
      for (int b = 0; b < P; ++b) acc = fma(Sq[q * P + b], v[b], acc);
      d[q * Q] = acc;
    }
  }
  __syncthreads();
  // stage 10: LLF flux times the face weights, in place of the own values
  for (int l = threadIdx.x; l < cpb * 6 * Q2; l += NT) {
    const int lc = l / (6 * Q2), r = l % (6 * Q2), f = r / Q2, j = r % Q2, d = f >> 1;
    const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
    const T* wj = WJ(lc);
    const T wt = wj[t1 * Q + j % Q] * wj[t2 * Q + j / Q];
    T* qo = XB(lc) + (f * 6) * Q2 + j;  // own values, components at stride Q2
    const T* qn = qo + 3 * Q2;           // neighbour values
    const int kind = fkind[lc * 6 + f];
    const T sg = (f & 1) ? T(1) : T(-1);
    const T um[3] = {qo[0], qo[Q2], qo[2 * Q2]};
    const T un = sg * qo[d * Q2];
    const T lm = T(2) * (un > T(0) ? un : -un);
    if (kind == 0) {
      const T up[3] = {qn[0], qn[Q2], qn[2 * Q2]};
      const T unb = sg * qn[d * Q2];
      const T lp = T(2) * (unb > T(0) ? unb : -unb);
      const T hl = T(0.5) * (lm > lp ? lm : lp);
#pragma unroll
      for (int c = 0; c < 3; ++c) qo[c * Q2] = wt * (T(0.5) * (um[c] * un + up[c] * unb) + hl * (um[c] - up[c]));
    } else if (kind == SIPG_BC_DIRICHLET) {
#pragma unroll
      for (int c = 0; c < 3; ++c) qo[c * Q2] = wt * (um[c] * un + lm * um[c]);
    } else {
#pragma unroll
      for (int c = 0; c < 3; ++c) qo[c * Q2] = wt * (um[c] * un);
    }
  }
  __syncthreads();
  // stages 11-12: test with S^T along t1, then t2; h2[f*3+c][a2*P+a1]
  for (int l = threadIdx.x; l < cpb * 18 * Q; l += NT) {
    const int lc = l / (18 * Q), r = l % (18 * Q), fc = r / Q, q2 = r % Q, f = fc / 3, c = fc % 3;
    const T* s = XB(lc) + (f * 6 + c) * Q2 + q2 * Q;
    T v[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) v[q] = s[q];
    T* d = XB(lc) + 36 * Q2 + fc * P * Q + q2 * P;
#pragma unroll
    for (int a = 0; a < P; ++a) {
      T acc = T(0);
#pragma unroll
      for (int q = 0; q < Q; ++q) acc = fma(Sq[q * P + a], v[q], acc);
      d[a] = acc;
    }
  }
  __syncthreads();
  for (int l = threadIdx.x; l < cpb * 18 * P; l += NT) {
    const int lc = l / (18 * P), r = l % (18 * P), fc = r / P, a1 = r % P;
    const T* s = XB(lc) + 36 * Q2 + fc * P * Q + a1;
    T v[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) v[q] = s[q * P];
    T* d = XB(lc) + fc * P2 + a1;
#pragma unroll
    for (int a = 0; a < P; ++a) {
      T acc = T(0);
#pragma unroll
      for (int q = 0; q < Q; ++q) acc = fma(Sq[q * P + a], v[q], acc);
      d[a * P] = acc;
    }
  }
  __syncthreads();
  // stage 13: y = cell term - face terms on the boundary nodes
  for (int l = threadIdx.x; l < cpb * 3 * P3; l += NT) {
    const int lc = l / (3 * P3), r = l % (3 * P3), c = r / P3, node = r % P3, e = e0 + lc;
    if (e >= g.ncell) continue;
    const int ax[3] = {node % P, (node / P) % P, node / P2};
    T v = SO(lc)[r];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int f = ax[d] == 0 ? 2 * d : (ax[d] == P - 1 ? 2 * d + 1 : -1);
      if (f < 0) continue;
      const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
      v = v - XB(lc)[(f * 3 + c) * P2 + ax[t2] * P + ax[t1]];
    }
    y[c * N + (long long)e * P3 + node] = cvt_out<double, T>(v, 2 * sc);  // quadratic in u
  }
#undef SU
#undef SO
#undef UQ
#undef WJ
#undef XB
}

template <int P>
size_t conv_smem(int cpb) {
  using Dm = ConvDims<P>;
  return ((size_t)Dm::shared + (size_t)cpb * Dm::per_cell) * sizeof(double) + (size_t)12 * cpb * sizeof(int);
}

template <int P>
int conv_default_cpb() {
  // about 64 KB of shared memory per block (3 cells at k = 3), at most 8
  const int c = (int)(64 * 1024 / conv_smem<P>(1));
  return c < 1 ? 1 : (c > 8 ? 8 : c);
}

template <int P>
int conv_max_cpb() {
  int c = 1;
  while (c < 64 && conv_smem<P>(c + 1) <= 200 * 1024) ++c;
  return c;
}

template <int P>
int launch_convective_p(const Mesh& m, const double* u, double* y, cudaStream_t s) {
  const int cpb = m.cpb_conv > 0 ? m.cpb_conv : conv_default_cpb<P>();
  const size_t smem = conv_smem<P>(cpb);
  const bool df = m.f64_arith == SIPG_F64_DOUBLE_FLOAT;
  cudaError_t e;
  if (smem > 48 * 1024) {
    e = df ? cudaFuncSetAttribute(convective_kernel<dfl, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
           : cudaFuncSetAttribute(convective_kernel<double, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(convective)");
  }
  const unsigned blocks = (unsigned)((m.ncell + cpb - 1) / cpb);
  if (df) {
    const int st = launch_df_scale(m, u, 3 * m.ncell * P * P * P, nullptr, 0, nullptr, s);
    if (st) return st;
  }
  if (df)
    convective_kernel<dfl, P><<<blocks, kConvThreads, smem, s>>>(
        make_geo<dfl>(m), m.dconvdf, (int)m.conv_off[1], (int)m.conv_off[2], (int)m.conv_off[3],
        (int)m.conv_off[4], u, y, cpb);
  else
    convective_kernel<double, P><<<blocks, kConvThreads, smem, s>>>(
        make_geo<double>(m), m.dconv64, (int)m.conv_off[1], (int)m.conv_off[2], (int)m.conv_off[3],
        (int)m.conv_off[4], u, y, cpb);
  const_cast<Mesh&>(m).launches++;
  e = cudaGetLastError();
  return e == cudaSuccess ? SIPG_OK : cuda_fail(e, "convective launch");
}

}  // namespace

int launch_convective(const Mesh& m, const double* u, double* y, cudaStream_t s) {
  switch (m.p) {
    case 2: return launch_convective_p<2>(m, u, y, s);
    case 3: return launch_convective_p<3>(m, u, y, s);
    case 4: return launch_convective_p<4>(m, u, y, s);
    case 5: return launch_convective_p<5>(m, u, y, s);
    case 6: return launch_convective_p<6>(m, u, y, s);
    case 7: return launch_convective_p<7>(m, u, y, s);
    case 8: return launch_convective_p<8>(m, u, y, s);
    default: return fail(SIPG_EINVAL, "unsupported degree");
  }
}

int convective_cpb(const Mesh& m, int* max_cpb) {
  int def = 1, mx = 1;
  switch (m.p) {
#define SIPG_CONV_CASE(P)      \
  case P:                      \
    def = conv_default_cpb<P>(); \
    mx = conv_max_cpb<P>();    \
    break;
    SIPG_CONV_CASE(2)
    SIPG_CONV_CASE(3)
    SIPG_CONV_CASE(4)
    SIPG_CONV_CASE(5)
    SIPG_CONV_CASE(6)
    SIPG_CONV_CASE(7)
    SIPG_CONV_CASE(8)
#undef SIPG_CONV_CASE
    default: break;
  }
  if (max_cpb) *max_cpb = mx;
  return m.cpb_conv > 0 ? m.cpb_conv : def;
}

}  // namespace sipg
