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
// On the separable map: u at the quadrature points is three 1D
// interpolations (Sq[q][a] = l_a(z_q)); (d_k phi_a, f) = sum over the points
// of Dq[a][q] = w_q l_a'(z_q) along k (the Jacobian cancels) and
// W[a][q] = l_a(z_q) w_q J(z_q) along the other two directions; a face
// integral over a d-face uses W along its two tangential directions.  One
// thread block per cell; all intermediate tensors in shared memory; the
// arithmetic in FP64 or double-float (the mesh's FP64 arithmetic).
#include "apply.cuh"

namespace sipg {

namespace {

constexpr int kConvThreads = 128;

// dst (op)= scale * contraction along `dir` of src with Mtx[o * NI + i];
// src extents e[0..2] (x fastest, e[dir] == NI), dst extents equal except
// NO along dir; op: 0 store, 1 add.  All threads of the block take part.
template <typename T, int NI, int NO>
__device__ void contract(const T* src, T* dst, int e0, int e1, int e2, int dir, const T* Mtx, int op) {
  const int ein[3] = {e0, e1, e2};
  const int eo0 = dir == 0 ? NO : e0, eo1 = dir == 1 ? NO : e1;
  const int sin[3] = {1, e0, e0 * e1};
  const int sout[3] = {1, eo0, eo0 * eo1};
  const int da = dir == 0 ? 1 : 0, db = dir == 2 ? 1 : 2;
  const int na = ein[da];
  const int nl = na * ein[db];
  for (int l = threadIdx.x; l < nl; l += blockDim.x) {
    const int ia = l % na, ib = l / na;
    const T* s = src + ia * sin[da] + ib * sin[db];
    T* d = dst + ia * sout[da] + ib * sout[db];
    T v[NI];
#pragma unroll
    for (int i = 0; i < NI; ++i) v[i] = s[i * sin[dir]];
#pragma unroll
    for (int o = 0; o < NO; ++o) {
      T acc = T(0);
#pragma unroll
      for (int i = 0; i < NI; ++i) acc = fma(Mtx[o * NI + i], v[i], acc);
      T* t = d + o * sout[dir];
      *t = op ? *t + acc : acc;
    }
  }
  __syncthreads();
}

template <typename T, int P>
__global__ void __launch_bounds__(kConvThreads) convective_kernel(Geo<T> g, const T* __restrict__ tabs,
                                                                  long long off_D, long long off_W0,
                                                                  long long off_W1, long long off_W2,
                                                                  const double* __restrict__ u,
                                                                  double* __restrict__ y) {
  constexpr int Q = (3 * (P - 1)) / 2 + 1;
  constexpr int P2 = P * P, P3 = P * P * P, Q2 = Q * Q, Q3 = Q * Q * Q;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* su = reinterpret_cast<T*>(smraw);  // [3][P3] nodal input
  T* so = su + 3 * P3;                   // [3][P3] result
  T* uq = so + 3 * P3;                   // [3][Q3] values at the quadrature points
  T* ta = uq + 3 * Q3;                   // [Q3]
  T* tb = ta + Q3;                       // [Q3]
  T* Sq = tb + Q3;                       // [Q][P]
  T* Dq = Sq + Q * P;                    // [P][Q]
  T* W = Dq + P * Q;                     // [3][P][Q] layer-weighted values
  T* fo = W + 3 * P * Q;                 // face: own nodal values [3][P2]
  T* fn = fo + 3 * P2;                   // neighbour nodal values [3][P2]
  T* qo = fn + 3 * P2;                   // own values at face points [3][Q2]
  T* qn = qo + 3 * Q2;                   // neighbour values at face points [3][Q2]
  T* fl = qn + 3 * Q2;                   // flux [3][Q2]
  T* f1 = fl + 3 * Q2;                   // [P][Q] scratch
  T* f2 = f1 + P * Q;                    // [P][P] scratch
  const int e = blockIdx.x;
  const long long N = (long long)g.ncell * P3;
  const int id[3] = {e % g.n[0], (e / g.n[0]) % g.n[1], e / (g.n[0] * g.n[1])};
  for (int i = threadIdx.x; i < 3 * P3; i += blockDim.x) {
    su[i] = cvt_in<T, double>(u[(i / P3) * N + (long long)e * P3 + i % P3]);
    so[i] = T(0);
  }
  for (int i = threadIdx.x; i < Q * P; i += blockDim.x) {
    Sq[i] = tabs[i];
    Dq[i] = tabs[off_D + i];
    const int a = i / Q, q = i % Q;  // W[d][a][q] = Sq[q][a] * w_q J_d(z_q) of the cell's layer
    W[0 * P * Q + i] = tabs[q * P + a] * tabs[off_W0 + (long long)id[0] * Q + q];
    W[1 * P * Q + i] = tabs[q * P + a] * tabs[off_W1 + (long long)id[1] * Q + q];
    W[2 * P * Q + i] = tabs[q * P + a] * tabs[off_W2 + (long long)id[2] * Q + q];
  }
  __syncthreads();
  // u at the quadrature points
  for (int c = 0; c < 3; ++c) {
    contract<T, P, Q>(su + c * P3, ta, P, P, P, 0, Sq, 0);
    contract<T, P, Q>(ta, tb, Q, P, P, 1, Sq, 0);
    contract<T, P, Q>(tb, uq + c * Q3, Q, Q, P, 2, Sq, 0);
  }
  // cell part: y_i += sum_k (D_k (x) W (x) W) (u_i u_k)
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k) {
      for (int j = threadIdx.x; j < Q3; j += blockDim.x) ta[j] = uq[i * Q3 + j] * uq[k * Q3 + j];
      __syncthreads();
      contract<T, Q, P>(ta, tb, Q, Q, Q, 0, k == 0 ? Dq : W + 0 * P * Q, 0);
      contract<T, Q, P>(tb, ta, P, Q, Q, 1, k == 1 ? Dq : W + 1 * P * Q, 0);
      contract<T, Q, P>(ta, so + i * P3, P, P, Q, 2, k == 2 ? Dq : W + 2 * P * Q, 1);
    }
  // faces
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
    const int sd = d == 0 ? 1 : (d == 1 ? P : P2);
    const int s1 = t1 == 0 ? 1 : (t1 == 1 ? P : P2);
    const int s2 = t2 == 0 ? 1 : (t2 == 1 ? P : P2);
    for (int side = 0; side < 2; ++side) {
      int nb, kind, jl;
      face_neighbor(g, d, side, id[d], e, nb, kind, jl);
      const T s = side ? T(1) : T(-1);
      const int aend = side ? P - 1 : 0, nend = P - 1 - aend;
      for (int i = threadIdx.x; i < 3 * P2; i += blockDim.x) {
        const int c = i / P2, f = i % P2, b = f % P, cc = f / P;
        fo[i] = su[c * P3 + aend * sd + b * s1 + cc * s2];
        if (kind == 0) fn[i] = cvt_in<T, double>(u[c * N + (long long)nb * P3 + nend * sd + b * s1 + cc * s2]);
      }
      __syncthreads();
      for (int c = 0; c < 3; ++c) {
        contract<T, P, Q>(fo + c * P2, f1, P, P, 1, 0, Sq, 0);
        contract<T, P, Q>(f1, qo + c * Q2, Q, P, 1, 1, Sq, 0);
        if (kind == 0) {
          contract<T, P, Q>(fn + c * P2, f1, P, P, 1, 0, Sq, 0);
          contract<T, P, Q>(f1, qn + c * Q2, Q, P, 1, 1, Sq, 0);
        }
      }
      for (int j = threadIdx.x; j < Q2; j += blockDim.x) {
        const T um[3] = {qo[j], qo[Q2 + j], qo[2 * Q2 + j]};
        const T un = s * um[d];
        const T lm = T(2) * (un > T(0) ? un : -un);
        if (kind == 0) {
          const T up[3] = {qn[j], qn[Q2 + j], qn[2 * Q2 + j]};
          const T unb = s * up[d];
          const T lp = T(2) * (unb > T(0) ? unb : -unb);
          const T lam = lm > lp ? lm : lp;
#pragma unroll
          for (int c = 0; c < 3; ++c)
            fl[c * Q2 + j] = T(0.5) * (um[c] * un + up[c] * unb) + T(0.5) * lam * (um[c] - up[c]);
        } else if (kind == SIPG_BC_DIRICHLET) {
#pragma unroll
          for (int c = 0; c < 3; ++c) fl[c * Q2 + j] = um[c] * un + lm * um[c];
        } else {
#pragma unroll
          for (int c = 0; c < 3; ++c) fl[c * Q2 + j] = um[c] * un;
        }
      }
      __syncthreads();
      for (int c = 0; c < 3; ++c) {
        contract<T, Q, P>(fl + c * Q2, f1, Q, Q, 1, 0, W + t1 * P * Q, 0);
        contract<T, Q, P>(f1, f2, P, Q, 1, 1, W + t2 * P * Q, 0);
        for (int f = threadIdx.x; f < P2; f += blockDim.x) {
          const int b = f % P, cc = f / P;
          T* t = so + c * P3 + aend * sd + b * s1 + cc * s2;
          *t = *t - f2[f];
        }
        __syncthreads();
      }
    }
  }
  for (int i = threadIdx.x; i < 3 * P3; i += blockDim.x)
    y[(i / P3) * N + (long long)e * P3 + i % P3] = cvt_out<double, T>(so[i]);
}

template <int P>
int launch_convective_p(const Mesh& m, const double* u, double* y, cudaStream_t s) {
  constexpr int Q = (3 * (P - 1)) / 2 + 1;
  constexpr int P2 = P * P, P3 = P * P * P, Q2 = Q * Q, Q3 = Q * Q * Q;
  const size_t smem = (size_t)(6 * P3 + 5 * Q3 + 5 * P * Q + 6 * P2 + 9 * Q2 + P * Q + P2) * sizeof(double);
  const bool df = m.f64_arith == SIPG_F64_DOUBLE_FLOAT;
  cudaError_t e;
  if (smem > 48 * 1024) {
    e = df ? cudaFuncSetAttribute(convective_kernel<dfl, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
           : cudaFuncSetAttribute(convective_kernel<double, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(convective)");
  }
  if (df)
    convective_kernel<dfl, P><<<(unsigned)m.ncell, kConvThreads, smem, s>>>(
        make_geo<dfl>(m), m.dconvdf, m.conv_off[1], m.conv_off[2], m.conv_off[3], m.conv_off[4], u, y);
  else
    convective_kernel<double, P><<<(unsigned)m.ncell, kConvThreads, smem, s>>>(
        make_geo<double>(m), m.dconv64, m.conv_off[1], m.conv_off[2], m.conv_off[3], m.conv_off[4], u, y);
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

}  // namespace sipg
