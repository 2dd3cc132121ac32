// Velocity-pressure coupling operators of the pressure-projection step,
// variant V3c (Sec. 3.3), in FP64:
//
//   divergence, Eq. (av3):  y_i = (grad phi_i, u)_e - (phi_i, {{u}}^ND . n)_de
//   gradient,   Eq. (bv3):  y_(d,i) = (d phi_i / dx_d, p)_e - (phi_i, {{p}}^ND n_d)_de
//   div-div local projection, Eq. (div-div):  (M + tau_e B) w = rhs cell by cell,
//       B_(d,d') = (d phi_i / dx_d, d phi_j / dx_d')_e,  tau_e of Eq. (tauD)
//
// ({{.}}^ND: the average on interior and periodic faces, the own trace on
// boundary faces, Sec. 3.1.)  On the separable map every one of these
// factorises into 1D matrices per direction and layer:
//   (d phi_i / dx, phi_j) = C (x) M_y (x) M_z  with C[a][b] = int l_a' l_b, the
//   same matrix for every layer (the Jacobian cancels);
//   the face integral over an x-face is M_y (x) M_z applied to the face values;
//   B_(x,x) = K_x (x) M_y (x) M_z,  B_(x,y) = C (x) C^T (x) M_z, ... .
// So the divergence and gradient are, per direction d, the 1D operator
// "C v plus the central-flux end terms" along d followed by the layer mass
// matrices along the other two directions; the end terms need one value of
// the neighbour's line (its value at the shared face).  Cells are processed
// cell-centrically (each cell writes only its own outputs, no atomics).
//
// The local projection is solved per cell by CG preconditioned with the
// tensorial inverse mass matrix (one thread block per cell, all vectors in
// shared memory); Sec. 3.3 solves these local problems iteratively.
#include <cmath>

#include "apply.cuh"

namespace sipg {

namespace {

constexpr int kDgThreads = 256;

// 1D line operator of the divergence / gradient along one direction:
// w = C v, then the central-flux end terms: the high face (n = +e_d) subtracts
// {{v}} there, the low face (n = -e_d) adds it; {{v}} = (v_own + v_nb) / 2 on an
// interior face, v_own on a boundary face.
template <int P>
__device__ __forceinline__ void line_divgrad(double (&w)[P], const double (&v)[P], const double* __restrict__ C,
                                             int kL, double vL, int kR, double vR) {
  matvec(w, C, v);
  w[P - 1] -= kR == 0 ? 0.5 * (v[P - 1] + vR) : v[P - 1];
  w[0] += kL == 0 ? 0.5 * (v[0] + vL) : v[0];
}

// MODE 0: divergence (3 components in, 1 out); MODE 1: gradient (1 in, 3 out).
template <int P, int MODE>
__global__ void __launch_bounds__(kDgThreads) divgrad_kernel(Geo<double> g, const double* __restrict__ C,
                                                             const double* __restrict__ x, double* __restrict__ y,
                                                             int cpb) {
  using O = LayerOff<P>;
  constexpr int P2 = P * P, P3 = P * P * P;
  constexpr int NIN = MODE == 0 ? 3 : 1;
  extern __shared__ __align__(16) unsigned char smraw[];
  double* sv = reinterpret_cast<double*>(smraw);  // inputs [NIN][cpb][P3]
  double* w1 = sv + (size_t)NIN * cpb * P3;        // [cpb][P3]
  double* w2 = w1 + (size_t)cpb * P3;              // [cpb][P3]
  double* acc = w2 + (size_t)cpb * P3;             // MODE 0: [cpb][P3]
  const int cs = threadIdx.x / P2;
  const int t = threadIdx.x - cs * P2;
  const int ti = t % P, tj = t / P;
  const long long cell0 = (long long)blockIdx.x * cpb;
  const int e = (int)(cell0 + cs);
  const bool active = cs < cpb && e < g.ncell;
  const int nc = (int)min((long long)cpb, (long long)g.ncell - cell0);
  const long long N = (long long)g.ncell * P3;
  for (int c = 0; c < NIN; ++c)
    for (int idx = threadIdx.x; idx < nc * P3; idx += blockDim.x)
      sv[(size_t)c * cpb * P3 + idx] = x[c * N + cell0 * P3 + idx];
  if (MODE == 0)
    for (int idx = threadIdx.x; idx < nc * P3; idx += blockDim.x) acc[idx] = 0.0;
  __syncthreads();
  int id[3] = {0, 0, 0};
  if (active) {
    id[0] = e % g.n[0];
    id[1] = (e / g.n[0]) % g.n[1];
    id[2] = e / (g.n[0] * g.n[1]);
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int d2 = d == 0 ? 1 : 0;  // the two other directions, d3 last
    const int d3 = d == 2 ? 1 : 2;
    const int comp = MODE == 0 ? d : 0;
    if (active) {
      int start, step;
      line_geom<P>(d, ti, tj, start, step);
      double v[P], w[P];
      load_line<double, P>(v, sv + (size_t)comp * cpb * P3 + (size_t)cs * P3, start, step);
      int nbL, nbR, kL, kR, jl, jr;
      face_neighbor(g, d, 0, id[d], e, nbL, kL, jl);
      face_neighbor(g, d, 1, id[d], e, nbR, kR, jr);
      const double* xc = x + comp * N;
      const double vL = kL == 0 ? xc[(long long)nbL * P3 + start + (P - 1) * step] : 0.0;
      const double vR = kR == 0 ? xc[(long long)nbR * P3 + start] : 0.0;
      line_divgrad<P>(w, v, C, kL, vL, kR, vR);
      store_line<double, P>(w1 + (size_t)cs * P3, w, start, step);
    }
    __syncthreads();
    if (active) {
      int start, step;
      line_geom<P>(d2, ti, tj, start, step);
      double v[P], r[P];
      load_line<double, P>(v, w1 + (size_t)cs * P3, start, step);
      matvec(r, g.tab[d2] + id[d2] * O::stride + O::M, v);
      store_line<double, P>(w2 + (size_t)cs * P3, r, start, step);
    }
    __syncthreads();
    if (active) {
      int start, step;
      line_geom<P>(d3, ti, tj, start, step);
      double v[P], r[P];
      load_line<double, P>(v, w2 + (size_t)cs * P3, start, step);
      matvec(r, g.tab[d3] + id[d3] * O::stride + O::M, v);
      double* dst = (MODE == 0 ? acc : w1) + (size_t)cs * P3 + start;
#pragma unroll
      for (int a = 0; a < P; ++a) dst[a * step] = MODE == 0 ? dst[a * step] + r[a] : r[a];
    }
    __syncthreads();
    if (MODE == 1) {
      for (int idx = threadIdx.x; idx < nc * P3; idx += blockDim.x) y[d * N + cell0 * P3 + idx] = w1[idx];
      __syncthreads();
    }
  }
  if (MODE == 0)
    for (int idx = threadIdx.x; idx < nc * P3; idx += blockDim.x) y[cell0 * P3 + idx] = acc[idx];
}

// tau_D of Eq. (tauD), one warp per cell: the volume average of each velocity
// component (the cell integral of phi_i is the product of the 1D mass
// matrices' row sums), tau = zeta |ubar| V^(1/3) dt.
template <int P>
__global__ void tau_div_kernel(Geo<double> g, const double* __restrict__ u, double zeta, double dt,
                               double* __restrict__ tau) {
  using O = LayerOff<P>;
  constexpr int P3 = P * P * P;
  __shared__ double rs[8][3][P];  // row sums per warp of the block (blockDim = 256)
  const int wib = threadIdx.x >> 5;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const bool valid = warp < g.ncell;
  const int e = valid ? warp : 0;
  const int id[3] = {e % g.n[0], (e / g.n[0]) % g.n[1], e / (g.n[0] * g.n[1])};
  if (lane < 3 * P) {
    const int d = lane / P, a = lane % P;
    const double* Md = (d == 0 ? g.tab[0] + id[0] * O::stride : (d == 1 ? g.tab[1] + id[1] * O::stride
                                                                       : g.tab[2] + id[2] * O::stride)) + O::M;
    double r = 0.0;
#pragma unroll
    for (int q = 0; q < P; ++q) r += Md[a * P + q];
    rs[wib][d][a] = r;
  }
  __syncwarp();
  if (!valid) return;
  const long long N = (long long)g.ncell * P3;
  double s[3] = {0.0, 0.0, 0.0}, vol = 0.0;
  for (int i = lane; i < P3; i += 32) {
    const int a = i % P, b = (i / P) % P, c = i / (P * P);
    const double m = rs[wib][0][a] * rs[wib][1][b] * rs[wib][2][c];
    vol += m;
#pragma unroll
    for (int d = 0; d < 3; ++d) s[d] += m * u[d * N + (long long)e * P3 + i];
  }
  for (int o = 16; o > 0; o >>= 1) {
    vol += __shfl_down_sync(0xffffffffu, vol, o);
#pragma unroll
    for (int d = 0; d < 3; ++d) s[d] += __shfl_down_sync(0xffffffffu, s[d], o);
  }
  if (lane == 0) {
    const double ux = s[0] / vol, uy = s[1] / vol, uz = s[2] / vol;
    tau[e] = zeta * sqrt(ux * ux + uy * uy + uz * uz) * cbrt(vol) * dt;
  }
}

// ------------------------------------------------------ one-cell operators
// One thread block per cell; thread t < P^2 owns line t of each phase.
template <typename T>
struct CellCtxT {
  const T* L[3];  // the cell's layer table per direction
  const T* C;     // C (shared memory)
  const T* Ct;    // C^T (shared memory)
  int t;
  bool active;    // t < P^2
};
using CellCtx = CellCtxT<double>;

// out (op)= scale * (A_x (x) A_y (x) A_z) in, where direction r's matrix is
// A_r + c_r B_r (B_r may be null); in, out: [P3]; t1, t2: [P3] scratch.
// op: 0 store, 1 add.
template <int P, typename T>
__device__ void cell_chain(const CellCtxT<T>& cc, const T* const (&A)[3], const T* const (&B)[3], const T (&cB)[3],
                           const T* in, T* out, T* t1, T* t2, int op, T scale) {
  const int ti = cc.t % P, tj = cc.t / P;
  const T* src[3] = {in, t1, t2};
  T* dst[3] = {t1, t2, out};
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    if (cc.active) {
      int start, step;
      line_geom<P>(r, ti, tj, start, step);
      T v[P], w[P];
      load_line<T, P>(v, src[r], start, step);
      matvec(w, A[r], v);
      if (B[r]) {
        T w2[P];
        matvec(w2, B[r], v);
#pragma unroll
        for (int a = 0; a < P; ++a) w[a] = fma(cB[r], w2[a], w[a]);
      }
      if (r < 2) {
        store_line<T, P>(dst[r], w, start, step);
      } else {
#pragma unroll
        for (int a = 0; a < P; ++a) {
          const T val = scale * w[a];
          dst[r][start + a * step] = op ? dst[r][start + a * step] + val : val;
        }
      }
    }
    __syncthreads();
  }
}

// y = (M + tau B) u on one cell: u, y: [3][P3]
template <int P, typename T>
__device__ void divdiv_cell(const CellCtxT<T>& cc, T tau, const T* u, T* y, T* t1, T* t2) {
  using O = LayerOff<P>;
  constexpr int P3 = P * P * P;
  const T* Mr[3] = {cc.L[0] + O::M, cc.L[1] + O::M, cc.L[2] + O::M};
  const T* Kr[3] = {cc.L[0] + O::K, cc.L[1] + O::K, cc.L[2] + O::K};
  for (int d = 0; d < 3; ++d) {
    // diagonal block: (M_d + tau K_d) along d, M along the others
    {
      const T* A[3] = {Mr[0], Mr[1], Mr[2]};
      const T* B[3] = {nullptr, nullptr, nullptr};
      T cB[3] = {T(0), T(0), T(0)};
      B[d] = Kr[d];
      cB[d] = tau;
      cell_chain<P>(cc, A, B, cB, u + d * P3, y + d * P3, t1, t2, 0, T(1));
    }
    // off-diagonal blocks: C along d (test derivative), C^T along d' (trial derivative)
    for (int dp = 0; dp < 3; ++dp) {
      if (dp == d) continue;
      const T* A[3] = {Mr[0], Mr[1], Mr[2]};
      A[d] = cc.C;
      A[dp] = cc.Ct;
      const T* B[3] = {nullptr, nullptr, nullptr};
      const T cB[3] = {T(0), T(0), T(0)};
      cell_chain<P>(cc, A, B, cB, u + dp * P3, y + d * P3, t1, t2, 1, tau);
    }
  }
}

// z = P^-1 r per component with the block preconditioner of (M + tau B):
// component d's diagonal block (M_d + tau K_d) (x) M (x) M is a tensor
// product, so its inverse is Pk[d] = (M_d + tau K_d)^-1 along d and the 1D
// inverse mass along the other two directions.
template <int P, typename T>
__device__ void blockprec_cell(const CellCtxT<T>& cc, const T* Pk, const T* r, T* z, T* t1, T* t2) {
  using O = LayerOff<P>;
  constexpr int P2 = P * P, P3 = P * P * P;
  for (int d = 0; d < 3; ++d) {
    const T* A[3] = {cc.L[0] + O::Mi, cc.L[1] + O::Mi, cc.L[2] + O::Mi};
    A[d] = Pk + d * P2;
    const T* B[3] = {nullptr, nullptr, nullptr};
    const T cB[3] = {T(0), T(0), T(0)};
    cell_chain<P>(cc, A, B, cB, r + d * P3, z + d * P3, t1, t2, 0, T(1));
  }
}

// Pk[d] = (M_d + tau K_d)^-1 for d < 3 (FP64 Gauss-Jordan of an SPD P x P
// matrix, one thread per direction); the caller synchronises.
template <int P, typename T>
__device__ void blockprec_setup(const CellCtxT<T>& cc, double tau, T* Pk) {
  using O = LayerOff<P>;
  constexpr int P2 = P * P;
  if (threadIdx.x < 3) {
    const int d = threadIdx.x;
    double a[P2], inv[P2];
    for (int i = 0; i < P2; ++i) {
      a[i] = cvt_out<double, T>(cc.L[d][O::M + i]) + tau * cvt_out<double, T>(cc.L[d][O::K + i]);
      inv[i] = (i / P == i % P) ? 1.0 : 0.0;
    }
    for (int c = 0; c < P; ++c) {
      const double piv = 1.0 / a[c * P + c];
      for (int j = 0; j < P; ++j) {
        a[c * P + j] *= piv;
        inv[c * P + j] *= piv;
      }
      for (int r = 0; r < P; ++r) {
        if (r == c) continue;
        const double f = a[r * P + c];
        for (int j = 0; j < P; ++j) {
          a[r * P + j] -= f * a[c * P + j];
          inv[r * P + j] -= f * inv[c * P + j];
        }
      }
    }
    for (int i = 0; i < P2; ++i) Pk[d * P2 + i] = cvt_in<T, double>(inv[i]);
  }
}

// sum of v over the block (blockDim <= 1024), result broadcast to all threads
__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) s += red[w];
  return s;
}

template <int P, typename T>
__device__ CellCtxT<T> cell_ctx(const Geo<T>& g, int e, const T* C, const T* Ct) {
  using O = LayerOff<P>;
  CellCtxT<T> cc;
  const int id[3] = {e % g.n[0], (e / g.n[0]) % g.n[1], e / (g.n[0] * g.n[1])};
  for (int d = 0; d < 3; ++d) cc.L[d] = g.tab[d] + id[d] * O::stride;
  cc.C = C;
  cc.Ct = Ct;
  cc.t = threadIdx.x;
  cc.active = threadIdx.x < P * P;
  return cc;
}

// stage C and C^T in shared memory
template <int P, typename T>
__device__ void stage_c(const T* __restrict__ Cg, T* C, T* Ct) {
  for (int i = threadIdx.x; i < P * P; i += blockDim.x) {
    const int a = i / P, b = i % P;
    C[i] = Cg[i];
    Ct[b * P + a] = Cg[i];
  }
}

template <int P>
__global__ void divdiv_apply_kernel(Geo<double> g, const double* __restrict__ Cg, const double* __restrict__ tau,
                                    const double* __restrict__ u, double* __restrict__ y) {
  constexpr int P3 = P * P * P;
  extern __shared__ __align__(16) unsigned char smraw[];
  double* su = reinterpret_cast<double*>(smraw);  // [3][P3]
  double* sy = su + 3 * P3;                        // [3][P3]
  double* t1 = sy + 3 * P3;
  double* t2 = t1 + P3;
  double* C = t2 + P3;
  double* Ct = C + P * P;
  const int e = blockIdx.x;
  const long long N = (long long)g.ncell * P3;
  for (int i = threadIdx.x; i < 3 * P3; i += blockDim.x) su[i] = u[(i / P3) * N + (long long)e * P3 + i % P3];
  stage_c<P>(Cg, C, Ct);
  __syncthreads();
  const CellCtx cc = cell_ctx<P>(g, e, C, Ct);
  divdiv_cell<P>(cc, tau[e], su, sy, t1, t2);
  for (int i = threadIdx.x; i < 3 * P3; i += blockDim.x) y[(i / P3) * N + (long long)e * P3 + i % P3] = sy[i];
}

// Per-cell CG on (M + tau B) x = rhs, preconditioned by the inverse of its
// component-diagonal blocks (blockprec_cell; M^-1 when tau = 0); x holds the
// initial guess.  status[0] |= 1 if a cell stops at maxit, |= 2 on breakdown;
// status[1] = max iterations over the cells.  T = double or dfl: the vectors
// and contractions in T, the dot products summed per thread in T and over the
// block in FP64, the CG scalars in FP64.
template <typename T, int P>
__global__ void divdiv_solve_kernel(Geo<T> g, const T* __restrict__ Cg, const double* __restrict__ tau,
                                    const double* __restrict__ rhs, double* __restrict__ x, double rtol, int maxit,
                                    int* __restrict__ status) {
  constexpr int P3 = P * P * P, V = 3 * P3;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sx = reinterpret_cast<T*>(smraw);
  T* sr = sx + V;
  T* sp = sr + V;
  T* sq = sp + V;  // A p, and after the updates z = M^-1 r (one buffer)
  T* sz = sq;
  T* t1 = sq + V;
  T* t2 = t1 + P3;
  T* C = t2 + P3;
  T* Ct = C + P * P;
  T* Pk = Ct + P * P;  // [3][P2] block preconditioner
  double* red = reinterpret_cast<double*>(Pk + 3 * P * P);  // 32
  const int e = blockIdx.x;
  const long long N = (long long)g.ncell * P3;
  // the call's scale exponent covers rhs and the initial x: vectors in T hold
  // v 2^-sc; r.r is compared with the unscaled bb (2 sc), the other dot
  // products only enter ratios
  const int sc = call_scale(g);
  double bb = 0.0;
  for (int i0 = threadIdx.x; i0 < V; i0 += 2 * blockDim.x) {
    double xv[2], bv[2];  // the loads of two entries issued before their conversions
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int i = i0 + j * blockDim.x;
      const long long gi = (i / P3) * N + (long long)e * P3 + i % P3;
      xv[j] = i < V ? __ldg(x + gi) : 0.0;
      bv[j] = i < V ? __ldg(rhs + gi) : 0.0;
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int i = i0 + j * blockDim.x;
      if (i < V) {
        sx[i] = cvt_in<T, double>(xv[j], sc);
        sr[i] = cvt_in<T, double>(bv[j], sc);
        bb += bv[j] * bv[j];
      }
    }
  }
  stage_c<P>(Cg, C, Ct);
  const CellCtxT<T> cc = cell_ctx<P>(g, e, (const T*)C, (const T*)Ct);
  blockprec_setup<P>(cc, tau[e], Pk);
  __syncthreads();
  bb = block_sum(bb, red);
  const T te = cvt_in<T, double>(tau[e]);
  // r = rhs - A x
  divdiv_cell<P>(cc, te, sx, sq, t1, t2);
  T acc = T(0);
  for (int i = threadIdx.x; i < V; i += blockDim.x) {
    sr[i] = sr[i] - sq[i];
    acc = fma(sr[i], sr[i], acc);
  }
  __syncthreads();
  double rr = block_sum(cvt_out<double, T>(acc, 2 * sc), red);
  blockprec_cell<P>(cc, Pk, sr, sz, t1, t2);
  acc = T(0);
  for (int i = threadIdx.x; i < V; i += blockDim.x) {
    sp[i] = sz[i];
    acc = fma(sr[i], sz[i], acc);
  }
  __syncthreads();
  double rz = block_sum(cvt_out<double, T>(acc), red);
  const double tol2 = rtol * rtol * bb;
  int it = 0;
  bool broke = false;
  while (rr > tol2 && it < maxit) {
    divdiv_cell<P>(cc, te, sp, sq, t1, t2);
    acc = T(0);
    for (int i = threadIdx.x; i < V; i += blockDim.x) acc = fma(sp[i], sq[i], acc);
    const double pq = block_sum(cvt_out<double, T>(acc), red);
    if (!(pq > 0.0)) {
      broke = true;
      break;
    }
    const double alpha = rz / pq;
    const T ap = cvt_in<T, double>(alpha), am = cvt_in<T, double>(-alpha);
    acc = T(0);
    for (int i = threadIdx.x; i < V; i += blockDim.x) {
      sx[i] = fma(ap, sp[i], sx[i]);
      sr[i] = fma(am, sq[i], sr[i]);
      acc = fma(sr[i], sr[i], acc);
    }
    __syncthreads();
    rr = block_sum(cvt_out<double, T>(acc, 2 * sc), red);
    blockprec_cell<P>(cc, Pk, sr, sz, t1, t2);
    acc = T(0);
    for (int i = threadIdx.x; i < V; i += blockDim.x) acc = fma(sr[i], sz[i], acc);
    const double rzn = block_sum(cvt_out<double, T>(acc), red);
    const T bt = cvt_in<T, double>(rzn / rz);
    rz = rzn;
    for (int i = threadIdx.x; i < V; i += blockDim.x) sp[i] = fma(bt, sp[i], sz[i]);
    __syncthreads();
    ++it;
  }
  for (int i = threadIdx.x; i < V; i += blockDim.x)
    x[(i / P3) * N + (long long)e * P3 + i % P3] = cvt_out<double, T>(sx[i], sc);
  if (threadIdx.x == 0) {
    if (broke) atomicOr(status, 2);
    else if (rr > tol2) atomicOr(status, 1);
    atomicMax(status + 1, it);
  }
}

// ------------------------------------------------- viscous operator coupling
// The divergence-form viscous operator of Sec. 3.2 (iii) is nu (L + T) plus
// the mass term: 2 eps(v):eps(u) = grad v : grad u + grad v : grad u^T and
// 2 eps(u) n = (grad u) n + (grad u)^T n, so the component-wise SIPG Laplacian
// L carries the grad u parts and the penalty, and T the transposed-gradient
// parts:
//   T(v, u) = sum_e (grad v : grad u^T)_e
//           - sum_F int ( {{(grad u)^T n}} . [v] + {{(grad v)^T n}} . [u] )
//           - sum_{F Dirichlet} int ( (grad u)^T n . v + (grad v)^T n . u ).
// On a face of cell e with outward normal s e_d, ((grad u)^T n)_m = s d_m u_d,
// so for a test function phi e_i of e the face contributes
//   (A) -s (phi, {{d_i u_d}})_F      ({{.}}: the own value on a Dirichlet face)
//   (B) only for i = d: -w s sum_m (d_m phi, J_m)_F with J = u_own - u_nb,
//       w = 1/2 on an interior face, J = u_own, w = 1 on a Dirichlet face;
// Neumann faces contribute nothing.  The cell part of output i is
// sum_j B_(j,i) u_j, B_(j,i) = (d_j phi_a, d_i phi_b): K along i for j = i,
// else C along j (test derivative) and C^T along i (trial derivative), M along
// the third direction.  On a d-face, in-face integrals are M / C / C^T along
// the two tangential directions t1 < t2 (the Jacobians cancel as in C).
template <typename T, int P>
__global__ void viscous_t_kernel(Geo<T> g, const T* __restrict__ Cg, const double* __restrict__ u,
                                 double* __restrict__ y, double scale, const int* __restrict__ skip) {
  if (skip && *skip) return;
  using O = LayerOff<P>;
  constexpr int P2 = P * P, P3 = P * P * P;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* su = reinterpret_cast<T*>(smraw);  // [3][P3] input
  T* so = su + 3 * P3;                   // [3][P3] T u
  T* t1 = so + 3 * P3;
  T* t2 = t1 + P3;
  T* C = t2 + P3;
  T* Ct = C + P2;
  T* fb = Ct + P2;  // face arrays [11][P2]
  const int e = blockIdx.x;
  const long long N = (long long)g.ncell * P3;
  const int xsc = call_scale(g);  // the call's scale exponent (double-float)
  for (int c = 0; c < 3; ++c) stage_cvt<T, double>(su + c * P3, u + c * N + (long long)e * P3, P3, xsc);
  stage_c<P>(Cg, C, Ct);
  __syncthreads();
  const CellCtxT<T> cc = cell_ctx<P>(g, e, (const T*)C, (const T*)Ct);
  // cell part
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      const T* A[3] = {cc.L[0] + O::M, cc.L[1] + O::M, cc.L[2] + O::M};
      if (i == j) {
        A[i] = cc.L[i] + O::K;
      } else {
        A[i] = Ct;
        A[j] = C;
      }
      const T* B[3] = {nullptr, nullptr, nullptr};
      const T cB[3] = {T(0), T(0), T(0)};
      cell_chain<P>(cc, A, B, cB, su + j * P3, so + i * P3, t1, t2, j == 0 ? 0 : 1, T(1));
    }
  // faces
  const int id[3] = {e % g.n[0], (e / g.n[0]) % g.n[1], e / (g.n[0] * g.n[1])};
  const bool act = threadIdx.x < P2;
  const int fb_ = threadIdx.x % P, fc_ = threadIdx.x / P;  // face node along (t1, t2)
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int ta = d == 0 ? 1 : 0;  // t1
    const int tb = d == 2 ? 1 : 2;  // t2
    const int sd = d == 0 ? 1 : (d == 1 ? P : P2);
    const int sa = ta == 0 ? 1 : (ta == 1 ? P : P2);
    const int sb = tb == 0 ? 1 : (tb == 1 ? P : P2);
    for (int side = 0; side < 2; ++side) {
      int nb, kind, jl;
      face_neighbor(g, d, side, id[d], e, nb, kind, jl);
      if (kind == SIPG_BC_NEUMANN) continue;  // the same for the whole block
      const T s = side ? T(1) : T(-1);
      const T w = kind == 0 ? T(0.5) : T(1);
      const int aend = side ? P - 1 : 0;
      const T* dEnd = cc.L[d] + (side ? O::dR : O::dL);
      const int base = fb_ * sa + fc_ * sb;  // node (a = 0, b, c)
      if (act) {
        T g_own = T(0);
#pragma unroll
        for (int a = 0; a < P; ++a) g_own = fma(dEnd[a], su[d * P3 + base + a * sd], g_own);
        const T ud = su[d * P3 + base + aend * sd];
        const T ua = su[ta * P3 + base + aend * sd];
        const T ub = su[tb * P3 + base + aend * sd];
        T avgN, avgU, Jd, Ja, Jb;
        if (kind == 0) {
          const int nend = P - 1 - aend;
          const T* dN = g.tab[d] + jl * O::stride + (side ? O::dL : O::dR);
          const double* un = u + (long long)nb * P3 + base;
          double r[P + 2];  // all loads issued before the conversions
#pragma unroll
          for (int a = 0; a < P; ++a) r[a] = __ldg(un + d * N + a * sd);
          r[P] = __ldg(un + ta * N + nend * sd);
          r[P + 1] = __ldg(un + tb * N + nend * sd);
          T g_nb = T(0);
#pragma unroll
          for (int a = 0; a < P; ++a) g_nb = fma(dN[a], cvt_in<T, double>(r[a], xsc), g_nb);
          const T udn = cvt_in<T, double>(nend ? r[P - 1] : r[0], xsc);
          const T uan = cvt_in<T, double>(r[P], xsc);
          const T ubn = cvt_in<T, double>(r[P + 1], xsc);
          avgN = T(0.5) * (g_own + g_nb);
          avgU = T(0.5) * (ud + udn);
          Jd = ud - udn;
          Ja = ua - uan;
          Jb = ub - ubn;
        } else {  // Dirichlet
          avgN = g_own;
          avgU = ud;
          Jd = ud;
          Ja = ua;
          Jb = ub;
        }
        const int f = fb_ + P * fc_;
        fb[0 * P2 + f] = avgN;
        fb[1 * P2 + f] = avgU;
        fb[2 * P2 + f] = Jd;
        fb[3 * P2 + f] = Ja;
        fb[4 * P2 + f] = Jb;
      }
      __syncthreads();
      if (act) {  // contractions along t1 (over b')
        const T* Ma = cc.L[ta] + O::M;
        T f1 = T(0), f2 = T(0), f3 = T(0), f4 = T(0), f5 = T(0), f6 = T(0);
#pragma unroll
        for (int q = 0; q < P; ++q) {
          const int src = q + P * fc_;
          f1 = fma(Ma[fb_ * P + q], fb[0 * P2 + src], f1);
          f2 = fma(Ct[fb_ * P + q], fb[1 * P2 + src], f2);
          f3 = fma(Ma[fb_ * P + q], fb[1 * P2 + src], f3);
          f4 = fma(Ma[fb_ * P + q], fb[2 * P2 + src], f4);
          f5 = fma(C[fb_ * P + q], fb[3 * P2 + src], f5);
          f6 = fma(Ma[fb_ * P + q], fb[4 * P2 + src], f6);
        }
        const int f = fb_ + P * fc_;
        fb[5 * P2 + f] = f1;
        fb[6 * P2 + f] = f2;
        fb[7 * P2 + f] = f3;
        fb[8 * P2 + f] = f4;
        fb[9 * P2 + f] = f5;
        fb[10 * P2 + f] = f6;
      }
      __syncthreads();
      if (act) {  // contractions along t2 (over c') and scatter to the own face node / line
        const T* Mb = cc.L[tb] + O::M;
        T r1 = T(0), r5 = T(0), r6 = T(0), r2 = T(0), r3 = T(0), r4 = T(0);
#pragma unroll
        for (int q = 0; q < P; ++q) {
          const int src = fb_ + P * q;
          r1 = fma(Mb[fc_ * P + q], fb[5 * P2 + src], r1);
          r2 = fma(Mb[fc_ * P + q], fb[6 * P2 + src], r2);
          r3 = fma(Ct[fc_ * P + q], fb[7 * P2 + src], r3);
          r4 = fma(Mb[fc_ * P + q], fb[8 * P2 + src], r4);
          r5 = fma(Mb[fc_ * P + q], fb[9 * P2 + src], r5);
          r6 = fma(C[fc_ * P + q], fb[10 * P2 + src], r6);
        }
        const int endn = base + aend * sd;
        so[d * P3 + endn] = so[d * P3 + endn] + (-(s * r1) - w * s * (r5 + r6));
        so[ta * P3 + endn] = so[ta * P3 + endn] + (-(s * r2));
        so[tb * P3 + endn] = so[tb * P3 + endn] + (-(s * r3));
        const T rall = -(w * s * r4);
#pragma unroll
        for (int a = 0; a < P; ++a) so[d * P3 + base + a * sd] = fma(dEnd[a], rall, so[d * P3 + base + a * sd]);
      }
      __syncthreads();
    }
  }
  // the final accumulation in FP64 (keeps the Laplace part's precision)
  const T sc = T(scale);
  for (int i = threadIdx.x; i < 3 * P3; i += blockDim.x) {
    const long long gi = (i / P3) * N + (long long)e * P3 + i % P3;
    y[gi] = y[gi] + cvt_out<double, T>(sc * so[i], xsc);
  }
}

int cell_threads(int p) { return (p * p + 31) / 32 * 32; }

int proj_cpb(int p) {
  const int c = kDgThreads / (p * p);
  return c < 1 ? 1 : c;
}

template <int P>
int launch_divgrad_p(const Mesh& m, const double* x, double* y, int mode, cudaStream_t s) {
  const int cpb = proj_cpb(P);
  const int threads = (cpb * P * P + 31) / 32 * 32;
  const int nbuf = mode == 0 ? 3 + 3 : 1 + 2;
  const size_t smem = (size_t)nbuf * cpb * P * P * P * sizeof(double);
  const unsigned blocks = (unsigned)((m.ncell + cpb - 1) / cpb);
  const Geo<double> g = make_geo<double>(m);
  cudaError_t e;
  if (mode == 0) {
    if (smem > 48 * 1024 &&
        (e = cudaFuncSetAttribute(divgrad_kernel<P, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess)
      return cuda_fail(e, "cudaFuncSetAttribute(divergence)");
    divgrad_kernel<P, 0><<<blocks, threads, smem, s>>>(g, m.dC64, x, y, cpb);
  } else {
    if (smem > 48 * 1024 &&
        (e = cudaFuncSetAttribute(divgrad_kernel<P, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess)
      return cuda_fail(e, "cudaFuncSetAttribute(gradient)");
    divgrad_kernel<P, 1><<<blocks, threads, smem, s>>>(g, m.dC64, x, y, cpb);
  }
  const_cast<Mesh&>(m).launches++;
  e = cudaGetLastError();
  return e == cudaSuccess ? SIPG_OK : cuda_fail(e, "divergence / gradient launch");
}

template <int P>
int launch_tau_p(const Mesh& m, const double* u, double zeta, double dt, double* tau, cudaStream_t s) {
  const int threads = 256;
  const unsigned blocks = (unsigned)((m.ncell * 32 + threads - 1) / threads);
  tau_div_kernel<P><<<blocks, threads, 0, s>>>(make_geo<double>(m), u, zeta, dt, tau);
  const_cast<Mesh&>(m).launches++;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SIPG_OK : cuda_fail(e, "tau_D launch");
}

template <int P>
int launch_divdiv_apply_p(const Mesh& m, const double* tau, const double* u, double* y, cudaStream_t s) {
  constexpr int P3 = P * P * P;
  const size_t smem = (size_t)(8 * P3 + 2 * P * P) * sizeof(double);
  cudaError_t e;
  if (smem > 48 * 1024 &&
      (e = cudaFuncSetAttribute(divdiv_apply_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
          cudaSuccess)
    return cuda_fail(e, "cudaFuncSetAttribute(div-div apply)");
  divdiv_apply_kernel<P><<<(unsigned)m.ncell, cell_threads(P), smem, s>>>(make_geo<double>(m), m.dC64, tau, u, y);
  const_cast<Mesh&>(m).launches++;
  e = cudaGetLastError();
  return e == cudaSuccess ? SIPG_OK : cuda_fail(e, "div-div apply launch");
}

template <int P>
int launch_divdiv_solve_p(const Mesh& m, const double* tau, const double* rhs, double* x, double rtol, int maxit,
                          int* status, cudaStream_t s) {
  constexpr int P3 = P * P * P;
  const size_t smem = (size_t)(12 * P3 + 2 * P3 + 5 * P * P + 32) * sizeof(double);
  const bool df = m.f64_arith == SIPG_F64_DOUBLE_FLOAT;
  cudaError_t e;
  if (smem > 48 * 1024) {
    e = df ? cudaFuncSetAttribute(divdiv_solve_kernel<dfl, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)
           : cudaFuncSetAttribute(divdiv_solve_kernel<double, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(div-div solve)");
  }
  if (df) {
    const int st = launch_df_scale(m, rhs, 3 * m.ncell * P3, x, 3 * m.ncell * P3, nullptr, s);
    if (st) return st;
  }
  if (df)
    divdiv_solve_kernel<dfl, P><<<(unsigned)m.ncell, cell_threads(P), smem, s>>>(make_geo<dfl>(m), m.dCdf, tau,
                                                                                 rhs, x, rtol, maxit, status);
  else
    divdiv_solve_kernel<double, P><<<(unsigned)m.ncell, cell_threads(P), smem, s>>>(make_geo<double>(m), m.dC64, tau,
                                                                                    rhs, x, rtol, maxit, status);
  const_cast<Mesh&>(m).launches++;
  e = cudaGetLastError();
  return e == cudaSuccess ? SIPG_OK : cuda_fail(e, "div-div solve launch");
}

template <int P>
int launch_viscous_t_p(const Mesh& m, const double* u, double* y, double scale, const int* skip, bool prescaled,
                       cudaStream_t s) {
  constexpr int P3 = P * P * P;
  const size_t smem = (size_t)(8 * P3 + 2 * P * P + 11 * P * P) * sizeof(double);
  cudaError_t e;
  if (smem > 48 * 1024) {
    e = m.f64_arith == SIPG_F64_DOUBLE_FLOAT
            ? cudaFuncSetAttribute(viscous_t_kernel<dfl, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
            : cudaFuncSetAttribute(viscous_t_kernel<double, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(viscous coupling)");
  }
  if (m.f64_arith == SIPG_F64_DOUBLE_FLOAT) {
    if (!df_coef_ok(scale)) return fail(SIPG_EINVAL, "double-float arithmetic needs nu in [2^-100, 2^100]");
    if (!prescaled) {
      const int st = launch_df_scale(m, u, 3 * m.ncell * P3, nullptr, 0, skip, s);
      if (st) return st;
    }
  }
  if (m.f64_arith == SIPG_F64_DOUBLE_FLOAT)
    viscous_t_kernel<dfl, P><<<(unsigned)m.ncell, cell_threads(P), smem, s>>>(make_geo<dfl>(m), m.dCdf, u, y, scale,
                                                                              skip);
  else
    viscous_t_kernel<double, P><<<(unsigned)m.ncell, cell_threads(P), smem, s>>>(make_geo<double>(m), m.dC64, u, y,
                                                                                 scale, skip);
  const_cast<Mesh&>(m).launches++;
  e = cudaGetLastError();
  return e == cudaSuccess ? SIPG_OK : cuda_fail(e, "viscous coupling launch");
}

}  // namespace

#define SIPG_PROJ_DISPATCH(CALL)                               \
  switch (m.p) {                                               \
    case 2: return CALL(2);                                    \
    case 3: return CALL(3);                                    \
    case 4: return CALL(4);                                    \
    case 5: return CALL(5);                                    \
    case 6: return CALL(6);                                    \
    case 7: return CALL(7);                                    \
    case 8: return CALL(8);                                    \
    default: return fail(SIPG_EINVAL, "unsupported degree");  \
  }

int launch_divergence(const Mesh& m, const double* u, double* y, cudaStream_t s) {
#define CALL(P) launch_divgrad_p<P>(m, u, y, 0, s)
  SIPG_PROJ_DISPATCH(CALL)
#undef CALL
}

int launch_gradient(const Mesh& m, const double* p, double* y, cudaStream_t s) {
#define CALL(P) launch_divgrad_p<P>(m, p, y, 1, s)
  SIPG_PROJ_DISPATCH(CALL)
#undef CALL
}

int launch_tau_div(const Mesh& m, const double* u, double zeta, double dt, double* tau, cudaStream_t s) {
#define CALL(P) launch_tau_p<P>(m, u, zeta, dt, tau, s)
  SIPG_PROJ_DISPATCH(CALL)
#undef CALL
}

int launch_divdiv_apply(const Mesh& m, const double* tau, const double* u, double* y, cudaStream_t s) {
#define CALL(P) launch_divdiv_apply_p<P>(m, tau, u, y, s)
  SIPG_PROJ_DISPATCH(CALL)
#undef CALL
}

int launch_viscous_t(const Mesh& m, const double* u, double* y, double scale, const int* skip, bool prescaled,
                     cudaStream_t s) {
#define CALL(P) launch_viscous_t_p<P>(m, u, y, scale, skip, prescaled, s)
  SIPG_PROJ_DISPATCH(CALL)
#undef CALL
}

int launch_divdiv_solve(const Mesh& m, const double* tau, const double* rhs, double* x, double rtol, int maxit,
                        int* status, cudaStream_t s) {
#define CALL(P) launch_divdiv_solve_p<P>(m, tau, rhs, x, rtol, maxit, status, s)
  SIPG_PROJ_DISPATCH(CALL)
#undef CALL
}

#undef SIPG_PROJ_DISPATCH

}  // namespace sipg
