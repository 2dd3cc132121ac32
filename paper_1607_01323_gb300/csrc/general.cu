// The SIPG Laplace / Helmholtz operator on a general (non-separable) map:
// SIPG_MAP_PERTURBED, the box plus a smooth displacement that vanishes on the
// box boundary.  With no separable structure the geometry is stored per
// quadrature point (Sec. 5: the iso-parametric degree-k map, Gauss k+1):
//   cell:  G = det J w J^-1 J^-T (6 values) and det J w (1), per Gauss point;
//   face:  g = w_F det J J^-1 J^-T e_d s  (= w dA J^-1 n, 3 values) and w dA,
//          per face Gauss point of each of the six faces, n = s J^-T e_d / |.|;
//   cell:  tau_e of Eq. (taue) from the quadrature volume and face areas.
// Cell term, per cell: reference gradients at the Gauss points by sum
// factorisation (interpolation S and derivative D at the Gauss points along
// x, y, z), f = nu G grad + c det J w u, and the transposed sweeps.  Faces,
// cell-centric as in the separable kernels: the traces and reference
// gradients of both sides at the face points, the flux terms of Sec. 3.2 (ii)
//   -(v, {{d_n u}}) - (d_n v, [u]/2) + tau [u] v        interior (and periodic),
//   -(v, d_n u) - (d_n v, u) + 2 tau_e u v              Dirichlet,
// nothing on Neumann faces, and the transposed contractions into the cell's
// own outputs (no atomics).  FP64 data; the arithmetic in FP64 or in
// double-float with the mesh's setting; one cell and component per block.
// The diagonal (Jacobi) sums a(phi_i, phi_i) directly per node.
#include <cmath>
#include <vector>

#include "apply.cuh"

namespace sipg {

// ------------------------------------------------------------------ host
void map_point(const sipg_mesh_desc& d, const double s[3], double x[3]) {
  for (int i = 0; i < 3; ++i) x[i] = map_coord(d, i, s[i]);
  if (d.map != SIPG_MAP_PERTURBED) return;
  double c[3];
  for (int i = 0; i < 3; ++i) c[i] = 2.0 * (double)((d.seed >> (16 * i)) & 0xFFFFull) / 65535.0 - 1.0;
  const double pi = 3.14159265358979323846;
  const double b = std::sin(pi * s[0]) * std::sin(pi * s[1]) * std::sin(pi * s[2]);
  for (int i = 0; i < 3; ++i)
    x[i] += d.amplitude * (d.hi[i] - d.lo[i]) * c[i] * b * std::cos(pi * (s[(i + 1) % 3] - s[(i + 2) % 3]));
}

namespace {

// out[qz][qy][qx] = sum M_z[qz][c] M_y[qy][b] M_x[qx][a] in[c][b][a]; M_r has
// n_r rows and p columns.
void contract3(const std::vector<double>& in, int p, const double* Mx, int nx, const double* My, int ny,
               const double* Mz, int nz, std::vector<double>& out) {
  std::vector<double> t1((size_t)p * p * nx), t2((size_t)p * ny * nx);
  for (int c = 0; c < p; ++c)
    for (int b = 0; b < p; ++b)
      for (int q = 0; q < nx; ++q) {
        double s = 0.0;
        for (int a = 0; a < p; ++a) s += Mx[q * p + a] * in[((size_t)c * p + b) * p + a];
        t1[((size_t)c * p + b) * nx + q] = s;
      }
  for (int c = 0; c < p; ++c)
    for (int q = 0; q < ny; ++q)
      for (int r = 0; r < nx; ++r) {
        double s = 0.0;
        for (int b = 0; b < p; ++b) s += My[q * p + b] * t1[((size_t)c * p + b) * nx + r];
        t2[((size_t)c * ny + q) * nx + r] = s;
      }
  out.assign((size_t)nz * ny * nx, 0.0);
  for (int q = 0; q < nz; ++q)
    for (int r = 0; r < ny * nx; ++r) {
      double s = 0.0;
      for (int c = 0; c < p; ++c) s += Mz[q * p + c] * t2[(size_t)c * ny * nx + r];
      out[(size_t)q * ny * nx + r] = s;
    }
}

bool inv3(const double J[3][3], double Ji[3][3], double& det) {
  det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
        J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  if (!(det > 0.0)) return false;
  const double id = 1.0 / det;
  Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) * id;
  Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * id;
  Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * id;
  Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) * id;
  Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * id;
  Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * id;
  Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) * id;
  Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * id;
  Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * id;
  return true;
}

}  // namespace

int build_general(Mesh& m) {
  const int p = m.p, P2 = p * p, P3 = p * p * p;
  std::vector<double> zn, wn, zq, wq;
  gll_rule(p, zn, wn);
  gauss_rule(p, zq, wq);
  std::vector<double> S(P2), D(P2), e0(p, 0.0), e1(p, 0.0), d0, d1, v;
  for (int q = 0; q < p; ++q) {
    std::vector<double> val, der;
    lagrange_eval(zn, zq[q], val, der);
    for (int a = 0; a < p; ++a) {
      S[q * p + a] = val[a];
      D[q * p + a] = der[a];
    }
  }
  lagrange_eval(zn, 0.0, v, d0);
  lagrange_eval(zn, 1.0, v, d1);
  e0[0] = 1.0;
  e1[p - 1] = 1.0;
  m.hgen_head.clear();
  m.hgen_head.insert(m.hgen_head.end(), S.begin(), S.end());
  m.hgen_head.insert(m.hgen_head.end(), D.begin(), D.end());
  m.hgen_head.insert(m.hgen_head.end(), d0.begin(), d0.end());
  m.hgen_head.insert(m.hgen_head.end(), d1.begin(), d1.end());
  const long long nc = m.ncell;
  std::vector<double> geo((size_t)nc * 7 * P3), face((size_t)nc * 6 * 4 * P2);
  m.htau_gen.assign((size_t)nc, 0.0);
  const int* n = m.desc.n;
  const double tsc = m.penalty * (m.k + 1) * (m.k + 1);
  std::vector<double> X[3], dJ[3][3];
  for (long long e = 0; e < nc; ++e) {
    const int id[3] = {(int)(e % n[0]), (int)((e / n[0]) % n[1]), (int)(e / ((long long)n[0] * n[1]))};
    for (int i = 0; i < 3; ++i) X[i].assign(P3, 0.0);
    for (int c = 0; c < p; ++c)
      for (int b = 0; b < p; ++b)
        for (int a = 0; a < p; ++a) {
          const double s[3] = {(id[0] + zn[a]) / n[0], (id[1] + zn[b]) / n[1], (id[2] + zn[c]) / n[2]};
          double x[3];
          map_point(m.desc, s, x);
          for (int i = 0; i < 3; ++i) X[i][((size_t)c * p + b) * p + a] = x[i];
        }
    // cell: J at the Gauss points
    double vol = 0.0;
    for (int i = 0; i < 3; ++i) {
      contract3(X[i], p, D.data(), p, S.data(), p, S.data(), p, dJ[i][0]);
      contract3(X[i], p, S.data(), p, D.data(), p, S.data(), p, dJ[i][1]);
      contract3(X[i], p, S.data(), p, S.data(), p, D.data(), p, dJ[i][2]);
    }
    double* G = &geo[(size_t)e * 7 * P3];
    for (int q = 0; q < P3; ++q) {
      const int qa = q % p, qb = (q / p) % p, qc = q / P2;
      double J[3][3], Ji[3][3], det;
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) J[i][j] = dJ[i][j][q];
      if (!inv3(J, Ji, det)) return fail(SIPG_EINVAL, "perturbed map is not invertible: reduce the amplitude");
      const double w = wq[qa] * wq[qb] * wq[qc] * det;
      vol += w;
      double K[3][3];  // J^-1 J^-T
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) K[i][j] = Ji[i][0] * Ji[j][0] + Ji[i][1] * Ji[j][1] + Ji[i][2] * Ji[j][2];
      G[0 * P3 + q] = w * K[0][0];
      G[1 * P3 + q] = w * K[0][1];
      G[2 * P3 + q] = w * K[0][2];
      G[3 * P3 + q] = w * K[1][1];
      G[4 * P3 + q] = w * K[1][2];
      G[5 * P3 + q] = w * K[2][2];
      G[6 * P3 + q] = w;
    }
    // faces: J at the face Gauss points (the end node along d)
    double area_sum = 0.0;
    for (int f = 0; f < 6; ++f) {
      const int d = f >> 1, side = f & 1;
      const double sg = side ? 1.0 : -1.0;
      const double* val_d = side ? e1.data() : e0.data();
      const double* der_d = side ? d1.data() : d0.data();
      std::vector<double> fJ[3][3];
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          const double* M[3];
          int nq[3];
          for (int r = 0; r < 3; ++r) {
            if (r == d) {
              M[r] = j == r ? der_d : val_d;
              nq[r] = 1;
            } else {
              M[r] = j == r ? D.data() : S.data();
              nq[r] = p;
            }
          }
          contract3(X[i], p, M[0], nq[0], M[1], nq[1], M[2], nq[2], fJ[i][j]);
        }
      // face points in (t1 fastest, t2) order; contract3 orders them z, y, x
      const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
      double* F = &face[((size_t)e * 6 + f) * 4 * P2];
      double area = 0.0;
      for (int q2 = 0; q2 < p; ++q2)
        for (int q1 = 0; q1 < p; ++q1) {
          int qi[3];
          qi[d] = 0;
          qi[t1] = q1;
          qi[t2] = q2;
          const int nqy = d == 1 ? 1 : p, nqx = d == 0 ? 1 : p;
          const int idx = (qi[2] * nqy + qi[1]) * nqx + qi[0];
          double J[3][3], Ji[3][3], det;
          for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) J[i][j] = fJ[i][j][idx];
          if (!inv3(J, Ji, det)) return fail(SIPG_EINVAL, "perturbed map is not invertible: reduce the amplitude");
          // J^-T e_d = row d of J^-1
          const double nr = std::sqrt(Ji[d][0] * Ji[d][0] + Ji[d][1] * Ji[d][1] + Ji[d][2] * Ji[d][2]);
          const double wt = wq[q1] * wq[q2] * det;
          const int pt = q2 * p + q1;
          for (int i = 0; i < 3; ++i)
            F[i * P2 + pt] = sg * wt * (Ji[i][0] * Ji[d][0] + Ji[i][1] * Ji[d][1] + Ji[i][2] * Ji[d][2]);
          F[3 * P2 + pt] = wt * nr;
          area += wt * nr;
        }
      const bool periodic = (side ? m.desc.bc_hi[d] : m.desc.bc_lo[d]) == SIPG_BC_PERIODIC;
      const bool boundary = !periodic && id[d] == (side ? n[d] - 1 : 0);
      area_sum += boundary ? area : 0.5 * area;
    }
    m.htau_gen[(size_t)e] = tsc * area_sum / vol;
  }
  for (double** ptr : {&m.dgen_geo, &m.dgen_face, &m.dgen_tau, &m.dgen_head}) {
    if (*ptr) cudaFree(*ptr);
    *ptr = nullptr;
  }
  cudaError_t err = cudaMalloc(&m.dgen_geo, geo.size() * sizeof(double));
  if (err == cudaSuccess) err = cudaMalloc(&m.dgen_face, face.size() * sizeof(double));
  if (err == cudaSuccess) err = cudaMalloc(&m.dgen_tau, m.htau_gen.size() * sizeof(double));
  if (err == cudaSuccess) err = cudaMalloc(&m.dgen_head, m.hgen_head.size() * sizeof(double));
  if (err != cudaSuccess) return fail(SIPG_ENOMEM, "cudaMalloc of the general geometry store failed");
  err = cudaMemcpy(m.dgen_geo, geo.data(), geo.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (err == cudaSuccess)
    err = cudaMemcpy(m.dgen_face, face.data(), face.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (err == cudaSuccess)
    err = cudaMemcpy(m.dgen_tau, m.htau_gen.data(), m.htau_gen.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (err == cudaSuccess)
    err = cudaMemcpy(m.dgen_head, m.hgen_head.data(), m.hgen_head.size() * sizeof(double), cudaMemcpyHostToDevice);
  return err == cudaSuccess ? SIPG_OK : cuda_fail(err, "upload general geometry store");
}

// ---------------------------------------------------------------- device
namespace {

constexpr int kGenThreads = 64;  // >= (k+1)^2 for k <= 7

struct GenArgs {
  Geo<double> g;
  const double* head;  // S [P2], D [P2], d0 [P], d1 [P]
  const double* geo;   // [cell][7][P3]
  const double* face;  // [cell][6][4][P2]
  const double* tau;   // [cell]
  const double* x;
  double* y;
  double cm, nu;
  int stiffness;
  const int* skip;
};

// unscaled conversion of geometry and coefficients (their range is the mesh's;
// inline, no out-of-line rare path: about 2,000 of them per cell)
template <typename T>
__device__ __forceinline__ T geo_in(double v) {
  if constexpr (std::is_same<T, dfl>::value)
    return df_from_double(v);
  else
    return (T)v;
}

template <int P>
__host__ __device__ constexpr int gstride(int dir) {
  return dir == 0 ? 1 : (dir == 1 ? P : P * P);
}

template <typename T, int P>
__global__ void __launch_bounds__(kGenThreads, 6) apply_general_kernel(GenArgs a) {
  constexpr int P2 = P * P, P3 = P2 * P;
  if (a.skip && *a.skip) return;
  __shared__ T su[P3], A1[P3], B1[P3], AA[P3], AB[P3], BA[P3], W[P3];
  __shared__ T sS[P2], sD[P2], sd0[P], sd1[P];
  __shared__ T fv[8][P2];
  __shared__ T ih[6][P2];  // face intermediates
  const int e = blockIdx.x, comp = blockIdx.y;
  const int nt = blockDim.x, tid = threadIdx.x;
  const long long N = (long long)a.g.ncell * P3;
  const double* x = a.x + comp * N;
  int sc = 0;  // the call's scale exponent (double-float)
  if constexpr (std::is_same<T, dfl>::value) sc = a.g.dsc ? *a.g.dsc : 0;
  stage_cvt<T, double>(su, x + (long long)e * P3, P3, sc);
  for (int i = tid; i < P2; i += nt) {
    sS[i] = geo_in<T>(a.head[i]);
    sD[i] = geo_in<T>(a.head[P2 + i]);
  }
  for (int i = tid; i < P; i += nt) {
    sd0[i] = geo_in<T>(a.head[2 * P2 + i]);
    sd1[i] = geo_in<T>(a.head[2 * P2 + P + i]);
  }
  __syncthreads();
  const T cnu = geo_in<T>(a.stiffness ? a.nu : 0.0), ccm = geo_in<T>(a.cm);
  const T fnu = geo_in<T>(a.nu);
  const double* G = a.geo + (long long)e * 7 * P3;
  // x: A1 = S u, B1 = D u
  for (int l = tid; l < P2; l += nt) {
    T v[P];
    for (int i = 0; i < P; ++i) v[i] = su[l * P + i];
    for (int q = 0; q < P; ++q) {
      T s = T(0), t = T(0);
      for (int i = 0; i < P; ++i) {
        s = fma(sS[q * P + i], v[i], s);
        t = fma(sD[q * P + i], v[i], t);
      }
      A1[l * P + q] = s;
      B1[l * P + q] = t;
    }
  }
  __syncthreads();
  // y: AA = S A1, AB = D A1, BA = S B1
  for (int l = tid; l < P2; l += nt) {
    const int qx = l % P, z = l / P, base = z * P2 + qx;
    T va[P], vb[P];
    for (int i = 0; i < P; ++i) {
      va[i] = A1[base + i * P];
      vb[i] = B1[base + i * P];
    }
    for (int q = 0; q < P; ++q) {
      T s = T(0), t = T(0), r = T(0);
      for (int i = 0; i < P; ++i) {
        s = fma(sS[q * P + i], va[i], s);
        t = fma(sD[q * P + i], va[i], t);
        r = fma(sS[q * P + i], vb[i], r);
      }
      AA[base + q * P] = s;
      AB[base + q * P] = t;
      BA[base + q * P] = r;
    }
  }
  __syncthreads();
  // z: gradients and value at the points, the metric, the transposed z sweep
  for (int l = tid; l < P2; l += nt) {
    T vaa[P], vab[P], vba[P];
    for (int i = 0; i < P; ++i) {
      vaa[i] = AA[l + i * P2];
      vab[i] = AB[l + i * P2];
      vba[i] = BA[l + i * P2];
    }
    T fx[P], fy[P], fz[P], fm[P];
    for (int q = 0; q < P; ++q) {
      T gx = T(0), gy = T(0), gz = T(0), uq = T(0);
      for (int i = 0; i < P; ++i) {
        gx = fma(sS[q * P + i], vba[i], gx);
        gy = fma(sS[q * P + i], vab[i], gy);
        gz = fma(sD[q * P + i], vaa[i], gz);
        uq = fma(sS[q * P + i], vaa[i], uq);
      }
      const int pt = q * P2 + l;
      const T g0 = geo_in<T>(G[0 * P3 + pt]), g1 = geo_in<T>(G[1 * P3 + pt]);
      const T g2 = geo_in<T>(G[2 * P3 + pt]), g3 = geo_in<T>(G[3 * P3 + pt]);
      const T g4 = geo_in<T>(G[4 * P3 + pt]), g5 = geo_in<T>(G[5 * P3 + pt]);
      fx[q] = cnu * fma(g0, gx, fma(g1, gy, g2 * gz));
      fy[q] = cnu * fma(g1, gx, fma(g3, gy, g4 * gz));
      fz[q] = cnu * fma(g2, gx, fma(g4, gy, g5 * gz));
      fm[q] = ccm * geo_in<T>(G[6 * P3 + pt]) * uq;
    }
    for (int i = 0; i < P; ++i) {
      T s1 = T(0), s2 = T(0), s3 = T(0);
      for (int q = 0; q < P; ++q) {
        s1 = fma(sS[q * P + i], fx[q], s1);
        s2 = fma(sS[q * P + i], fy[q], s2);
        s3 = fma(sD[q * P + i], fz[q], fma(sS[q * P + i], fm[q], s3));
      }
      BA[l + i * P2] = s1;
      AB[l + i * P2] = s2;
      AA[l + i * P2] = s3;
    }
  }
  __syncthreads();
  // transposed y: A1 = S^T AA + D^T AB, B1 = S^T BA
  for (int l = tid; l < P2; l += nt) {
    const int qx = l % P, z = l / P, base = z * P2 + qx;
    T va[P], vb[P], vc[P];
    for (int i = 0; i < P; ++i) {
      va[i] = AA[base + i * P];
      vb[i] = AB[base + i * P];
      vc[i] = BA[base + i * P];
    }
    for (int i = 0; i < P; ++i) {
      T s = T(0), t = T(0);
      for (int q = 0; q < P; ++q) {
        s = fma(sS[q * P + i], va[q], fma(sD[q * P + i], vb[q], s));
        t = fma(sS[q * P + i], vc[q], t);
      }
      A1[base + i * P] = s;
      B1[base + i * P] = t;
    }
  }
  __syncthreads();
  // transposed x: W = S^T A1 + D^T B1
  for (int l = tid; l < P2; l += nt) {
    T va[P], vb[P];
    for (int i = 0; i < P; ++i) {
      va[i] = A1[l * P + i];
      vb[i] = B1[l * P + i];
    }
    for (int i = 0; i < P; ++i) {
      T s = T(0);
      for (int q = 0; q < P; ++q) s = fma(sS[q * P + i], va[q], fma(sD[q * P + i], vb[q], s));
      W[l * P + i] = s;
    }
  }
  __syncthreads();
  // faces
  if (a.stiffness) {
    const int id[3] = {e % a.g.n[0], (e / a.g.n[0]) % a.g.n[1], e / (a.g.n[0] * a.g.n[1])};
    const double tau_e = a.tau[e];  // penalties stay FP64 (one conversion per face)
#pragma unroll 1
    for (int f = 0; f < 6; ++f) {
      const int d = f >> 1, side = f & 1;
      int nb, kind, jl;
      face_neighbor(a.g, d, side, d == 0 ? id[0] : (d == 1 ? id[1] : id[2]), e, nb, kind, jl);
      if (kind == SIPG_BC_NEUMANN) continue;  // uniform over the block
      const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
      const int sd = gstride<P>(d), s1 = gstride<P>(t1), s2 = gstride<P>(t2);
      const int end = side ? P - 1 : 0, nend = P - 1 - end;
      const T* dend = side ? sd1 : sd0;
      const T* dnb = side ? sd0 : sd1;
      // plane values and normal reference derivatives of both sides
      for (int j = tid; j < P2; j += nt) {
        const int b = j % P, cc = j / P, tr = b * s1 + cc * s2;
        fv[0][j] = su[end * sd + tr];
        T nd = T(0);
        for (int i = 0; i < P; ++i) nd = fma(dend[i], su[i * sd + tr], nd);
        fv[1][j] = nd;
        if (kind == 0) {
          const double* xn = x + (long long)nb * P3;
          double xv[P];  // all loads issued before the conversions
#pragma unroll
          for (int i = 0; i < P; ++i) xv[i] = __ldg(xn + i * sd + tr);
          fv[2][j] = cvt_in<T, double>(nend ? xv[P - 1] : xv[0], sc);
          T nn = T(0);
#pragma unroll
          for (int i = 0; i < P; ++i) nn = fma(dnb[i], cvt_in<T, double>(xv[i], sc), nn);
          fv[3][j] = nn;
        }
      }
      __syncthreads();
      // to the face points in two 1D stages: along t1 (S for all four plane
      // arrays, D for the two value planes), then along t2
      for (int l = tid; l < 6 * P; l += nt) {
        const int k = l / P, cc = l % P;  // k < 4: S of plane k; k = 4, 5: D of planes 0, 2
        const T* src = fv[k < 4 ? k : (k == 4 ? 0 : 2)] + cc * P;
        const T* M = k < 4 ? sS : sD;
        if (k < 4 && kind != 0 && k >= 2) continue;
        if (k == 5 && kind != 0) continue;
        for (int q1 = 0; q1 < P; ++q1) {
          T t = T(0);
          for (int b = 0; b < P; ++b) t = fma(M[q1 * P + b], src[b], t);
          ih[k][cc * P + q1] = t;
        }
      }
      __syncthreads();
      // flux at the face points
      const double* Fo = a.face + ((long long)e * 6 + f) * 4 * P2;
      const double* Fn = kind == 0 ? a.face + ((long long)nb * 6 + (2 * d + 1 - side)) * 4 * P2 : nullptr;
      const T tau_f = geo_in<T>(kind == 0 ? fmax(tau_e, a.tau[nb]) : tau_e), tau_o = geo_in<T>(tau_e);
      for (int q = tid; q < P2; q += nt) {
        const int q1 = q % P, q2 = q / P;
        // val: u, d_d u of both sides; d1: t1-derivative; d2: t2-derivative
        T val[4] = {T(0), T(0), T(0), T(0)}, d1v[2] = {T(0), T(0)}, d2v[2] = {T(0), T(0)};
        const int nv = kind == 0 ? 4 : 2;
        for (int cc = 0; cc < P; ++cc) {
          const T ws = sS[q2 * P + cc], wd = sD[q2 * P + cc];
          const int j = cc * P + q1;
          for (int k = 0; k < nv; ++k) val[k] = fma(ws, ih[k][j], val[k]);
          d1v[0] = fma(ws, ih[4][j], d1v[0]);
          d2v[0] = fma(wd, ih[0][j], d2v[0]);
          if (kind == 0) {
            d1v[1] = fma(ws, ih[5][j], d1v[1]);
            d2v[1] = fma(wd, ih[2][j], d2v[1]);
          }
        }
        // reference gradients (x, y, z order) and d_n u w dA = grad . g
        T go[3], gn[3];
        go[d] = val[1];
        go[t1] = d1v[0];
        go[t2] = d2v[0];
        const T fo0 = geo_in<T>(Fo[0 * P2 + q]), fo1 = geo_in<T>(Fo[1 * P2 + q]);
        const T fo2 = geo_in<T>(Fo[2 * P2 + q]);
        const T dn_own = fma(go[0], fo0, fma(go[1], fo1, go[2] * fo2));
        const T wda = geo_in<T>(Fo[3 * P2 + q]);
        T rv, rg;
        if (kind == 0) {
          gn[d] = val[3];
          gn[t1] = d1v[1];
          gn[t2] = d2v[1];
          // the neighbour's g carries its own outward normal, -n
          const T dn_nb = fma(gn[0], geo_in<T>(Fn[0 * P2 + q]),
                              fma(gn[1], geo_in<T>(Fn[1 * P2 + q]), gn[2] * geo_in<T>(Fn[2 * P2 + q])));
          const T jump = val[0] - val[2];
          rv = tau_f * wda * jump - T(0.5) * (dn_own - dn_nb);
          rg = -(T(0.5) * jump);
        } else {  // Dirichlet
          rv = T(2) * tau_o * wda * val[0] - dn_own;
          rg = -val[0];
        }
        const T fo[3] = {fo0, fo1, fo2};
        fv[4][q] = fnu * rv;
        fv[5][q] = fnu * rg * fo[d];
        fv[6][q] = fnu * rg * fo[t1];
        fv[7][q] = fnu * rg * fo[t2];
      }
      __syncthreads();
      // test functions in two 1D stages: along t2 (q2 -> cc), then along t1
      // (q1 -> b); values and tangential derivatives land on the end plane,
      // the normal derivative on the lines through it
      for (int l = tid; l < P2; l += nt) {
        const int q1 = l % P, cc = l / P;
        T tv = T(0), tn = T(0), tt1 = T(0), tt2 = T(0);
        for (int q2 = 0; q2 < P; ++q2) {
          const int q = q2 * P + q1;
          const T ws = sS[q2 * P + cc];
          tv = fma(ws, fv[4][q], tv);
          tn = fma(ws, fv[5][q], tn);
          tt1 = fma(ws, fv[6][q], tt1);
          tt2 = fma(sD[q2 * P + cc], fv[7][q], tt2);
        }
        ih[0][cc * P + q1] = tv + tt2;
        ih[1][cc * P + q1] = tn;
        ih[2][cc * P + q1] = tt1;
      }
      __syncthreads();
      for (int j = tid; j < P2; j += nt) {
        const int b = j % P, cc = j / P, tr = b * s1 + cc * s2;
        T pv = T(0), pn = T(0);
        for (int q1 = 0; q1 < P; ++q1) {
          const int t = cc * P + q1;
          pv = fma(sS[q1 * P + b], ih[0][t], pv);
          pv = fma(sD[q1 * P + b], ih[2][t], pv);
          pn = fma(sS[q1 * P + b], ih[1][t], pn);
        }
        W[end * sd + tr] = W[end * sd + tr] + pv;
        for (int i = 0; i < P; ++i) W[i * sd + tr] = fma(dend[i], pn, W[i * sd + tr]);
      }
      __syncthreads();
    }
  }
  double* y = a.y + comp * N;
  for (int i = tid; i < P3; i += nt) y[(long long)e * P3 + i] = cvt_out<double, T>(W[i], sc);
}

// diag(A)_i = a(phi_i, phi_i) on a general map: the cell term summed over the
// Gauss points, and per face the flux of phi_i tested with phi_i, with phi_i
// also as the neighbour's trace when a periodic direction has one cell (the
// cell is its own neighbour).  One thread per node.
template <int P>
__global__ void __launch_bounds__(kGenThreads) general_diag_kernel(GenArgs a) {
  constexpr int P2 = P * P, P3 = P2 * P;
  __shared__ double sS[P2], sD[P2], sd0[P], sd1[P];
  const int e = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < P2; i += nt) {
    sS[i] = a.head[i];
    sD[i] = a.head[P2 + i];
  }
  for (int i = tid; i < P; i += nt) {
    sd0[i] = a.head[2 * P2 + i];
    sd1[i] = a.head[2 * P2 + P + i];
  }
  __syncthreads();
  const double* G = a.geo + (long long)e * 7 * P3;
  const int id[3] = {e % a.g.n[0], (e / a.g.n[0]) % a.g.n[1], e / (a.g.n[0] * a.g.n[1])};
  const double tau_e = a.tau[e];
  for (int node = tid; node < P3; node += nt) {
    const int ia[3] = {node % P, (node / P) % P, node / P2};
    double acc = 0.0;
    for (int qc = 0; qc < P; ++qc)
      for (int qb = 0; qb < P; ++qb)
        for (int qa = 0; qa < P; ++qa) {
          const int pt = (qc * P + qb) * P + qa;
          const double sx = sS[qa * P + ia[0]], sy = sS[qb * P + ia[1]], sz = sS[qc * P + ia[2]];
          const double gx = sD[qa * P + ia[0]] * sy * sz, gy = sx * sD[qb * P + ia[1]] * sz,
                       gz = sx * sy * sD[qc * P + ia[2]];
          double v = 0.0;
          if (a.stiffness)
            v = a.nu * (G[0 * P3 + pt] * gx * gx + G[3 * P3 + pt] * gy * gy + G[5 * P3 + pt] * gz * gz +
                        2.0 * (G[1 * P3 + pt] * gx * gy + G[2 * P3 + pt] * gx * gz + G[4 * P3 + pt] * gy * gz));
          const double ph = sx * sy * sz;
          acc += v + a.cm * G[6 * P3 + pt] * ph * ph;
        }
    if (a.stiffness) {
      for (int f = 0; f < 6; ++f) {
        const int d = f >> 1, side = f & 1;
        int nb, kind, jl;
        face_neighbor(a.g, d, side, d == 0 ? id[0] : (d == 1 ? id[1] : id[2]), e, nb, kind, jl);
        if (kind == SIPG_BC_NEUMANN) continue;
        const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
        const int end = side ? P - 1 : 0, nend = P - 1 - end;
        const double* dend = side ? sd1 : sd0;
        const double* dnb = side ? sd0 : sd1;
        const int ad = d == 0 ? ia[0] : (d == 1 ? ia[1] : ia[2]);
        const int b = t1 == 0 ? ia[0] : ia[1], cc = t2 == 2 ? ia[2] : ia[1];
        const bool self = kind == 0 && nb == e;  // one cell along a periodic direction
        const double* Fo = a.face + ((long long)e * 6 + f) * 4 * P2;
        const double* Fn = kind == 0 ? a.face + ((long long)nb * 6 + (2 * d + 1 - side)) * 4 * P2 : nullptr;
        const double tau_f = kind == 0 ? fmax(tau_e, a.tau[nb]) : tau_e;
        const double own = ad == end ? 1.0 : 0.0, oth = (self && ad == nend) ? 1.0 : 0.0;
        for (int q2 = 0; q2 < P; ++q2)
          for (int q1 = 0; q1 < P; ++q1) {
            const int q = q2 * P + q1;
            const double s1 = sS[q1 * P + b], s2 = sS[q2 * P + cc];
            const double t1v = sD[q1 * P + b] * s2, t2v = s1 * sD[q2 * P + cc];
            // phi on the own face and its reference gradient there
            double go[3];
            go[d] = dend[ad] * s1 * s2;
            go[t1] = own * t1v;
            go[t2] = own * t2v;
            const double um = own * s1 * s2;
            const double gdot = go[0] * Fo[0 * P2 + q] + go[1] * Fo[1 * P2 + q] + go[2] * Fo[2 * P2 + q];
            const double wda = Fo[3 * P2 + q];
            double rv, rg;
            if (kind == 0) {
              double gn[3] = {0.0, 0.0, 0.0};
              double up = 0.0, dnn = 0.0;
              if (self) {  // phi as the neighbour's trace on the opposite face
                gn[d] = dnb[ad] * s1 * s2;
                gn[t1] = oth * t1v;
                gn[t2] = oth * t2v;
                up = oth * s1 * s2;
                dnn = gn[0] * Fn[0 * P2 + q] + gn[1] * Fn[1 * P2 + q] + gn[2] * Fn[2 * P2 + q];
              }
              const double jump = um - up;
              rv = tau_f * wda * jump - 0.5 * (gdot - dnn);
              rg = -0.5 * jump;
            } else {
              rv = 2.0 * tau_e * wda * um - gdot;
              rg = -um;
            }
            acc += a.nu * (rv * um + rg * gdot);
          }
      }
    }
    a.y[(long long)e * P3 + node] = acc;
  }
}

}  // namespace

int launch_general(const Mesh& m, const double* x, double* y, int ncomp, double cm, double nu, bool stiffness,
                   const int* skip, cudaStream_t s) {
  GenArgs a{};
  a.g = make_geo<double>(m);
  a.head = m.dgen_head;
  a.geo = m.dgen_geo;
  a.face = m.dgen_face;
  a.tau = m.dgen_tau;
  a.x = x;
  a.y = y;
  a.cm = cm;
  a.nu = nu;
  a.stiffness = stiffness ? 1 : 0;
  a.skip = skip;
  const dim3 grid((unsigned)m.ncell, (unsigned)ncomp);
  if (m.f64_arith == SIPG_F64_DOUBLE_FLOAT) {
    if (!df_coef_ok(cm) || !df_coef_ok(nu))
      return fail(SIPG_EINVAL, "double-float arithmetic needs mass_coef and nu in [2^-100, 2^100]");
    const int st = launch_df_scale(m, x, m.ncell * m.p * m.p * m.p * ncomp, nullptr, 0, skip, s);
    if (st) return st;
  }
  switch (m.p) {
#define SIPG_GEN_CASE(P) \
  case P:                \
    if (m.f64_arith == SIPG_F64_DOUBLE_FLOAT)             \
      apply_general_kernel<dfl, P><<<grid, kGenThreads, 0, s>>>(a); \
    else                                                  \
      apply_general_kernel<double, P><<<grid, kGenThreads, 0, s>>>(a); \
    break;
    SIPG_GEN_CASE(2)
    SIPG_GEN_CASE(3)
    SIPG_GEN_CASE(4)
    SIPG_GEN_CASE(5)
    SIPG_GEN_CASE(6)
    SIPG_GEN_CASE(7)
    SIPG_GEN_CASE(8)
#undef SIPG_GEN_CASE
    default: return fail(SIPG_EINVAL, "unsupported degree");
  }
  const_cast<Mesh&>(m).launches++;
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SIPG_OK : cuda_fail(e, "general operator launch");
}

}  // namespace sipg

namespace sipg {

int launch_general_diagonal(const Mesh& m, bool stiffness, double cm, double nu, double* diag, cudaStream_t s) {
  GenArgs a{};
  a.g = make_geo<double>(m);
  a.head = m.dgen_head;
  a.geo = m.dgen_geo;
  a.face = m.dgen_face;
  a.tau = m.dgen_tau;
  a.y = diag;
  a.cm = cm;
  a.nu = nu;
  a.stiffness = stiffness ? 1 : 0;
  switch (m.p) {
#define SIPG_GEN_CASE(P) \
  case P:                \
    general_diag_kernel<P><<<(unsigned)m.ncell, kGenThreads, 0, s>>>(a); break;
    SIPG_GEN_CASE(2)
    SIPG_GEN_CASE(3)
    SIPG_GEN_CASE(4)
    SIPG_GEN_CASE(5)
    SIPG_GEN_CASE(6)
    SIPG_GEN_CASE(7)
    SIPG_GEN_CASE(8)
#undef SIPG_GEN_CASE
    default: return fail(SIPG_EINVAL, "unsupported degree");
  }
  const_cast<Mesh&>(m).launches++;
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SIPG_OK : cuda_fail(e, "general diagonal launch");
}

}  // namespace sipg
