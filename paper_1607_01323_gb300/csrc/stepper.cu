// The dual-splitting time step (Sec. 2.2) in the V3c variant (Sec. 4): the
// stepper object, its two kernels (the pressure data on the no-slip walls and
// a fused linear combination of vectors) and the sequence of library calls
// of one step.  Every vector stays on the device; the host only sequences
// kernels and reads the solvers' convergence data.
//
// Wall data, Eq. (ipflux): on a wall face with outward normal s e_d,
//   H = s (div F^c(u) + nu curl omega)_d,
//   (div F^c)_d = u_j d_j u_d + u_d div u,
//   (curl omega)_d = d_e1 omega_e2 - d_e2 omega_e1   (e1, e2 = d+1, d+2 cyclic),
// at the (k+1)^2 Gauss points of the face, from the wall cell alone.  omega is
// the cell-wise L2 projection of curl u (Sec. 3.2 (ii)); with the separable
// map the projection of d_j u is (M_j^-1 C^T) u along j (the mass matrices of
// the other two directions cancel), tabulated per layer as Dv_j.  Only the
// trace of omega on the face plane enters (its derivatives are tangential);
// the derivative d_d u_d normal to the face uses the full lines through it.
// The right-hand side contribution of a face is (q, h)_F with
// h = -sum_i beta_i H^(n-i) + s f_d, integrated with the Gauss weights and
// the tangential Jacobians (the separable face's area element).
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "sipg_internal.h"

namespace sipg {

namespace {

constexpr int kLinThreads = 256;
constexpr int kWallThreads = 64;  // >= (k+1)^2 for k <= 7

struct LinTerms {
  const double* x[4];
  double c[4];
};

// y[i] = sum_j c_j x_j[i] + add_(i / len); y may be one of the x_j.
__global__ void __launch_bounds__(kLinThreads) lincomb_kernel(long long n, long long len, int m, LinTerms t,
                                                              double a0, double a1, double a2, double* y) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) {
    double v = 0.0;
    for (int j = 0; j < m; ++j) v = fma(t.c[j], t.x[j][i], v);
    const long long comp = i / len;
    y[i] = v + (comp == 0 ? a0 : (comp == 1 ? a1 : a2));
  }
}

struct WallArgs {
  const int* wcell;   // wall cells
  const int* wmask;   // bit f (= 2 d + side) set for each no-slip face of the cell
  const int* wfirst;  // index of the cell's first wall face
  const double* tab;  // wall tables (Mesh::dns64)
  long long off[3];   // per-direction layer blocks in tab
  int n[3];
  long long ncell;
  double nu;
  const double* u;    // 3 components of the velocity
  double* hnew;       // wall data of u, [face][P^2]
  const double* hold[3];  // older wall data (hold[0] unused: the new values)
  double beta[3];
  int nbeta;          // 0: wall data only; else add the face terms to rhs
  double f[3];
  double* rhs;        // pressure right-hand side
};

template <int P>
__host__ __device__ constexpr int wstride(int dir) {
  return dir == 0 ? 1 : (dir == 1 ? P : P * P);
}

template <int P>
__global__ void __launch_bounds__(kWallThreads) wall_kernel(WallArgs a) {
  constexpr int P2 = P * P, P3 = P * P * P, LB = P + 2 + P2;
  __shared__ double su[3 * P3];
  __shared__ double sS[P2], sD[P2], sd0[P], sd1[P], sw[P];
  __shared__ double sL[3 * LB];  // the cell's layer block in each direction
  __shared__ double U[3][P2], Nd[P2], W[2][P2], hw[P2];
  const int e = a.wcell[blockIdx.x];
  const int mask = a.wmask[blockIdx.x];
  const long long N = a.ncell * P3;
  const int id[3] = {e % a.n[0], (e / a.n[0]) % a.n[1], e / (a.n[0] * a.n[1])};
  for (int i = threadIdx.x; i < 3 * P3; i += blockDim.x) su[i] = a.u[(i / P3) * N + (long long)e * P3 + i % P3];
  for (int i = threadIdx.x; i < P2; i += blockDim.x) {
    sS[i] = a.tab[i];
    sD[i] = a.tab[P2 + i];
  }
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    sd0[i] = a.tab[2 * P2 + i];
    sd1[i] = a.tab[2 * P2 + P + i];
    sw[i] = a.tab[2 * P2 + 2 * P + i];
  }
  for (int i = threadIdx.x; i < 3 * LB; i += blockDim.x) {
    const int d = i / LB;
    const int layer = d == 0 ? id[0] : (d == 1 ? id[1] : id[2]);
    sL[i] = a.tab[(d == 0 ? a.off[0] : (d == 1 ? a.off[1] : a.off[2])) + (long long)layer * LB + i % LB];
  }
  __syncthreads();
  int face = a.wfirst[blockIdx.x];
#pragma unroll 1
  for (int f = 0; f < 6; ++f) {
    if (!(mask >> f & 1)) continue;
    const int d = f >> 1, side = f & 1;
    const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
    const int e1 = (d + 1) % 3, e2 = (d + 2) % 3;
    const int end = side ? P - 1 : 0;
    const double sg = side ? 1.0 : -1.0;
    const double* dend = side ? sd1 : sd0;
    const double Jend = sL[d * LB + P + side];
    // plane values: u, the normal derivative of u_d, and the two tangential
    // components of omega
    for (int j = threadIdx.x; j < P2; j += blockDim.x) {
      const int b = j % P, cc = j / P;
      const int tr = b * wstride<P>(t1) + cc * wstride<P>(t2);
      const int node = end * wstride<P>(d) + tr;
      for (int c = 0; c < 3; ++c) U[c][j] = su[c * P3 + node];
      double nd = 0.0;
      for (int q = 0; q < P; ++q) nd = fma(dend[q], su[d * P3 + q * wstride<P>(d) + tr], nd);
      Nd[j] = nd / Jend;
      // (Dv_dir u_k) at this plane node
      auto dproj = [&](int dir, int k) {
        const double* Dv = sL + dir * LB + P + 2;
        double v = 0.0;
        if (dir == d) {
          for (int q = 0; q < P; ++q) v = fma(Dv[end * P + q], su[k * P3 + q * wstride<P>(d) + tr], v);
        } else if (dir == t1) {
          for (int q = 0; q < P; ++q)
            v = fma(Dv[b * P + q], su[k * P3 + end * wstride<P>(d) + q * wstride<P>(t1) + cc * wstride<P>(t2)], v);
        } else {
          for (int q = 0; q < P; ++q)
            v = fma(Dv[cc * P + q], su[k * P3 + end * wstride<P>(d) + b * wstride<P>(t1) + q * wstride<P>(t2)], v);
        }
        return v;
      };
      // omega_m = Dv_(m+1) u_(m+2) - Dv_(m+2) u_(m+1)
      W[0][j] = dproj((e1 + 1) % 3, (e1 + 2) % 3) - dproj((e1 + 2) % 3, (e1 + 1) % 3);
      W[1][j] = dproj((e2 + 1) % 3, (e2 + 2) % 3) - dproj((e2 + 2) % 3, (e2 + 1) % 3);
    }
    __syncthreads();
    // values and tangential derivatives at the Gauss points
    for (int q = threadIdx.x; q < P2; q += blockDim.x) {
      const int q1 = q % P, q2 = q / P;
      const double J1 = sL[t1 * LB + q1], J2 = sL[t2 * LB + q2];
      auto val = [&](const double* X) {
        double v = 0.0;
#pragma unroll 1
        for (int cc = 0; cc < P; ++cc) {
          double r = 0.0;
          for (int b = 0; b < P; ++b) r = fma(sS[q1 * P + b], X[cc * P + b], r);
          v = fma(sS[q2 * P + cc], r, v);
        }
        return v;
      };
      auto der1 = [&](const double* X) {
        double v = 0.0;
#pragma unroll 1
        for (int cc = 0; cc < P; ++cc) {
          double r = 0.0;
          for (int b = 0; b < P; ++b) r = fma(sD[q1 * P + b], X[cc * P + b], r);
          v = fma(sS[q2 * P + cc], r, v);
        }
        return v / J1;
      };
      auto der2 = [&](const double* X) {
        double v = 0.0;
#pragma unroll 1
        for (int cc = 0; cc < P; ++cc) {
          double r = 0.0;
          for (int b = 0; b < P; ++b) r = fma(sS[q1 * P + b], X[cc * P + b], r);
          v = fma(sD[q2 * P + cc], r, v);
        }
        return v / J2;
      };
      const double ud = val(U[d]), ut1 = val(U[t1]), ut2 = val(U[t2]), ndd = val(Nd);
      const double d1ud = der1(U[d]), d2ud = der2(U[d]);
      const double divu = ndd + der1(U[t1]) + der2(U[t2]);
      const double divF = ud * ndd + ut1 * d1ud + ut2 * d2ud + ud * divu;
      const double de1w2 = e1 == t1 ? der1(W[1]) : der2(W[1]);
      const double de2w1 = e2 == t1 ? der1(W[0]) : der2(W[0]);
      const double H = sg * (divF + a.nu * (de1w2 - de2w1));
      a.hnew[(long long)face * P2 + q] = H;
      if (a.nbeta > 0) {
        double hs = a.beta[0] * H;
        for (int i = 1; i < a.nbeta; ++i) hs = fma(a.beta[i], a.hold[i][(long long)face * P2 + q], hs);
        const double fd = d == 0 ? a.f[0] : (d == 1 ? a.f[1] : a.f[2]);
        hw[q] = (sg * fd - hs) * sw[q1] * sw[q2] * J1 * J2;
      }
    }
    __syncthreads();
    if (a.nbeta > 0) {
      for (int j = threadIdx.x; j < P2; j += blockDim.x) {
        const int b = j % P, cc = j / P;
        double v = 0.0;
        for (int q2 = 0; q2 < P; ++q2) {
          double r = 0.0;
          for (int q1 = 0; q1 < P; ++q1) r = fma(sS[q1 * P + b], hw[q2 * P + q1], r);
          v = fma(sS[q2 * P + cc], r, v);
        }
        const long long node = (long long)e * P3 + end * wstride<P>(d) + b * wstride<P>(t1) + cc * wstride<P>(t2);
        a.rhs[node] += v;
      }
      __syncthreads();
    }
    ++face;
  }
}

int launch_lincomb(long long n, long long len, int m, const double* const* x, const double* c, const double* add,
                   double* y, cudaStream_t s) {
  LinTerms t{};
  for (int j = 0; j < m; ++j) {
    t.x[j] = x[j];
    t.c[j] = c[j];
  }
  long long blocks = (n + kLinThreads - 1) / kLinThreads;
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (blocks < 1) blocks = 1;
  lincomb_kernel<<<(unsigned)blocks, kLinThreads, 0, s>>>(n, len, m, t, add ? add[0] : 0.0, add ? add[1] : 0.0,
                                                           add ? add[2] : 0.0, y);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SIPG_OK : cuda_fail(e, "linear-combination launch");
}

int launch_wall(int p, int nw, const WallArgs& a, cudaStream_t s) {
  if (nw == 0) return SIPG_OK;
  switch (p) {
#define SIPG_WALL_CASE(P) \
  case P:                 \
    wall_kernel<P><<<(unsigned)nw, kWallThreads, 0, s>>>(a); break;
    SIPG_WALL_CASE(3)
    SIPG_WALL_CASE(4)
    SIPG_WALL_CASE(5)
    SIPG_WALL_CASE(6)
    SIPG_WALL_CASE(7)
    SIPG_WALL_CASE(8)
#undef SIPG_WALL_CASE
    default: return fail(SIPG_EINVAL, "wall data need 2 <= k <= 7");
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SIPG_OK : cuda_fail(e, "wall-data launch");
}

// (gamma0, alpha_i, beta_i) of the order-J BDF / extrapolation pair
// (Karniadakis, Israeli and Orszag 1991)
void bdf_ex(int J, double& g0, double al[3], double be[3]) {
  const double G[3] = {1.0, 1.5, 11.0 / 6.0};
  const double A[3][3] = {{1.0, 0.0, 0.0}, {2.0, -0.5, 0.0}, {3.0, -1.5, 1.0 / 3.0}};
  const double B[3][3] = {{1.0, 0.0, 0.0}, {2.0, -1.0, 0.0}, {3.0, -3.0, 1.0}};
  g0 = G[J - 1];
  for (int i = 0; i < 3; ++i) {
    al[i] = A[J - 1][i];
    be[i] = B[J - 1][i];
  }
}

}  // namespace

}  // namespace sipg

using namespace sipg;

struct sipg_ns {
  sipg_mesh* mv = nullptr;  // velocity mesh (walls Dirichlet)
  sipg_mesh* mp = nullptr;  // pressure mesh (walls Neumann)
  sipg_ns_params prm{};
  long long N = 0;          // nodes per component
  int P = 0;
  int device = 0;
  // history ring: level i lives in slot lev[i]
  double* u[3] = {nullptr, nullptr, nullptr};
  double* c[3] = {nullptr, nullptr, nullptr};
  double* h[3] = {nullptr, nullptr, nullptr};
  int lev[3] = {0, 1, 2};
  int nlev = 0;
  double *uhat = nullptr, *uhh = nullptr, *t1 = nullptr, *t2 = nullptr;
  double *rhs_p = nullptr, *tau = nullptr;
  // pressure history for the extrapolated initial guess (Sec. 5.1)
  double* pr[3] = {nullptr, nullptr, nullptr};
  int plev[3] = {0, 1, 2};
  int npl = 0;
  int *dwcell = nullptr, *dwmask = nullptr, *dwfirst = nullptr;
  int nw = 0, nwf = 0;
  std::vector<void*> owned;
  ~sipg_ns() {
    for (void* q : owned) cudaFree(q);
    if (mv) sipg_destroy_mesh(mv);
    if (mp) sipg_destroy_mesh(mp);
  }
};

namespace {

int ns_alloc(sipg_ns& ns, void** ptr, size_t bytes) {
  cudaError_t e = cudaMalloc(ptr, bytes ? bytes : 8);
  if (e != cudaSuccess) return fail(SIPG_ENOMEM, "stepper buffers: cudaMalloc failed");
  ns.owned.push_back(*ptr);
  cudaMemset(*ptr, 0, bytes ? bytes : 8);
  return SIPG_OK;
}

int ns_device(const sipg_ns& ns) {
  int cur = -1;
  cudaError_t e = cudaGetDevice(&cur);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (cur != ns.device && (e = cudaSetDevice(ns.device)) != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  return SIPG_OK;
}

// Wall data of level `slot` only (nbeta = 0) or with the pressure face terms.
int ns_wall(const sipg_ns& ns, int slot, int nbeta, const double* beta, const double* f, cudaStream_t s) {
  const Mesh& m = *ns.mv;
  WallArgs a{};
  a.wcell = ns.dwcell;
  a.wmask = ns.dwmask;
  a.wfirst = ns.dwfirst;
  a.tab = m.dns64;
  for (int d = 0; d < 3; ++d) {
    a.off[d] = m.ns_off[d];
    a.n[d] = m.desc.n[d];
  }
  a.ncell = m.ncell;
  a.nu = ns.prm.nu;
  a.u = ns.u[slot];
  a.hnew = ns.h[slot];
  a.nbeta = nbeta;
  for (int i = 0; i < 3; ++i) {
    a.hold[i] = i < ns.nlev ? ns.h[ns.lev[i]] : nullptr;
    a.beta[i] = (beta && i < nbeta) ? beta[i] : 0.0;
    a.f[i] = f ? f[i] : 0.0;
  }
  a.rhs = ns.rhs_p;
  const int st = launch_wall(ns.P, ns.nw, a, s);
  if (st == SIPG_OK) const_cast<sipg_mesh*>(ns.mv)->launches += ns.nw ? 1 : 0;
  return st;
}

// Convective term and wall data of the level in `slot`.
int ns_level_terms(sipg_ns& ns, int slot, cudaStream_t s) {
  int st = sipg_apply_convective_f64(ns.mv, ns.u[slot], ns.c[slot], s);
  if (st) return st;
  return ns_wall(ns, slot, 0, nullptr, nullptr, s);
}

int ns_lincomb(sipg_ns& ns, long long n, int m, const double* const* x, const double* c, const double* add, double* y,
               cudaStream_t s) {
  const int st = launch_lincomb(n, ns.N, m, x, c, add, y, s);
  if (st == SIPG_OK) ns.mv->launches++;
  return st;
}

}  // namespace

extern "C" {

int sipg_ns_default_params(sipg_ns_params* prm) {
  if (!prm) return fail(SIPG_EINVAL, "params is NULL");
  std::memset(prm, 0, sizeof(*prm));
  prm->k = 3;
  prm->penalty = 1.0;
  prm->nu = 1.0 / 180.0;
  prm->dt = 1e-3;
  prm->order = 3;
  prm->zeta = 1.0;
  prm->pressure_precond = SIPG_PC_JACOBI;
  prm->rtol_pressure = 1e-10;
  prm->rtol_viscous = 1e-10;
  prm->rtol_projection = 1e-10;
  prm->maxit = 10000;
  prm->maxit_projection = 500;
  return SIPG_OK;
}

int sipg_ns_create(const sipg_mesh_desc* desc, const sipg_ns_params* prm, sipg_ns** out) {
  if (!desc || !prm || !out) return fail(SIPG_EINVAL, "NULL argument");
  *out = nullptr;
  if (prm->k < 2 || prm->k > 7) return fail(SIPG_EINVAL, "the stepper needs 2 <= k <= 7 (pressure wall data)");
  if (desc->map == SIPG_MAP_PERTURBED) return fail(SIPG_EINVAL, "the stepper needs a separable map");
  if (!(prm->nu > 0.0) || !std::isfinite(prm->nu)) return fail(SIPG_EINVAL, "nu must be finite and > 0");
  if (!(prm->dt > 0.0) || !std::isfinite(prm->dt)) return fail(SIPG_EINVAL, "dt must be finite and > 0");
  if (prm->order < 1 || prm->order > 3) return fail(SIPG_EINVAL, "order must be 1, 2 or 3");
  if (!(prm->zeta >= 0.0) || !std::isfinite(prm->zeta)) return fail(SIPG_EINVAL, "zeta must be finite and >= 0");
  if (prm->pressure_precond != SIPG_PC_JACOBI && prm->pressure_precond != SIPG_PC_GMG_F32)
    return fail(SIPG_EINVAL, "pressure_precond must be SIPG_PC_JACOBI or SIPG_PC_GMG_F32");
  if (!(prm->rtol_pressure > 0.0) || !(prm->rtol_viscous > 0.0) || !(prm->rtol_projection > 0.0) ||
      prm->maxit < 1 || prm->maxit_projection < 1)
    return fail(SIPG_EINVAL, "tolerances must be > 0 and iteration bounds >= 1");
  sipg_mesh_desc dp = *desc;
  for (int d = 0; d < 3; ++d) {
    if (desc->bc_lo[d] == SIPG_BC_NEUMANN || desc->bc_hi[d] == SIPG_BC_NEUMANN)
      return fail(SIPG_EINVAL, "the stepper supports periodic sides and no-slip walls only");
    if (dp.bc_lo[d] == SIPG_BC_DIRICHLET) dp.bc_lo[d] = SIPG_BC_NEUMANN;
    if (dp.bc_hi[d] == SIPG_BC_DIRICHLET) dp.bc_hi[d] = SIPG_BC_NEUMANN;
  }
  sipg_ns* ns = new (std::nothrow) sipg_ns();
  if (!ns) return fail(SIPG_ENOMEM, "host allocation");
  int st;
  auto bail = [&](int code) {
    delete ns;
    return code;
  };
  ns->prm = *prm;
  if ((st = sipg_create_mesh(desc, &ns->mv)) || (st = sipg_create_mesh(&dp, &ns->mp))) return bail(st);
  if ((st = sipg_set_degree(ns->mv, prm->k)) || (st = sipg_set_degree(ns->mp, prm->k))) return bail(st);
  if ((st = sipg_set_penalty(ns->mv, prm->penalty)) || (st = sipg_set_penalty(ns->mp, prm->penalty)))
    return bail(st);
  ns->device = ns->mv->device;
  ns->P = prm->k + 1;
  ns->N = ns->mv->ncell * ns->P * ns->P * ns->P;
  // wall cells and faces
  std::vector<int> wc, wm, wf;
  const int* n = desc->n;
  for (long long e = 0; e < ns->mv->ncell; ++e) {
    const int id[3] = {(int)(e % n[0]), (int)((e / n[0]) % n[1]), (int)(e / ((long long)n[0] * n[1]))};
    int mask = 0;
    for (int d = 0; d < 3; ++d) {
      if (id[d] == 0 && desc->bc_lo[d] == SIPG_BC_DIRICHLET) mask |= 1 << (2 * d);
      if (id[d] == n[d] - 1 && desc->bc_hi[d] == SIPG_BC_DIRICHLET) mask |= 1 << (2 * d + 1);
    }
    if (mask) {
      wc.push_back((int)e);
      wm.push_back(mask);
      wf.push_back(ns->nwf);
      ns->nwf += __builtin_popcount(mask);
    }
  }
  ns->nw = (int)wc.size();
  const size_t V = (size_t)3 * ns->N * sizeof(double), S = (size_t)ns->N * sizeof(double);
  const size_t H = (size_t)ns->nwf * ns->P * ns->P * sizeof(double);
  for (int i = 0; i < 3; ++i) {
    if ((st = ns_alloc(*ns, (void**)&ns->u[i], V)) || (st = ns_alloc(*ns, (void**)&ns->c[i], V)) ||
        (st = ns_alloc(*ns, (void**)&ns->h[i], H)))
      return bail(st);
  }
  if ((st = ns_alloc(*ns, (void**)&ns->uhat, V)) || (st = ns_alloc(*ns, (void**)&ns->uhh, V)) ||
      (st = ns_alloc(*ns, (void**)&ns->t1, V)) || (st = ns_alloc(*ns, (void**)&ns->t2, V)) ||
      (st = ns_alloc(*ns, (void**)&ns->rhs_p, S)) || (st = ns_alloc(*ns, (void**)&ns->pr[0], S)) ||
      (st = ns_alloc(*ns, (void**)&ns->pr[1], S)) || (st = ns_alloc(*ns, (void**)&ns->pr[2], S)) ||
      (st = ns_alloc(*ns, (void**)&ns->tau, (size_t)ns->mv->ncell * sizeof(double))) ||
      (st = ns_alloc(*ns, (void**)&ns->dwcell, wc.size() * sizeof(int))) ||
      (st = ns_alloc(*ns, (void**)&ns->dwmask, wm.size() * sizeof(int))) ||
      (st = ns_alloc(*ns, (void**)&ns->dwfirst, wf.size() * sizeof(int))))
    return bail(st);
  cudaError_t e = cudaSuccess;
  if (ns->nw) {
    e = cudaMemcpy(ns->dwcell, wc.data(), wc.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(ns->dwmask, wm.data(), wm.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(ns->dwfirst, wf.data(), wf.size() * sizeof(int), cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) return bail(cuda_fail(e, "stepper wall lists"));
  *out = ns;
  return SIPG_OK;
}

int sipg_ns_destroy(sipg_ns* ns) {
  if (!ns) return fail(SIPG_EINVAL, "stepper is NULL");
  ns_device(*ns);
  delete ns;
  return SIPG_OK;
}

int sipg_ns_mesh(sipg_ns* ns, int which, sipg_mesh** out) {
  if (!ns || !out || (which != 0 && which != 1)) return fail(SIPG_EINVAL, "bad argument");
  *out = which == 0 ? ns->mv : ns->mp;
  return SIPG_OK;
}

int sipg_ns_set_velocity(sipg_ns* ns, int level, const double* u, void* stream) {
  if (!ns || !u) return fail(SIPG_EINVAL, "NULL argument");
  if (level < 0 || level >= ns->prm.order) return fail(SIPG_EINVAL, "level must be in [0, order)");
  if (level > ns->nlev) return fail(SIPG_EINVAL, "set the levels in order: 0, then 1, then 2");
  int st;
  if ((st = ns_device(*ns))) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if (level == 0) {
    ns->nlev = 0;
    for (int i = 0; i < 3; ++i) ns->lev[i] = i;
  }
  const int slot = ns->lev[level];
  cudaError_t e = cudaMemcpyAsync(ns->u[slot], u, (size_t)3 * ns->N * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return cuda_fail(e, "copy velocity");
  ns->nlev = level + 1;
  if ((st = ns_level_terms(*ns, slot, s))) return st;
  if (level == 0) {
    ns->npl = 0;
    for (int i = 0; i < 3; ++i) ns->plev[i] = i;
    cudaMemsetAsync(ns->pr[0], 0, (size_t)ns->N * sizeof(double), s);
  }
  e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? SIPG_OK : cuda_fail(e, "set velocity");
}

static int ns_step(sipg_ns* ns, const double* f, void* stream, sipg_ns_stats* stats);

int sipg_ns_step(sipg_ns* ns, const double* f, void* stream, sipg_ns_stats* stats) {
  if (!ns) return fail(SIPG_EINVAL, "stepper is NULL");
  const int st = ns_step(ns, f, stream, stats);
  if (st != SIPG_OK && st != SIPG_MAXITER && ns->nlev > 0) {
    // a slot may already hold part of the new level: forget the history
    ns->nlev = 0;
    ns->npl = 0;
  }
  return st;
}

static int ns_step(sipg_ns* ns, const double* f, void* stream, sipg_ns_stats* stats) {
  if (ns->nlev < 1) return fail(SIPG_EINVAL, "set the velocity (level 0) before stepping");
  int st;
  if ((st = ns_device(*ns))) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const sipg_ns_params& q = ns->prm;
  const double fz[3] = {0.0, 0.0, 0.0};
  const double* fv = f ? f : fz;
  const int J = ns->nlev < q.order ? ns->nlev : q.order;
  double g0, al[3], be[3];
  bdf_ex(J, g0, al, be);
  const double dt = q.dt;
  const long long N = ns->N, N3 = 3 * N;
  // (i) u_hat = (sum alpha_i u^(n-i) + dt M^-1 sum beta_i C^(n-i) + dt f) / gamma0
  {
    const double* x[3];
    for (int i = 0; i < J; ++i) x[i] = ns->c[ns->lev[i]];
    if ((st = ns_lincomb(*ns, N3, J, x, be, nullptr, ns->t1, s))) return st;
    if ((st = sipg_apply_inverse_mass_f64(ns->mv, ns->t1, ns->t2, 3, s))) return st;
    const double* y[4];
    double c[4];
    for (int i = 0; i < J; ++i) {
      y[i] = ns->u[ns->lev[i]];
      c[i] = al[i] / g0;
    }
    y[J] = ns->t2;
    c[J] = dt / g0;
    const double add[3] = {dt * fv[0] / g0, dt * fv[1] / g0, dt * fv[2] / g0};
    if ((st = ns_lincomb(*ns, N3, J + 1, y, c, add, ns->uhat, s))) return st;
  }
  // (ii) pressure: rhs = (gamma0/dt) D u_hat + wall terms, zero-mean CG
  {
    if ((st = sipg_apply_divergence_f64(ns->mv, ns->uhat, ns->rhs_p, s))) return st;
    const double* x[1] = {ns->rhs_p};
    const double c[1] = {g0 / dt};
    if ((st = ns_lincomb(*ns, N, 1, x, c, nullptr, ns->rhs_p, s))) return st;
    // (recomputes level 0's wall data in place: the same values)
    if ((st = ns_wall(*ns, ns->lev[0], J, be, fv, s))) return st;
  }
  sipg_cg_opts po;
  sipg_cg_default_opts(&po);
  po.op = SIPG_OP_LAPLACE;
  po.precond = q.pressure_precond;
  po.flexible = q.pressure_precond == SIPG_PC_GMG_F32 ? 1 : 0;
  po.zero_mean = 1;
  po.rtol = q.rtol_pressure;
  po.maxit = q.maxit;
  int pit = 0, vit = 0, jit = 0;
  double prr = 0.0, vrr = 0.0;
  // initial guess: the pressure extrapolated with the beta of the order the
  // known pressure levels allow (Sec. 5.1)
  const int Jp = ns->npl < J ? ns->npl : J;
  const int new_p = ns->npl < q.order ? ns->plev[ns->npl] : ns->plev[q.order - 1];
  if (Jp > 0) {
    double gp, ap[3], bp[3];
    bdf_ex(Jp, gp, ap, bp);
    const double* x[3];
    for (int i = 0; i < Jp; ++i) x[i] = ns->pr[ns->plev[i]];
    if ((st = ns_lincomb(*ns, N, Jp, x, bp, nullptr, ns->pr[new_p], s))) return st;
  } else {
    cudaMemsetAsync(ns->pr[new_p], 0, (size_t)N * sizeof(double), s);
  }
  const int pst = sipg_cg_solve(ns->mp, &po, ns->rhs_p, ns->pr[new_p], 1, s, &pit, &prr);
  if (pst != SIPG_OK && pst != SIPG_MAXITER) return pst;
  // (iii) projection: (M + tau_D B) u_hathat = M u_hat + (dt/gamma0) G p
  if ((st = sipg_tau_div_f64(ns->mv, ns->u[ns->lev[0]], q.zeta, dt, ns->tau, s))) return st;
  if ((st = sipg_apply_mass_f64(ns->mv, ns->uhat, ns->t1, 3, s))) return st;
  if ((st = sipg_apply_gradient_f64(ns->mv, ns->pr[new_p], ns->t2, s))) return st;
  {
    const double* x[2] = {ns->t1, ns->t2};
    const double c[2] = {1.0, dt / g0};
    if ((st = ns_lincomb(*ns, N3, 2, x, c, nullptr, ns->t1, s))) return st;
  }
  cudaError_t e = cudaMemcpyAsync(ns->uhh, ns->uhat, (size_t)N3 * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return cuda_fail(e, "copy u_hat");
  const int jst = sipg_project_divdiv_f64(ns->mv, ns->tau, ns->t1, ns->uhh, q.rtol_projection, q.maxit_projection, s,
                                          &jit);
  if (jst != SIPG_OK && jst != SIPG_MAXITER) return jst;
  // (iv) viscous step into the oldest slot, from u_hathat
  if ((st = sipg_apply_mass_f64(ns->mv, ns->uhh, ns->t1, 3, s))) return st;
  {
    const double* x[1] = {ns->t1};
    const double c[1] = {g0 / dt};
    if ((st = ns_lincomb(*ns, N3, 1, x, c, nullptr, ns->t1, s))) return st;
  }
  // a free slot while fewer than `order` levels are known, else the oldest
  // level's (its data were last used in (ii))
  const int new_slot = (ns->nlev < q.order) ? ns->lev[ns->nlev] : ns->lev[q.order - 1];
  {
    // initial guess: the velocity extrapolated with beta (Sec. 5.1); the slot
    // may hold the oldest level, read and overwritten element by element
    const double* x[3];
    for (int i = 0; i < J; ++i) x[i] = ns->u[ns->lev[i]];
    if ((st = ns_lincomb(*ns, N3, J, x, be, nullptr, ns->u[new_slot], s))) return st;
  }
  sipg_cg_opts vo;
  sipg_cg_default_opts(&vo);
  vo.op = SIPG_OP_VISCOUS;
  vo.mass_coef = g0 / dt;
  vo.nu = q.nu;
  vo.precond = SIPG_PC_INVMASS;
  vo.rtol = q.rtol_viscous;
  vo.maxit = q.maxit;
  const int vst = sipg_cg_solve(ns->mv, &vo, ns->t1, ns->u[new_slot], 3, s, &vit, &vrr);
  if (vst != SIPG_OK && vst != SIPG_MAXITER) return vst;
  // rotate: the new level becomes level 0
  const int keep = ns->nlev < q.order ? ns->nlev + 1 : q.order;
  int nl[3] = {new_slot, 0, 0};
  int w = 1;
  for (int i = 0; i < 3 && w < 3; ++i)
    if (ns->lev[i] != new_slot) nl[w++] = ns->lev[i];
  for (int i = 0; i < 3; ++i) ns->lev[i] = nl[i];
  ns->nlev = keep;
  int pl[3] = {new_p, 0, 0};
  w = 1;
  for (int i = 0; i < 3 && w < 3; ++i)
    if (ns->plev[i] != new_p) pl[w++] = ns->plev[i];
  for (int i = 0; i < 3; ++i) ns->plev[i] = pl[i];
  ns->npl = ns->npl < q.order ? ns->npl + 1 : q.order;
  if ((st = ns_level_terms(*ns, new_slot, s))) return st;
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "step");
  if (stats) {
    stats->order = J;
    stats->pressure_iters = pit;
    stats->viscous_iters = vit;
    stats->projection_iters = jit;
    stats->pressure_relres = prr;
    stats->viscous_relres = vrr;
  }
  if (pst == SIPG_MAXITER) return fail(SIPG_MAXITER, "pressure CG reached maxit");
  if (jst == SIPG_MAXITER) return fail(SIPG_MAXITER, "a cell's projection CG reached maxit");
  if (vst == SIPG_MAXITER) return fail(SIPG_MAXITER, "viscous CG reached maxit");
  return SIPG_OK;
}

int sipg_ns_velocity(const sipg_ns* ns, double* u, void* stream) {
  if (!ns || !u) return fail(SIPG_EINVAL, "NULL argument");
  if (ns->nlev < 1) return fail(SIPG_EINVAL, "no velocity set");
  int st;
  if ((st = ns_device(*ns))) return st;
  const cudaError_t e = cudaMemcpyAsync(u, ns->u[ns->lev[0]], (size_t)3 * ns->N * sizeof(double),
                                        cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
  return e == cudaSuccess ? SIPG_OK : cuda_fail(e, "copy velocity");
}

int sipg_ns_pressure(const sipg_ns* ns, double* p, void* stream) {
  if (!ns || !p) return fail(SIPG_EINVAL, "NULL argument");
  int st;
  if ((st = ns_device(*ns))) return st;
  const cudaError_t e = cudaMemcpyAsync(p, ns->pr[ns->plev[0]], (size_t)ns->N * sizeof(double),
                                        cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
  return e == cudaSuccess ? SIPG_OK : cuda_fail(e, "copy pressure");
}

int sipg_ns_wall_data(const sipg_ns* ns, double* h, long long* count, void* stream) {
  if (!ns || !count) return fail(SIPG_EINVAL, "NULL argument");
  *count = (long long)ns->nwf * ns->P * ns->P;
  if (!h) return SIPG_OK;
  if (ns->nlev < 1) return fail(SIPG_EINVAL, "no velocity set");
  int st;
  if ((st = ns_device(*ns))) return st;
  if (*count == 0) return SIPG_OK;
  const cudaError_t e = cudaMemcpyAsync(h, ns->h[ns->lev[0]], (size_t)*count * sizeof(double),
                                        cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
  return e == cudaSuccess ? SIPG_OK : cuda_fail(e, "copy wall data");
}

}  // extern "C"
