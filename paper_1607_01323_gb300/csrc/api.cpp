// C ABI of libsipg: argument validation, mesh lifetime, profiling and the
// cells-per-block autotuner.  Every entry point returns a status and never
// aborts; CUDA errors become SIPG_ECUDA with the runtime's message.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <sstream>
#include <string>
#include <type_traits>

#include "sipg_internal.h"

namespace sipg {

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }

int fail(int status, const std::string& msg) {
  g_err = msg;
  return status;
}

int cuda_fail(cudaError_t e, const char* where) {
  g_err = std::string(where) + ": " + cudaGetErrorString(e);
  cudaGetLastError();
  return SIPG_ECUDA;
}

Mesh::~Mesh() {
  mg_release(*this);
  for (int d = 0; d < 3; ++d) {
    if (dtab64[d]) cudaFree(dtab64[d]);
    if (dtab32[d]) cudaFree(dtab32[d]);
  }
  for (int d = 0; d < 3; ++d)
    if (dtabdf[d]) cudaFree(dtabdf[d]);
  if (ws) cudaFree(ws);
  if (dC64) cudaFree(dC64);
  if (dC32) cudaFree(dC32);
  if (dCdf) cudaFree(dCdf);
  if (dconv64) cudaFree(dconv64);
  if (dconvdf) cudaFree(dconvdf);
  if (dns64) cudaFree(dns64);
  if (dscale) cudaFree(dscale);
  for (double* q : {dgen_head, dgen_geo, dgen_face, dgen_tau})
    if (q) cudaFree(q);
  for (auto& pr : pending) {
    cudaEventDestroy(pr.first);
    cudaEventDestroy(pr.second);
  }
}

template <typename T>
Geo<T> make_geo(const Mesh& m) {
  Geo<T> g;
  for (int d = 0; d < 3; ++d) {
    g.n[d] = m.desc.n[d];
    g.bc_lo[d] = m.desc.bc_lo[d];
    g.bc_hi[d] = m.desc.bc_hi[d];
  }
  g.ncell = (int)m.ncell;
  for (int d = 0; d < 3; ++d) {
    if (std::is_same<T, double>::value)
      g.tab[d] = reinterpret_cast<const T*>(m.dtab64[d]);
    else if (std::is_same<T, float>::value)
      g.tab[d] = reinterpret_cast<const T*>(m.dtab32[d]);
    else
      g.tab[d] = reinterpret_cast<const T*>(m.dtabdf[d]);
  }
  g.tau_scale = T(m.penalty * (m.k + 1) * (m.k + 1));
  g.dsc = m.dscale ? m.dscale + 2 : nullptr;
  for (int d = 0; d < 3; ++d) g.lm[d] = m.lay_same[d] ? 0 : -1;
  return g;
}
template Geo<double> make_geo<double>(const Mesh&);
template Geo<float> make_geo<float>(const Mesh&);
template Geo<dfl> make_geo<dfl>(const Mesh&);

// Default cells per block: the largest count whose p^2 threads per cell fill a
// 256-thread block with the fewest idle lanes (blocks are rounded up to whole
// warps): 64, 28, 16, 10, 7, 5, 4 cells for p = 2..8.
int default_cpb(int p, int precision) {
  (void)precision;
  switch (p) {
    case 2: return 64;
    case 3: return 28;
    case 4: return 16;
    case 5: return 10;
    case 6: return 7;
    case 7: return 5;
    default: return 4;
  }
}

// Plane mapping (P threads per cell): as many cells as fit 256 threads and
// about 100 KB of shared memory (three FP32 buffers of p^3 per cell).
int default_cpb_plane(int p) {
  int c = 256 / p;
  const int smem_cap = 100 * 1024 / (3 * p * p * p * 4);
  return c < smem_cap ? c : smem_cap;
}

int cells_per_block(const Mesh& m, int precision) {
  if (m.cpb[precision] > 0) return m.cpb[precision];
  return (precision == 1 && m.f32_mapping == 1) ? default_cpb_plane(m.p) : default_cpb(m.p, precision);
}

void prof_begin(Mesh& m, cudaStream_t s, cudaEvent_t* e0) {
  *e0 = nullptr;
  if (!m.profile) return;
  cudaEventCreate(e0);
  cudaEventRecord(*e0, s);
}

void prof_end(Mesh& m, cudaStream_t s, cudaEvent_t e0) {
  if (!m.profile || !e0) return;
  cudaEvent_t e1;
  cudaEventCreate(&e1);
  cudaEventRecord(e1, s);
  m.pending.emplace_back(e0, e1);
}

}  // namespace sipg

using namespace sipg;


namespace {

bool valid_bc(int b) { return b == SIPG_BC_PERIODIC || b == SIPG_BC_DIRICHLET || b == SIPG_BC_NEUMANN; }

int check_mesh(const sipg_mesh* m) {
  if (!m) return fail(SIPG_EINVAL, "mesh is NULL");
  return SIPG_OK;
}

// Entry points built on the separable 1D tables reject the general map.
int check_separable(const sipg_mesh* m) {
  int st;
  if ((st = check_mesh(m))) return st;
  if (m->general()) return fail(SIPG_EINVAL, "this operation needs a separable map (not SIPG_MAP_PERTURBED)");
  return SIPG_OK;
}

int check_vec(const void* x, const void* y, int ncomp) {
  if (!x || !y) return fail(SIPG_EINVAL, "vector pointer is NULL");
  if (ncomp < 1) return fail(SIPG_EINVAL, "ncomp must be >= 1");
  if (x == y) return fail(SIPG_EINVAL, "x and y must not alias");
  return SIPG_OK;
}

int set_device(const Mesh& m) {
  int cur = -1;
  cudaError_t e = cudaGetDevice(&cur);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (cur != m.device) {
    e = cudaSetDevice(m.device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  }
  return SIPG_OK;
}

long long n_dofs(const Mesh& m) { return m.ncell * m.p * m.p * m.p; }

template <typename T>
int apply_common(const sipg_mesh* mc, T cm, T nu, const T* nu_cell, bool stiffness, const T* x, T* y, int ncomp,
                 void* stream) {
  int st;
  if ((st = check_mesh(mc))) return st;
  if ((st = check_vec(x, y, ncomp))) return st;
  if (!(cm >= T(0)) || !std::isfinite((double)cm)) return fail(SIPG_EINVAL, "mass_coef must be finite and >= 0");
  if (stiffness && !nu_cell && !(nu > T(0))) return fail(SIPG_EINVAL, "nu must be > 0");
  Mesh& m = const_cast<sipg_mesh&>(*mc);
  if ((st = set_device(m))) return st;
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0;
  if (m.general()) {
    if (!std::is_same<T, double>::value || nu_cell)
      return fail(SIPG_EINVAL, "a perturbed mesh supports FP64 applies with a constant viscosity only");
    prof_begin(m, s, &e0);
    st = launch_general(m, reinterpret_cast<const double*>(x), reinterpret_cast<double*>(y), ncomp, (double)cm,
                        (double)nu, stiffness, nullptr, s);
    prof_end(m, s, e0);
    if (st == SIPG_OK && m.profile) m.prof_applies++;
    return st;
  }
  prof_begin(m, s, &e0);
  st = launch_apply<T>(m, x, y, ncomp, cm, nu, nu_cell, stiffness, nullptr, nullptr, s);
  prof_end(m, s, e0);
  if (st == SIPG_OK && m.profile) m.prof_applies++;
  return st;
}

}  // namespace

extern "C" {

const char* sipg_last_error(void) { return g_err.c_str(); }

int sipg_create_mesh(const sipg_mesh_desc* d, sipg_mesh** out) {
  if (!d || !out) return fail(SIPG_EINVAL, "NULL argument");
  *out = nullptr;
  for (int i = 0; i < 3; ++i) {
    if (d->n[i] < 1) return fail(SIPG_EINVAL, "cells per direction must be >= 1");
    if (!(d->hi[i] > d->lo[i]) || !std::isfinite(d->lo[i]) || !std::isfinite(d->hi[i]))
      return fail(SIPG_EINVAL, "box needs finite lo < hi");
    if (!valid_bc(d->bc_lo[i]) || !valid_bc(d->bc_hi[i])) return fail(SIPG_EINVAL, "unknown boundary condition");
    if ((d->bc_lo[i] == SIPG_BC_PERIODIC) != (d->bc_hi[i] == SIPG_BC_PERIODIC))
      return fail(SIPG_EINVAL, "periodic sides must be paired");
  }
  if (d->map != SIPG_MAP_AFFINE && d->map != SIPG_MAP_CHANNEL_TANH && d->map != SIPG_MAP_CHANNEL_LINEAR &&
      d->map != SIPG_MAP_PERTURBED)
    return fail(SIPG_EINVAL, "unknown map");
  if ((d->map == SIPG_MAP_CHANNEL_TANH || d->map == SIPG_MAP_CHANNEL_LINEAR) &&
      !(d->gamma > 0.0 && std::isfinite(d->gamma)))
    return fail(SIPG_EINVAL, "channel map needs gamma > 0");
  if (d->map == SIPG_MAP_PERTURBED && !(d->amplitude >= 0.0 && std::isfinite(d->amplitude)))
    return fail(SIPG_EINVAL, "perturbed map needs a finite amplitude >= 0");
  long long nc = (long long)d->n[0] * d->n[1] * d->n[2];
  if (nc * 512 >= (1LL << 31) * 8LL) return fail(SIPG_EINVAL, "mesh too large");
  if (nc >= (1LL << 31)) return fail(SIPG_EINVAL, "too many cells");
  sipg_mesh* m = new (std::nothrow) sipg_mesh();
  if (!m) return fail(SIPG_ENOMEM, "host allocation failed");
  m->desc = *d;
  m->ncell = nc;
  cudaError_t e = cudaGetDevice(&m->device);
  if (e != cudaSuccess) {
    delete m;
    return cuda_fail(e, "cudaGetDevice");
  }
  m->k = 3;
  m->p = 4;
  e = cudaMalloc(&m->dscale, 4 * sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(m->dscale, 0, 4 * sizeof(int));
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete m;
    return fail(SIPG_ENOMEM, "cudaMalloc of the mesh's scale word failed");
  }
  int st = build_tables(*m);
  if (st) {
    delete m;
    return st;
  }
  *out = m;
  return SIPG_OK;
}

int sipg_destroy_mesh(sipg_mesh* m) {
  if (!m) return SIPG_OK;
  set_device(*m);
  cudaDeviceSynchronize();
  delete m;
  return SIPG_OK;
}

int sipg_set_degree(sipg_mesh* m, int k) {
  int st;
  if ((st = check_mesh(m))) return st;
  if (k < 1 || k > 7) return fail(SIPG_EINVAL, "degree must be 1 <= k <= 7");
  if ((st = set_device(*m))) return st;
  cudaDeviceSynchronize();
  mg_release(*m);
  const int k0 = m->k;
  m->k = k;
  m->p = k + 1;
  st = build_tables(*m);
  if (st) {
    m->k = k0;
    m->p = k0 + 1;
    build_tables(*m);
    return st;
  }
  m->cpb[0] = m->cpb[1] = 0;
  return SIPG_OK;
}

int sipg_set_penalty(sipg_mesh* m, double f) {
  int st;
  if ((st = check_mesh(m))) return st;
  if (!(f > 0.0) || !std::isfinite(f)) return fail(SIPG_EINVAL, "penalty factor must be > 0");
  if ((st = set_device(*m))) return st;
  cudaDeviceSynchronize();  // the tables hold the penalty shares: no launch may still read them
  mg_release(*m);
  const double f0 = m->penalty;
  m->penalty = f;
  st = build_tables(*m);
  if (st) {
    m->penalty = f0;
    build_tables(*m);
  }
  return st;
}

int sipg_n_dofs(const sipg_mesh* m, long long* n) {
  int st;
  if ((st = check_mesh(m))) return st;
  if (!n) return fail(SIPG_EINVAL, "NULL output");
  *n = n_dofs(*m);
  return SIPG_OK;
}

int sipg_n_cells(const sipg_mesh* m, long long* n) {
  int st;
  if ((st = check_mesh(m))) return st;
  if (!n) return fail(SIPG_EINVAL, "NULL output");
  *n = m->ncell;
  return SIPG_OK;
}

int sipg_node_coordinates(const sipg_mesh* m, double* xyz) {
  int st;
  if ((st = check_mesh(m))) return st;
  if (!xyz) return fail(SIPG_EINVAL, "NULL output");
  const int p = m->p;
  std::vector<double> zn, wn;
  gll_rule(p, zn, wn);
  std::vector<double> X[3];
  for (int d = 0; d < 3; ++d) {
    const int n = m->desc.n[d];
    X[d].resize((size_t)n * p);
    for (int i = 0; i < n; ++i)
      for (int a = 0; a < p; ++a) X[d][(size_t)i * p + a] = map_coord(m->desc, d, (i + zn[a]) / n);
  }
  const int nx = m->desc.n[0], ny = m->desc.n[1];
  long long idx = 0;
  if (m->general()) {
    const int* n = m->desc.n;
    for (long long e = 0; e < m->ncell; ++e) {
      const int ix = (int)(e % nx), iy = (int)((e / nx) % ny), iz = (int)(e / ((long long)nx * ny));
      for (int c = 0; c < p; ++c)
        for (int b = 0; b < p; ++b)
          for (int a = 0; a < p; ++a, ++idx) {
            const double s[3] = {(ix + zn[a]) / n[0], (iy + zn[b]) / n[1], (iz + zn[c]) / n[2]};
            map_point(m->desc, s, xyz + 3 * idx);
          }
    }
    return SIPG_OK;
  }
  for (long long e = 0; e < m->ncell; ++e) {
    const int ix = (int)(e % nx), iy = (int)((e / nx) % ny), iz = (int)(e / ((long long)nx * ny));
    for (int c = 0; c < p; ++c)
      for (int b = 0; b < p; ++b)
        for (int a = 0; a < p; ++a, ++idx) {
          xyz[3 * idx + 0] = X[0][(size_t)ix * p + a];
          xyz[3 * idx + 1] = X[1][(size_t)iy * p + b];
          xyz[3 * idx + 2] = X[2][(size_t)iz * p + c];
        }
  }
  return SIPG_OK;
}

int sipg_penalty_values(const sipg_mesh* m, double* tau) {
  int st;
  if ((st = check_mesh(m))) return st;
  if (!tau) return fail(SIPG_EINVAL, "NULL output");
  if (m->general()) {
    for (long long e = 0; e < m->ncell; ++e) tau[e] = m->htau_gen[(size_t)e];
    return SIPG_OK;
  }
  const int p = m->p, nx = m->desc.n[0], ny = m->desc.n[1];
  const double s = m->penalty * (m->k + 1) * (m->k + 1);
  const int st_ = lstride(p);
  for (long long e = 0; e < m->ncell; ++e) {
    const int ix = (int)(e % nx), iy = (int)((e / nx) % ny), iz = (int)(e / ((long long)nx * ny));
    tau[e] = s * (m->htab[0][(size_t)ix * st_ + lay_t(p)] + m->htab[1][(size_t)iy * st_ + lay_t(p)] +
                  m->htab[2][(size_t)iz * st_ + lay_t(p)]);
  }
  return SIPG_OK;
}

int sipg_apply_laplace_f64(const sipg_mesh* m, const double* x, double* y, int ncomp, void* stream) {
  return apply_common<double>(m, 0.0, 1.0, nullptr, true, x, y, ncomp, stream);
}

int sipg_apply_laplace_f32(const sipg_mesh* m, const float* x, float* y, int ncomp, void* stream) {
  return apply_common<float>(m, 0.f, 1.f, nullptr, true, x, y, ncomp, stream);
}

int sipg_apply_helmholtz_f64(const sipg_mesh* m, double cm, double nu, const double* nu_cell, const double* x,
                             double* y, int ncomp, void* stream) {
  return apply_common<double>(m, cm, nu, nu_cell, true, x, y, ncomp, stream);
}

int sipg_apply_helmholtz_f32(const sipg_mesh* m, float cm, float nu, const float* nu_cell, const float* x, float* y,
                             int ncomp, void* stream) {
  return apply_common<float>(m, cm, nu, nu_cell, true, x, y, ncomp, stream);
}

int sipg_apply_mass_f64(const sipg_mesh* m, const double* x, double* y, int ncomp, void* stream) {
  return apply_common<double>(m, 1.0, 0.0, nullptr, false, x, y, ncomp, stream);
}

int sipg_apply_inverse_mass_f64(const sipg_mesh* mc, const double* x, double* y, int ncomp, void* stream) {
  int st;
  if ((st = check_separable(mc))) return st;
  if ((st = check_vec(x, y, ncomp))) return st;
  Mesh& m = const_cast<sipg_mesh&>(*mc);
  if ((st = set_device(m))) return st;
  return launch_inverse_mass(m, x, y, ncomp, nullptr, false, (cudaStream_t)stream);
}

int sipg_diagonal_f64(const sipg_mesh* mc, int op, double cm, double nu, const double* nu_cell, double* diag,
                      void* stream) {
  int st;
  if ((st = check_mesh(mc))) return st;
  if (!diag) return fail(SIPG_EINVAL, "diag is NULL");
  if (op != SIPG_OP_LAPLACE && op != SIPG_OP_HELMHOLTZ) return fail(SIPG_EINVAL, "unknown operator");
  Mesh& m = const_cast<sipg_mesh&>(*mc);
  if ((st = set_device(m))) return st;
  if (op == SIPG_OP_LAPLACE) return launch_diagonal(m, true, 0.0, 1.0, nullptr, diag, (cudaStream_t)stream);
  if (!(cm >= 0.0) || (!nu_cell && !(nu > 0.0))) return fail(SIPG_EINVAL, "need mass_coef >= 0 and nu > 0");
  return launch_diagonal(m, true, cm, nu, nu_cell, diag, (cudaStream_t)stream);
}

int sipg_cg_default_opts(sipg_cg_opts* o) {
  if (!o) return fail(SIPG_EINVAL, "NULL opts");
  std::memset(o, 0, sizeof(*o));
  o->op = SIPG_OP_LAPLACE;
  o->mass_coef = 0.0;
  o->nu = 1.0;
  o->nu_cell = nullptr;
  o->precond = SIPG_PC_JACOBI;
  o->cheb_degree = 4;
  o->cheb_range = 20.0;
  o->cheb_lmax = 0.0;
  o->cheb_lanczos_steps = 20;
  o->zero_mean = 0;
  o->rtol = 1e-10;
  o->maxit = 10000;
  o->flexible = 0;
  o->use_graph = 1;
  o->check_every = 16;
  o->mg_degree = 5;
  o->mg_range = 20.0;
  o->mg_coarse_tol = 1e-3;
  o->mg_coarse_maxdeg = 200;
  return SIPG_OK;
}

int sipg_cg_solve(sipg_mesh* m, const sipg_cg_opts* o, const double* b, double* x, int ncomp, void* stream,
                  int* iters, double* relres) {
  int st;
  if ((st = check_mesh(m))) return st;
  if (!o) return fail(SIPG_EINVAL, "opts is NULL");
  if ((st = check_vec(b, x, ncomp))) return st;
  if (o->op != SIPG_OP_LAPLACE && o->op != SIPG_OP_HELMHOLTZ && o->op != SIPG_OP_VISCOUS)
    return fail(SIPG_EINVAL, "unknown operator");
  if (o->op == SIPG_OP_HELMHOLTZ && (!(o->mass_coef >= 0.0) || (!o->nu_cell && !(o->nu > 0.0))))
    return fail(SIPG_EINVAL, "Helmholtz needs mass_coef >= 0 and nu > 0");
  if (o->op == SIPG_OP_VISCOUS) {
    if (!(o->mass_coef >= 0.0) || !(o->nu > 0.0) || o->nu_cell)
      return fail(SIPG_EINVAL, "the viscous operator needs mass_coef >= 0, a constant nu > 0 and no nu_cell");
    if (ncomp != 3) return fail(SIPG_EINVAL, "the viscous operator couples exactly 3 components");
    if (o->precond != SIPG_PC_NONE && o->precond != SIPG_PC_INVMASS)
      return fail(SIPG_EINVAL, "the viscous operator supports the preconditioners none and invmass");
    if (o->zero_mean) return fail(SIPG_EINVAL, "zero_mean applies to the Laplace operator only");
  }
  if (o->precond < SIPG_PC_NONE || o->precond > SIPG_PC_GMG_F32) return fail(SIPG_EINVAL, "unknown preconditioner");
  if (m->general() && (o->op == SIPG_OP_VISCOUS || (o->precond != SIPG_PC_NONE && o->precond != SIPG_PC_JACOBI) ||
                       o->nu_cell))
    return fail(SIPG_EINVAL, "on a perturbed mesh CG supports the Laplace / Helmholtz operator with a constant nu "
                             "and SIPG_PC_NONE or SIPG_PC_JACOBI");
  if (o->precond == SIPG_PC_GMG_F32) {
    if (o->op != SIPG_OP_LAPLACE) return fail(SIPG_EINVAL, "the multigrid preconditioner supports the Laplace operator");
    if (ncomp != 1) return fail(SIPG_EINVAL, "the multigrid preconditioner supports one component");
  }
  if (o->precond == SIPG_PC_CHEB_F32) {
    if (o->cheb_degree < 1 || o->cheb_degree > 64) return fail(SIPG_EINVAL, "cheb_degree must be in [1, 64]");
    if (!(o->cheb_range > 1.0)) return fail(SIPG_EINVAL, "cheb_range must be > 1");
    if (!(o->cheb_lmax > 0.0) && (o->cheb_lanczos_steps < 2 || o->cheb_lanczos_steps > 128))
      return fail(SIPG_EINVAL, "cheb_lanczos_steps must be in [2, 128]");
    if (o->op == SIPG_OP_HELMHOLTZ && o->nu_cell)
      return fail(SIPG_EINVAL, "the FP32 Chebyshev preconditioner supports a constant nu only");
  }
  if (!(o->rtol >= 0.0) || o->maxit < 1) return fail(SIPG_EINVAL, "need rtol >= 0 and maxit >= 1");
  if (o->check_every < 1 || o->check_every > 4096) return fail(SIPG_EINVAL, "check_every must be in [1, 4096]");
  bool all_bc_free = true;  // singular operator: all sides periodic or Neumann, Laplace
  for (int d = 0; d < 3; ++d)
    if (m->desc.bc_lo[d] == SIPG_BC_DIRICHLET || m->desc.bc_hi[d] == SIPG_BC_DIRICHLET) all_bc_free = false;
  if (all_bc_free && o->op == SIPG_OP_LAPLACE && !o->zero_mean)
    return fail(SIPG_EINVAL, "singular Laplace problem (no Dirichlet side): set zero_mean");
  if ((st = set_device(*m))) return st;
  // The solve runs on a private non-blocking stream joined to the caller's
  // stream with events, so that graph capture also works when the caller uses
  // the legacy default stream.
  cudaStream_t cs = (cudaStream_t)stream, s = nullptr;
  cudaEvent_t ev = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
  e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    cudaStreamDestroy(s);
    return cuda_fail(e, "cudaEventCreate");
  }
  cudaEventRecord(ev, cs);
  cudaStreamWaitEvent(s, ev, 0);
  st = cg_solve(*m, *o, b, x, ncomp, s, iters, relres);
  cudaEventRecord(ev, s);
  cudaStreamWaitEvent(cs, ev, 0);
  cudaStreamSynchronize(s);
  cudaEventDestroy(ev);
  cudaStreamDestroy(s);
  return st;
}

int sipg_cg_solve_noalloc(sipg_mesh* m, const sipg_cg_opts* o, const double* b, double* x, int ncomp, void* stream,
                          int* iters, double* relres) {
  int st;
  if ((st = check_separable(m))) return st;
  if (!o) return fail(SIPG_EINVAL, "opts is NULL");
  if ((st = check_vec(b, x, ncomp))) return st;
  if (o->op != SIPG_OP_LAPLACE && o->op != SIPG_OP_HELMHOLTZ) return fail(SIPG_EINVAL, "unknown operator");
  if (o->op == SIPG_OP_HELMHOLTZ && (!(o->mass_coef >= 0.0) || (!o->nu_cell && !(o->nu > 0.0))))
    return fail(SIPG_EINVAL, "Helmholtz needs mass_coef >= 0 and nu > 0");
  if (o->precond < SIPG_PC_NONE || o->precond > SIPG_PC_INVMASS)
    return fail(SIPG_EINVAL, "the allocation-free solve supports preconditioners none, jacobi and invmass");
  if (!(o->rtol >= 0.0) || o->maxit < 1) return fail(SIPG_EINVAL, "need rtol >= 0 and maxit >= 1");
  if (o->check_every < 1 || o->check_every > 4096) return fail(SIPG_EINVAL, "check_every must be in [1, 4096]");
  bool all_bc_free = true;
  for (int d = 0; d < 3; ++d)
    if (m->desc.bc_lo[d] == SIPG_BC_DIRICHLET || m->desc.bc_hi[d] == SIPG_BC_DIRICHLET) all_bc_free = false;
  if (all_bc_free && o->op == SIPG_OP_LAPLACE && !o->zero_mean)
    return fail(SIPG_EINVAL, "singular Laplace problem (no Dirichlet side): set zero_mean");
  if ((st = set_device(*m))) return st;
  return cg_solve_noalloc(*m, *o, b, x, ncomp, (cudaStream_t)stream, iters, relres);
}

int sipg_mg_setup(sipg_mesh* m, const sipg_cg_opts* o, void* stream) {
  int st;
  if ((st = check_separable(m))) return st;
  if (!o) return fail(SIPG_EINVAL, "opts is NULL");
  bool all_bc_free = true;
  for (int d = 0; d < 3; ++d)
    if (m->desc.bc_lo[d] == SIPG_BC_DIRICHLET || m->desc.bc_hi[d] == SIPG_BC_DIRICHLET) all_bc_free = false;
  if (all_bc_free && !o->zero_mean)
    return fail(SIPG_EINVAL, "singular Laplace problem (no Dirichlet side): set zero_mean");
  if ((st = set_device(*m))) return st;
  return mg_setup(*m, *o, (cudaStream_t)stream);
}

int sipg_mg_info(const sipg_mesh* m, int max_levels, int* nlevels, int* n_cells, double* lmax, double* coarse_lmin,
                 int* coarse_degree) {
  int st;
  if ((st = check_mesh(m))) return st;
  if (max_levels < 0) return fail(SIPG_EINVAL, "max_levels must be >= 0");
  return mg_info(*m, max_levels, nlevels, n_cells, lmax, coarse_lmin, coarse_degree);
}

int sipg_mg_vcycle(sipg_mesh* m, const double* r, double* z, void* stream) {
  int st;
  if ((st = check_separable(m))) return st;
  if (!r || !z) return fail(SIPG_EINVAL, "NULL vector");
  if (r == z) return fail(SIPG_EINVAL, "r and z must not overlap");
  if (!m->mg) return fail(SIPG_EINVAL, "no multigrid hierarchy set up on this mesh (sipg_mg_setup)");
  if ((st = set_device(*m))) return st;
  return mg_vcycle(*m, r, z, nullptr, nullptr, nullptr, nullptr, (cudaStream_t)stream);
}

int sipg_apply_divergence_f64(const sipg_mesh* m, const double* u, double* y, void* stream) {
  int st;
  if ((st = check_separable(m))) return st;
  if (!u || !y) return fail(SIPG_EINVAL, "NULL vector");
  if (u == y) return fail(SIPG_EINVAL, "u and y must not overlap");
  if ((st = set_device(const_cast<sipg_mesh&>(*m)))) return st;
  return launch_divergence(*m, u, y, (cudaStream_t)stream);
}

int sipg_apply_gradient_f64(const sipg_mesh* m, const double* p, double* y, void* stream) {
  int st;
  if ((st = check_separable(m))) return st;
  if (!p || !y) return fail(SIPG_EINVAL, "NULL vector");
  if (p == y) return fail(SIPG_EINVAL, "p and y must not overlap");
  if ((st = set_device(const_cast<sipg_mesh&>(*m)))) return st;
  return launch_gradient(*m, p, y, (cudaStream_t)stream);
}

int sipg_apply_viscous_f64(const sipg_mesh* m, double mass_coef, double nu, const double* u, double* y,
                           void* stream) {
  int st;
  if ((st = check_separable(m))) return st;
  if (!u || !y) return fail(SIPG_EINVAL, "NULL vector");
  if (u == y) return fail(SIPG_EINVAL, "u and y must not overlap");
  if (!(mass_coef >= 0.0) || !std::isfinite(mass_coef)) return fail(SIPG_EINVAL, "mass_coef must be finite and >= 0");
  if (!(nu > 0.0) || !std::isfinite(nu)) return fail(SIPG_EINVAL, "nu must be finite and > 0");
  if ((st = set_device(*m))) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = launch_apply<double>(*m, u, y, 3, mass_coef, nu, nullptr, true, nullptr, nullptr, s))) return st;
  // in double-float the operator's scale pass over u left u's scale in the mesh's word
  return launch_viscous_t(*m, u, y, nu, nullptr, m->f64_arith == SIPG_F64_DOUBLE_FLOAT, s);
}

int sipg_apply_convective_f64(const sipg_mesh* m, const double* u, double* y, void* stream) {
  int st;
  if ((st = check_separable(m))) return st;
  if (!u || !y) return fail(SIPG_EINVAL, "NULL vector");
  if (u == y) return fail(SIPG_EINVAL, "u and y must not overlap");
  if ((st = set_device(*m))) return st;
  return launch_convective(*m, u, y, (cudaStream_t)stream);
}

int sipg_tau_div_f64(const sipg_mesh* m, const double* u, double zeta, double dt, double* tau, void* stream) {
  int st;
  if ((st = check_separable(m))) return st;
  if (!u || !tau) return fail(SIPG_EINVAL, "NULL vector");
  if (!(zeta >= 0.0) || !(dt >= 0.0) || !std::isfinite(zeta) || !std::isfinite(dt))
    return fail(SIPG_EINVAL, "zeta and dt must be finite and >= 0");
  if ((st = set_device(const_cast<sipg_mesh&>(*m)))) return st;
  return launch_tau_div(*m, u, zeta, dt, tau, (cudaStream_t)stream);
}

int sipg_apply_divdiv_f64(const sipg_mesh* m, const double* tau, const double* u, double* y, void* stream) {
  int st;
  if ((st = check_separable(m))) return st;
  if (!tau || !u || !y) return fail(SIPG_EINVAL, "NULL vector");
  if (u == y) return fail(SIPG_EINVAL, "u and y must not overlap");
  if ((st = set_device(const_cast<sipg_mesh&>(*m)))) return st;
  return launch_divdiv_apply(*m, tau, u, y, (cudaStream_t)stream);
}

int sipg_project_divdiv_f64(sipg_mesh* m, const double* tau, const double* rhs, double* x, double rtol, int maxit,
                            void* stream, int* iters_out) {
  int st;
  if ((st = check_separable(m))) return st;
  if (!tau || !rhs || !x) return fail(SIPG_EINVAL, "NULL vector");
  if (rhs == x) return fail(SIPG_EINVAL, "rhs and x must not overlap");
  if (!(rtol >= 0.0) || maxit < 1) return fail(SIPG_EINVAL, "need rtol >= 0 and maxit >= 1");
  if ((st = set_device(*m))) return st;
  cudaStream_t s = (cudaStream_t)stream;
  int* status = nullptr;
  cudaError_t e = cudaMalloc(&status, 2 * sizeof(int));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(SIPG_ENOMEM, "cudaMalloc of the solve status failed");
  }
  e = cudaMemsetAsync(status, 0, 2 * sizeof(int), s);
  if (e != cudaSuccess) {
    cudaFree(status);
    return cuda_fail(e, "clear solve status");
  }
  st = launch_divdiv_solve(*m, tau, rhs, x, rtol, maxit, status, s);
  int h[2] = {0, 0};
  if (!st) {
    e = cudaMemcpyAsync(h, status, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_fail(e, "read solve status");
  }
  cudaFree(status);
  if (st) return st;
  if (iters_out) *iters_out = h[1];
  if (h[0] & 2) return fail(SIPG_BREAKDOWN, "local projection CG: non-positive curvature (tau < 0?)");
  if (h[0] & 1) return fail(SIPG_MAXITER, "local projection CG: a cell did not converge within maxit");
  return SIPG_OK;
}

int sipg_cg_noalloc_capacity(long long* bytes) {
  if (!bytes) return fail(SIPG_EINVAL, "NULL output");
  *bytes = (long long)noalloc_scratch_bytes();
  return SIPG_OK;
}

int sipg_adjoint_grad_nu(const sipg_mesh* mc, const double* nu_cell, const double* u, const double* lam,
                         double* grad, void* stream) {
  int st;
  if ((st = check_separable(mc))) return st;
  if (!nu_cell || !u || !lam || !grad) return fail(SIPG_EINVAL, "NULL argument");
  Mesh& m = const_cast<sipg_mesh&>(*mc);
  if ((st = set_device(m))) return st;
  return launch_adjoint(m, nu_cell, u, lam, grad, (cudaStream_t)stream);
}

int sipg_set_f64_arithmetic(sipg_mesh* m, int mode) {
  int st;
  if ((st = check_mesh(m))) return st;
  if (mode != SIPG_F64_NATIVE && mode != SIPG_F64_DOUBLE_FLOAT) return fail(SIPG_EINVAL, "unknown FP64 arithmetic");
  m->f64_arith = mode;
  return SIPG_OK;
}

int sipg_get_f64_arithmetic(const sipg_mesh* m, int* mode) {
  int st;
  if ((st = check_mesh(m))) return st;
  if (!mode) return fail(SIPG_EINVAL, "NULL output");
  *mode = m->f64_arith;
  return SIPG_OK;
}

int sipg_get_cells_per_block(const sipg_mesh* m, int precision, int* cpb) {
  int st;
  if ((st = check_mesh(m))) return st;
  if (!cpb || precision < 0 || precision > 2) return fail(SIPG_EINVAL, "bad argument");
  *cpb = precision == 2 ? convective_cpb(*m, nullptr) : cells_per_block(*m, precision);
  return SIPG_OK;
}

int sipg_set_f32_mapping(sipg_mesh* m, int mapping) {
  int st;
  if ((st = check_mesh(m))) return st;
  if (mapping != SIPG_THREADS_LINE && mapping != SIPG_THREADS_PLANE) return fail(SIPG_EINVAL, "unknown mapping");
  m->f32_mapping = mapping;
  m->cpb[1] = 0;
  return SIPG_OK;
}

int sipg_set_cells_per_block(sipg_mesh* m, int precision, int cpb) {
  int st;
  if ((st = check_mesh(m))) return st;
  if (precision == 2) {
    int mx = 1;
    convective_cpb(*m, &mx);
    if (cpb < 1 || cpb > mx) return fail(SIPG_EINVAL, "cells per block out of range for this degree");
    m->cpb_conv = cpb;
    return SIPG_OK;
  }
  if (precision != 0 && precision != 1) return fail(SIPG_EINVAL, "precision must be 0, 1 or 2");
  const size_t elt = precision == 0 ? 8 : 4;
  if (cpb < 1 || (cpb * m->p * m->p + 31) / 32 * 32 > kMaxCellThreads || (size_t)3 * cpb * m->p * m->p * m->p * elt > 200 * 1024)
    return fail(SIPG_EINVAL, "cells per block out of range for this degree");
  m->cpb[precision] = cpb;
  return SIPG_OK;
}

// Autotuner cache: a JSON object of entries
//   "<key>": {"cpb": <cells per block>, "mapping": <FP32 thread mapping>}
// Only files of this shape are read (written by cache_store); anything else
// counts as an empty cache and is replaced on the next store.
static std::map<std::string, std::pair<int, int>> cache_read(const char* path) {
  std::map<std::string, std::pair<int, int>> out;
  std::ifstream f(path);
  if (!f) return out;
  std::stringstream ss;
  ss << f.rdbuf();
  const std::string s = ss.str();
  size_t pos = s.find('{');
  if (pos == std::string::npos) return out;
  ++pos;
  auto int_after = [&](size_t from, size_t to, const char* name, int* v) {
    const size_t k = s.find(name, from);
    if (k == std::string::npos || k > to) return false;
    const size_t c = s.find(':', k);
    if (c == std::string::npos || c > to) return false;
    *v = std::atoi(s.c_str() + c + 1);
    return true;
  };
  while (true) {
    const size_t q0 = s.find('"', pos);
    if (q0 == std::string::npos) break;
    const size_t q1 = s.find('"', q0 + 1);
    const size_t o0 = q1 == std::string::npos ? q1 : s.find('{', q1);
    const size_t o1 = o0 == std::string::npos ? o0 : s.find('}', o0);
    if (o1 == std::string::npos) break;
    int cpb = 0, mapping = 0;
    if (int_after(o0, o1, "\"cpb\"", &cpb) && cpb > 0) {
      int_after(o0, o1, "\"mapping\"", &mapping);
      out[s.substr(q0 + 1, q1 - q0 - 1)] = {cpb, mapping};
    }
    pos = o1 + 1;
  }
  return out;
}

static void cache_store(const char* path, const std::string& key, int cpb, int mapping) {
  auto entries = cache_read(path);
  entries[key] = {cpb, mapping};
  const std::string tmp = std::string(path) + ".tmp";
  {
    std::ofstream f(tmp, std::ios::trunc);
    if (!f) return;
    f << "{\n";
    size_t i = 0;
    for (const auto& kv : entries)
      f << "  \"" << kv.first << "\": {\"cpb\": " << kv.second.first << ", \"mapping\": " << kv.second.second
        << "}" << (++i < entries.size() ? "," : "") << "\n";
    f << "}\n";
  }
  std::rename(tmp.c_str(), path);  // whole-file replacement (no partial file is ever read)
}

// Cells per block of the convective kernel: every feasible count, timed on a
// zero velocity field (the kernel's work does not depend on the values).
static int autotune_convective(sipg_mesh* m, int* best_out) {
  int st;
  if ((st = set_device(*m))) return st;
  int mx = 1;
  convective_cpb(*m, &mx);
  const long long n = 3 * n_dofs(*m);
  double *x = nullptr, *y = nullptr;
  cudaError_t e = cudaMalloc(&x, n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&y, n * sizeof(double));
  if (e != cudaSuccess) {
    if (x) cudaFree(x);
    return fail(SIPG_ENOMEM, "autotune buffers");
  }
  cudaMemset(x, 0, n * sizeof(double));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int old = m->cpb_conv;
  int best = 0;
  float best_ms = 1e30f;
  for (int c = 1; c <= mx; ++c) {
    m->cpb_conv = c;
    float tot = 0.f;
    bool ok = true;
    for (int rep = 0; rep < 3 && ok; ++rep) {
      cudaEventRecord(e0, 0);
      for (int it = 0; it < 2; ++it)
        if (launch_convective(*m, x, y, 0)) ok = false;
      cudaEventRecord(e1, 0);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) tot += ms;  // first repetition is warm-up
    }
    if (ok && tot < best_ms) {
      best_ms = tot;
      best = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(x);
  cudaFree(y);
  cudaGetLastError();
  m->cpb_conv = best ? best : old;
  if (!best) return fail(SIPG_ECUDA, "autotune: no candidate ran");
  *best_out = best;
  return SIPG_OK;
}

int sipg_autotune(sipg_mesh* m, int precision, const char* cache_path) {
  int st;
  if ((st = check_separable(m))) return st;
  if (precision < 0 || precision > 2) return fail(SIPG_EINVAL, "precision must be 0, 1 or 2");
  char key[160];
  std::snprintf(key, sizeof(key), "k=%d prec=%d map=%d n=%dx%dx%d%s", m->k, precision, m->desc.map, m->desc.n[0],
                m->desc.n[1], m->desc.n[2],
                precision != 1 ? (m->f64_arith == SIPG_F64_DOUBLE_FLOAT ? " arith=df" : " arith=native") : "");
  if (cache_path) {
    const auto entries = cache_read(cache_path);
    const auto it = entries.find(key);
    if (it != entries.end()) {
      const int old_map = m->f32_mapping;
      if (precision == 1 && (it->second.second == SIPG_THREADS_LINE || it->second.second == SIPG_THREADS_PLANE))
        m->f32_mapping = it->second.second;
      if (sipg_set_cells_per_block(m, precision, it->second.first) == SIPG_OK) return SIPG_OK;
      m->f32_mapping = old_map;
    }
  }
  if (precision == 2) {
    int best = 0;
    if ((st = autotune_convective(m, &best))) return st;
    if (cache_path) cache_store(cache_path, key, best, 0);
    return SIPG_OK;
  }
  if ((st = set_device(*m))) return st;
  const size_t elt = precision == 0 ? 8 : 4;
  const long long n = n_dofs(*m);
  void *x = nullptr, *y = nullptr;
  cudaError_t e = cudaMalloc(&x, n * elt);
  if (e == cudaSuccess) e = cudaMalloc(&y, n * elt);
  if (e != cudaSuccess) {
    if (x) cudaFree(x);
    return fail(SIPG_ENOMEM, "autotune buffers");
  }
  cudaMemset(x, 0, n * elt);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int best = 0;
  float best_ms = 1e30f;
  const int old = m->cpb[precision];
  const int old_map = m->f32_mapping;
  int best_map = old_map;
  for (int cand = 0; cand < (precision == 1 ? 2 * 128 : 128); ++cand) {
    const int c = cand % 128 + 1;
    if (precision == 1) m->f32_mapping = cand < 128 ? 0 : 1;  // FP32: both thread mappings
    // every feasible count whose block wastes at most 1/8 of its lanes
    const int per_cell = (precision == 1 && m->f32_mapping == 1) ? m->p : m->p * m->p;
    const int thr = c * per_cell, rounded = (thr + 31) / 32 * 32;
    if (8 * (rounded - thr) > rounded) continue;
    if (sipg_set_cells_per_block(m, precision, c) != SIPG_OK) continue;
    float tot = 0.f;
    bool ok = true;
    for (int rep = 0; rep < 4 && ok; ++rep) {
      cudaEventRecord(e0, 0);
      for (int it = 0; it < 3; ++it) {
        int s2 = precision == 0 ? launch_apply<double>(*m, (double*)x, (double*)y, 1, 0.0, 1.0, nullptr, true, nullptr,
                                                       nullptr, 0)
                                : launch_apply<float>(*m, (float*)x, (float*)y, 1, 0.f, 1.f, nullptr, true, nullptr,
                                                      nullptr, 0);
        if (s2) ok = false;
      }
      cudaEventRecord(e1, 0);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) tot += ms;  // first repetition is warm-up
    }
    if (ok && tot < best_ms) {
      best_ms = tot;
      best = c;
      best_map = m->f32_mapping;
    }
  }
  m->f32_mapping = best_map;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(x);
  cudaFree(y);
  cudaGetLastError();
  if (best == 0) {
    m->cpb[precision] = old;
    m->f32_mapping = old_map;
    return fail(SIPG_ECUDA, "autotune: no candidate ran");
  }
  m->cpb[precision] = best;
  if (cache_path) cache_store(cache_path, key, best, precision == 1 ? m->f32_mapping : 0);
  return SIPG_OK;
}

int sipg_profile_enable(sipg_mesh* m, int on) {
  int st;
  if ((st = check_mesh(m))) return st;
  m->profile = on != 0;
  return SIPG_OK;
}

int sipg_profile_read(sipg_mesh* m, int reset, double* apply_ms, long long* applies, long long* launches) {
  int st;
  if ((st = check_mesh(m))) return st;
  for (auto& pr : m->pending) {
    float ms = 0.f;
    cudaEventSynchronize(pr.second);
    if (cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess) m->prof_ms += ms;
    cudaEventDestroy(pr.first);
    cudaEventDestroy(pr.second);
  }
  m->pending.clear();
  cudaGetLastError();
  if (apply_ms) *apply_ms = m->prof_ms;
  if (applies) *applies = m->prof_applies;
  if (launches) *launches = m->launches;
  if (reset) {
    m->prof_ms = 0.0;
    m->prof_applies = 0;
    m->launches = 0;
  }
  return SIPG_OK;
}

}  // extern "C"
