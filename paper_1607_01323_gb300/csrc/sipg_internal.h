// Internal declarations of libsipg (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "dfloat.cuh"
#include "sipg.h"

namespace sipg {

constexpr int PMIN = 2, PMAX = 8;  // p = k + 1, 1 <= k <= 7
constexpr int kMaxCellThreads = 256;  // block size limit of the cell kernels (register budget)

// One "layer" is one cell index along one direction.  Because the map is
// separable (x = X(xi), y = Y(eta), z = Z(zeta)), every cell integral and every
// face integral factorises into 1D matrices per direction and layer:
//   M  = S^T diag(w J) S        (1D mass, Gauss rule with p points)
//   K  = D^T diag(w / J) D      (1D stiffness)
//   Mi = M^-1                   (1D inverse mass)
//   dL = l'(0) / J(0), dR = l'(1) / J(1)   (normal derivative at the ends)
//   h  = extent of the layer,  t = (c_lo + c_hi) / h with c = 1/2 on an
//        interior or periodic face and 1 on a boundary face, so that
//        tau_e = f (k+1)^2 (t_x + t_y + t_z) is Eq. (taue) for the cell.
// For the uniform-viscosity kernel the own-face consistency terms of a layer are
// folded into one matrix and the averages' 1/2 into the derivative vectors:
//   Kc  = K - c_hi (e_R dR^T + dR e_R^T) + c_lo (e_L dL^T + dL e_L^T)
//         (c = 1/2 on an interior or periodic face, 1 on a Dirichlet face,
//         0 on a Neumann face),
//   dLh = dL / 2, dRh = dR / 2,
//   ts  = f (k+1)^2 t (this layer's share of tau_e),
//   dTL, dTR = max(0, ts of the low / high neighbour layer - ts), so that the
//   face penalty max(tau_e, tau_neighbour) of Eq. (tau) is tau_e + dT.
// The uniform-viscosity kernel evaluates the cell operator as
// (Mx x My x Mz) sum_d (M_d^-1 along d) w_d, so it also keeps the line operator
// premultiplied by the inverse mass:
//   Qc = Mi Kc,  mL = Mi e_0, mR = Mi e_(p-1),  qL = Mi dLh, qR = Mi dRh.
// Table layout per layer, stride lstride(p); every matrix block is padded to
// lmat(p) = p*p rounded up to a multiple of 4 entries and every vector block to
// lvec(p) = p rounded up to 4, so that each block starts 16-byte aligned (FP32
// kernels read the blocks with 128-bit loads):
//   [M][K][Mi][Kc] (lmat each) [dL][dR][dLh][dRh] (lvec each) [h][t][ts][dTL][dTR][cs][0][0]
//   [Qc] (lmat) [mL][mR][qL][qR] (lvec each) [EQc][EKc][EM] (lmat each)
// cs = 1 marks a centrosymmetric layer (M, Kc and Qc unchanged by reversing
// both indices: a uniform layer away from non-periodic boundaries); for p >= 5
// the E* blocks then hold the even-odd form of Qc, Kc and M (eo_pack), with
// which a contraction takes h (h + p mod 2) + h^2 + (p odd ? h + 1 : 0)
// multiply-adds plus 2p additions instead of p^2 (h = p / 2).
inline int lmat(int p) { return (p * p + 3) / 4 * 4; }
inline int lvec(int p) { return (p + 3) / 4 * 4; }
inline int lstride(int p) { return 8 * lmat(p) + 8 * lvec(p) + 8; }
inline int lay_M(int) { return 0; }
inline int lay_K(int p) { return lmat(p); }
inline int lay_Mi(int p) { return 2 * lmat(p); }
inline int lay_Kc(int p) { return 3 * lmat(p); }
inline int lay_dL(int p) { return 4 * lmat(p); }
inline int lay_dR(int p) { return 4 * lmat(p) + lvec(p); }
inline int lay_dLh(int p) { return 4 * lmat(p) + 2 * lvec(p); }
inline int lay_dRh(int p) { return 4 * lmat(p) + 3 * lvec(p); }
inline int lay_h(int p) { return 4 * lmat(p) + 4 * lvec(p); }
inline int lay_t(int p) { return 4 * lmat(p) + 4 * lvec(p) + 1; }
inline int lay_ts(int p) { return 4 * lmat(p) + 4 * lvec(p) + 2; }
inline int lay_dTL(int p) { return 4 * lmat(p) + 4 * lvec(p) + 3; }
inline int lay_dTR(int p) { return 4 * lmat(p) + 4 * lvec(p) + 4; }
inline int lay_Qc(int p) { return 4 * lmat(p) + 4 * lvec(p) + 8; }
inline int lay_mL(int p) { return 5 * lmat(p) + 4 * lvec(p) + 8; }
inline int lay_mR(int p) { return 5 * lmat(p) + 5 * lvec(p) + 8; }
inline int lay_qL(int p) { return 5 * lmat(p) + 6 * lvec(p) + 8; }
inline int lay_qR(int p) { return 5 * lmat(p) + 7 * lvec(p) + 8; }
inline int lay_cs(int p) { return 4 * lmat(p) + 4 * lvec(p) + 5; }
inline int lay_EQc(int p) { return 5 * lmat(p) + 8 * lvec(p) + 8; }
inline int lay_EKc(int p) { return 6 * lmat(p) + 8 * lvec(p) + 8; }
inline int lay_EM(int p) { return 7 * lmat(p) + 8 * lvec(p) + 8; }

// Geometry arguments shared by all cell kernels (passed by value).
template <typename T>
struct Geo {
  int n[3];
  int bc_lo[3], bc_hi[3];
  int ncell;
  const T* tab[3];  // per-direction layer tables on the device
  T tau_scale;      // penalty factor * (k+1)^2
  const int* dsc;   // scale exponent of the call (double-float kernels; see launch_df_scale)
  int lm[3];        // layer-index mask of the uniform operator: 0 where every layer of the
                    // direction has the same table (all cells read layer 0's copy), else -1
};

// Host-side state of one mesh.
struct Mesh {
  sipg_mesh_desc desc{};
  int k = 3, p = 4;
  double penalty = 1.0;
  int device = 0;
  long long ncell = 0;
  std::vector<double> htab[3];  // host layer tables (double)
  double* dtab64[3] = {nullptr, nullptr, nullptr};
  float* dtab32[3] = {nullptr, nullptr, nullptr};
  dfl* dtabdf[3] = {nullptr, nullptr, nullptr};  // double-float copies (hi, lo)
  // reference derivative-mass matrix C[a][b] = int_0^1 l_a'(s) l_b(s) ds (Gauss
  // k+1, exact); the same for every layer: the map's Jacobian cancels in
  // (d phi_a / dx, phi_b) on a separable map
  std::vector<double> hC;
  double* dC64 = nullptr;
  float* dC32 = nullptr;
  dfl* dCdf = nullptr;
  // over-integration tables of the convective term (Sec. 5: floor(3k/2)+1
  // Gauss points): [Sq: Q x P, l_a(z_q)] [Dq: P x Q, w_q l_a'(z_q)]
  // [WJ_x: nx x Q] [WJ_y: ny x Q] [WJ_z: nz x Q] with WJ = w_q J(z_q) per layer
  int nqc = 0;
  long long conv_off[5] = {0, 0, 0, 0, 0};
  std::vector<double> hconv;
  double* dconv64 = nullptr;
  dfl* dconvdf = nullptr;
  // wall tables of the dual-splitting step (stepper.cu): header S, D, d0, d1,
  // w (Gauss k+1), then per direction (from ns_off[d]) and layer: J at the
  // Gauss points, J at both ends, Dv = M^-1 C^T
  std::vector<double> hns;
  long long ns_off[3] = {0, 0, 0};
  double* dns64 = nullptr;
  // general-metric store of SIPG_MAP_PERTURBED (general.cu): per cell G and
  // det J w at the Gauss points, per face point w dA J^-1 n and w dA, tau_e
  std::vector<double> hgen_head, htau_gen;
  double* dgen_head = nullptr;
  double* dgen_geo = nullptr;
  double* dgen_face = nullptr;
  double* dgen_tau = nullptr;
  bool general() const { return desc.map == SIPG_MAP_PERTURBED; }
  bool eo_xz = false;  // every x- and z-layer centrosymmetric (even-odd contractions, p >= 5)
  int f64_arith = 0;  // FP64 operator arithmetic: 0 native FP64, 1 double-float
  int lay_same[3] = {0, 0, 0};  // every layer of the direction has a bitwise equal table
  int f32_mapping = 0;  // FP32 uniform operator: 0 one line per thread, 1 one plane per thread
  int cpb[2] = {0, 0};  // cells per block, [0] FP64, [1] FP32 (0 = default)
  int cpb_conv = 0;     // cells per block of the convective kernel (0 = default)
  // profiling
  bool profile = false;
  double prof_ms = 0.0;
  long long prof_applies = 0;
  long long launches = 0;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;  // unread event pairs
  // double-float scale word [key accumulator, block counter, scale exponent, -]
  // written by launch_df_scale before every double-float kernel of a call
  int* dscale = nullptr;
  // cached CG workspace
  void* ws = nullptr;
  size_t ws_bytes = 0;
  // cached multigrid hierarchy (mg.cu), dropped when degree or penalty change
  void* mg = nullptr;
  ~Mesh();
};

// ---------------------------------------------------------------- errors
void set_error(const std::string& msg);
int fail(int status, const std::string& msg);
int cuda_fail(cudaError_t e, const char* where);

// ---------------------------------------------------------------- tables
// 1D rules on [0, 1] (independent Newton iterations on Legendre polynomials).
void gll_rule(int p, std::vector<double>& z, std::vector<double>& w);
void gauss_rule(int n, std::vector<double>& z, std::vector<double>& w);
// Value and derivative of all Lagrange polynomials on nodes z at point x.
void lagrange_eval(const std::vector<double>& z, double x, std::vector<double>& val, std::vector<double>& der);
// Analytic separable map along direction d at global reference coordinate s in [0,1].
double map_coord(const sipg_mesh_desc& d, int dir, double s);
// Rebuild host layer tables and upload them.
int build_tables(Mesh& m);
// The full map at global reference coordinates s (general.cu).
void map_point(const sipg_mesh_desc& d, const double s[3], double x[3]);
// The general-metric store of SIPG_MAP_PERTURBED (general.cu).
int build_general(Mesh& m);
// y = cm M x + nu A x on a general map, ncomp components (general.cu); the
// kernel returns at once when *skip != 0.
int launch_general(const Mesh& m, const double* x, double* y, int ncomp, double cm, double nu, bool stiffness,
                   const int* skip, cudaStream_t s);
// diag(cm M + nu A) on a general map (general.cu).
int launch_general_diagonal(const Mesh& m, bool stiffness, double cm, double nu, double* diag, cudaStream_t s);

// ---------------------------------------------------------------- kernels
template <typename T>
Geo<T> make_geo(const Mesh& m);

// Where an operator kernel sends its dot products (x.y, sum y, sum x):
// per-block partials to partials[3 * block]; if counter is set, the last block
// to finish adds all partials in a fixed order into totals[0..2] and resets the
// counter (no waiting: each block only increments it once).  If skip is set
// and *skip != 0 the kernel returns at once (a finished solver's flag).
struct DotSink {
  double* partials = nullptr;
  unsigned* counter = nullptr;
  double* totals = nullptr;
  const int* skip = nullptr;
  int sums = 1;  // 0: only x.y is needed (sum y, sum x are left 0)
  int prescaled = 0;  // 1: the kernel that wrote x already left its double-float scale in the mesh's word
};

// Chebyshev-step epilogue of the FP32 Laplace operator (multigrid smoother):
// with t = A d for the block's own unknowns, r -= t, dnew = c1 d + c2 dinv r,
// x += dnew; t is not stored.  dnew must not alias d, which neighbouring blocks
// still read.
struct ChebEpi {
  float* r = nullptr;
  const float* dinv = nullptr;
  float* x = nullptr;
  float* dnew = nullptr;
  float c1 = 0.f, c2 = 0.f;
};
int launch_cheb_step(const Mesh& m, const float* d, const ChebEpi& epi, const int* skip, cudaStream_t s);

// Operator apply: y = mass_coef M x + nu (L x) [stiffness on/off]; nu_cell
// replaces nu when not null.  Dot products go to `sink` (may be null); the
// number of blocks is written to *nblocks.
template <typename T>
int launch_apply(const Mesh& m, const T* x, T* y, int ncomp, T mass_coef, T nu, const T* nu_cell, bool stiffness,
                 const DotSink* sink, int* nblocks, cudaStream_t s);
template <>
int launch_apply<double>(const Mesh& m, const double* x, double* y, int ncomp, double mass_coef, double nu,
                         const double* nu_cell, bool stiffness, const DotSink* sink, int* nblocks, cudaStream_t s);
template <>
int launch_apply<float>(const Mesh& m, const float* x, float* y, int ncomp, float mass_coef, float nu,
                        const float* nu_cell, bool stiffness, const DotSink* sink, int* nblocks, cudaStream_t s);

// Scale pass of a double-float call: the scale exponent s of the finite
// entries of v[0..n) and v2[0..n2) (v2 may be null) into m.dscale[2], so that
// the call's kernels evaluate v 2^-s and scale their results back exactly.
// Returns at once when skip is set and *skip != 0.  Calls on one mesh share
// the word, so double-float calls on one mesh must be stream-ordered.
int launch_df_scale(const Mesh& m, const double* v, long long n, const double* v2, long long n2, const int* skip,
                    cudaStream_t s);
// A scalar coefficient of a double-float call must be 0 or lie in
// [2^-100, 2^100] in magnitude (the FP32 exponent range with room to spare).
bool df_coef_ok(double v);

// prescaled: x's double-float scale is already in the mesh's word (set by the
// kernel that wrote x), so the scale pass is skipped
int launch_inverse_mass(const Mesh& m, const double* x, double* y, int ncomp, double* dots, bool prescaled,
                        cudaStream_t s);
int launch_diagonal(const Mesh& m, bool stiffness, double mass_coef, double nu, const double* nu_cell, double* diag,
                    cudaStream_t s);
int launch_adjoint(const Mesh& m, const double* nu_cell, const double* u, const double* lam, double* grad,
                   cudaStream_t s);

int cg_solve(Mesh& m, const sipg_cg_opts& o, const double* b, double* x, int ncomp, cudaStream_t s, int* iters,
             double* relres);

// Pressure-projection operators (projection.cu, FP64): divergence of Eq. (av3)
// (3 components in, 1 out), gradient of Eq. (bv3) (1 in, 3 out), tau_D of
// Eq. (tauD), the div-div operator of Eq. (div-div) and its batched per-cell
// CG solve with the inverse-mass preconditioner.
int launch_divergence(const Mesh& m, const double* u, double* y, cudaStream_t s);
int launch_gradient(const Mesh& m, const double* p, double* y, cudaStream_t s);
int launch_tau_div(const Mesh& m, const double* u, double zeta, double dt, double* tau, cudaStream_t s);
int launch_divdiv_apply(const Mesh& m, const double* tau, const double* u, double* y, cudaStream_t s);
int launch_divdiv_solve(const Mesh& m, const double* tau, const double* rhs, double* x, double rtol, int maxit,
                        int* status_dev, cudaStream_t s);
// y = convective term of Eq. (convstepspat) (LLF flux, over-integration;
// 3 components in and out; convective.cu)
int launch_convective(const Mesh& m, const double* u, double* y, cudaStream_t s);
// cells per block the convective kernel uses; *max_cpb = the largest that fits
int convective_cpb(const Mesh& m, int* max_cpb);
// y += scale * T u, the transposed-gradient part of the divergence-form
// viscous operator (3 components in and out; projection.cu); returns at once
// when skip is set and *skip != 0
int launch_viscous_t(const Mesh& m, const double* u, double* y, double scale, const int* skip, bool prescaled,
                     cudaStream_t s);

int cg_solve_noalloc(Mesh& m, const sipg_cg_opts& o, const double* b, double* x, int ncomp, cudaStream_t s,
                     int* iters, double* relres);
size_t noalloc_scratch_bytes();

// Extreme Ritz values of D^-1 A (A as selected by o.op, D = diag(A)) from
// `steps` Jacobi-PCG iterations on A y = b (Lanczos from the CG coefficients);
// stops early when ||r|| <= rtol ||b||.  Uses the mesh's CG workspace.
int lanczos_extremes(Mesh& m, const sipg_cg_opts& o, const double* b, int ncomp, int steps, double rtol,
                     cudaStream_t s, double* ritz_min, double* ritz_max);

// Geometric multigrid (mg.cu): set-up (cached on the mesh), one V-cycle
// z = V(r) (skip / mean / ap / part as for the CG preconditioner, may be null),
// hierarchy description and release.
int mg_setup(Mesh& m, const sipg_cg_opts& o, cudaStream_t s);
int mg_vcycle(Mesh& m, const double* r, double* z, const double* ap, const int* skip, const double* mean,
              double* part, cudaStream_t s);
int mg_info(const Mesh& m, int max_levels, int* nlevels, int* n_cells, double* lmax, double* coarse_lmin,
            int* coarse_degree);
void mg_release(Mesh& m);

// profiling helpers (api.cpp)
void prof_begin(Mesh& m, cudaStream_t s, cudaEvent_t* e0);
void prof_end(Mesh& m, cudaStream_t s, cudaEvent_t e0);

int default_cpb(int p, int precision);
int default_cpb_plane(int p);
int cells_per_block(const Mesh& m, int precision);  // current setting or default for the mapping

}  // namespace sipg

// The opaque handle of the C ABI is the mesh itself.
struct sipg_mesh : public sipg::Mesh {};

