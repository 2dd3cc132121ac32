// 1D bases, quadrature and the per-layer geometry tables of the separable
// iso-parametric mapping (host code).
//
// Sec. 3.1: nodal Lagrange polynomials on the Legendre-Gauss-Lobatto points.
// Sec. 5:   Gauss quadrature with n_q = k+1 points per direction; the mapping
//           is the degree-k interpolant of the analytic map (iso-parametric);
//           the inverse mass matrix is the tensor product of inverted 1D
//           node-to-quadrature transforms (square because n_q = k+1).
// Sec. 3.2, Eq. (taue): tau_e = (k+1)^2 (A(dOmega_e^Gamma)/2 + A(dOmega_e^bdy)) / V(Omega_e).
// Sec. 7.1: the tanh grading of the wall-normal coordinate.
#include <cmath>
#include <cstring>

#include "sipg_internal.h"

namespace sipg {

namespace {

// P_n(t) and P_n'(t) by the three-term recurrence (long double).
void legendre(int n, long double t, long double& P, long double& dP, long double& d2P) {
  long double p0 = 1.0L, p1 = t;
  if (n == 0) {
    P = 1.0L;
    dP = 0.0L;
    d2P = 0.0L;
    return;
  }
  for (int j = 2; j <= n; ++j) {
    long double p2 = ((2.0L * j - 1.0L) * t * p1 - (j - 1.0L) * p0) / j;
    p0 = p1;
    p1 = p2;
  }
  P = p1;
  // derivatives from the Legendre ODE / the identity (1-t^2) P' = n (P_{n-1} - t P_n)
  long double one_m = 1.0L - t * t;
  dP = n * (p0 - t * p1) / one_m;
  d2P = (2.0L * t * dP - n * (n + 1.0L) * P) / one_m;
}

}  // namespace

void gauss_rule(int n, std::vector<double>& z, std::vector<double>& w) {
  z.assign(n, 0.0);
  w.assign(n, 0.0);
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int i = 0; i < n; ++i) {
    // Newton on P_n from the Chebyshev-like initial guess, roots in increasing order
    long double t = -std::cos(pi * (i + 0.75L) / (n + 0.5L));
    long double P, dP, d2P;
    for (int it = 0; it < 100; ++it) {
      legendre(n, t, P, dP, d2P);
      long double dt = P / dP;
      t -= dt;
      if (std::fabs(dt) < 1e-19L) break;
    }
    legendre(n, t, P, dP, d2P);
    z[i] = (double)(0.5L * (t + 1.0L));
    w[i] = (double)(1.0L / ((1.0L - t * t) * dP * dP));  // 2/((1-t^2)P'^2) halved
  }
}

void gll_rule(int p, std::vector<double>& z, std::vector<double>& w) {
  int k = p - 1;
  z.assign(p, 0.0);
  w.assign(p, 0.0);
  const long double pi = 3.141592653589793238462643383279502884L;
  std::vector<long double> t(p);
  t[0] = -1.0L;
  t[k] = 1.0L;
  for (int i = 1; i < k; ++i) {
    // Newton on P_k' (interior GLL nodes), started at the Chebyshev-Lobatto point
    long double x = -std::cos(pi * i / k);
    long double P, dP, d2P;
    for (int it = 0; it < 100; ++it) {
      legendre(k, x, P, dP, d2P);
      long double dx = dP / d2P;
      x -= dx;
      if (std::fabs(dx) < 1e-19L) break;
    }
    t[i] = x;
  }
  for (int i = 0; i < p; ++i) {
    long double P = 1, dP, d2P;
    if (i == 0 || i == k) {
      P = (i == 0 && (k % 2 == 1)) ? -1.0L : 1.0L;  // P_k(+-1) = (+-1)^k
    } else {
      legendre(k, t[i], P, dP, d2P);
    }
    z[i] = (double)(0.5L * (t[i] + 1.0L));
    w[i] = (double)(1.0L / (k * (k + 1.0L) * P * P));
  }
}

void lagrange_eval(const std::vector<double>& z, double x, std::vector<double>& val, std::vector<double>& der) {
  // barycentric form: l_a(x) = (lambda_a / (x - z_a)) / sum_b lambda_b / (x - z_b)
  const int p = (int)z.size();
  val.assign(p, 0.0);
  der.assign(p, 0.0);
  std::vector<long double> lam(p, 1.0L);
  for (int a = 0; a < p; ++a)
    for (int b = 0; b < p; ++b)
      if (b != a) lam[a] /= ((long double)z[a] - (long double)z[b]);
  int hit = -1;
  for (int a = 0; a < p; ++a)
    if (std::fabs((long double)x - z[a]) < 1e-15L) hit = a;
  if (hit >= 0) {
    // x is node `hit`: values are a unit vector, derivatives the row of the
    // differentiation matrix D_ij = (lambda_j / lambda_i) / (z_i - z_j), D_ii = -sum.
    val[hit] = 1.0;
    long double diag = 0.0L;
    for (int b = 0; b < p; ++b) {
      if (b == hit) continue;
      long double d = (lam[b] / lam[hit]) / ((long double)z[hit] - (long double)z[b]);
      der[b] = (double)d;
      diag -= d;
    }
    der[hit] = (double)diag;
    return;
  }
  long double s = 0.0L;
  std::vector<long double> q(p);
  for (int a = 0; a < p; ++a) {
    q[a] = lam[a] / ((long double)x - z[a]);
    s += q[a];
  }
  for (int a = 0; a < p; ++a) {
    long double la = q[a] / s;
    // l_a'(x) = l_a(x) * sum_{m != a} 1 / (x - z_m)
    long double sd = 0.0L;
    for (int m = 0; m < p; ++m)
      if (m != a) sd += 1.0L / ((long double)x - z[m]);
    val[a] = (double)la;
    der[a] = (double)(la * sd);
  }
}

double map_coord(const sipg_mesh_desc& d, int dir, double s) {
  const double lo = d.lo[dir], hi = d.hi[dir];
  if (d.map == SIPG_MAP_CHANNEL_TANH && dir == 1) {
    double t = std::tanh(d.gamma * (2.0 * s - 1.0)) / std::tanh(d.gamma);
    return lo + (hi - lo) * 0.5 * (1.0 + t);
  }
  if (d.map == SIPG_MAP_CHANNEL_LINEAR && dir == 1) {
    // graded vertices eta_j = j / n, straight in between
    const int n = d.n[1];
    int j = (int)std::floor(s * n);
    j = j < 0 ? 0 : (j > n - 1 ? n - 1 : j);
    const double e0 = (double)j / n, e1 = (double)(j + 1) / n;
    const double y0 = std::tanh(d.gamma * (2.0 * e0 - 1.0)) / std::tanh(d.gamma);
    const double y1 = std::tanh(d.gamma * (2.0 * e1 - 1.0)) / std::tanh(d.gamma);
    const double t = y0 + (y1 - y0) * (s - e0) * n;
    return lo + (hi - lo) * 0.5 * (1.0 + t);
  }
  return lo + (hi - lo) * s;
}

namespace {

// Gauss-Jordan inverse of a small SPD matrix (long double).
bool invert(int p, const std::vector<long double>& A, std::vector<long double>& Ainv) {
  std::vector<long double> a(A);
  Ainv.assign(p * p, 0.0L);
  for (int i = 0; i < p; ++i) Ainv[i * p + i] = 1.0L;
  for (int c = 0; c < p; ++c) {
    int piv = c;
    for (int r = c + 1; r < p; ++r)
      if (std::fabs(a[r * p + c]) > std::fabs(a[piv * p + c])) piv = r;
    if (a[piv * p + c] == 0.0L) return false;
    if (piv != c)
      for (int j = 0; j < p; ++j) {
        std::swap(a[c * p + j], a[piv * p + j]);
        std::swap(Ainv[c * p + j], Ainv[piv * p + j]);
      }
    long double inv = 1.0L / a[c * p + c];
    for (int j = 0; j < p; ++j) {
      a[c * p + j] *= inv;
      Ainv[c * p + j] *= inv;
    }
    for (int r = 0; r < p; ++r) {
      if (r == c) continue;
      long double f = a[r * p + c];
      if (f == 0.0L) continue;
      for (int j = 0; j < p; ++j) {
        a[r * p + j] -= f * a[c * p + j];
        Ainv[r * p + j] -= f * Ainv[c * p + j];
      }
    }
  }
  return true;
}

}  // namespace

// A[a][b] = A[p-1-a][p-1-b] up to the rounding of the table computation
// (about 1e-15 of the largest entry for a uniform layer, whose nodes are
// taken relative to its start; graded layers are far from symmetric): the
// test allows 1e-12, and eo_pack symmetrises.
static bool centrosymmetric(int p, const double* A) {
  double mx = 0.0, d = 0.0;
  for (int i = 0; i < p * p; ++i) mx = std::fmax(mx, std::fabs(A[i]));
  for (int a = 0; a < p; ++a)
    for (int b = 0; b < p; ++b) d = std::fmax(d, std::fabs(A[a * p + b] - A[(p - 1 - a) * p + (p - 1 - b)]));
  return d <= 1e-12 * mx;
}

// Even-odd form of a centrosymmetric p x p matrix A (Solomonoff's splitting):
// with h = p / 2, e_b = v_b + v_(p-1-b), o_b = v_b - v_(p-1-b) (b < h) and,
// for odd p, the middle value v_h, the product y = A v is
//   s_a = sum_b E[a][b] e_b (+ E[a][h] v_h),  d_a = sum_b O[a][b] o_b,
//   y_a = s_a + d_a,  y_(p-1-a) = s_a - d_a  (a < h),
//   y_h = sum_b Z[b] e_b + Z[h] v_h  (odd p),
// E[a][b] = (A[a][b] + A[a][p-1-b]) / 2, E[a][h] = A[a][h], O[a][b] =
// (A[a][b] - A[a][p-1-b]) / 2, Z = the middle row.  Packed as E (h x (h + odd)),
// O (h x h), Z (h + 1 for odd p), from the symmetrised A.
static void eo_pack(int p, const double* A, double* out) {
  const int h = p / 2, odd = p & 1;
  auto S = [&](int a, int b) { return 0.5L * ((long double)A[a * p + b] + A[(p - 1 - a) * p + (p - 1 - b)]); };
  int k = 0;
  for (int a = 0; a < h; ++a) {
    for (int b = 0; b < h; ++b) out[k++] = (double)(0.5L * (S(a, b) + S(a, p - 1 - b)));
    if (odd) out[k++] = (double)S(a, h);
  }
  for (int a = 0; a < h; ++a)
    for (int b = 0; b < h; ++b) out[k++] = (double)(0.5L * (S(a, b) - S(a, p - 1 - b)));
  if (odd) {
    for (int b = 0; b < h; ++b) out[k++] = (double)S(h, b);
    out[k++] = (double)S(h, h);
  }
}

int build_tables(Mesh& m) {
  const int p = m.p;
  std::vector<double> zn, wn, zq, wq;
  gll_rule(p, zn, wn);
  gauss_rule(p, zq, wq);
  // S[q][a] = l_a(x_q), D[q][a] = l_a'(x_q); end derivatives d0, d1
  std::vector<double> S(p * p), D(p * p), d0, d1, v;
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
  // C[a][b] = sum_q w_q l_a'(z_q) l_b(z_q)
  m.hC.assign((size_t)p * p, 0.0);
  for (int a = 0; a < p; ++a)
    for (int b = 0; b < p; ++b) {
      long double sc = 0.0L;
      for (int q = 0; q < p; ++q) sc += (long double)wq[q] * D[q * p + a] * S[q * p + b];
      m.hC[a * p + b] = (double)sc;
    }
  const int st = lstride(p);
  for (int dir = 0; dir < 3; ++dir) {
    const int n = m.desc.n[dir];
    std::vector<double>& tab = m.htab[dir];
    tab.assign((size_t)n * st, 0.0);
    for (int i = 0; i < n; ++i) {
      double* L = &tab[(size_t)i * st];
      std::vector<long double> X(p);
      // every entry depends on the layer's own geometry only: affine directions
      // take the nodes relative to the layer's start (exact, the same for every
      // uniform layer), the graded direction the map's global values
      const bool affine_dir =
          !(dir == 1 && (m.desc.map == SIPG_MAP_CHANNEL_TANH || m.desc.map == SIPG_MAP_CHANNEL_LINEAR));
      for (int a = 0; a < p; ++a)
        X[a] = affine_dir ? (long double)(m.desc.hi[dir] - m.desc.lo[dir]) * zn[a] / n
                          : (long double)map_coord(m.desc, dir, (i + zn[a]) / n);
      // derivative of the degree-k interpolant of the map at the Gauss points and ends
      std::vector<long double> J(p, 0.0L);
      long double J0 = 0.0L, J1 = 0.0L;
      for (int q = 0; q < p; ++q)
        for (int a = 0; a < p; ++a) J[q] += X[a] * D[q * p + a];
      for (int a = 0; a < p; ++a) {
        J0 += X[a] * d0[a];
        J1 += X[a] * d1[a];
      }
      for (int q = 0; q < p; ++q)
        if (!(J[q] > 0.0L)) return fail(SIPG_EINVAL, "mapping is not monotone: degenerate cell");
      std::vector<long double> Mm(p * p, 0.0L), Mi;
      for (int a = 0; a < p; ++a)
        for (int b = 0; b < p; ++b) {
          long double sm = 0.0L, sk = 0.0L;
          for (int q = 0; q < p; ++q) {
            sm += (long double)wq[q] * J[q] * S[q * p + a] * S[q * p + b];
            sk += (long double)wq[q] / J[q] * D[q * p + a] * D[q * p + b];
          }
          Mm[a * p + b] = sm;
          L[lay_M(p) + a * p + b] = (double)sm;
          L[lay_K(p) + a * p + b] = (double)sk;
        }
      if (!invert(p, Mm, Mi)) return fail(SIPG_EINVAL, "singular 1D mass matrix");
      for (int j = 0; j < p * p; ++j) L[lay_Mi(p) + j] = (double)Mi[j];
      for (int a = 0; a < p; ++a) {
        L[lay_dL(p) + a] = (double)(d0[a] / J0);
        L[lay_dR(p) + a] = (double)(d1[a] / J1);
      }
      double h = (double)(X[p - 1] - X[0]);
      bool per = m.desc.bc_lo[dir] == SIPG_BC_PERIODIC;
      double clo = (i == 0 && !per) ? 1.0 : 0.5;
      double chi = (i == n - 1 && !per) ? 1.0 : 0.5;
      L[lay_h(p)] = h;
      L[lay_t(p)] = (clo + chi) / h;
      // own-face consistency weights of the precombined matrix Kc
      const double wlo = (i == 0 && !per) ? (m.desc.bc_lo[dir] == SIPG_BC_DIRICHLET ? 1.0 : 0.0) : 0.5;
      const double whi = (i == n - 1 && !per) ? (m.desc.bc_hi[dir] == SIPG_BC_DIRICHLET ? 1.0 : 0.0) : 0.5;
      const double* dL = L + lay_dL(p);
      const double* dR = L + lay_dR(p);
      for (int a = 0; a < p; ++a)
        for (int b = 0; b < p; ++b) {
          double v = L[lay_K(p) + a * p + b];
          v -= whi * ((a == p - 1 ? dR[b] : 0.0) + (b == p - 1 ? dR[a] : 0.0));
          v += wlo * ((a == 0 ? dL[b] : 0.0) + (b == 0 ? dL[a] : 0.0));
          L[lay_Kc(p) + a * p + b] = v;
        }
      for (int a = 0; a < p; ++a) {
        L[lay_dLh(p) + a] = 0.5 * dL[a];
        L[lay_dRh(p) + a] = 0.5 * dR[a];
      }
      // the line operator premultiplied by the inverse mass (extended precision)
      for (int a = 0; a < p; ++a) {
        long double q = 0.0L, ql = 0.0L, qr = 0.0L;
        for (int b = 0; b < p; ++b) {
          ql += Mi[a * p + b] * (long double)L[lay_dLh(p) + b];
          qr += Mi[a * p + b] * (long double)L[lay_dRh(p) + b];
        }
        for (int c = 0; c < p; ++c) {
          q = 0.0L;
          for (int b = 0; b < p; ++b) q += Mi[a * p + b] * (long double)L[lay_Kc(p) + b * p + c];
          L[lay_Qc(p) + a * p + c] = (double)q;
        }
        L[lay_mL(p) + a] = (double)Mi[a * p];
        L[lay_mR(p) + a] = (double)Mi[a * p + p - 1];
        L[lay_qL(p) + a] = (double)ql;
        L[lay_qR(p) + a] = (double)qr;
      }
      // centrosymmetric layers: the even-odd forms of Qc, Kc and M
      const bool cs = p >= 5 && centrosymmetric(p, L + lay_M(p)) && centrosymmetric(p, L + lay_Kc(p)) &&
                      centrosymmetric(p, L + lay_Qc(p));
      L[lay_cs(p)] = cs ? 1.0 : 0.0;
      if (cs) {
        eo_pack(p, L + lay_Qc(p), L + lay_EQc(p));
        eo_pack(p, L + lay_Kc(p), L + lay_EKc(p));
        eo_pack(p, L + lay_M(p), L + lay_EM(p));
      }
    }
    // penalty shares and face increments (Eq. (taue), Eq. (tau))
    const double s = m.penalty * (m.k + 1) * (m.k + 1);
    const bool per = m.desc.bc_lo[dir] == SIPG_BC_PERIODIC;
    for (int i = 0; i < n; ++i) tab[(size_t)i * st + lay_ts(p)] = s * tab[(size_t)i * st + lay_t(p)];
    for (int i = 0; i < n; ++i) {
      const double ts = tab[(size_t)i * st + lay_ts(p)];
      const int jl = i > 0 ? i - 1 : (per ? n - 1 : -1);
      const int jr = i < n - 1 ? i + 1 : (per ? 0 : -1);
      const double tl = jl >= 0 ? tab[(size_t)jl * st + lay_ts(p)] : ts;
      const double tr = jr >= 0 ? tab[(size_t)jr * st + lay_ts(p)] : ts;
      tab[(size_t)i * st + lay_dTL(p)] = tl > ts ? tl - ts : 0.0;
      tab[(size_t)i * st + lay_dTR(p)] = tr > ts ? tr - ts : 0.0;
    }
  }
  // directions whose layers all have the same table (equal widths of an
  // affine direction: the tables depend on the local nodes only)
  for (int dir = 0; dir < 3; ++dir) {
    m.lay_same[dir] = 1;
    for (int i = 1; i < m.desc.n[dir] && m.lay_same[dir]; ++i)
      if (std::memcmp(&m.htab[dir][(size_t)i * st], &m.htab[dir][0], st * sizeof(double)) != 0) m.lay_same[dir] = 0;
  }
  // even-odd contractions along x and z when all their layers allow it
  m.eo_xz = p >= 5;
  for (int dir : {0, 2})
    for (int i = 0; i < m.desc.n[dir]; ++i)
      if (m.htab[dir][(size_t)i * st + lay_cs(p)] == 0.0) m.eo_xz = false;
  // over-integration tables of the convective term
  {
    const int Q = (3 * m.k) / 2 + 1;
    m.nqc = Q;
    std::vector<double> zo, wo;
    gauss_rule(Q, zo, wo);
    std::vector<double> So(Q * p), Dqo(p * Q);
    for (int q = 0; q < Q; ++q) {
      std::vector<double> val, der;
      lagrange_eval(zn, zo[q], val, der);
      for (int a = 0; a < p; ++a) {
        So[q * p + a] = val[a];
        Dqo[a * Q + q] = wo[q] * der[a];
      }
    }
    m.hconv.clear();
    m.conv_off[0] = 0;
    m.hconv.insert(m.hconv.end(), So.begin(), So.end());
    m.conv_off[1] = (long long)m.hconv.size();
    m.hconv.insert(m.hconv.end(), Dqo.begin(), Dqo.end());
    for (int dir = 0; dir < 3; ++dir) {
      m.conv_off[2 + dir] = (long long)m.hconv.size();
      const int n = m.desc.n[dir];
      for (int i = 0; i < n; ++i) {
        std::vector<long double> X(p);
        for (int a = 0; a < p; ++a) X[a] = map_coord(m.desc, dir, (i + zn[a]) / n);
        for (int q = 0; q < Q; ++q) {
          std::vector<double> val, der;
          lagrange_eval(zn, zo[q], val, der);
          long double J = 0.0L;
          for (int a = 0; a < p; ++a) J += X[a] * der[a];
          m.hconv.push_back((double)(wo[q] * J));
        }
      }
    }
  }
  // wall tables of the dual-splitting step: S, D (Gauss k+1), the end
  // derivatives d0, d1 and the Gauss weights; per direction and layer the map
  // derivative J at the Gauss points and both ends, and Dv = M^-1 C^T, the
  // cell-wise L2 projection of a derivative along that direction (the other
  // two directions' mass matrices cancel against the inverse mass).
  {
    m.hns.clear();
    m.hns.insert(m.hns.end(), S.begin(), S.end());
    m.hns.insert(m.hns.end(), D.begin(), D.end());
    m.hns.insert(m.hns.end(), d0.begin(), d0.end());
    m.hns.insert(m.hns.end(), d1.begin(), d1.end());
    m.hns.insert(m.hns.end(), wq.begin(), wq.end());
    for (int dir = 0; dir < 3; ++dir) {
      m.ns_off[dir] = (long long)m.hns.size();
      const int n = m.desc.n[dir];
      for (int i = 0; i < n; ++i) {
        std::vector<long double> X(p);
        for (int a = 0; a < p; ++a) X[a] = map_coord(m.desc, dir, (i + zn[a]) / n);
        long double J0 = 0.0L, J1 = 0.0L;
        for (int q = 0; q < p; ++q) {
          long double J = 0.0L;
          for (int a = 0; a < p; ++a) J += X[a] * D[q * p + a];
          m.hns.push_back((double)J);
        }
        for (int a = 0; a < p; ++a) {
          J0 += X[a] * d0[a];
          J1 += X[a] * d1[a];
        }
        m.hns.push_back((double)J0);
        m.hns.push_back((double)J1);
        const double* Mi = &m.htab[dir][(size_t)i * lstride(p) + lay_Mi(p)];
        for (int a = 0; a < p; ++a)
          for (int b = 0; b < p; ++b) {
            long double v = 0.0L;
            for (int c = 0; c < p; ++c) v += (long double)Mi[a * p + c] * m.hC[b * p + c];
            m.hns.push_back((double)v);
          }
      }
    }
  }
  // upload (double, float and double-float copies)
  {
    if (m.dC64) cudaFree(m.dC64);
    if (m.dC32) cudaFree(m.dC32);
    if (m.dCdf) cudaFree(m.dCdf);
    m.dC64 = nullptr;
    m.dC32 = nullptr;
    m.dCdf = nullptr;
    std::vector<dfl> cd(m.hC.size());
    for (size_t j = 0; j < cd.size(); ++j) cd[j] = dfl(m.hC[j]);
    std::vector<float> cf(m.hC.begin(), m.hC.end());
    cudaError_t e = cudaMalloc(&m.dC64, m.hC.size() * sizeof(double));
    if (e != cudaSuccess) return fail(SIPG_ENOMEM, "cudaMalloc of the derivative-mass table failed");
    e = cudaMalloc(&m.dC32, cf.size() * sizeof(float));
    if (e != cudaSuccess) return fail(SIPG_ENOMEM, "cudaMalloc of the derivative-mass table failed");
    e = cudaMemcpy(m.dC64, m.hC.data(), m.hC.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m.dC32, cf.data(), cf.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&m.dCdf, cd.size() * sizeof(dfl));
    if (e == cudaSuccess) e = cudaMemcpy(m.dCdf, cd.data(), cd.size() * sizeof(dfl), cudaMemcpyHostToDevice);
    if (m.dconv64) cudaFree(m.dconv64);
    if (m.dconvdf) cudaFree(m.dconvdf);
    m.dconv64 = nullptr;
    m.dconvdf = nullptr;
    std::vector<dfl> cvd(m.hconv.size());
    for (size_t j = 0; j < cvd.size(); ++j) cvd[j] = dfl(m.hconv[j]);
    if (e == cudaSuccess) e = cudaMalloc(&m.dconv64, m.hconv.size() * sizeof(double));
    if (e == cudaSuccess)
      e = cudaMemcpy(m.dconv64, m.hconv.data(), m.hconv.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&m.dconvdf, cvd.size() * sizeof(dfl));
    if (e == cudaSuccess) e = cudaMemcpy(m.dconvdf, cvd.data(), cvd.size() * sizeof(dfl), cudaMemcpyHostToDevice);
    if (m.dns64) cudaFree(m.dns64);
    m.dns64 = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&m.dns64, m.hns.size() * sizeof(double));
    if (e == cudaSuccess)
      e = cudaMemcpy(m.dns64, m.hns.data(), m.hns.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "upload derivative-mass table");
  }
  for (int dir = 0; dir < 3; ++dir) {
    if (m.dtab64[dir]) cudaFree(m.dtab64[dir]);
    if (m.dtab32[dir]) cudaFree(m.dtab32[dir]);
    if (m.dtabdf[dir]) cudaFree(m.dtabdf[dir]);
    m.dtab64[dir] = nullptr;
    m.dtab32[dir] = nullptr;
    m.dtabdf[dir] = nullptr;
    size_t cnt = m.htab[dir].size();
    cudaError_t e = cudaMalloc(&m.dtab64[dir], cnt * sizeof(double));
    if (e != cudaSuccess) return fail(SIPG_ENOMEM, "cudaMalloc of geometry tables failed");
    e = cudaMalloc(&m.dtab32[dir], cnt * sizeof(float));
    if (e != cudaSuccess) return fail(SIPG_ENOMEM, "cudaMalloc of geometry tables failed");
    std::vector<float> f(cnt);
    for (size_t j = 0; j < cnt; ++j) f[j] = (float)m.htab[dir][j];
    e = cudaMemcpy(m.dtab64[dir], m.htab[dir].data(), cnt * sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "upload geometry tables");
    e = cudaMemcpy(m.dtab32[dir], f.data(), cnt * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "upload geometry tables");
    std::vector<dfl> dd(cnt);
    for (size_t j = 0; j < cnt; ++j) dd[j] = dfl(m.htab[dir][j]);
    e = cudaMalloc(&m.dtabdf[dir], cnt * sizeof(dfl));
    if (e != cudaSuccess) return fail(SIPG_ENOMEM, "cudaMalloc of geometry tables failed");
    e = cudaMemcpy(m.dtabdf[dir], dd.data(), cnt * sizeof(dfl), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "upload geometry tables");
  }
  return m.general() ? build_general(m) : SIPG_OK;
}

}  // namespace sipg
