// Reference-element matrices by quadrature (see tables.h).
#include "tables.h"

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <stdexcept>

namespace yt {
namespace {

// Forward-mode dual number with three partial derivatives.
struct Dual {
  double v;
  double d[3];
};
inline Dual dconst(double c) { return Dual{c, {0.0, 0.0, 0.0}}; }
inline Dual operator+(Dual a, Dual b) { return Dual{a.v + b.v, {a.d[0] + b.d[0], a.d[1] + b.d[1], a.d[2] + b.d[2]}}; }
inline Dual operator-(Dual a, Dual b) { return Dual{a.v - b.v, {a.d[0] - b.d[0], a.d[1] - b.d[1], a.d[2] - b.d[2]}}; }
inline Dual operator*(Dual a, Dual b) {
  return Dual{a.v * b.v, {a.d[0] * b.v + a.v * b.d[0], a.d[1] * b.v + a.v * b.d[1], a.d[2] * b.v + a.v * b.d[2]}};
}
inline Dual operator*(double s, Dual a) { return Dual{s * a.v, {s * a.d[0], s * a.d[1], s * a.d[2]}}; }
inline Dual operator/(Dual a, Dual b) {
  double inv = 1.0 / b.v;
  double q = a.v * inv;
  return Dual{q, {(a.d[0] - q * b.d[0]) * inv, (a.d[1] - q * b.d[1]) * inv, (a.d[2] - q * b.d[2]) * inv}};
}

inline double dconst_like(double, double c) { return c; }
inline Dual dconst_like(const Dual&, double c) { return dconst(c); }
inline Dual operator+(Dual a, double c) { a.v += c; return a; }
inline Dual operator*(Dual a, double s) { return s * a; }

// Jacobi polynomial P_n^{(alpha,0)}(x) by the three-term recurrence
// 2n(n+a)(2n+a-2) P_n = (2n+a-1)[(2n+a)(2n+a-2) x + a^2] P_{n-1} - 2(n+a-1)(n-1)(2n+a) P_{n-2}.
template <typename T>
T jacobi(int n, int alpha, T x) {
  T p0 = dconst_like(x, 1.0);
  if (n == 0) return p0;
  const double a = alpha;
  T p1 = 0.5 * ((a + 2.0) * x + dconst_like(x, a));
  for (int k = 2; k <= n; ++k) {
    const double kk = k;
    const double c0 = 2.0 * kk * (kk + a) * (2.0 * kk + a - 2.0);
    const double c1 = (2.0 * kk + a - 1.0) * (2.0 * kk + a) * (2.0 * kk + a - 2.0);
    const double c2 = (2.0 * kk + a - 1.0) * a * a;
    const double c3 = 2.0 * (kk + a - 1.0) * (kk - 1.0) * (2.0 * kk + a);
    T p2 = (1.0 / c0) * (c1 * (x * p1) + c2 * p1 - c3 * p0);
    p0 = p1;
    p1 = p2;
  }
  return p1;
}

template <typename T>
T ipow(T x, int n) {
  T r = dconst_like(x, 1.0);
  for (int i = 0; i < n; ++i) r = r * x;
  return r;
}

struct Idx3 { int p, q, r; };
std::vector<Idx3> tet_indices(int N) {
  std::vector<Idx3> out;
  for (int d = 0; d <= N; ++d)
    for (int p = 0; p <= d; ++p)
      for (int q = 0; q <= d - p; ++q) out.push_back({p, q, d - p - q});
  return out;
}
std::vector<std::pair<int, int>> tri_indices(int N) {
  std::vector<std::pair<int, int>> out;
  for (int d = 0; d <= N; ++d)
    for (int p = 0; p <= d; ++p) out.push_back({p, d - p});
  return out;
}

// Dubiner function phi_pqr at (xi, eta, zeta) (as duals: value and gradient).
Dual phi_dual(const Idx3& t, Dual xi, Dual eta, Dual zeta) {
  Dual s1 = dconst(1.0) - eta - zeta;
  Dual s2 = dconst(1.0) - zeta;
  Dual u = (2.0 * xi) / s1 - dconst(1.0);
  Dual v = (2.0 * eta) / s2 - dconst(1.0);
  Dual w = 2.0 * zeta - dconst(1.0);
  return jacobi(t.p, 0, u) * ipow(s1, t.p) * jacobi(t.q, 2 * t.p + 1, v) * ipow(s2, t.q) *
         jacobi(t.r, 2 * t.p + 2 * t.q + 2, w);
}
double phi(const Idx3& t, double xi, double eta, double zeta) {
  double s1 = 1.0 - eta - zeta, s2 = 1.0 - zeta;
  return jacobi(t.p, 0, 2.0 * xi / s1 - 1.0) * ipow(s1, t.p) *
         jacobi(t.q, 2 * t.p + 1, 2.0 * eta / s2 - 1.0) * ipow(s2, t.q) *
         jacobi(t.r, 2 * t.p + 2 * t.q + 2, 2.0 * zeta - 1.0);
}
double psi(const std::pair<int, int>& t, double c1, double c2) {
  double s = 1.0 - c2;
  return jacobi(t.first, 0, 2.0 * c1 / s - 1.0) * ipow(s, t.first) *
         jacobi(t.second, 2 * t.first + 1, 2.0 * c2 - 1.0);
}

// Gauss-Legendre rule on [0,1] by Newton iteration on P_n.
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    double z = std::cos(pi * (i + 0.75) / (n + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      double pn = n == 1 ? z : p1;
      double pm = n == 1 ? 1.0 : p0;
      dp = n * (z * pn - pm) / (z * z - 1.0);
      double dz = pn / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = 0.5 * (1.0 - z);
    w[i] = 1.0 / ((1.0 - z * z) * dp * dp);  // 2/((1-z^2)P'^2) scaled by 1/2
  }
}

const int kFaceVerts[4][3] = {{0, 2, 1}, {0, 1, 3}, {0, 3, 2}, {1, 2, 3}};
const double kTetVerts[4][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};

void face_point(int s, double c1, double c2, double out[3]) {
  const double* a = kTetVerts[kFaceVerts[s][0]];
  const double* b = kTetVerts[kFaceVerts[s][1]];
  const double* c = kTetVerts[kFaceVerts[s][2]];
  for (int x = 0; x < 3; ++x) out[x] = a[x] + c1 * (b[x] - a[x]) + c2 * (c[x] - a[x]);
}
void orient(int h, double c1, double c2, double& o1, double& o2) {
  double rest = 1.0 - c1 - c2;
  if (h == 0) { o1 = c2; o2 = c1; }
  else if (h == 1) { o1 = rest; o2 = c2; }
  else { o1 = c1; o2 = rest; }
}

void clean(std::vector<double>& m, size_t off, size_t n) {
  double mx = 0.0;
  for (size_t i = 0; i < n; ++i) mx = std::max(mx, std::fabs(m[off + i]));
  for (size_t i = 0; i < n; ++i)
    if (std::fabs(m[off + i]) <= 1e-12 * mx) m[off + i] = 0.0;
}

RefMatrices build(int N) {
  RefMatrices r;
  r.N = N;
  r.B = n_basis(N);
  r.BT = n_face_basis(N);
  r.BM = binom3(N + 2);
  const int B = r.B, BT = r.BT;
  auto ti = tet_indices(N);
  auto fi = tri_indices(N);

  std::vector<double> gx, gw;
  gauss_legendre(N + 3, gx, gw);
  const int ng = static_cast<int>(gx.size());

  // volume: mass and stiffness
  std::vector<double> M(B, 0.0), K(3 * B * B, 0.0);
  std::vector<Dual> vals(B);
  for (int ia = 0; ia < ng; ++ia)
    for (int ib = 0; ib < ng; ++ib)
      for (int ic = 0; ic < ng; ++ic) {
        double a = gx[ia], b = gx[ib], c = gx[ic];
        double zeta = c, eta = b * (1.0 - c), xi = a * (1.0 - b) * (1.0 - c);
        double wt = gw[ia] * gw[ib] * gw[ic] * (1.0 - b) * (1.0 - c) * (1.0 - c);
        Dual X{xi, {1, 0, 0}}, Y{eta, {0, 1, 0}}, Z{zeta, {0, 0, 1}};
        for (int k = 0; k < B; ++k) vals[k] = phi_dual(ti[k], X, Y, Z);
        for (int k = 0; k < B; ++k) {
          M[k] += wt * vals[k].v * vals[k].v;
          for (int d = 0; d < 3; ++d) {
            double g = wt * vals[k].d[d];
            if (g == 0.0) continue;
            for (int l = 0; l < B; ++l) K[(size_t)d * B * B + k + (size_t)l * B] += g * vals[l].v;
          }
        }
      }
  r.M = M;
  r.Khat.assign(3 * B * B, 0.0);
  r.Ktilde.assign(3 * B * B, 0.0);
  for (int d = 0; d < 3; ++d) {
    clean(K, (size_t)d * B * B, (size_t)B * B);
    for (int k = 0; k < B; ++k)
      for (int l = 0; l < B; ++l) {
        r.Khat[(size_t)d * B * B + k + (size_t)l * B] = K[(size_t)d * B * B + k + (size_t)l * B] / M[k];
        r.Ktilde[(size_t)d * B * B + k + (size_t)l * B] = -K[(size_t)d * B * B + l + (size_t)k * B] / M[k];
      }
  }

  // faces: W, R, f
  std::vector<double> fw, f1, f2;
  for (int ia = 0; ia < ng; ++ia)
    for (int ib = 0; ib < ng; ++ib) {
      double a = gx[ia], b = gx[ib];
      f2.push_back(b);
      f1.push_back(a * (1.0 - b));
      fw.push_back(gw[ia] * gw[ib] * (1.0 - b));
    }
  const int nf = static_cast<int>(fw.size());
  r.W.assign(BT, 0.0);
  std::vector<double> psiv((size_t)nf * BT);
  for (int q = 0; q < nf; ++q)
    for (int m = 0; m < BT; ++m) {
      psiv[(size_t)q * BT + m] = psi(fi[m], f1[q], f2[q]);
      r.W[m] += fw[q] * psiv[(size_t)q * BT + m] * psiv[(size_t)q * BT + m];
    }
  r.R.assign((size_t)4 * B * BT, 0.0);
  for (int s = 0; s < 4; ++s) {
    for (int q = 0; q < nf; ++q) {
      double x[3];
      face_point(s, f1[q], f2[q], x);
      for (int l = 0; l < B; ++l) {
        double pv = fw[q] * phi(ti[l], x[0], x[1], x[2]);
        for (int m = 0; m < BT; ++m) r.R[(size_t)s * B * BT + l + (size_t)m * B] += pv * psiv[(size_t)q * BT + m];
      }
    }
    for (int l = 0; l < B; ++l)
      for (int m = 0; m < BT; ++m) r.R[(size_t)s * B * BT + l + (size_t)m * B] /= r.W[m];
    clean(r.R, (size_t)s * B * BT, (size_t)B * BT);
  }
  r.Rhat.assign(r.R.size(), 0.0);
  for (int s = 0; s < 4; ++s)
    for (int l = 0; l < B; ++l)
      for (int m = 0; m < BT; ++m) {
        size_t i = (size_t)s * B * BT + l + (size_t)m * B;
        r.Rhat[i] = r.R[i] * r.W[m] / M[l];
      }
  r.f.assign((size_t)3 * BT * BT, 0.0);
  for (int h = 0; h < 3; ++h) {
    for (int q = 0; q < nf; ++q) {
      double o1, o2;
      orient(h, f1[q], f2[q], o1, o2);
      for (int n = 0; n < BT; ++n) {
        double pn = fw[q] * psi(fi[n], o1, o2);
        for (int m = 0; m < BT; ++m) r.f[(size_t)h * BT * BT + m + (size_t)n * BT] += pn * psiv[(size_t)q * BT + m];
      }
    }
    for (int m = 0; m < BT; ++m)
      for (int n = 0; n < BT; ++n) r.f[(size_t)h * BT * BT + m + (size_t)n * BT] /= r.W[m];
    clean(r.f, (size_t)h * BT * BT, (size_t)BT * BT);
  }
  return r;
}

}  // namespace

const RefMatrices& reference_matrices(int N) {
  static std::mutex mu;
  static std::map<int, RefMatrices> cache;
  if (N < 1 || N > 6) throw std::invalid_argument("polynomial degree must be 1..6");
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(N);
  if (it == cache.end()) it = cache.emplace(N, build(N)).first;
  return it->second;
}

}  // namespace yt
