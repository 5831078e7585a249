// 1D nodes, weights and operator tables (host, setup only), and the
// deformed-box mesh helper.
//
// Sec. 4 (after Eq. (18)): nodal points are the p+1 Gauss-Lobatto-Legendre
// points; Table 1: BP1-BP4 integrate with q = p+2 Gauss-Legendre points,
// BP5-BP6 with the GLL points themselves.  Eq. (22) needs the 1D
// interpolation J (q x p1) and derivative D (q x p1) matrices; the quadrature-
// point derivative Dq (q x q) serves the interpolate-then-differentiate form
// of the gradient (Sec. 5, Eqs. (31)-(33)).
//
// Nodes come from Newton iteration on the Legendre recurrence in double;
// derivative and interpolation matrices from barycentric Lagrange formulas
// (Berrut and Trefethen, SIAM Review 2004).
#include <cmath>
#include <cstring>

#include "internal.h"

namespace ceedbp {
namespace {

// P_n(x) and P_n'(x) by (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}, P'_{k+1} = P'_{k-1} + (2k+1) P_k.
void legendre(int n, double x, double* p, double* dp, double* ddp) {
  double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0, dd0 = 0.0, dd1 = 0.0;
  if (n == 0) { *p = 1.0; *dp = 0.0; *ddp = 0.0; return; }
  for (int k = 1; k < n; ++k) {
    double p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1);
    double d2 = d0 + (2 * k + 1) * p1;
    double dd2 = dd0 + (2 * k + 1) * d1;
    p0 = p1; p1 = p2; d0 = d1; d1 = d2; dd0 = dd1; dd1 = dd2;
  }
  *p = p1; *dp = d1; *ddp = dd1;
}

void symmetrize(std::vector<double>& x) {
  int n = int(x.size());
  for (int i = 0; i < n / 2; ++i) {
    double v = 0.5 * (x[n - 1 - i] - x[i]);
    x[i] = -v;
    x[n - 1 - i] = v;
  }
  if (n % 2) x[n / 2] = 0.0;
}

void gll_rule(int N, std::vector<double>& x, std::vector<double>& w) {
  x.assign(N + 1, 0.0);
  w.assign(N + 1, 0.0);
  x[0] = -1.0;
  x[N] = 1.0;
  for (int j = 1; j < N; ++j) {
    double t = -std::cos(M_PI * j / N);
    for (int it = 0; it < 100; ++it) {
      double p, dp, ddp;
      legendre(N, t, &p, &dp, &ddp);
      double step = dp / ddp;
      t -= step;
      if (std::fabs(step) < 1e-16) break;
    }
    x[j] = t;
  }
  symmetrize(x);
  for (int j = 0; j <= N; ++j) {
    double p, dp, ddp;
    legendre(N, x[j], &p, &dp, &ddp);
    w[j] = 2.0 / (N * (N + 1.0) * p * p);
  }
  for (int j = 0; j <= N / 2; ++j) {
    double v = 0.5 * (w[j] + w[N - j]);
    w[j] = w[N - j] = v;
  }
}

void gauss_rule(int q, std::vector<double>& x, std::vector<double>& w) {
  x.assign(q, 0.0);
  w.assign(q, 0.0);
  for (int i = 0; i < q; ++i) {
    double t = -std::cos(M_PI * (i + 0.75) / (q + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p, dp, ddp;
      legendre(q, t, &p, &dp, &ddp);
      double step = p / dp;
      t -= step;
      if (std::fabs(step) < 1e-16) break;
    }
    x[i] = t;
  }
  symmetrize(x);
  for (int i = 0; i < q; ++i) {
    double p, dp, ddp;
    legendre(q, x[i], &p, &dp, &ddp);
    w[i] = 2.0 / ((1.0 - x[i] * x[i]) * dp * dp);
  }
  for (int i = 0; i < q / 2; ++i) {
    double v = 0.5 * (w[i] + w[q - 1 - i]);
    w[i] = w[q - 1 - i] = v;
  }
}

std::vector<double> bary_weights(const std::vector<double>& z) {
  int n = int(z.size());
  std::vector<double> lam(n, 1.0);
  for (int j = 0; j < n; ++j)
    for (int m = 0; m < n; ++m)
      if (m != j) lam[j] /= (z[j] - z[m]);
  return lam;
}

// Differentiation matrix of the Lagrange basis on nodes z (barycentric form,
// diagonal by the negative-sum rule).
std::vector<double> diff_matrix(const std::vector<double>& z) {
  int n = int(z.size());
  std::vector<double> lam = bary_weights(z), D(size_t(n) * n, 0.0);
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      double v = (lam[j] / lam[i]) / (z[i] - z[j]);
      D[size_t(i) * n + j] = v;
      s += v;
    }
    D[size_t(i) * n + i] = -s;
  }
  return D;
}

// Interpolation matrix L[r][j] = h_j(x_r) of the Lagrange basis on nodes z.
std::vector<double> interp_matrix(const std::vector<double>& z, const std::vector<double>& x) {
  int n = int(z.size()), m = int(x.size());
  std::vector<double> lam = bary_weights(z), L(size_t(m) * n, 0.0);
  for (int r = 0; r < m; ++r) {
    int hit = -1;
    for (int j = 0; j < n; ++j)
      if (x[r] == z[j]) hit = j;
    if (hit >= 0) {
      L[size_t(r) * n + hit] = 1.0;
      continue;
    }
    double den = 0.0;
    for (int j = 0; j < n; ++j) den += lam[j] / (x[r] - z[j]);
    for (int j = 0; j < n; ++j) L[size_t(r) * n + j] = (lam[j] / (x[r] - z[j])) / den;
  }
  return L;
}

}  // namespace

bool build_basis(int order, int q, bool gll_quad, Basis1D* out, std::string* err) {
  if (order < 1 || order > kMaxOrder) {
    *err = "order must be in 1..15";
    return false;
  }
  int p1 = order + 1;
  if (gll_quad) q = p1;
  if (q < p1 || q > kMaxQ) {
    *err = "quadrature points per direction must satisfy N+1 <= q <= 17";
    return false;
  }
  Basis1D& b = *out;
  b.p1 = p1;
  b.q = q;
  b.colloc = gll_quad;
  gll_rule(order, b.xi, b.rho);
  if (gll_quad) {
    b.eta = b.xi;
    b.w = b.rho;
  } else {
    gauss_rule(q, b.eta, b.w);
  }
  std::vector<double> Dn = diff_matrix(b.xi);  // p1 x p1 at the nodes
  b.J = interp_matrix(b.xi, b.eta);            // q x p1
  b.Dh.assign(size_t(q) * p1, 0.0);            // derivative at quadrature points: J * Dn (exact, degree N-1)
  for (int r = 0; r < q; ++r)
    for (int j = 0; j < p1; ++j) {
      double s = 0.0;
      for (int i = 0; i < p1; ++i) s += b.J[size_t(r) * p1 + i] * Dn[size_t(i) * p1 + j];
      b.Dh[size_t(r) * p1 + j] = s;
    }
  if (gll_quad) {
    b.Dh = Dn;
    b.Dq = Dn;
  } else {
    b.Dq = diff_matrix(b.eta);
  }
  return true;
}

}  // namespace ceedbp

extern "C" ceedbp_status ceedbp_mesh_box(int Ex, int Ey, int Ez, int order, double amp, double* coords,
                                         int64_t* l2g, uint8_t* dirichlet, int64_t* nglobal_out) {
  using namespace ceedbp;
  if (Ex < 1 || Ey < 1 || Ez < 1 || order < 1 || order > kMaxOrder) return CEEDBP_EINVAL;
  const int N = order, p1 = N + 1;
  const int64_t nx = int64_t(N) * Ex + 1, ny = int64_t(N) * Ey + 1, nz = int64_t(N) * Ez + 1;
  if (nglobal_out) *nglobal_out = nx * ny * nz;
  std::vector<double> xi, rho;
  gll_rule(N, xi, rho);
  // Undeformed 1D coordinates and their sines per global line index.
  auto line = [&](int E1, int64_t n1, std::vector<double>& c, std::vector<double>& s) {
    c.assign(n1, 0.0);
    s.assign(n1, 0.0);
    for (int e = 0; e < E1; ++e)
      for (int i = 0; i < p1; ++i) {
        int64_t I = int64_t(e) * N + i;
        c[I] = (e + (xi[i] + 1.0) / 2.0) / E1;
        s[I] = std::sin(M_PI * c[I]);
      }
  };
  std::vector<double> cx, sx, cy, sy, cz, sz;
  line(Ex, nx, cx, sx);
  line(Ey, ny, cy, sy);
  line(Ez, nz, cz, sz);
  const int64_t nloc = int64_t(p1) * p1 * p1;
  if (coords || l2g) {
    for (int64_t e = 0; e < int64_t(Ex) * Ey * Ez; ++e) {
      const int64_t ex = e % Ex, ey = (e / Ex) % Ey, ez = e / (int64_t(Ex) * Ey);
      for (int k = 0; k < p1; ++k)
        for (int j = 0; j < p1; ++j)
          for (int i = 0; i < p1; ++i) {
            const int64_t a = i + p1 * (j + int64_t(p1) * k);
            const int64_t I = ex * N + i, J = ey * N + j, K = ez * N + k;
            if (coords) {
              const double s = amp * sx[I] * sy[J] * sz[K];
              double* c = coords + (e * nloc + a) * 3;
              c[0] = cx[I] + s;
              c[1] = cy[J] + s;
              c[2] = cz[K] + s;
            }
            if (l2g) l2g[e * nloc + a] = I + nx * (J + ny * K);
          }
    }
  }
  if (dirichlet) {
    for (int64_t K = 0; K < nz; ++K)
      for (int64_t J = 0; J < ny; ++J)
        for (int64_t I = 0; I < nx; ++I)
          dirichlet[I + nx * (J + ny * K)] =
              (I == 0 || I == nx - 1 || J == 0 || J == ny - 1 || K == 0 || K == nz - 1) ? 1 : 0;
  }
  return CEEDBP_OK;
}
