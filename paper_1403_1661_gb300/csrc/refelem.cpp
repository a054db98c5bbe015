// Reference triangle construction (host, FP64). See refelem.hpp.
#include "refelem.hpp"

#include <algorithm>
#include <cmath>
#include <stdexcept>

namespace swe {
namespace {

const double kPi = 3.14159265358979323846;

// Jacobi P_n^(a,b)(x), unnormalised, by the three-term recurrence
// 2n(n+a+b)(2n+a+b-2) P_n = (2n+a+b-1)[(2n+a+b)(2n+a+b-2) x + a^2-b^2] P_{n-1}
//                           - 2(n+a-1)(n+b-1)(2n+a+b) P_{n-2}.
double jacobi_raw(double x, double a, double b, int n) {
  if (n == 0) return 1.0;
  double p0 = 1.0;
  double p1 = 0.5 * ((a + b + 2.0) * x + (a - b));
  for (int k = 2; k <= n; ++k) {
    double c = 2.0 * k + a + b;
    double p2 = ((c - 1.0) * (c * (c - 2.0) * x + a * a - b * b) * p1 -
                 2.0 * (k + a - 1.0) * (k + b - 1.0) * c * p0) /
                (2.0 * k * (k + a + b) * (c - 2.0));
    p0 = p1;
    p1 = p2;
  }
  return p1;
}

double jacobi_norm(double a, double b, int n) {
  // squared L2 norm of P_n^(a,b) under (1-x)^a (1+x)^b
  double lg = (a + b + 1.0) * std::log(2.0) - std::log(2.0 * n + a + b + 1.0) +
              std::lgamma(n + a + 1.0) + std::lgamma(n + b + 1.0) -
              std::lgamma(n + a + b + 1.0) - std::lgamma(n + 1.0);
  return std::exp(lg);
}

double jacobi_raw_deriv(double x, double a, double b, int n) {
  if (n == 0) return 0.0;
  return 0.5 * (n + a + b + 1.0) * jacobi_raw(x, a + 1.0, b + 1.0, n - 1);
}

double jacobi_orthonormal_deriv(double x, double a, double b, int n) {
  return jacobi_raw_deriv(x, a, b, n) / std::sqrt(jacobi_norm(a, b, n));
}

std::vector<double> inverse(const std::vector<double>& A, int n) {
  std::vector<double> M(A), I(n * n, 0.0);
  for (int i = 0; i < n; ++i) I[i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(M[r * n + c]) > std::fabs(M[p * n + c])) p = r;
    if (M[p * n + c] == 0.0) throw std::runtime_error("singular matrix");
    if (p != c)
      for (int k = 0; k < n; ++k) {
        std::swap(M[p * n + k], M[c * n + k]);
        std::swap(I[p * n + k], I[c * n + k]);
      }
    double d = 1.0 / M[c * n + c];
    for (int k = 0; k < n; ++k) {
      M[c * n + k] *= d;
      I[c * n + k] *= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      double f = M[r * n + c];
      if (f == 0.0) continue;
      for (int k = 0; k < n; ++k) {
        M[r * n + k] -= f * M[c * n + k];
        I[r * n + k] -= f * I[c * n + k];
      }
    }
  }
  return I;
}

// C = A (m x k) * B (k x n)
std::vector<double> matmul(const std::vector<double>& A, const std::vector<double>& B, int m, int k,
                           int n) {
  std::vector<double> C(m * n, 0.0);
  for (int i = 0; i < m; ++i)
    for (int l = 0; l < k; ++l) {
      double a = A[i * k + l];
      if (a == 0.0) continue;
      for (int j = 0; j < n; ++j) C[i * n + j] += a * B[l * n + j];
    }
  return C;
}

std::vector<double> transpose(const std::vector<double>& A, int m, int n) {
  std::vector<double> T(n * m);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < n; ++j) T[j * m + i] = A[i * n + j];
  return T;
}

// collapsed coordinates of the reference triangle
void collapse(double r, double s, double& a, double& b) {
  a = (std::fabs(1.0 - s) > 1e-14) ? 2.0 * (1.0 + r) / (1.0 - s) - 1.0 : -1.0;
  b = s;
}

// orthonormal PKDO basis psi_ij and its gradient
double basis(double r, double s, int i, int j) {
  double a, b;
  collapse(r, s, a, b);
  return std::sqrt(2.0) * jacobi_orthonormal(a, 0, 0, i) * jacobi_orthonormal(b, 2.0 * i + 1.0, 0, j) *
         std::pow(1.0 - b, i);
}

void grad_basis(double r, double s, int i, int j, double& dr, double& ds) {
  double a, b;
  collapse(r, s, a, b);
  double fa = jacobi_orthonormal(a, 0, 0, i), dfa = jacobi_orthonormal_deriv(a, 0, 0, i);
  double gb = jacobi_orthonormal(b, 2.0 * i + 1.0, 0, j);
  double dgb = jacobi_orthonormal_deriv(b, 2.0 * i + 1.0, 0, j);
  if (i == 0) {
    dr = 0.0;
    ds = fa * dgb;
  } else {
    double pm = std::pow(1.0 - b, i - 1);
    dr = 2.0 * dfa * gb * pm;
    ds = dfa * gb * (1.0 + a) * pm + fa * (dgb * std::pow(1.0 - b, i) - i * gb * pm);
  }
  dr *= std::sqrt(2.0);
  ds *= std::sqrt(2.0);
}

// Vandermonde-type matrices: rows = points, columns = modes (i outer, j inner)
void vander(int N, const std::vector<double>& r, const std::vector<double>& s, std::vector<double>& V,
            std::vector<double>* Vr, std::vector<double>* Vs) {
  int np = (N + 1) * (N + 2) / 2, m = (int)r.size();
  V.assign(m * np, 0.0);
  if (Vr) Vr->assign(m * np, 0.0);
  if (Vs) Vs->assign(m * np, 0.0);
  for (int p = 0; p < m; ++p) {
    int c = 0;
    for (int i = 0; i <= N; ++i)
      for (int j = 0; j <= N - i; ++j, ++c) {
        V[p * np + c] = basis(r[p], s[p], i, j);
        if (Vr) {
          double dr, ds;
          grad_basis(r[p], s[p], i, j, dr, ds);
          (*Vr)[p * np + c] = dr;
          (*Vs)[p * np + c] = ds;
        }
      }
  }
}

std::vector<double> gauss_lobatto(int N) {
  std::vector<double> x(N + 1);
  x[0] = -1.0;
  x[N] = 1.0;
  if (N >= 2) {
    std::vector<double> xi, wi;
    jacobi_gauss(N - 1, 1.0, 1.0, xi, wi);
    for (int i = 0; i < N - 1; ++i) x[i + 1] = xi[i];
  }
  return x;
}

// Warburton (2006) optimised blend parameters, as tabulated by Hesthaven &
// Warburton (2008), N = 1..15.
const double kAlphaOpt[15] = {0.0000, 0.0000, 1.4152, 0.1001, 0.2751, 0.9800, 1.0999, 1.2832,
                              1.3648, 1.4773, 1.4959, 1.5743, 1.5770, 1.6223, 1.6258};

// 1D warp (GLL minus equidistant) at r, divided by 1 - r^2 (zero at the ends)
double warp_factor(int N, double rr, const std::vector<double>& gll) {
  double w = 0.0;
  for (int i = 0; i <= N; ++i) {
    double xi = -1.0 + 2.0 * i / N;
    double li = 1.0;
    for (int j = 0; j <= N; ++j) {
      if (j == i) continue;
      double xj = -1.0 + 2.0 * j / N;
      li *= (rr - xj) / (xi - xj);
    }
    w += (gll[i] - xi) * li;
  }
  if (std::fabs(rr) < 1.0 - 1e-10) return w / (1.0 - rr * rr);
  return 0.0;
}

void warp_blend(int N, std::vector<double>& r, std::vector<double>& s) {
  double alpha = (N <= 15) ? kAlphaOpt[N - 1] : 5.0 / 3.0;
  std::vector<double> gll = gauss_lobatto(N);
  int np = (N + 1) * (N + 2) / 2;
  r.assign(np, 0.0);
  s.assign(np, 0.0);
  const double sq3 = std::sqrt(3.0);
  for (int i = 0; i <= N; ++i)
    for (int j = 0; j <= N - i; ++j) {
      double L1 = (double)i / N, L3 = (double)j / N, L2 = 1.0 - L1 - L3;
      double x = -L2 + L3, y = (-L2 - L3 + 2.0 * L1) / sq3;
      double w1 = 4.0 * L2 * L3 * warp_factor(N, L3 - L2, gll) * (1.0 + (alpha * L1) * (alpha * L1));
      double w2 = 4.0 * L1 * L3 * warp_factor(N, L1 - L3, gll) * (1.0 + (alpha * L2) * (alpha * L2));
      double w3 = 4.0 * L1 * L2 * warp_factor(N, L2 - L1, gll) * (1.0 + (alpha * L3) * (alpha * L3));
      x += w1 + std::cos(2.0 * kPi / 3.0) * w2 + std::cos(4.0 * kPi / 3.0) * w3;
      y += std::sin(2.0 * kPi / 3.0) * w2 + std::sin(4.0 * kPi / 3.0) * w3;
      double l1 = (sq3 * y + 1.0) / 3.0;
      double l2 = (-3.0 * x - sq3 * y + 2.0) / 6.0;
      double l3 = (3.0 * x - sq3 * y + 2.0) / 6.0;
      int k = lattice_index(N, i, j);
      r[k] = -l2 + l3 - l1;
      s[k] = -l2 - l3 + l1;
    }
}

}  // namespace

double jacobi_orthonormal(double x, double alpha, double beta, int n) {
  return jacobi_raw(x, alpha, beta, n) / std::sqrt(jacobi_norm(alpha, beta, n));
}

void jacobi_gauss(int n, double a, double b, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int k = 0; k < n; ++k) {
    double xk = -std::cos((2.0 * k + 1.0) * kPi / (2.0 * n));
    if (k > 0) xk = 0.5 * (xk + x[k - 1]);
    for (int it = 0; it < 200; ++it) {
      double p = jacobi_raw(xk, a, b, n), dp = jacobi_raw_deriv(xk, a, b, n);
      double defl = 0.0;
      for (int i = 0; i < k; ++i) defl += 1.0 / (xk - x[i]);
      double dx = p / (dp - p * defl);
      xk -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    x[k] = xk;
  }
  std::sort(x.begin(), x.end());
  for (int k = 0; k < n; ++k) {
    double sum = 0.0;
    for (int m = 0; m < n; ++m) {
      double p = jacobi_orthonormal(x[k], a, b, m);
      sum += p * p;
    }
    w[k] = 1.0 / sum;
  }
}

int ref_num_cubature(int N) {
  int q = (3 * N + 1) / 2;  // ceil(3N/2)
  return q * q;
}

int ref_num_gauss(int N) { return (3 * N + 2) / 2; }  // ceil((3N+1)/2)

RefElem RefElem::build(int N, int q_in, int ng_in) {
  if (N < 1 || N > 7) throw std::runtime_error("order out of range");
  RefElem e;
  e.N = N;
  e.Np = (N + 1) * (N + 2) / 2;
  e.Nfp = N + 1;
  const int np = e.Np;
  warp_blend(N, e.r, e.s);
  vander(N, e.r, e.s, e.V, nullptr, nullptr);
  e.invV = inverse(e.V, np);
  std::vector<double> VVt = matmul(e.V, transpose(e.V, np, np), np, np, np);  // M^{-1}
  std::vector<double> Mmat = inverse(VVt, np);

  // volume cubature: conical product, Gauss-Legendre (a) x Gauss-Jacobi(1,0) (b)
  const int q = q_in > 0 ? q_in : (3 * N + 1) / 2;
  std::vector<double> xa, wa, xb, wb;
  jacobi_gauss(q, 0.0, 0.0, xa, wa);
  jacobi_gauss(q, 1.0, 0.0, xb, wb);
  for (int i = 0; i < q; ++i)
    for (int j = 0; j < q; ++j) {
      e.rc.push_back((1.0 + xa[i]) * (1.0 - xb[j]) / 2.0 - 1.0);
      e.sc.push_back(xb[j]);
      e.wc.push_back(wa[i] * wb[j] / 2.0);
    }
  e.Ncub = (int)e.rc.size();
  const int nc = e.Ncub;
  std::vector<double> Vc, Vcr, Vcs;
  vander(N, e.rc, e.sc, Vc, &Vcr, &Vcs);
  e.Ic = matmul(Vc, e.invV, nc, np, np);
  e.Icr = matmul(Vcr, e.invV, nc, np, np);
  e.Ics = matmul(Vcs, e.invV, nc, np, np);
  auto project = [&](const std::vector<double>& I) {
    std::vector<double> It = transpose(I, nc, np);  // np x nc
    for (int i = 0; i < np; ++i)
      for (int c = 0; c < nc; ++c) It[i * nc + c] *= e.wc[c];
    return matmul(VVt, It, np, np, nc);
  };
  e.Pr = project(e.Icr);
  e.Ps = project(e.Ics);
  e.P = project(e.Ic);

  // faces: Gauss-Legendre, lift and the 1D face interpolation
  e.Ng = ng_in > 0 ? ng_in : ref_num_gauss(N);
  const int ng = e.Ng;
  jacobi_gauss(ng, 0.0, 0.0, e.tg, e.wg);
  const double vr[3] = {-1.0, 1.0, -1.0}, vs[3] = {-1.0, -1.0, 1.0};
  e.Lg.assign(np * 3 * ng, 0.0);
  for (int f = 0; f < 3; ++f) {
    int a = f, b = (f + 1) % 3;
    std::vector<double> fr(ng), fs(ng);
    for (int g = 0; g < ng; ++g) {
      double t = 0.5 * (1.0 + e.tg[g]);
      fr[g] = vr[a] + t * (vr[b] - vr[a]);
      fs[g] = vs[a] + t * (vs[b] - vs[a]);
    }
    std::vector<double> Vg;
    vander(N, fr, fs, Vg, nullptr, nullptr);
    std::vector<double> Ig = matmul(Vg, e.invV, ng, np, np);  // ng x np
    std::vector<double> IgT = transpose(Ig, ng, np);           // np x ng
    for (int i = 0; i < np; ++i)
      for (int g = 0; g < ng; ++g) IgT[i * ng + g] *= e.wg[g];
    std::vector<double> L = matmul(VVt, IgT, np, np, ng);
    for (int i = 0; i < np; ++i)
      for (int g = 0; g < ng; ++g) e.Lg[i * 3 * ng + f * ng + g] = L[i * ng + g];
  }
  std::vector<double> gll = gauss_lobatto(N);
  e.I1d.assign(ng * e.Nfp, 0.0);
  for (int g = 0; g < ng; ++g)
    for (int m = 0; m <= N; ++m) {
      double l = 1.0;
      for (int k = 0; k <= N; ++k)
        if (k != m) l *= (e.tg[g] - gll[k]) / (gll[m] - gll[k]);
      e.I1d[g * e.Nfp + m] = l;
    }
  for (int f = 0; f < 3; ++f)
    for (int m = 0; m <= N; ++m) e.face_node[f][m] = face_node_index(N, f, m);

  // element mean, P1 projection at the vertices, barycentric coordinates
  e.mean_w.assign(np, 0.0);
  for (int i = 0; i < np; ++i)
    for (int j = 0; j < np; ++j) e.mean_w[j] += 0.5 * Mmat[i * np + j];
  e.vertex_node[0] = lattice_index(N, 0, 0);
  e.vertex_node[1] = lattice_index(N, 0, N);
  e.vertex_node[2] = lattice_index(N, N, 0);
  std::vector<double> keep(np * np, 0.0);
  {
    int c = 0;
    for (int i = 0; i <= N; ++i)
      for (int j = 0; j <= N - i; ++j, ++c) keep[c * np + c] = (i + j <= 1) ? 1.0 : 0.0;
  }
  std::vector<double> Pi1 = matmul(matmul(e.V, keep, np, np, np), e.invV, np, np, np);
  e.T1.assign(3 * np, 0.0);
  for (int v = 0; v < 3; ++v)
    for (int j = 0; j < np; ++j) e.T1[v * np + j] = Pi1[e.vertex_node[v] * np + j];
  e.bary.assign(np * 3, 0.0);
  for (int j = 0; j < np; ++j) {
    e.bary[j * 3 + 0] = -(e.r[j] + e.s[j]) / 2.0;
    e.bary[j * 3 + 1] = (1.0 + e.r[j]) / 2.0;
    e.bary[j * 3 + 2] = (1.0 + e.s[j]) / 2.0;
  }
  return e;
}

}  // namespace swe
