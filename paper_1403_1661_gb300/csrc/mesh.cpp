// Mesh connectivity, geometry, time steps and levels (host). See mesh.hpp.
#include <algorithm>
#include <cmath>
#include <string>
#include <tuple>

#include "mesh.hpp"

namespace swe {

std::string Mesh::create(const double* vx, const double* vy, int32_t nv, const int32_t* EToV,
                         int32_t K, Mesh& m) {
  if (!vx || !vy || !EToV || nv < 3 || K < 1) return "mesh: empty or NULL input";
  m.K = K;
  m.nv = nv;
  m.vx.assign(vx, vx + nv);
  m.vy.assign(vy, vy + nv);
  m.EToV.assign(EToV, EToV + 3 * (size_t)K);
  for (int32_t k = 0; k < K; ++k) {
    int32_t* v = &m.EToV[3 * (size_t)k];
    for (int a = 0; a < 3; ++a)
      if (v[a] < 0 || v[a] >= nv) return "mesh: vertex index out of range";
    if (v[0] == v[1] || v[1] == v[2] || v[0] == v[2]) return "mesh: repeated vertex in a triangle";
    double a2 = (vx[v[1]] - vx[v[0]]) * (vy[v[2]] - vy[v[0]]) -
                (vx[v[2]] - vx[v[0]]) * (vy[v[1]] - vy[v[0]]);
    if (!(a2 != 0.0) || !std::isfinite(a2)) return "mesh: degenerate triangle";
    if (a2 < 0) std::swap(v[1], v[2]);
  }
  // connectivity: sort (min vertex, max vertex, element, face) and pair equal keys
  std::vector<std::tuple<int64_t, int32_t, int32_t>> keys;
  keys.reserve(3 * (size_t)K);
  for (int32_t k = 0; k < K; ++k)
    for (int f = 0; f < 3; ++f) {
      int64_t a = m.EToV[3 * (size_t)k + f], b = m.EToV[3 * (size_t)k + (f + 1) % 3];
      int64_t lo = std::min(a, b), hi = std::max(a, b);
      keys.emplace_back(lo * (int64_t)nv + hi, k, f);
    }
  std::sort(keys.begin(), keys.end());
  m.EToE.assign(3 * (size_t)K, -1);
  m.EToF.assign(3 * (size_t)K, -1);
  for (size_t i = 0; i < keys.size();) {
    size_t j = i + 1;
    while (j < keys.size() && std::get<0>(keys[j]) == std::get<0>(keys[i])) ++j;
    if (j - i > 2) return "mesh: a face is shared by more than two triangles";
    if (j - i == 2) {
      int32_t k1 = std::get<1>(keys[i]), f1 = std::get<2>(keys[i]);
      int32_t k2 = std::get<1>(keys[i + 1]), f2 = std::get<2>(keys[i + 1]);
      if (k1 == k2) return "mesh: triangle adjacent to itself";
      m.EToE[3 * (size_t)k1 + f1] = k2;
      m.EToF[3 * (size_t)k1 + f1] = f2;
      m.EToE[3 * (size_t)k2 + f2] = k1;
      m.EToF[3 * (size_t)k2 + f2] = f1;
    }
    i = j;
  }
  // affine geometry
  m.rx.resize(K); m.ry.resize(K); m.sx.resize(K); m.sy.resize(K); m.J.resize(K);
  m.cx.resize(K); m.cy.resize(K); m.flen.resize(3 * (size_t)K);
  for (int32_t k = 0; k < K; ++k) {
    const int32_t* v = &m.EToV[3 * (size_t)k];
    double x0 = vx[v[0]], x1 = vx[v[1]], x2 = vx[v[2]];
    double y0 = vy[v[0]], y1 = vy[v[1]], y2 = vy[v[2]];
    double xr = 0.5 * (x1 - x0), xs = 0.5 * (x2 - x0), yr = 0.5 * (y1 - y0), ys = 0.5 * (y2 - y0);
    double J = xr * ys - xs * yr;
    m.J[k] = J;
    m.rx[k] = ys / J;
    m.ry[k] = -xs / J;
    m.sx[k] = -yr / J;
    m.sy[k] = xr / J;
    m.cx[k] = (x0 + x1 + x2) / 3.0;
    m.cy[k] = (y0 + y1 + y2) / 3.0;
    double X[3] = {x0, x1, x2}, Y[3] = {y0, y1, y2};
    for (int f = 0; f < 3; ++f)
      m.flen[3 * (size_t)k + f] = std::hypot(X[(f + 1) % 3] - X[f], Y[(f + 1) % 3] - Y[f]);
  }
  return std::string();
}

void tvb_stencil(const Mesh& m, std::vector<double>& alpha, std::vector<double>& beta,
                 std::vector<int32_t>& jsel) {
  const int32_t K = m.K;
  alpha.assign(3 * (size_t)K, 0.0);
  beta.assign(3 * (size_t)K, 0.0);
  jsel.assign(3 * (size_t)K, 0);
  for (int32_t k = 0; k < K; ++k) {
    const int32_t* v = &m.EToV[3 * (size_t)k];
    double X[3] = {m.vx[v[0]], m.vx[v[1]], m.vx[v[2]]};
    double Y[3] = {m.vy[v[0]], m.vy[v[1]], m.vy[v[2]]};
    double bx = m.cx[k], by = m.cy[k];
    double dmx[3], dmy[3], dbx[3], dby[3];
    for (int f = 0; f < 3; ++f) {
      double mx = 0.5 * (X[f] + X[(f + 1) % 3]), my = 0.5 * (Y[f] + Y[(f + 1) % 3]);
      dmx[f] = mx - bx;
      dmy[f] = my - by;
      int32_t nb = m.EToE[3 * (size_t)k + f];
      if (nb >= 0) {
        dbx[f] = m.cx[nb] - bx;
        dby[f] = m.cy[nb] - by;
      } else {
        // ghost centroid: b0 reflected across the face line
        double ex = X[(f + 1) % 3] - X[f], ey = Y[(f + 1) % 3] - Y[f];
        double L = std::hypot(ex, ey);
        double nx = ey / L, ny = -ex / L;
        double d = dmx[f] * nx + dmy[f] * ny;
        dbx[f] = 2.0 * d * nx;
        dby[f] = 2.0 * d * ny;
      }
    }
    for (int i = 0; i < 3; ++i) {
      double best = -1e300, ba = 0, bb = 0;
      int bj = (i + 1) % 3;
      for (int t = 1; t <= 2; ++t) {
        int j = (i + t) % 3;
        double det = dbx[i] * dby[j] - dbx[j] * dby[i];
        double al = (dmx[i] * dby[j] - dbx[j] * dmy[i]) / det;
        double be = (dbx[i] * dmy[i] - dby[i] * dmx[i]) / det;
        double score = std::min(al, be);
        if (score > best) {
          best = score;
          ba = al;
          bb = be;
          bj = j;
        }
      }
      alpha[3 * (size_t)k + i] = ba;
      beta[3 * (size_t)k + i] = bb;
      jsel[3 * (size_t)k + i] = bj;
    }
  }
}

void element_dt(const Mesh& m, int N, const double* h, const double* hu, const double* hv, double g,
                double cfl, std::vector<double>& dt) {
  const int np = (N + 1) * (N + 2) / 2;
  const size_t n = (size_t)m.K * np;
  double hmax = -1e300;
  for (size_t i = 0; i < n; ++i) hmax = std::max(hmax, h[i]);
  double href = 1e-2 * hmax;
  double C = cfl / ((N + 1.0) * (N + 1.0));
  dt.resize(m.K);
  for (int32_t k = 0; k < m.K; ++k) {
    double amax = 0.0;
    for (int j = 0; j < np; ++j) {
      size_t i = (size_t)k * np + j;
      double hh = std::max(h[i], href);
      double u = 0.0, v = 0.0;
      if (h[i] > href) {
        u = hu[i] / h[i];
        v = hv[i] / h[i];
      }
      amax = std::max(amax, std::hypot(u, v) + std::sqrt(g * hh));
    }
    const double* L = &m.flen[3 * (size_t)k];
    double area = 2.0 * m.J[k];
    double H = 2.0 * area / (L[0] + L[1] + L[2]);  // inradius
    dt[k] = C * H / amax;
  }
}

double assign_levels(const std::vector<double>& dt, int nlevels, std::vector<int32_t>& level) {
  double dtmin = 1e300;
  for (double d : dt) dtmin = std::min(dtmin, d);
  level.resize(dt.size());
  for (size_t k = 0; k < dt.size(); ++k) {
    int e;
    std::frexp(dt[k] / dtmin, &e);  // ratio = m 2^e, m in [0.5, 1): 2^{e-1} <= ratio < 2^e
    level[k] = std::min(std::max(e, 1), nlevels);
  }
  return dtmin;
}

double regroup_levels(const std::vector<double>& dt, double dt_min, const std::vector<int32_t>& old_level,
                      int64_t k, int nlevels, std::vector<int32_t>& level) {
  int v2 = 62;   // the power of two in k
  if (k > 0) {
    v2 = 0;
    while (((k >> v2) & 1) == 0) ++v2;
  }
  const int cap = v2 + 1 < nlevels ? v2 + 1 : nlevels;
  level.resize(dt.size());
  double margin = 1e300;
  for (size_t i = 0; i < dt.size(); ++i) {
    int e;
    std::frexp(dt[i] / dt_min, &e);
    int l = std::min(std::max(e, 1), nlevels);
    l = std::min(l, old_level[i] + 1);
    l = std::min(l, cap);
    level[i] = l;
    margin = std::min(margin, dt[i] / std::ldexp(dt_min, l - 1));
  }
  return margin;
}

}  // namespace swe
