// Triangle mesh: connectivity, affine geometry, CFL time step and MRAB levels.
//
// Section 3 (conforming triangles, affine elements) and Section 4 (Eq. cfl and the
// level rule 2^{l-1} dt_min <= dt_k < 2^l dt_min) of arXiv:1403.1661.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace swe {

struct Mesh {
  int32_t K = 0, nv = 0;
  std::vector<double> vx, vy;       // vertices
  std::vector<int32_t> EToV;        // K x 3, counter-clockwise
  std::vector<int32_t> EToE, EToF;  // K x 3, -1 on boundary faces
  // affine geometry (FP64)
  std::vector<double> rx, ry, sx, sy, J;  // K
  std::vector<double> cx, cy;              // centroids
  std::vector<double> flen;                // K x 3 face lengths

  // Builds connectivity and geometry; returns an error message or empty string.
  static std::string create(const double* vx, const double* vy, int32_t nv, const int32_t* EToV,
                            int32_t K, Mesh& out);
};

// Per element and edge i the TVB stencil (Cockburn & Shu 1998, triangles):
// m_i - b0 = alpha_i (b_i - b0) + beta_i (b_j - b0), j = jsel_i, where b_i is the
// centroid of the neighbour across face i (a wall face uses b0 reflected across it).
void tvb_stencil(const Mesh& m, std::vector<double>& alpha, std::vector<double>& beta,
                 std::vector<int32_t>& jsel);

// dt_k = cfl/(N+1)^2 * H_k / a_k (Eq. cfl) with H_k = the inradius and
// a_k = max over the element's nodes of |u| + sqrt(g max(h, 1e-2 max h)),
// u = hu/h where h exceeds that reference depth and 0 elsewhere.
void element_dt(const Mesh& m, int N, const double* h, const double* hu, const double* hv, double g,
                double cfl, std::vector<double>& dt);

// Level 1..nlevels (Section 4) from dt; returns dt_min.
double assign_levels(const std::vector<double>& dt, int nlevels, std::vector<int32_t>& level);
// Levels for a regroup with dt_min kept (Section 4): the largest l with
// 2^{l-1} dt_min <= dt_k in 1..nlevels, at most old + 1, at most 1 + (the power
// of two in k). Returns min_k dt_k / (2^{l_k - 1} dt_min).
double regroup_levels(const std::vector<double>& dt, double dt_min, const std::vector<int32_t>& old_level,
                      int64_t k, int nlevels, std::vector<int32_t>& level);

}  // namespace swe
