// Reference triangle of the nodal DG method (host, FP64).
//
// Section 3 of arXiv:1403.1661: Lagrange basis on Warp & Blend nodes, cubature
// for volume integrals, Gauss-Legendre rules for surface integrals; Section 7:
// projection matrices Pr, Ps, P (weights folded in) and the lift L^g.
// Built from first principles here (orthonormal Jacobi polynomials by their
// three-term recurrence, Gauss rules by Newton iteration) and independent of any
// other implementation in this repository.
#pragma once

#include <vector>

namespace swe {

struct RefElem {
  int N = 0, Np = 0, Nfp = 0, Ncub = 0, Ng = 0;
  std::vector<double> r, s;                 // nodes (Np), lattice order
  std::vector<double> V, invV;              // Np x Np, row-major
  std::vector<double> rc, sc, wc;           // cubature points and weights
  std::vector<double> Ic, Icr, Ics;         // Ncub x Np
  std::vector<double> Pr, Ps, P;            // Np x Ncub
  std::vector<double> tg, wg;               // Gauss-Legendre on [-1, 1] (Ng)
  std::vector<double> Lg;                   // Np x (3 Ng): face f columns f*Ng..f*Ng+Ng-1
  std::vector<double> I1d;                  // Ng x Nfp: face-node values -> Gauss points
  std::vector<double> mean_w;               // Np: element mean = sum_j mean_w[j] q_j
  std::vector<double> T1;                   // 3 x Np: nodal values -> vertex values of Pi1 q
  std::vector<double> bary;                 // Np x 3: barycentric coordinates of the nodes
  int vertex_node[3] = {0, 0, 0};
  int face_node[3][8] = {};                 // face f, position m (from vertex f to f+1)

  // q: points per direction of the conical-product volume rule (exact to degree
  // 2q - 1), ng: Gauss points per face; 0 = the defaults ceil(3N/2) and
  // ceil((3N+1)/2) (degrees 3N - 1 and 3N)
  static RefElem build(int N, int q = 0, int ng = 0);
};

// Library node index of lattice point (i, j): i = N * weight of vertex 2,
// j = N * weight of vertex 1.
inline int lattice_index(int N, int i, int j) { return i * (N + 1) - i * (i - 1) / 2 + j; }

// Node index of position m (0..N) along face f, traversed from vertex f to f+1.
inline int face_node_index(int N, int f, int m) {
  if (f == 0) return lattice_index(N, 0, m);
  if (f == 1) return lattice_index(N, m, N - m);
  return lattice_index(N, N - m, 0);
}

void jacobi_gauss(int n, double alpha, double beta, std::vector<double>& x, std::vector<double>& w);
double jacobi_orthonormal(double x, double alpha, double beta, int n);

int ref_num_cubature(int N);   // Ncub of the default rule (degree 3N-1)
int ref_num_gauss(int N);      // Ng of the default face rule (degree 3N)

}  // namespace swe
