// Reference elements for the nodal DG solver (host, double precision).
//
// Line: GLL nodes (Section 3.1), mass M^1D, derivative D^1D, lift vectors
// (M^1D)^{-1} e_0 and (M^1D)^{-1} e_N, barycentric-weighted edge masses.
// Triangle: Warp & Blend nodes taken as the tetrahedron's face distribution
// (Section 3.1), mass, D_r, D_s and the barycentric-weighted masses
// M_a = int l_i l_j lambda_a from which M^{tri,k} = sum_a J_a M_a (Section 4.2).
// Tetrahedron: Warp & Blend nodes, D_r, D_s, D_t, mass and the reference lift.
//
// All operators come from orthonormal (Proriol-Koornwinder-Dubiner) modal
// bases: M = (V V^T)^{-1}, D = V_r V^{-1}, and weighted masses by Gauss
// quadrature of the modal basis in collapsed coordinates.
#pragma once
#include <array>
#include <cstdint>
#include <string>
#include <vector>

namespace dgw {

struct Mat {
  int r = 0, c = 0;
  std::vector<double> a;
  Mat() = default;
  Mat(int r_, int c_) : r(r_), c(c_), a(size_t(r_) * c_, 0.0) {}
  double& operator()(int i, int j) { return a[size_t(i) * c + j]; }
  double operator()(int i, int j) const { return a[size_t(i) * c + j]; }
};

Mat matmul(const Mat& A, const Mat& B);
Mat transpose(const Mat& A);
bool invert(const Mat& A, Mat& Ainv);  // Gauss-Jordan, partial pivoting

struct RefElems {
  int N = 0, Nt = 0, Nq = 0, Npw = 0, Npt = 0;
  // line
  std::vector<double> gll;
  Mat M1, D1, Mea, Meb;  // Mea: int l_m l_n (1-x)/2, Meb: (1+x)/2
  std::vector<double> ell0, ellN;
  // triangle
  std::vector<double> tri_r, tri_s;
  Mat Dr, Ds, Mt, Ma[3];
  std::vector<std::vector<int>> edge_nodes;  // 3 x (N+1), from first to second edge vertex
  // tet
  std::vector<double> tet_r, tet_s, tet_t;
  Mat tDr, tDs, tDt, tM, tLIFT;               // LIFT: Npt x (4 Nt), faces in order
  std::vector<std::vector<int>> tet_face_nodes;  // 4 x Nt, element node order
  // wedge faces: 0 bottom, 1 top, 2..4 quads; element node ids, face order
  std::vector<std::vector<int>> wedge_face_nodes;
  // triangle-face symmetries: perm[code][k] = index (in the neighbour face's
  // own order) of the node that coincides with own face node k.  code encodes
  // pos[m] = position in the own face vertex list of the neighbour's m-th
  // face vertex, code = pos[0]*3 + pos[1] (a permutation of 0,1,2).
  std::vector<std::vector<int>> tri_perm;  // 9 x Nt (invalid codes empty)
  // inverse Vandermonde matrices (Lagrange basis = modal basis x Vinv)
  Mat line_Vinv, tri_Vinv, tet_Vinv;
};

// Lagrange basis values at a reference point
void line_lagrange(const RefElems& R, double t, double* out);
void tri_lagrange(const RefElems& R, double r, double s, double* out);
void tet_lagrange(const RefElems& R, double r, double s, double t, double* out);

RefElems build_reference(int N);

// triangle lattice index of barycentric integer weights (a, b): node order
// for b = 0..N, for a = 0..N-b.
inline int tri_index(int N, int a, int b) { return b * (N + 1) - (b * (b - 1)) / 2 + a; }

// Carpenter-Kennedy five-stage fourth-order 2N-storage Runge-Kutta.
extern const double kLSRK_A[5];
extern const double kLSRK_B[5];
extern const double kLSRK_C[5];

}  // namespace dgw
