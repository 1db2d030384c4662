// Reference-element matrices of tetrahedral ADER-DG (host code of the library).
//
// Computed by Gauss quadrature in collapsed coordinates with the Dubiner basis evaluated
// through Jacobi three-term recurrences; gradients by forward-mode dual numbers.  All
// matrices are column-major.  Entries below 1e-12 of the matrix's largest magnitude are
// set to exactly zero, so the stored sparsity pattern is the structural one.
#pragma once
#include <vector>

namespace yt {

struct RefMatrices {
  int N = 0;     // polynomial degree
  int B = 0;     // C(N+3,3) basis functions on the tetrahedron
  int BT = 0;    // C(N+2,2) basis functions on a face
  int BM = 0;    // C(N+2,3): basis functions of degree < N
  std::vector<double> M;       // B             diagonal of the mass matrix
  std::vector<double> Khat;    // 3 x B x B     M^-1 K^x,  K^x_kl = int dphi_k/dxi_x phi_l
  std::vector<double> Ktilde;  // 3 x B x B     -M^-1 (K^x)^T
  std::vector<double> R;       // 4 x B x BT    trace of phi_l on face s in the face basis
  std::vector<double> Rhat;    // 4 x B x BT    M^-1 R^s W
  std::vector<double> f;       // 3 x BT x BT   f^h_mn = <psi_n o Theta_h, psi_m> / W_m
  std::vector<double> W;       // BT            <psi_m, psi_m>
};

// Cached per degree N (1..6); thread-safe.
const RefMatrices& reference_matrices(int N);

inline int binom3(int n) { return n < 3 ? 0 : n * (n - 1) * (n - 2) / 6; }
inline int n_basis(int N) { return (N + 1) * (N + 2) * (N + 3) / 6; }
inline int n_face_basis(int N) { return (N + 1) * (N + 2) / 2; }

}  // namespace yt
