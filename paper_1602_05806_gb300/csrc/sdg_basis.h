// 1D reference-element algebra of degree N on [0,1] (Sec. 2.1, Eq. matrices;
// Sec. 2.2, L2 projections).  All matrices row-major n1 x n1, entry [p][q] at
// p*n1 + q, with p the test-function index and q the unknown index.
#pragma once

namespace sdg {

constexpr int kMaxN = 11;
constexpr int kMaxN1 = kMaxN + 1;

struct Basis1D {
  int N, n1;
  double xi[kMaxN1], w[kMaxN1];           // GL nodes / weights on [0,1]
  double phi0[kMaxN1], phi1[kMaxN1];      // phi_m(0), phi_m(1)
  double M[kMaxN1 * kMaxN1];              // mass matrix (diagonal = w)
  double Rt[kMaxN1 * kMaxN1], Lt[kMaxN1 * kMaxN1];   // R~, L~
  double Rb[kMaxN1 * kMaxN1], Lb[kMaxN1 * kMaxN1];   // R-bar, L-bar
  double ML[kMaxN1 * kMaxN1], MR[kMaxN1 * kMaxN1];   // M^L, M^R
  double HR[kMaxN1 * kMaxN1], HL[kMaxN1 * kMaxN1], HC[kMaxN1 * kMaxN1];
  double Dn[kMaxN1 * kMaxN1];             // Dn[k][m] = phi_m'(xi_k)
};

// n-point Gauss-Legendre rule on [0,1], nodes ascending.
void gauss_legendre(int n, double* xi, double* w);

// Fill every matrix of degree N (0 <= N <= kMaxN).  Returns 0 or -1.
int build_basis(int N, Basis1D* b);

// Orthogonal projector (n1 x n1, row-major) onto the kernel of R~ - L~, the
// local patterns whose weak gradient vanishes when repeated in every cell;
// the kernel of the periodic pressure operator is the tensor product of this
// space over the directions, repeated in every element.  Returns its
// dimension (1 for even N: the constants; 2 for odd N).
int kernel_projector(const Basis1D& b, double* proj);

// Orthonormal basis of the same space: basis[j*n1 + l], j < returned dim.
int kernel_basis(const Basis1D& b, double* basis);

// 1D blocks of the operator kernel as stored in one compute precision (all
// values exactly representable in it, kept here as doubles):
//   HR; HL = HR^T; HC symmetrised                      (exactly symmetric)
//   rho[m] = row sum of [HL HC HR]                     (zero up to rounding)
//   kz = 1 for odd N: z = stored local sawtooth pattern (orthogonal to the
//        constants, max |z| = 1), zn = z / (z.z), and C the symmetric matrix
//        with (HL + HC + HR + C) q = 0 for q in span{1, z} (exact arithmetic).
struct CoefSet {
  double HL[kMaxN1 * kMaxN1], HC[kMaxN1 * kMaxN1], HR[kMaxN1 * kMaxN1], C[kMaxN1 * kMaxN1];
  double rho[kMaxN1], z[kMaxN1], zn[kMaxN1];
  int kz;
};

// fp32 != 0: round every stored value to float first.
void build_coefs(const Basis1D& b, int fp32, CoefSet* out);

}  // namespace sdg
