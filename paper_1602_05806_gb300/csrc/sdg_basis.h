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

constexpr int kMaxHalf = (kMaxN1 + 1) / 2;

// 1D line operator of the pressure / viscous kernels as stored in one
// compute precision (every value exactly representable in it, kept here as
// doubles), in the even/odd basis of the line.
//
// The Gauss-Legendre nodes are symmetric about 1/2, so with J the reversal
// of a line the blocks satisfy H^L = J H^R J and J H^C J = H^C.  A line x of
// n nodes maps to x^ = P x:  x^_k = x_k + x_{n-1-k} (k < h, even part),
// x^_h = x_h (middle node, odd n only), x^_{hE+k} = x_k - x_{n-1-k} (k < h,
// odd part), with h = floor(n/2), hE = ceil(n/2).  Every line operator X
// acts as X^ = Q X Q^T on x^, Q = G^-1 P, G = P P^T = diag(2, .., [1], .., 2),
// and the result returns through out = P^T y^ (out_k = y^_k + y^_{hE+k},
// out_{n-1-k} = y^_k - y^_{hE+k}).  In this basis H^C is block diagonal
// (CE, CO) and H^R = [[A, B], [-B^T, D]], H^L = [[A, -B], [B^T, D]] with A,
// D, CE, CO symmetric: the n x n contractions shrink to six blocks of about
// (n/2)^2, and the stored operator is exactly symmetric (H^L_eff =
// (H^R_eff)^T, H^C_eff symmetric) because the blocks are stored that way.
//
// Correction making the stored operator annihilate the local kernel
// (constants; for odd N also the antisymmetric sawtooth z):
//   even N (kz = 0): -diag(rho), rho the row sums of H^L + H^C + H^R in the
//     natural basis; in the even/odd basis rho_e (even part, middle node
//     included) and rho_o (odd part).
//   odd N (kz = 1): with q = mu 1 + dz z the orthogonal fit of the centre
//     line onto {1, z} (mu = sum(c^_E) / n, dz = zn . c^_O) removed from the
//     three lines, the correction is -k0 (S0 . c'_E) - k1 (S1 . c'_O) on the
//     even / odd outputs, S = (H^L + H^C + H^R) [k0, k1] on the orthonormal
//     kernel basis; in exact arithmetic this is the symmetric rank-4
//     correction C with (H^L + H^C + H^R + C) q = 0 on span{1, z}.
struct CoefSet {
  int n, hE, h;
  double A[kMaxHalf * kMaxHalf], B[kMaxHalf * kMaxHalf], D[kMaxHalf * kMaxHalf];
  double CE[kMaxHalf * kMaxHalf], CO[kMaxHalf * kMaxHalf];
  double rho_e[kMaxHalf], rho_o[kMaxHalf];
  double zn[kMaxHalf], z2[kMaxHalf];   // dz = zn . c^_O ; the odd part of z is 2 z_k = z2[k]
  double S0[kMaxHalf], S1[kMaxHalf], k1[kMaxHalf];
  double k0, inv_n;
  int kz;
};

// fp32 != 0: round every stored value to float first.
void build_coefs(const Basis1D& b, int fp32, CoefSet* out);

// The line operator the stored set applies, in the natural basis, evaluated
// in long double from the stored values: HL, HR the neighbour blocks and Mc
// the centre block including the kernel correction (n x n row-major each).
void line_operator(const CoefSet& c, double* HL, double* Mc, double* HR);

}  // namespace sdg
