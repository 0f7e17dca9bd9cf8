// Host-side FP64 set-up of the 1D reference-element algebra (Sec. 2.1):
// Gauss-Legendre nodes by Newton iteration on the Legendre three-term
// recurrence, the Lagrange basis in barycentric form, and every 1D matrix of
// Eq. matrices / Sec. 2.2 by Gauss-Legendre quadrature of its integral.
#include "sdg_basis.h"

#include <cmath>
#include <vector>

namespace sdg {

namespace {

constexpr double kPi = 3.14159265358979323846;

// P_n(x) and P_n'(x) by the recurrence (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}.
void legendre(int n, double x, double* p, double* dp) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { *p = 1.0; *dp = 0.0; return; }
  for (int k = 1; k < n; ++k) {
    double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
    p0 = p1;
    p1 = p2;
  }
  *p = p1;
  *dp = n * (x * p1 - p0) / (x * x - 1.0);
}

}  // namespace

void gauss_legendre(int n, double* xi, double* w) {
  // Roots of P_n on (-1,1), refined from the asymptotic initial guess.
  for (int k = 0; k < n; ++k) {
    double x = std::cos(kPi * (k + 0.75) / (n + 0.5));
    double p, dp;
    for (int it = 0; it < 100; ++it) {
      legendre(n, x, &p, &dp);
      double dx = p / dp;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    legendre(n, x, &p, &dp);
    // node k counts from the right end; store ascending on [0,1]
    xi[n - 1 - k] = 0.5 * (1.0 - (-x));  // (x + 1) / 2
    w[n - 1 - k] = 1.0 / ((1.0 - x * x) * dp * dp);  // (2 / ((1-x^2) P'^2)) / 2
  }
  if (n == 1) { xi[0] = 0.5; w[0] = 1.0; }
  // exact symmetry of the rule about 1/2
  for (int k = 0; k < n / 2; ++k) {
    double a = 0.5 * (xi[k] + (1.0 - xi[n - 1 - k]));
    xi[k] = a;
    xi[n - 1 - k] = 1.0 - a;
    double b = 0.5 * (w[k] + w[n - 1 - k]);
    w[k] = b;
    w[n - 1 - k] = b;
  }
  if (n % 2 == 1) xi[n / 2] = 0.5;
}

namespace {

// Barycentric Lagrange basis through `nodes` (n points).
struct Lagrange {
  int n;
  std::vector<double> x, lam;   // nodes and barycentric weights
  std::vector<double> D;        // D[i*n+j] = phi_j'(x_i)

  explicit Lagrange(const std::vector<double>& nodes) : n((int)nodes.size()), x(nodes) {
    lam.assign(n, 1.0);
    for (int j = 0; j < n; ++j)
      for (int k = 0; k < n; ++k)
        if (k != j) lam[j] /= (x[j] - x[k]);
    D.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) {
      double diag = 0.0;
      for (int j = 0; j < n; ++j) {
        if (j == i) continue;
        double v = (lam[j] / lam[i]) / (x[i] - x[j]);
        D[i * n + j] = v;
        diag -= v;
      }
      D[i * n + i] = diag;
    }
  }
  // values phi_j(t) for all j
  void eval(double t, double* phi) const {
    for (int j = 0; j < n; ++j)
      if (t == x[j]) {
        for (int k = 0; k < n; ++k) phi[k] = (k == j) ? 1.0 : 0.0;
        return;
      }
    double s = 0.0;
    for (int j = 0; j < n; ++j) {
      phi[j] = lam[j] / (t - x[j]);
      s += phi[j];
    }
    for (int j = 0; j < n; ++j) phi[j] /= s;
  }
  // derivatives phi_j'(t): phi_j' has degree n-2 and is interpolated exactly
  // through the nodes, phi_j'(t) = sum_i phi_i(t) D[i][j].
  void deriv(double t, double* dphi) const {
    std::vector<double> phi(n);
    eval(t, phi.data());
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int i = 0; i < n; ++i) s += phi[i] * D[i * n + j];
      dphi[j] = s;
    }
  }
};

}  // namespace

int build_basis(int N, Basis1D* b) {
  if (N < 0 || N > kMaxN) return -1;
  const int n1 = N + 1;
  b->N = N;
  b->n1 = n1;
  gauss_legendre(n1, b->xi, b->w);
  std::vector<double> nodes(b->xi, b->xi + n1);
  Lagrange L(nodes);

  // quadrature for the integrals: n1 + 2 points is exact for degree 2N+3
  const int nq = n1 + 2;
  double qs[kMaxN1 + 2], qw[kMaxN1 + 2];
  gauss_legendre(nq, qs, qw);

  auto at = [&](double* m, int p, int q) -> double& { return m[p * n1 + q]; };
  for (int p = 0; p < n1 * n1; ++p) {
    b->M[p] = b->Rt[p] = b->Lt[p] = b->Rb[p] = b->Lb[p] = 0.0;
    b->ML[p] = b->MR[p] = 0.0;
  }
  std::vector<double> phiA(n1), phiB(n1), dA(n1), dB(n1), half(n1), zero(n1), one(n1);
  L.eval(0.5, half.data());
  L.eval(0.0, zero.data());
  L.eval(1.0, one.data());
  for (int j = 0; j < n1; ++j) { b->phi0[j] = zero[j]; b->phi1[j] = one[j]; }

  for (int k = 0; k < nq; ++k) {
    const double s = qs[k], wk = qw[k];
    // integrand pieces at the left half (s/2) and the right half (1/2 + s/2)
    L.eval(0.5 * s, phiA.data());
    L.eval(0.5 + 0.5 * s, phiB.data());
    L.deriv(0.5 * s, dA.data());
    L.deriv(0.5 + 0.5 * s, dB.data());
    std::vector<double> phiS(n1);
    L.eval(s, phiS.data());
    for (int p = 0; p < n1; ++p)
      for (int q = 0; q < n1; ++q) {
        at(b->M, p, q) += wk * phiS[p] * phiS[q];
        // R~: right half of the dual cell lies in main cell i+1 (its left half)
        at(b->Rt, p, q) += 0.5 * wk * phiB[p] * dA[q];
        // L~: left half of the dual cell lies in main cell i (its right half)
        at(b->Lt, p, q) -= 0.5 * wk * phiA[p] * dB[q];
        // R-bar / L-bar: main-cell test function, dual-cell unknown
        at(b->Rb, p, q) -= 0.5 * wk * dB[p] * phiA[q];
        at(b->Lb, p, q) += 0.5 * wk * dA[p] * phiB[q];
        at(b->ML, p, q) += 0.5 * wk * phiA[p] * phiB[q];
        at(b->MR, p, q) += 0.5 * wk * phiB[p] * phiA[q];
      }
  }
  // point (jump) terms of Eq. matrices
  for (int p = 0; p < n1; ++p)
    for (int q = 0; q < n1; ++q) {
      at(b->Rt, p, q) += half[p] * zero[q];
      at(b->Lt, p, q) += half[p] * one[q];
      at(b->Rb, p, q) += one[p] * half[q];
      at(b->Lb, p, q) += zero[p] * half[q];
    }
  // H blocks with M^-1 = diag(1/w) (the GL nodal mass matrix is diagonal)
  for (int p = 0; p < n1; ++p)
    for (int q = 0; q < n1; ++q) {
      double hr = 0, hl = 0, hc = 0;
      for (int k = 0; k < n1; ++k) {
        const double iw = 1.0 / b->w[k];
        hr -= at(b->Rb, p, k) * iw * at(b->Rt, k, q);
        hl -= at(b->Lb, p, k) * iw * at(b->Lt, k, q);
        hc += at(b->Rb, p, k) * iw * at(b->Lt, k, q) + at(b->Lb, p, k) * iw * at(b->Rt, k, q);
      }
      at(b->HR, p, q) = hr;
      at(b->HL, p, q) = hl;
      at(b->HC, p, q) = hc;
    }
  // nodal derivative Dn[k][m] = phi_m'(xi_k)
  for (int k = 0; k < n1; ++k)
    for (int m = 0; m < n1; ++m) b->Dn[k * n1 + m] = (n1 == 1) ? 0.0 : L.D[k * n1 + m];
  return 0;
}

namespace {

// Cyclic Jacobi eigen-decomposition of a symmetric n x n matrix A (row-major,
// destroyed); eigenvalues to lam[], eigenvectors to the columns of V.
void jacobi_eig(int n, double* A, double* lam, double* V) {
  for (int i = 0; i < n * n; ++i) V[i] = 0.0;
  for (int i = 0; i < n; ++i) V[i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += A[p * n + q] * A[p * n + q];
    if (off < 1e-300) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double app = A[p * n + p], aqq = A[q * n + q];
        const double tau = (aqq - app) / (2.0 * apq);
        const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        const double c = 1.0 / std::sqrt(1.0 + t * t), sn = t * c;
        for (int k = 0; k < n; ++k) {  // A <- A J (columns p, q)
          const double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - sn * akq;
          A[k * n + q] = sn * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // A <- J^T A (rows p, q)
          const double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - sn * aqk;
          A[q * n + k] = sn * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double vkp = V[k * n + p], vkq = V[k * n + q];
          V[k * n + p] = c * vkp - sn * vkq;
          V[k * n + q] = sn * vkp + c * vkq;
        }
      }
  }
  for (int i = 0; i < n; ++i) lam[i] = A[i * n + i];
}

}  // namespace

namespace {

int kernel_eig(const Basis1D& b, std::vector<double>& V, std::vector<double>& lam, double* tol_out) {
  const int n = b.n1;
  std::vector<double> G(n * n), A(n * n);
  V.assign(n * n, 0.0);
  lam.assign(n, 0.0);
  double scale = 0.0;  // size of R~ and L~ (R~ - L~ itself vanishes for N = 1)
  for (int i = 0; i < n * n; ++i) {
    G[i] = b.Rt[i] - b.Lt[i];
    scale = std::fmax(scale, std::fabs(b.Rt[i]) + std::fabs(b.Lt[i]));
  }
  scale *= scale;
  for (int p = 0; p < n; ++p)
    for (int q = 0; q < n; ++q) {
      double s = 0.0;
      for (int k = 0; k < n; ++k) s += G[k * n + p] * G[k * n + q];
      A[p * n + q] = s;
    }
  jacobi_eig(n, A.data(), lam.data(), V.data());
  *tol_out = 1e-12 * (scale > 0 ? scale : 1.0);
  return n;
}

}  // namespace

int kernel_basis(const Basis1D& b, double* basis) {
  const int n = b.n1;
  std::vector<double> V, lam;
  double tol;
  kernel_eig(b, V, lam, &tol);
  int dim = 0;
  for (int j = 0; j < n; ++j) {
    if (std::fabs(lam[j]) > tol) continue;
    for (int l = 0; l < n; ++l) basis[dim * n + l] = V[l * n + j];
    ++dim;
  }
  return dim;
}

int kernel_projector(const Basis1D& b, double* proj) {
  const int n = b.n1;
  double basis[kMaxN1 * kMaxN1];
  const int dim = kernel_basis(b, basis);
  for (int p = 0; p < n; ++p)
    for (int q = 0; q < n; ++q) {
      double s = 0.0;
      for (int j = 0; j < dim; ++j) s += basis[j * n + p] * basis[j * n + q];
      proj[p * n + q] = s;
    }
  return dim;
}

void build_coefs(const Basis1D& b, int fp32, CoefSet* c) {
  const int n = b.n1;
  auto rnd = [fp32](double v) { return fp32 ? (double)(float)v : v; };
  for (int i = 0; i < kMaxN1 * kMaxN1; ++i) c->HL[i] = c->HC[i] = c->HR[i] = c->C[i] = 0.0;
  for (int i = 0; i < kMaxN1; ++i) c->rho[i] = c->z[i] = c->zn[i] = 0.0;
  for (int m = 0; m < n; ++m)
    for (int k = 0; k < n; ++k) {
      c->HR[m * n + k] = rnd(b.HR[m * n + k]);
      c->HL[m * n + k] = rnd(b.HR[k * n + m]);
      c->HC[m * n + k] = rnd(0.5 * (b.HC[m * n + k] + b.HC[k * n + m]));
    }
  std::vector<double> G(n * n);
  for (int i = 0; i < n * n; ++i) G[i] = c->HL[i] + c->HC[i] + c->HR[i];
  for (int m = 0; m < n; ++m) {
    long double rs = 0.0L;
    for (int k = 0; k < n; ++k) rs += (long double)c->HL[m * n + k] + (long double)c->HC[m * n + k] +
                                      (long double)c->HR[m * n + k];
    c->rho[m] = rnd((double)rs);
  }
  double kb[kMaxN1 * kMaxN1];
  const int kd = kernel_basis(b, kb);
  c->kz = kd >= 2 ? 1 : 0;
  if (!c->kz) return;
  // z: the kernel direction orthogonal to the constants, scaled to max 1
  double best = -1.0;
  std::vector<double> z(n);
  for (int j = 0; j < kd; ++j) {
    double mean = 0.0;
    for (int l = 0; l < n; ++l) mean += kb[j * n + l];
    mean /= n;
    double nrm = 0.0;
    for (int l = 0; l < n; ++l) nrm += (kb[j * n + l] - mean) * (kb[j * n + l] - mean);
    if (nrm > best) {
      best = nrm;
      for (int l = 0; l < n; ++l) z[l] = kb[j * n + l] - mean;
    }
  }
  double zmax = 0.0;
  for (int l = 0; l < n; ++l) zmax = std::fmax(zmax, std::fabs(z[l]));
  double zz = 0.0;
  for (int l = 0; l < n; ++l) {
    c->z[l] = rnd(z[l] / zmax);
    zz += c->z[l] * c->z[l];
  }
  for (int l = 0; l < n; ++l) c->zn[l] = rnd(c->z[l] / zz);
  // orthonormal K = [k0, k1] spanning {1, z_stored} (Gram-Schmidt in FP64)
  std::vector<double> k0(n, 1.0 / std::sqrt((double)n)), k1(n);
  double d = 0.0;
  for (int l = 0; l < n; ++l) d += k0[l] * c->z[l];
  double nn = 0.0;
  for (int l = 0; l < n; ++l) { k1[l] = c->z[l] - d * k0[l]; nn += k1[l] * k1[l]; }
  nn = std::sqrt(nn);
  for (int l = 0; l < n; ++l) k1[l] /= nn;
  // S = G K; C = -(S K^T + K S^T - K (K^T S) K^T)
  std::vector<double> S0(n), S1(n);
  for (int m = 0; m < n; ++m) {
    double a = 0.0, bb = 0.0;
    for (int k = 0; k < n; ++k) { a += G[m * n + k] * k0[k]; bb += G[m * n + k] * k1[k]; }
    S0[m] = a;
    S1[m] = bb;
  }
  double KS[2][2] = {{0, 0}, {0, 0}};
  for (int l = 0; l < n; ++l) {
    KS[0][0] += k0[l] * S0[l]; KS[0][1] += k0[l] * S1[l];
    KS[1][0] += k1[l] * S0[l]; KS[1][1] += k1[l] * S1[l];
  }
  for (int p = 0; p < n; ++p)
    for (int q = 0; q < n; ++q) {
      const double skt = S0[p] * k0[q] + S1[p] * k1[q];
      const double kst = k0[p] * S0[q] + k1[p] * S1[q];
      const double kk = k0[p] * (KS[0][0] * k0[q] + KS[0][1] * k1[q]) + k1[p] * (KS[1][0] * k0[q] + KS[1][1] * k1[q]);
      c->C[p * n + q] = -(skt + kst - kk);
    }
  for (int p = 0; p < n; ++p)
    for (int q = p + 1; q < n; ++q) {
      const double v = rnd(0.5 * (c->C[p * n + q] + c->C[q * n + p]));
      c->C[p * n + q] = c->C[q * n + p] = v;
    }
  for (int p = 0; p < n; ++p) c->C[p * n + p] = rnd(c->C[p * n + p]);
}

}  // namespace sdg
