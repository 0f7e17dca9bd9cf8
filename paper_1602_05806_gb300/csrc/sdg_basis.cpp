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

namespace {

using LD = long double;

// Row-major n x n helpers in long double.
struct Mat {
  int n;
  LD v[kMaxN1 * kMaxN1];
  LD& at(int i, int j) { return v[i * n + j]; }
  LD at(int i, int j) const { return v[i * n + j]; }
};

Mat mat_zero(int n) {
  Mat m;
  m.n = n;
  for (int i = 0; i < n * n; ++i) m.v[i] = 0.0L;
  return m;
}

Mat mat_mul(const Mat& a, const Mat& b) {
  Mat c = mat_zero(a.n);
  for (int i = 0; i < a.n; ++i)
    for (int j = 0; j < a.n; ++j) {
      LD s = 0.0L;
      for (int k = 0; k < a.n; ++k) s += a.at(i, k) * b.at(k, j);
      c.at(i, j) = s;
    }
  return c;
}

Mat mat_t(const Mat& a) {
  Mat c = mat_zero(a.n);
  for (int i = 0; i < a.n; ++i)
    for (int j = 0; j < a.n; ++j) c.at(i, j) = a.at(j, i);
  return c;
}

// P (even/odd transform, rows: even part, middle, odd part) and Q = G^-1 P.
void eo_transforms(int n, Mat& P, Mat& Q) {
  const int h = n / 2, hE = (n + 1) / 2;
  P = mat_zero(n);
  Q = mat_zero(n);
  for (int k = 0; k < h; ++k) {
    P.at(k, k) = 1.0L;
    P.at(k, n - 1 - k) = 1.0L;
    P.at(hE + k, k) = 1.0L;
    P.at(hE + k, n - 1 - k) = -1.0L;
  }
  if (n % 2) P.at(h, h) = 1.0L;
  for (int i = 0; i < n; ++i) {
    const LD g = (n % 2 && i == h) ? 1.0L : 2.0L;
    for (int j = 0; j < n; ++j) Q.at(i, j) = P.at(i, j) / g;
  }
}

// Stored e/o blocks -> natural-basis H^L, H^C, H^R (long double).
void effective_blocks(const CoefSet& c, Mat& HL, Mat& HC, Mat& HR) {
  const int n = c.n, h = c.h, hE = c.hE;
  Mat P, Q;
  eo_transforms(n, P, Q);
  Mat R = mat_zero(n), L = mat_zero(n), C = mat_zero(n);
  for (int i = 0; i < hE; ++i)
    for (int j = 0; j < hE; ++j) {
      R.at(i, j) = L.at(i, j) = c.A[i * hE + j];
      C.at(i, j) = c.CE[i * hE + j];
    }
  for (int i = 0; i < hE; ++i)
    for (int j = 0; j < h; ++j) {
      const LD bij = c.B[i * h + j];
      R.at(i, hE + j) = bij;
      L.at(i, hE + j) = -bij;
      R.at(hE + j, i) = -bij;
      L.at(hE + j, i) = bij;
    }
  for (int i = 0; i < h; ++i)
    for (int j = 0; j < h; ++j) {
      R.at(hE + i, hE + j) = L.at(hE + i, hE + j) = c.D[i * h + j];
      C.at(hE + i, hE + j) = c.CO[i * h + j];
    }
  const Mat Pt = mat_t(P);
  HR = mat_mul(Pt, mat_mul(R, P));
  HL = mat_mul(Pt, mat_mul(L, P));
  HC = mat_mul(Pt, mat_mul(C, P));
}

}  // namespace

void build_coefs(const Basis1D& b, int fp32, CoefSet* c) {
  const int n = b.n1, h = n / 2, hE = (n + 1) / 2;
  auto rnd = [fp32](LD v) { return fp32 ? (double)(float)v : (double)v; };
  *c = CoefSet{};
  c->n = n;
  c->h = h;
  c->hE = hE;
  Mat P, Q;
  eo_transforms(n, P, Q);
  Mat HR = mat_zero(n), HC = mat_zero(n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      HR.at(i, j) = b.HR[i * n + j];
      HC.at(i, j) = 0.5L * ((LD)b.HC[i * n + j] + (LD)b.HC[j * n + i]);
    }
  const Mat Qt = mat_t(Q);
  const Mat R = mat_mul(Q, mat_mul(HR, Qt));  // [[A, B], [-B^T, D]] up to rounding
  const Mat C = mat_mul(Q, mat_mul(HC, Qt));  // diag(CE, CO) up to rounding
  for (int i = 0; i < hE; ++i)
    for (int j = 0; j < hE; ++j) {
      c->A[i * hE + j] = rnd(0.5L * (R.at(i, j) + R.at(j, i)));
      c->CE[i * hE + j] = rnd(0.5L * (C.at(i, j) + C.at(j, i)));
    }
  for (int i = 0; i < hE; ++i)
    for (int j = 0; j < h; ++j) c->B[i * h + j] = rnd(0.5L * (R.at(i, hE + j) - R.at(hE + j, i)));
  for (int i = 0; i < h; ++i)
    for (int j = 0; j < h; ++j) {
      c->D[i * h + j] = rnd(0.5L * (R.at(hE + i, hE + j) + R.at(hE + j, hE + i)));
      c->CO[i * h + j] = rnd(0.5L * (C.at(hE + i, hE + j) + C.at(hE + j, hE + i)));
    }
  // line sum of the stored operator in the natural basis
  Mat EL, EC, ER;
  effective_blocks(*c, EL, EC, ER);
  Mat G = mat_zero(n);
  for (int i = 0; i < n * n; ++i) G.v[i] = EL.v[i] + EC.v[i] + ER.v[i];
  double kb[kMaxN1 * kMaxN1];
  const int kd = kernel_basis(b, kb);
  c->kz = kd >= 2 ? 1 : 0;
  if (!c->kz) {
    // rho = G 1, made exactly symmetric under the reversal
    LD rho[kMaxN1];
    for (int i = 0; i < n; ++i) {
      LD s = 0.0L;
      for (int j = 0; j < n; ++j) s += G.at(i, j);
      rho[i] = s;
    }
    for (int k = 0; k < h; ++k) {
      const LD r = 0.5L * (rho[k] + rho[n - 1 - k]);
      c->rho_e[k] = rnd(0.5L * r);
      c->rho_o[k] = rnd(0.5L * r);
    }
    if (n % 2) c->rho_e[h] = rnd(rho[h]);
    return;
  }
  // odd N: z = the kernel direction orthogonal to the constants, made
  // exactly antisymmetric, max |z| = 1
  double best = -1.0;
  std::vector<LD> z(n, 0.0L);
  for (int j = 0; j < kd; ++j) {
    LD mean = 0.0L;
    for (int l = 0; l < n; ++l) mean += kb[j * n + l];
    mean /= n;
    LD nrm = 0.0L;
    for (int l = 0; l < n; ++l) nrm += (kb[j * n + l] - mean) * (kb[j * n + l] - mean);
    if ((double)nrm > best) {
      best = (double)nrm;
      for (int l = 0; l < n; ++l) z[l] = kb[j * n + l] - mean;
    }
  }
  LD zmax = 0.0L;
  for (int k = 0; k < h; ++k) {
    const LD a = 0.5L * (z[k] - z[n - 1 - k]);
    z[k] = a;
    z[n - 1 - k] = -a;
    zmax = std::fmax((double)zmax, std::fabs((double)a));
  }
  LD zz = 0.0L;
  for (int k = 0; k < h; ++k) {
    const double zk = rnd(z[k] / zmax);
    z[k] = zk;
    z[n - 1 - k] = -zk;
    zz += 2.0L * (LD)zk * (LD)zk;
  }
  for (int k = 0; k < h; ++k) {
    c->z2[k] = 2.0 * (double)z[k];  // exact
    c->zn[k] = rnd(z[k] / zz);
  }
  // orthonormal kernel basis k0 = 1/sqrt(n), k1 = z/|z|; S = G [k0, k1]
  const LD k0 = 1.0L / std::sqrt((LD)n), znorm = std::sqrt(zz);
  LD S0[kMaxN1], S1[kMaxN1];
  for (int i = 0; i < n; ++i) {
    LD a = 0.0L, bb = 0.0L;
    for (int j = 0; j < n; ++j) {
      a += G.at(i, j) * k0;
      bb += G.at(i, j) * (z[j] / znorm);
    }
    S0[i] = a;
    S1[i] = bb;
  }
  for (int k = 0; k < h; ++k) {
    c->S0[k] = rnd(0.5L * (S0[k] + S0[n - 1 - k]));
    c->S1[k] = rnd(0.5L * (S1[k] - S1[n - 1 - k]));
    c->k1[k] = rnd(z[k] / znorm);
  }
  c->k0 = rnd(k0);
  c->inv_n = rnd(1.0L / n);
}

void line_operator(const CoefSet& c, double* HLo, double* Mco, double* HRo) {
  const int n = c.n, h = c.h, hE = c.hE;
  Mat EL, EC, ER;
  effective_blocks(c, EL, EC, ER);
  Mat P, Q;
  eo_transforms(n, P, Q);
  for (int j = 0; j < n; ++j) {
    // centre line e_j: fit, shifted line, correction (as the kernel does)
    LD x[kMaxN1], q[kMaxN1];
    for (int i = 0; i < n; ++i) { x[i] = (i == j) ? 1.0L : 0.0L; q[i] = 0.0L; }
    LD xE[kMaxHalf], xO[kMaxHalf];
    for (int k = 0; k < h; ++k) { xE[k] = x[k] + x[n - 1 - k]; xO[k] = x[k] - x[n - 1 - k]; }
    if (n % 2) xE[h] = x[h];
    LD yE[kMaxHalf] = {0}, yO[kMaxHalf] = {0};
    if (c.kz) {
      LD sum = 0.0L, dz = 0.0L;
      for (int k = 0; k < h; ++k) { sum += xE[k]; dz += (LD)c.zn[k] * xO[k]; }
      const LD mu = sum * (LD)c.inv_n;
      for (int k = 0; k < h; ++k) {
        q[k] = mu + dz * 0.5L * (LD)c.z2[k];
        q[n - 1 - k] = mu - dz * 0.5L * (LD)c.z2[k];
        xE[k] -= 2.0L * mu;
        xO[k] -= dz * (LD)c.z2[k];
      }
      LD al = 0.0L, be = 0.0L;
      for (int k = 0; k < h; ++k) { al += (LD)c.S0[k] * xE[k]; be += (LD)c.S1[k] * xO[k]; }
      for (int k = 0; k < h; ++k) { yE[k] = -al * (LD)c.k0; yO[k] = -be * (LD)c.k1[k]; }
    } else {
      for (int k = 0; k < hE; ++k) yE[k] = -(LD)c.rho_e[k] * xE[k];
      for (int k = 0; k < h; ++k) yO[k] = -(LD)c.rho_o[k] * xO[k];
    }
    for (int i = 0; i < n; ++i) {
      LD s = 0.0L;
      for (int k = 0; k < n; ++k) s += EC.at(i, k) * (x[k] - q[k]) - (EL.at(i, k) + ER.at(i, k)) * q[k];
      // correction back to the natural basis
      LD corr;
      if (i < h) corr = yE[i] + yO[i];
      else if (n % 2 && i == h) corr = yE[h];
      else corr = yE[n - 1 - i] - yO[n - 1 - i];
      Mco[i * n + j] = (double)(s + corr);
    }
  }
  for (int i = 0; i < n * n; ++i) {
    HLo[i] = (double)EL.v[i];
    HRo[i] = (double)ER.v[i];
  }
}

}  // namespace sdg
