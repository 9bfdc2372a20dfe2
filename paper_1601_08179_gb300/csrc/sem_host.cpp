// Host-side 1D setup of the condensed spectral-element operator.
//
// Sec. 3: nodal Lagrange basis on the p+1 Gauss-Lobatto-Legendre (GLL) points;
//   lumped mass M = diag(w); stiffness K_ij = int phi_i' phi_j' = (D^T W D)_ij,
//   exact because the integrand has degree 2p-2.
// Sec. 5, Eq. generalized_eigenvalues: S_II M_II S_II^T = I,
//   S_II K_II S_II^T = Lambda.  M_II is diagonal, so the generalised problem is
//   the standard symmetric problem of C = W^-1/2 K_II W^-1/2 = Q Lambda Q^T,
//   solved here by cyclic Jacobi rotations; V = W^-1/2 Q, S_II = V^T.
// Sec. 6: transformed stiffness K~ = S K S^T with S = diag(1, S_II, 1): the
//   interior block is Lambda, the border vectors are K~_{I0} = S_II K_{I0} and
//   K~_{Ip} = S_II K_{Ip}; the corners equal those of K.
#include <cmath>
#include <cstdio>
#include <string>
#include <vector>

#include "sem_internal.h"

namespace {

// P_p(x) and P_p'(x) from the Legendre three-term recurrence.
void legendre_pd(int p, double x, double* P, double* dP) {
  double p0 = 1.0, p1 = x;
  if (p == 0) { *P = 1.0; *dP = 0.0; return; }
  for (int k = 1; k < p; ++k) {
    double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
    p0 = p1;
    p1 = p2;
  }
  *P = p1;
  // P_p' = p (x P_p - P_{p-1}) / (x^2 - 1), valid for |x| < 1
  *dP = (std::fabs(x) < 1.0) ? p * (x * p1 - p0) / (x * x - 1.0) : 0.5 * p * (p + 1.0) * (x > 0 ? 1.0 : (p % 2 ? 1.0 : -1.0));
}

// Interior GLL points: roots of P_p'.  Newton from the Chebyshev-Lobatto points,
// with P_p'' from Legendre's equation (1-x^2) P'' = 2x P' - p(p+1) P.
bool gll_points(int p, std::vector<double>* x, std::vector<double>* w) {
  const double pi = 3.14159265358979323846;
  x->assign(p + 1, 0.0);
  w->assign(p + 1, 0.0);
  (*x)[0] = -1.0;
  (*x)[p] = 1.0;
  for (int i = 1; i < p; ++i) {
    double t = -std::cos(pi * i / p);
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre_pd(p, t, &P, &dP);
      double ddP = (2.0 * t * dP - p * (p + 1.0) * P) / (1.0 - t * t);
      double step = dP / ddP;
      t -= step;
      if (std::fabs(step) < 1e-16) break;
    }
    (*x)[i] = t;
  }
  // symmetrise: the points are symmetric about 0
  for (int i = 1; i < p; ++i) {
    double s = 0.5 * ((*x)[i] - (*x)[p - i]);
    (*x)[i] = s;
    (*x)[p - i] = -s;
  }
  if (p % 2 == 0) (*x)[p / 2] = 0.0;
  for (int i = 0; i <= p; ++i) {
    double P, dP;
    legendre_pd(p, (*x)[i], &P, &dP);
    (*w)[i] = 2.0 / (p * (p + 1.0) * P * P);
  }
  for (int i = 1; i <= p; ++i)
    if (!((*x)[i] > (*x)[i - 1])) return false;
  return true;
}

// Lagrange differentiation matrix D_ij = phi_j'(x_i) from barycentric weights;
// the diagonal makes every row sum to zero (derivative of a constant).
std::vector<double> diff_matrix(const std::vector<double>& x) {
  const int q = (int)x.size();
  std::vector<double> bw(q, 1.0), D(q * q, 0.0);
  for (int j = 0; j < q; ++j)
    for (int m = 0; m < q; ++m)
      if (m != j) bw[j] *= (x[j] - x[m]);
  for (int j = 0; j < q; ++j) bw[j] = 1.0 / bw[j];
  for (int i = 0; i < q; ++i) {
    double s = 0.0;
    for (int j = 0; j < q; ++j) {
      if (j == i) continue;
      D[i * q + j] = (bw[j] / bw[i]) / (x[i] - x[j]);
      s += D[i * q + j];
    }
    D[i * q + i] = -s;
  }
  return D;
}

// Cyclic Jacobi eigenvalue iteration for a symmetric n x n matrix A (row-major,
// destroyed).  Returns eigenvalues in lam and eigenvectors as columns of Q.
void jacobi_eig(int n, std::vector<double> A, std::vector<double>* lam, std::vector<double>* Q) {
  Q->assign(n * n, 0.0);
  for (int i = 0; i < n; ++i) (*Q)[i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        tot += A[i * n + j] * A[i * n + j];
        if (i != j) off += A[i * n + j] * A[i * n + j];
      }
    if (off <= 1e-32 * tot) break;
    for (int r = 0; r < n - 1; ++r)
      for (int c = r + 1; c < n; ++c) {
        double arc = A[r * n + c];
        if (arc == 0.0) continue;
        double theta = (A[c * n + c] - A[r * n + r]) / (2.0 * arc);
        double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double cs = 1.0 / std::sqrt(t * t + 1.0), sn = t * cs;
        for (int k = 0; k < n; ++k) {   // A <- J^T A J, columns r and c
          double akr = A[k * n + r], akc = A[k * n + c];
          A[k * n + r] = cs * akr - sn * akc;
          A[k * n + c] = sn * akr + cs * akc;
        }
        for (int k = 0; k < n; ++k) {   // rows r and c
          double ark = A[r * n + k], ack = A[c * n + k];
          A[r * n + k] = cs * ark - sn * ack;
          A[c * n + k] = sn * ark + cs * ack;
        }
        for (int k = 0; k < n; ++k) {
          double qkr = (*Q)[k * n + r], qkc = (*Q)[k * n + c];
          (*Q)[k * n + r] = cs * qkr - sn * qkc;
          (*Q)[k * n + c] = sn * qkr + cs * qkc;
        }
      }
  }
  lam->resize(n);
  for (int i = 0; i < n; ++i) (*lam)[i] = A[i * n + i];
}

}  // namespace

bool sem_build_1d(int p, SemHost1D* out, std::string* err) {
  if (p < 2 || p > SEM_MAXN + 1) { *err = "p must be in [2, 32]"; return false; }
  const int q = p + 1, n = p - 1;
  out->p = p;
  if (!gll_points(p, &out->x, &out->w)) { *err = "GLL Newton iteration failed"; return false; }
  std::vector<double> D = diff_matrix(out->x);
  out->K.assign(q * q, 0.0);
  for (int i = 0; i < q; ++i)
    for (int j = 0; j < q; ++j) {
      double s = 0.0;
      for (int m = 0; m < q; ++m) s += D[m * q + i] * out->w[m] * D[m * q + j];
      out->K[i * q + j] = s;
    }
  for (int i = 0; i < q; ++i)     // exact symmetry
    for (int j = i + 1; j < q; ++j) {
      double s = 0.5 * (out->K[i * q + j] + out->K[j * q + i]);
      out->K[i * q + j] = out->K[j * q + i] = s;
    }
  // C = W^-1/2 K_II W^-1/2
  std::vector<double> C(n * n), rs(n);
  for (int i = 0; i < n; ++i) rs[i] = 1.0 / std::sqrt(out->w[i + 1]);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) C[i * n + j] = rs[i] * out->K[(i + 1) * q + (j + 1)] * rs[j];
  std::vector<double> lam, Q;
  jacobi_eig(n, C, &lam, &Q);
  // sort ascending
  std::vector<int> ord(n);
  for (int i = 0; i < n; ++i) ord[i] = i;
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j)
      if (lam[ord[j]] < lam[ord[i]]) { int t = ord[i]; ord[i] = ord[j]; ord[j] = t; }
  out->lam.resize(n);
  out->V.assign(n * n, 0.0);
  for (int c = 0; c < n; ++c) {
    int src = ord[c];
    out->lam[c] = lam[src];
    double sgn = (rs[0] * Q[0 * n + src] >= 0.0) ? 1.0 : -1.0;   // first entry positive
    for (int r = 0; r < n; ++r) out->V[r * n + c] = sgn * rs[r] * Q[r * n + src];
  }
  // transformed 1D operator
  SemBasis& b = out->basis;
  b.n = n;
  b.w0 = out->w[0];
  b.K[0][0] = out->K[0];
  b.K[0][1] = out->K[p];
  b.K[1][0] = out->K[p * q];
  b.K[1][1] = out->K[p * q + p];
  for (int i = 0; i < SEM_MAXN; ++i) { b.lam[i] = 0; b.k[0][i] = 0; b.k[1][i] = 0; }
  for (int i = 0; i < n; ++i) {
    b.lam[i] = out->lam[i];
    double s0 = 0.0, sp = 0.0;   // (V^T K_{I0})_i, (V^T K_{Ip})_i
    for (int r = 0; r < n; ++r) {
      s0 += out->V[r * n + i] * out->K[(r + 1) * q + 0];
      sp += out->V[r * n + i] * out->K[(r + 1) * q + p];
    }
    b.k[0][i] = s0;
    b.k[1][i] = sp;
  }
  return true;
}
