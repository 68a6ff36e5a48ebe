// Host-side set-up: GLL nodes, 1-D operator blocks, patch eigen-tables,
// interpolation matrices.  Runs once in pmg_hierarchy_build; nothing here is
// on the per-iteration path.
//
// Paper: Stiller, arXiv 1603.02524.  Sec. 2.4 (nodal operators), Eq.
// (L:generic) (block-tridiagonal global 1-D stiffness), Sec. 3.1 (subdomains,
// fast diagonalisation, weights), Sec. 3.2 (embedded interpolation).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <stdexcept>

#include "pmg_internal.h"

namespace pmg {

// Legendre polynomial L_P and its derivatives at x (three-term recurrence).
static void legendre(int P, double x, double& Lp, double& dLp, double& d2Lp) {
  double l0 = 1.0, l1 = x;
  if (P == 0) {
    Lp = 1.0; dLp = 0.0; d2Lp = 0.0;
    return;
  }
  for (int n = 1; n < P; ++n) {
    double l2 = ((2.0 * n + 1.0) * x * l1 - n * l0) / (n + 1.0);
    l0 = l1;
    l1 = l2;
  }
  Lp = l1;
  // derivative from (1 - x^2) L_P' = P (L_{P-1} - x L_P); away from +-1 only
  double one_m = 1.0 - x * x;
  dLp = P * (l0 - x * l1) / one_m;
  // Legendre ODE: (1 - x^2) L'' - 2 x L' + P (P+1) L = 0
  d2Lp = (2.0 * x * dLp - P * (P + 1.0) * Lp) / one_m;
}

// GLL nodes: -1, the roots of L_P' (Newton from Chebyshev-Gauss-Lobatto
// guesses), +1; weights rho_i = 2 / (P (P+1) L_P(eta_i)^2).
void gll_nodes(int P, std::vector<double>& eta, std::vector<double>& rho) {
  eta.assign(P + 1, 0.0);
  rho.assign(P + 1, 0.0);
  eta[0] = -1.0;
  eta[P] = 1.0;
  for (int i = 1; i < P; ++i) {
    double x = -std::cos(M_PI * i / P);
    for (int it = 0; it < 100; ++it) {
      double L, dL, d2L;
      legendre(P, x, L, dL, d2L);
      double dx = dL / d2L;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    eta[i] = x;
  }
  // exact symmetry of the node set
  for (int i = 0; i <= P / 2; ++i) {
    double a = 0.5 * (eta[P - i] - eta[i]);
    eta[i] = -a;
    eta[P - i] = a;
  }
  if (P % 2 == 0) eta[P / 2] = 0.0;
  for (int i = 0; i <= P; ++i) {
    double L, dL, d2L;
    double x = eta[i];
    // L_P(+-1) = (+-1)^P; otherwise use the recurrence value
    if (i == 0 || i == P) {
      L = (i == 0 && (P % 2)) ? -1.0 : 1.0;
    } else {
      legendre(P, x, L, dL, d2L);
    }
    rho[i] = 2.0 / (P * (P + 1.0) * L * L);
  }
}

// Classical GLL differentiation matrix D_ik = phi_k'(eta_i):
// L_P(eta_i) / (L_P(eta_k) (eta_i - eta_k)) off the diagonal,
// -P(P+1)/4 and P(P+1)/4 at the two corners, 0 elsewhere on the diagonal.
static void gll_diff(int P, const std::vector<double>& eta, std::vector<double>& D) {
  int NP = P + 1;
  std::vector<double> L(NP);
  for (int i = 0; i < NP; ++i) {
    if (i == 0) {
      L[i] = (P % 2) ? -1.0 : 1.0;
    } else if (i == P) {
      L[i] = 1.0;
    } else {
      double dL, d2L;
      legendre(P, eta[i], L[i], dL, d2L);
    }
  }
  D.assign(NP * NP, 0.0);
  for (int i = 0; i < NP; ++i)
    for (int k = 0; k < NP; ++k)
      if (i != k) D[i * NP + k] = L[i] / (L[k] * (eta[i] - eta[k]));
  D[0] = -P * (P + 1.0) / 4.0;
  D[P * NP + P] = P * (P + 1.0) / 4.0;
}

// Barycentric Lagrange interpolation matrix B[i][k] = phi_k(x_i) (nodes -> x).
void lagrange_matrix(const std::vector<double>& nodes, const std::vector<double>& x,
                     std::vector<double>& B) {
  int n = (int)nodes.size(), m = (int)x.size();
  std::vector<double> bw(n, 1.0);
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j)
      if (j != k) bw[k] /= (nodes[k] - nodes[j]);
  B.assign((size_t)m * n, 0.0);
  for (int i = 0; i < m; ++i) {
    int hit = -1;
    for (int k = 0; k < n; ++k)
      if (x[i] == nodes[k]) hit = k;
    if (hit >= 0) {
      B[(size_t)i * n + hit] = 1.0;
      continue;
    }
    double den = 0.0;
    for (int k = 0; k < n; ++k) den += bw[k] / (x[i] - nodes[k]);
    for (int k = 0; k < n; ++k) B[(size_t)i * n + k] = bw[k] / (x[i] - nodes[k]) / den;
  }
}

// Global 1-D operator blocks of one axis (Eq. L:generic, with the Delta x^m
// reading of the first L^-/L^+ terms and the Dirichlet ghost fold-in).
void build_axis(Axis1DHost& a, int P, const std::vector<double>& dx, bool periodic, double beta,
                double mu_star) {
  a.P = P;
  a.NP = P + 1;
  a.Ne = (int)dx.size();
  a.periodic = periodic;
  a.beta = beta;
  a.mu_star = mu_star;
  a.dx = dx;
  gll_nodes(P, a.eta, a.rho);
  gll_diff(P, a.eta, a.D);
  const int NP = a.NP, Ne = a.Ne;
  const auto& D = a.D;
  const auto& rho = a.rho;
  a.Ls.assign(NP * NP, 0.0);
  for (int i = 0; i < NP; ++i)
    for (int k = 0; k < NP; ++k) {
      double s = 0.0;
      for (int j = 0; j < NP; ++j) s += rho[j] * D[j * NP + i] * D[j * NP + k];
      a.Ls[i * NP + k] = s;
    }
  a.L0.assign((size_t)Ne * NP * NP, 0.0);
  a.Lm.assign((size_t)Ne * NP * NP, 0.0);
  a.Lp.assign((size_t)Ne * NP * NP, 0.0);
  a.M.assign((size_t)Ne * NP, 0.0);
  a.cpl.assign((size_t)Ne * 8, 0.0);
  auto width = [&](int m) {
    if (m >= 0 && m < Ne) return dx[m];
    if (periodic) return dx[((m % Ne) + Ne) % Ne];
    return m < 0 ? dx[0] : dx[Ne - 1];   // ghost element: mirrored width
  };
  auto wall = [&](int left_elem) {       // is the face (left_elem | left_elem+1) a wall?
    return !periodic && (left_elem < 0 || left_elem >= Ne - 1);
  };
  // bracket of Eq. (flux:num:sigma) on the face between elements l and l+1
  auto bracket = [&](int l) {
    double b = wall(l) ? 0.0 : beta;
    double ha = width(l), hb = width(l + 1);
    double mu0 = 1.0 / (2.0 * ha * rho[P]) + 1.0 / (2.0 * hb * rho[0]);
    return 2.0 * (b * b + b) / (ha * rho[P]) + 2.0 * (b * b - b) / (hb * rho[0]) +
           mu0 * (1.0 + mu_star);
  };
  for (int m = 0; m < Ne; ++m) {
    const double h = dx[m], hl = width(m - 1), hr = width(m + 1);
    const double bl = wall(m - 1) ? 0.0 : beta;
    const double br = wall(m) ? 0.0 : beta;
    const double cl = bracket(m - 1), cr = bracket(m);
    double* L0 = &a.L0[(size_t)m * NP * NP];
    double* Lm = &a.Lm[(size_t)m * NP * NP];
    double* Lp = &a.Lp[(size_t)m * NP * NP];
    for (int i = 0; i < NP; ++i)
      for (int k = 0; k < NP; ++k) {
        double v = 2.0 / h * a.Ls[i * NP + k];
        if (k == 0) v += (1 - 2 * bl) / h * D[0 * NP + i];
        if (i == 0) v += (1 - 2 * bl) / h * D[0 * NP + k];
        if (i == 0 && k == 0) v += cl;
        if (k == P) v -= (1 + 2 * br) / h * D[P * NP + i];
        if (i == P) v -= (1 + 2 * br) / h * D[P * NP + k];
        if (i == P && k == P) v += cr;
        L0[i * NP + k] = v;
        double vm = 0.0, vp = 0.0;
        if (k == P) vm -= (1 - 2 * bl) / h * D[0 * NP + i];
        if (i == 0) vm += (1 + 2 * bl) / hl * D[P * NP + k];
        if (i == 0 && k == P) vm -= cl;
        if (k == 0) vp += (1 + 2 * br) / h * D[P * NP + i];
        if (i == P) vp -= (1 - 2 * br) / hr * D[0 * NP + k];
        if (i == P && k == 0) vp -= cr;
        Lm[i * NP + k] = vm;
        Lp[i * NP + k] = vp;
      }
    double* c = &a.cpl[(size_t)m * 8];
    c[0] = (1 - 2 * bl) / h; c[1] = (1 + 2 * bl) / hl; c[2] = cl; c[3] = 1.0;
    c[4] = (1 + 2 * br) / h; c[5] = (1 - 2 * br) / hr; c[6] = cr; c[7] = 1.0;
    // Dirichlet walls (reading C2): the ghost element holds u_ghost,k = -u_{P-k};
    // fold L^- (resp. L^+) applied to the ghost into L0 and drop the coupling.
    if (!periodic && m == 0) {
      for (int i = 0; i < NP; ++i)
        for (int k = 0; k < NP; ++k) L0[i * NP + k] -= Lm[i * NP + (P - k)];
      std::fill(Lm, Lm + NP * NP, 0.0);
      c[0] = c[1] = c[2] = c[3] = 0.0;
    }
    if (!periodic && m == Ne - 1) {
      for (int i = 0; i < NP; ++i)
        for (int k = 0; k < NP; ++k) L0[i * NP + k] -= Lp[i * NP + (P - k)];
      std::fill(Lp, Lp + NP * NP, 0.0);
      c[4] = c[5] = c[6] = c[7] = 0.0;
    }
    for (int i = 0; i < NP; ++i) a.M[(size_t)m * NP + i] = 0.5 * h * rho[i];
  }
}

double Axis1DHost::entry(int I, int J) const {
  int ma = I / NP, ia = I % NP, mb = J / NP, jb = J % NP;
  double v = 0.0;
  for (int r = -1; r <= 1; ++r) {
    int mm = ma + r;
    if (periodic) {
      mm = ((mm % Ne) + Ne) % Ne;
    } else if (mm < 0 || mm >= Ne) {
      continue;
    }
    if (mm != mb) continue;
    const std::vector<double>& B = (r == -1) ? Lm : (r == 0 ? L0 : Lp);
    v += B[(size_t)ma * NP * NP + ia * NP + jb];
  }
  return v;
}

// Cyclic Jacobi eigen-solver for a symmetric n x n matrix A (row-major,
// destroyed).  V receives the eigenvectors as columns, lam the eigenvalues
// (ascending).  Returns the number of sweeps, -1 if not converged.
int sym_eig_jacobi(int n, std::vector<double>& A, std::vector<double>& V, std::vector<double>& lam) {
  V.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  double fro = 0.0;
  for (double x : A) fro += x * x;
  fro = std::sqrt(fro);
  int sweep = 0;
  double off = 0.0;
  for (; sweep < 60; ++sweep) {
    off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += A[(size_t)p * n + q] * A[(size_t)p * n + q];
    if (std::sqrt(off) <= 1e-16 * fro || off == 0.0) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        double apq = A[(size_t)p * n + q];
        if (apq == 0.0) continue;
        double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
        // rotation angle that annihilates a_pq: tan(2 theta) = 2 a_pq / (a_qq - a_pp)
        double theta = (aqq - app) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {        // columns p, q of A
          double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
          A[(size_t)k * n + p] = c * akp - s * akq;
          A[(size_t)k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {        // rows p, q of A
          double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
          A[(size_t)p * n + k] = c * apk - s * aqk;
          A[(size_t)q * n + k] = s * apk + c * aqk;
        }
        A[(size_t)p * n + q] = 0.0;
        A[(size_t)q * n + p] = 0.0;
        for (int k = 0; k < n; ++k) {        // accumulate V = V J
          double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
          V[(size_t)k * n + p] = c * vkp - s * vkq;
          V[(size_t)k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  lam.resize(n);
  for (int i = 0; i < n; ++i) lam[i] = A[(size_t)i * n + i];
  // sort ascending
  std::vector<int> ord(n);
  for (int i = 0; i < n; ++i) ord[i] = i;
  std::sort(ord.begin(), ord.end(), [&](int x, int y) { return lam[x] < lam[y]; });
  std::vector<double> l2(n), V2((size_t)n * n);
  for (int j = 0; j < n; ++j) {
    l2[j] = lam[ord[j]];
    for (int k = 0; k < n; ++k) V2[(size_t)k * n + j] = V[(size_t)k * n + ord[j]];
  }
  lam.swap(l2);
  V.swap(V2);
  return (sweep < 60 || std::sqrt(off) <= 1e-13 * fro) ? sweep : -1;
}

int overlap_nodes(int P_l, int policy) {
  if (policy == PMG_OVERLAP_ZERO) return 0;
  if (policy == PMG_OVERLAP_LEVEL_FLOOR) return 1 + P_l / 8;
  return 1 + (P_l + 4) / 8;
}

// Smoothed sign function phi (Sec. 3.1); sgn outside (-1, 1).
double transition(double x, int weighting) {
  if (weighting == PMG_WEIGHT_UNWEIGHTED) return 1.0;
  if (x >= 1.0) return 1.0;
  if (x <= -1.0) return -1.0;
  if (weighting == PMG_WEIGHT_ARITHMETIC) return 0.0;
  if (weighting == PMG_WEIGHT_CUBIC) return 0.5 * x * (3.0 - x * x);
  double x2 = x * x;
  return x * (15.0 + x2 * (-10.0 + 3.0 * x2)) / 8.0;
}

// Scaled 1-D patch matrix B = M^-1/2 L_s M^-1/2 with a decoupled identity for
// positions outside the domain (Dirichlet truncation); Msq = diag(M)^1/2.
static void patch_matrix(const Axis1DHost& a, const std::vector<int>& gidx, std::vector<double>& B,
                         std::vector<double>& Msq) {
  const int n = (int)gidx.size();
  B.assign((size_t)n * n, 0.0);
  Msq.assign(n, 1.0);
  for (int p = 0; p < n; ++p) Msq[p] = gidx[p] >= 0 ? std::sqrt(a.M[gidx[p]]) : 1.0;
  for (int p = 0; p < n; ++p)
    for (int q = 0; q < n; ++q) {
      double v = (gidx[p] < 0 || gidx[q] < 0) ? (p == q ? 1.0 : 0.0) : a.entry(gidx[p], gidx[q]);
      B[(size_t)p * n + q] = v / (Msq[p] * Msq[q]);
    }
  for (int p = 0; p < n; ++p)          // exact symmetry before the eigen-solver
    for (int q = p + 1; q < n; ++q) {
      double s = 0.5 * (B[(size_t)p * n + q] + B[(size_t)q * n + p]);
      B[(size_t)p * n + q] = s;
      B[(size_t)q * n + p] = s;
    }
}

static void jacobi_or_throw(int n, std::vector<double>& A, std::vector<double>& V, std::vector<double>& l) {
  if (sym_eig_jacobi(n, A, V, l) < 0) throw std::runtime_error("Jacobi eigen-solver did not converge");
}

// Is the patch centro-symmetric: every position inside the domain, and B, M and
// the weights unchanged under the reversal a -> n-1-a?
static bool centro_symmetric(const std::vector<int>& gidx, const std::vector<double>& B,
                             const std::vector<double>& Msq, const std::vector<double>& w) {
  const int n = (int)gidx.size();
  if (n < 2 || n > 64) return false;     // the kernels fold lines of at most 64 nodes
  double big = 0.0;
  for (double x : B) big = std::max(big, std::fabs(x));
  for (int p = 0; p < n; ++p) {
    if (gidx[p] < 0) return false;
    if (std::fabs(Msq[p] - Msq[n - 1 - p]) > 1e-14 * Msq[p]) return false;
    if (std::fabs(w[p] - w[n - 1 - p]) > 1e-15) return false;
    for (int q = 0; q < n; ++q)
      if (std::fabs(B[(size_t)p * n + q] - B[(size_t)(n - 1 - p) * n + (n - 1 - q)]) > 1e-13 * big)
        return false;
  }
  return true;
}

// Eigen-tables of one patch axis (fast diagonalisation, Sec. 3.1):
// L_s S = M_s S Lambda with S^T M_s S = I, forward table S, backward table
// W = diag(w) S stored transposed.  General form: S row-major n x n (node,
// mode), W^T row-major (mode, node), modes by ascending lambda.
// Centro-symmetric form (sym = 1, n <= 64): the problem splits into the
// symmetric and antisymmetric subspaces, solved separately; S holds the
// symmetric block (NE x NE, rows = nodes 0..NE-1) then the antisymmetric one
// (NO x NO, rows = nodes 0..NO-1); W^T the same blocks transposed (rows =
// modes); lambda in the same mode order.
static void patch_tables(const Axis1DHost& a, const std::vector<int>& gidx, const std::vector<double>& w,
                         double* S, double* W, double* lam, int* sym) {
  const int n = (int)gidx.size();
  std::vector<double> B, Msq;
  patch_matrix(a, gidx, B, Msq);
  if (!centro_symmetric(gidx, B, Msq, w)) {
    std::vector<double> V, l;
    jacobi_or_throw(n, B, V, l);
    for (int p = 0; p < n; ++p)
      for (int i = 0; i < n; ++i) {
        S[(size_t)p * n + i] = V[(size_t)p * n + i] / Msq[p];
        W[(size_t)i * n + p] = w[p] * S[(size_t)p * n + i];     // W^T: mode-major
      }
    for (int i = 0; i < n; ++i) lam[i] = l[i];
    *sym = 0;
    return;
  }
  const int H = n / 2, NE = n - H, NO = H;
  const double r2 = std::sqrt(0.5);
  // reduced matrices in the bases e_k = (d_k + d_{n-1-k})/sqrt2 (k < H), e_mid = d_H,
  // and o_k = (d_k - d_{n-1-k})/sqrt2
  std::vector<double> Be((size_t)NE * NE), Bo((size_t)NO * NO);
  auto Bat = [&](int p, int q) { return B[(size_t)p * n + q]; };
  for (int k = 0; k < NE; ++k)
    for (int l = 0; l < NE; ++l) {
      double v;
      if (k < H && l < H) v = Bat(k, l) + Bat(k, n - 1 - l);      // (1/2)(2 B_kl + 2 B_k,n-1-l)
      else if (k < H) v = (Bat(k, H) + Bat(n - 1 - k, H)) * r2;
      else if (l < H) v = (Bat(H, l) + Bat(H, n - 1 - l)) * r2;
      else v = Bat(H, H);
      Be[(size_t)k * NE + l] = v;
    }
  for (int k = 0; k < NO; ++k)
    for (int l = 0; l < NO; ++l) Bo[(size_t)k * NO + l] = Bat(k, l) - Bat(k, n - 1 - l);
  for (int k = 0; k < NE; ++k)
    for (int l = k + 1; l < NE; ++l) {
      double s = 0.5 * (Be[(size_t)k * NE + l] + Be[(size_t)l * NE + k]);
      Be[(size_t)k * NE + l] = Be[(size_t)l * NE + k] = s;
    }
  for (int k = 0; k < NO; ++k)
    for (int l = k + 1; l < NO; ++l) {
      double s = 0.5 * (Bo[(size_t)k * NO + l] + Bo[(size_t)l * NO + k]);
      Bo[(size_t)k * NO + l] = Bo[(size_t)l * NO + k] = s;
    }
  std::vector<double> Ve, le, Vo, lo;
  jacobi_or_throw(NE, Be, Ve, le);
  if (NO > 0) jacobi_or_throw(NO, Bo, Vo, lo);
  // nodal values of the modes: node a < H of a symmetric mode = Ve[a][i] / (sqrt2 Msq[a]),
  // middle node = Ve[H][i] / Msq[H]; antisymmetric: Vo[a][i] / (sqrt2 Msq[a]) (negated at n-1-a)
  double* Se = S;
  double* So = S + (size_t)NE * NE;
  double* We = W;
  double* Wo = W + (size_t)NE * NE;
  for (int p = 0; p < NE; ++p)
    for (int i = 0; i < NE; ++i) {
      double s = Ve[(size_t)p * NE + i] * ((p < H) ? r2 : 1.0) / Msq[p];
      Se[(size_t)p * NE + i] = s;
      We[(size_t)i * NE + p] = w[p] * s;                         // transposed

    }
  for (int p = 0; p < NO; ++p)
    for (int i = 0; i < NO; ++i) {
      double s = Vo[(size_t)p * NO + i] * r2 / Msq[p];
      So[(size_t)p * NO + i] = s;
      Wo[(size_t)i * NO + p] = w[p] * s;                         // transposed
    }
  for (int i = 0; i < NE; ++i) lam[i] = le[i];
  for (int i = 0; i < NO; ++i) lam[NE + i] = lo[i];
  *sym = 1;
}

static int wrap_index(const Axis1DHost& a, int I) {
  int N = a.Ne * a.NP;
  if (a.periodic) return ((I % N) + N) % N;
  return (I < 0 || I >= N) ? -1 : I;
}

static void alloc_tables(AxisTables& t) {
  t.S.assign((size_t)t.count * t.n * t.n, 0.0);
  t.W.assign((size_t)t.count * t.n * t.n, 0.0);
  t.lam.assign((size_t)t.count * t.n, 0.0);
  t.sym.assign(t.count, 0);
}

// Element-centred patches along one axis (Sec. 3.1): element m plus N_o node
// layers of each neighbour: global 1-D range [m NP - N_o, m NP + NP + N_o).
// Weights w_H (Eq. weight function:ec) with readings C6 and C18.
void ec_axis_tables(const Axis1DHost& a, int No, int weighting, double tau, AxisTables& t) {
  const int NP = a.NP, Ne = a.Ne, P = a.P;
  t.n = NP + 2 * No;
  t.count = Ne;
  t.start0 = -No;
  alloc_tables(t);
  const int n = t.n;
  const double dxi = (a.eta[No] + 1.0) * tau;      // tau < 1: narrower transition (learned knob)
  for (int m = 0; m < Ne; ++m) {
    std::vector<int> g(n);
    std::vector<double> w(n, 0.0);
    for (int s = 0; s < n; ++s) g[s] = wrap_index(a, m * NP - No + s);
    bool has_left = a.periodic || m > 0, has_right = a.periodic || m < Ne - 1;
    for (int s = 0; s < n; ++s) {
      if (g[s] < 0) continue;
      double xi;
      if (s < No) {
        xi = a.eta[P - No + 1 + s] - 2.0;
      } else if (s < No + NP) {
        xi = a.eta[s - No];
      } else {
        xi = a.eta[s - No - NP] + 2.0;
      }
      double wt = 1.0;
      if (No > 0) {
        double l = has_left ? transition((1.0 + xi) / dxi, weighting) : 1.0;
        double r = has_right ? transition((1.0 - xi) / dxi, weighting) : 1.0;
        wt = 0.5 * (l + r);
      }
      w[s] = wt;
    }
    patch_tables(a, g, w, &t.S[(size_t)m * n * n], &t.W[(size_t)m * n * n], &t.lam[(size_t)m * n],
                 &t.sym[m]);
  }
}

// Face-centred patches, normal axis (Sec. 3.1): face f between elements f-1
// and f, global 1-D range [f NP - P, f NP + P) (far-face layers excluded).
// Normal weight w_F = 1/2 [1 + phi(1 - |xi_F|)] (reading C5); walls: C13.
void fc_axis_tables(const Axis1DHost& a, int weighting, double tau, AxisTables& t) {
  const int NP = a.NP, Ne = a.Ne, P = a.P;
  t.n = 2 * P;
  t.count = a.periodic ? Ne : Ne + 1;
  t.start0 = -P;
  alloc_tables(t);
  const int n = t.n;
  for (int f = 0; f < t.count; ++f) {
    std::vector<int> g(n);
    std::vector<double> w(n, 0.0);
    for (int s = 0; s < n; ++s) g[s] = wrap_index(a, f * NP - P + s);
    for (int s = 0; s < n; ++s) {
      if (g[s] < 0) continue;
      // s < P: node s+1 of element f-1 (xi_F = eta - 1); else node s-P of element f (xi_F = eta + 1)
      double xiF = (s < P) ? a.eta[s + 1] - 1.0 : a.eta[s - P] + 1.0;
      w[s] = 0.5 * (1.0 + transition((1.0 - std::fabs(xiF)) / tau, weighting));
    }
    patch_tables(a, g, w, &t.S[(size_t)f * n * n], &t.W[(size_t)f * n * n], &t.lam[(size_t)f * n],
                 &t.sym[f]);
  }
}

// Generalised eigen-pairs of the whole global 1-D operator (coarse solve),
// general (unfolded) form.
void global_axis_eig(const Axis1DHost& a, std::vector<double>& S, std::vector<double>& lam) {
  const int N = a.Ne * a.NP;
  std::vector<int> g(N);
  for (int i = 0; i < N; ++i) g[i] = i;
  std::vector<double> B, Msq, V, l;
  patch_matrix(a, g, B, Msq);
  jacobi_or_throw(N, B, V, l);
  S.assign((size_t)N * N, 0.0);
  for (int p = 0; p < N; ++p)
    for (int i = 0; i < N; ++i) S[(size_t)p * N + i] = V[(size_t)p * N + i] / Msq[p];
  lam = l;
}

// Apply-kernel tables of one axis: per element m, Lt = M_m^-1 L^0_m (rows
// scaled by the inverse diagonal mass, so the kernel scales by the nodal mass
// product once per node), its centro-symmetry flag and, when symmetric, the
// even-odd folded form: E[i][a] = (Lt[i][a] + Lt[i][P-a]) / 2 for a < H and
// E[i][H] = Lt[i][H] (middle column, odd NP), rows i < NE; then
// O[i][a] = (Lt[i][a] - Lt[i][P-a]) / 2, i, a < H.  Coupling row (2 NP + 8):
// [-aL D0_i / M_i]_i, [aR DP_i / M_i]_i, bL/M_0, cL/M_0, hasL, bR/M_P, cR/M_P, hasR.
void apply_axis_tables(const Axis1DHost& a, ApplyAxisHost& t, bool fold_coupling) {
  const int NP = a.NP, Ne = a.Ne, P = a.P;
  const int H = NP / 2, NE = NP - H, NO = H;
  t.L0.assign((size_t)Ne * NP * NP, 0.0);
  t.cpl.assign((size_t)Ne * (2 * NP + 8), 0.0);
  t.sym.assign(Ne, 0);
  std::vector<double> Lt((size_t)NP * NP);
  for (int m = 0; m < Ne; ++m) {
    const double* M = &a.M[(size_t)m * NP];
    const double* L0 = &a.L0[(size_t)m * NP * NP];
    double big = 0.0;
    for (int i = 0; i < NP; ++i)
      for (int k = 0; k < NP; ++k) {
        Lt[(size_t)i * NP + k] = L0[(size_t)i * NP + k] / M[i];
        big = std::max(big, std::fabs(Lt[(size_t)i * NP + k]));
      }
    bool sym = NP >= 2;
    for (int i = 0; i < NP && sym; ++i)
      for (int k = 0; k < NP; ++k)
        if (std::fabs(Lt[(size_t)i * NP + k] - Lt[(size_t)(P - i) * NP + (P - k)]) > 1e-13 * big) {
          sym = false;
          break;
        }
    double* dst = &t.L0[(size_t)m * NP * NP];
    if (sym) {
      double* E = dst;
      double* O = dst + (size_t)NE * NE;
      for (int i = 0; i < NE; ++i)
        for (int c = 0; c < NE; ++c)
          E[(size_t)i * NE + c] = (c < H) ? 0.5 * (Lt[(size_t)i * NP + c] + Lt[(size_t)i * NP + (P - c)])
                                          : Lt[(size_t)i * NP + H];
      for (int i = 0; i < NO; ++i)
        for (int c = 0; c < NO; ++c)
          O[(size_t)i * NO + c] = 0.5 * (Lt[(size_t)i * NP + c] - Lt[(size_t)i * NP + (P - c)]);
    } else {
      std::copy(Lt.begin(), Lt.end(), dst);
    }
    t.sym[m] = sym ? 1 : 0;
    const double* c = &a.cpl[(size_t)m * 8];
    double* o = &t.cpl[(size_t)m * (2 * NP + 8)];
    for (int i = 0; i < NP; ++i) {
      o[i] = c[3] != 0.0 ? -c[0] * a.D[0 * NP + i] / M[i] : 0.0;
      o[NP + i] = c[7] != 0.0 ? c[4] * a.D[(size_t)P * NP + i] / M[i] : 0.0;
    }
    o[2 * NP + 0] = c[1] / M[0];
    o[2 * NP + 1] = c[2] / M[0];
    o[2 * NP + 2] = c[3];
    o[2 * NP + 3] = c[5] / M[P];
    o[2 * NP + 4] = c[6] / M[P];
    o[2 * NP + 5] = c[7];
    // both neighbours, a centro-symmetric block and mirrored coupling rows (c_R[P - i] =
    // c_L[i]: equal neighbour widths): the rows are stored folded, the even part of c_L
    // in o[0..NE), the odd part in o[NP..NP + NO), flagged in o[2 NP + 6], so that the
    // kernel adds c_L u_P + c_R u_0 inside the even-odd accumulation (half the products)
    bool csym = fold_coupling && sym && c[3] != 0.0 && c[7] != 0.0;
    double cbig = 0.0;
    for (int i = 0; i < NP; ++i) cbig = std::max(cbig, std::fabs(o[i]));
    for (int i = 0; i < NP && csym; ++i)
      if (std::fabs(o[NP + (P - i)] - o[i]) > 1e-13 * cbig) csym = false;
    if (csym) {
      std::vector<double> cl(o, o + NP);
      for (int i = 0; i < NE; ++i) o[i] = (i < H) ? 0.5 * (cl[i] + cl[P - i]) : cl[H];
      for (int i = NE; i < NP; ++i) o[i] = 0.0;
      for (int i = 0; i < NO; ++i) o[NP + i] = 0.5 * (cl[i] - cl[P - i]);
      for (int i = NO; i < NP; ++i) o[NP + i] = 0.0;
    }
    o[2 * NP + 6] = csym ? 1.0 : 0.0;
  }
}

// The apply tables in the kernel's accumulate form: per element, the M^-1 L^0
// block transposed (row a holds column a: general L^0[i][a] over i; even-odd:
// the folded E then O blocks, transposed), each row padded to W entries (16
// bytes of the device type), block stride NP * pad(NP); the coupling rows
// c[0..NP) and c[NP..2NP) padded likewise, then the 8 scalars.
void apply_rowform(const ApplyAxisHost& t, int NP, int W, std::vector<double>& L0r,
                   std::vector<double>& cplr) {
  auto pad = [W](int n) { return (n + W - 1) / W * W; };
  const int H = NP / 2, NE = NP - H, NO = H;
  const int PNP = pad(NP), PE = pad(NE), PO = pad(NO > 0 ? NO : 1);
  const size_t LB = (size_t)NP * PNP, CB = 2 * (size_t)PNP + 8;
  const int Ne = (int)t.sym.size();
  L0r.assign((size_t)Ne * LB, 0.0);
  cplr.assign((size_t)Ne * CB, 0.0);
  for (int m = 0; m < Ne; ++m) {
    const double* src = &t.L0[(size_t)m * NP * NP];
    double* dst = &L0r[(size_t)m * LB];
    if (t.sym[m]) {
      for (int i = 0; i < NE; ++i)
        for (int a = 0; a < NE; ++a) dst[(size_t)a * PE + i] = src[(size_t)i * NE + a];
      for (int i = 0; i < NO; ++i)
        for (int a = 0; a < NO; ++a) dst[(size_t)NE * PE + (size_t)a * PO + i] = src[(size_t)NE * NE + i * NO + a];
    } else {
      for (int i = 0; i < NP; ++i)
        for (int a = 0; a < NP; ++a) dst[(size_t)a * PNP + i] = src[(size_t)i * NP + a];
    }
    const double* c = &t.cpl[(size_t)m * (2 * NP + 8)];
    double* o = &cplr[(size_t)m * CB];
    for (int i = 0; i < NP; ++i) {
      o[i] = c[i];
      o[PNP + i] = c[NP + i];
    }
    for (int j = 0; j < 8; ++j) o[2 * PNP + j] = c[2 * NP + j];
  }
}

// Expand even-odd folded patch tables (sym = 1) into the general layout
// (S node-major, W^T mode-major, symmetric modes first), for the tensor-core
// line passes, which apply the full n x n tables.
void unfold_tables(AxisTables& t) {
  const int n = t.n, H = n / 2, NE = n - H, NO = H;
  std::vector<double> Sf((size_t)n * n), Wf((size_t)n * n);
  for (int p = 0; p < t.count; ++p) {
    if (!t.sym[p]) continue;
    const double* S = &t.S[(size_t)p * n * n];
    const double* W = &t.W[(size_t)p * n * n];
    std::fill(Sf.begin(), Sf.end(), 0.0);
    std::fill(Wf.begin(), Wf.end(), 0.0);
    for (int i = 0; i < NE; ++i)
      for (int a = 0; a < NE; ++a) {
        const double s = S[(size_t)a * NE + i], w = W[(size_t)i * NE + a];
        Sf[(size_t)a * n + i] = s;
        Sf[(size_t)(n - 1 - a) * n + i] = s;
        Wf[(size_t)i * n + a] = w;
        Wf[(size_t)i * n + (n - 1 - a)] = w;
      }
    const double* So = S + (size_t)NE * NE;
    const double* Wo = W + (size_t)NE * NE;
    for (int i = 0; i < NO; ++i)
      for (int a = 0; a < NO; ++a) {
        const double s = So[(size_t)a * NO + i], w = Wo[(size_t)i * NO + a];
        Sf[(size_t)a * n + NE + i] = s;
        Sf[(size_t)(n - 1 - a) * n + NE + i] = -s;
        Wf[(size_t)(NE + i) * n + a] = w;
        Wf[(size_t)(NE + i) * n + (n - 1 - a)] = -w;
      }
    std::copy(Sf.begin(), Sf.end(), t.S.begin() + (size_t)p * n * n);
    std::copy(Wf.begin(), Wf.end(), t.W.begin() + (size_t)p * n * n);
    t.sym[p] = 0;
  }
}

}  // namespace pmg

namespace pmg {

// k copies of a non-periodic axis one after the other: the 1-D operator becomes block
// diagonal (the wall elements of every copy keep their ghost fold-in and no coupling),
// so copy c of a vector on the stacked axis is the copy of that vector on the original.
void stack_axis(const Axis1DHost& a, int k, Axis1DHost& out) {
  out = a;
  out.Ne = a.Ne * k;
  out.dx.clear();
  out.L0.clear();
  out.Lm.clear();
  out.Lp.clear();
  out.M.clear();
  out.cpl.clear();
  for (int c = 0; c < k; ++c) {
    out.dx.insert(out.dx.end(), a.dx.begin(), a.dx.end());
    out.L0.insert(out.L0.end(), a.L0.begin(), a.L0.end());
    out.Lm.insert(out.Lm.end(), a.Lm.begin(), a.Lm.end());
    out.Lp.insert(out.Lp.end(), a.Lp.begin(), a.Lp.end());
    out.M.insert(out.M.end(), a.M.begin(), a.M.end());
    out.cpl.insert(out.cpl.end(), a.cpl.begin(), a.cpl.end());
  }
}

// The patch tables of one axis repeated for k stacked copies: the positions of copy c
// follow those of copy c - 1; skip = 1 where a copy holds one position more than
// elements (the faces normal to the axis).
void stack_tables(const AxisTables& t, int k, int skip, AxisTables& out) {
  out = t;
  out.count = t.count * k;
  out.bpos = t.count;
  out.bskip = skip;
  out.S.clear();
  out.W.clear();
  out.lam.clear();
  out.sym.clear();
  for (int c = 0; c < k; ++c) {
    out.S.insert(out.S.end(), t.S.begin(), t.S.end());
    out.W.insert(out.W.end(), t.W.begin(), t.W.end());
    out.lam.insert(out.lam.end(), t.lam.begin(), t.lam.end());
    out.sym.insert(out.sym.end(), t.sym.begin(), t.sym.end());
  }
}

}  // namespace pmg
