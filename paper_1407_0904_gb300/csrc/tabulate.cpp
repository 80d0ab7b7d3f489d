// Host-side reference-element tabulation and reference tensors (FP64).
//
// Section 2 of the paper (step 2 of the local-assembly kernel, Listing 1's static
// tables W, X_D10, X_D01, Y): basis functions and their reference derivatives at the
// points of a quadrature rule. Here:
//  * the quadrature rule is the collapsed (conical-product) Gauss-Jacobi rule:
//    triangle x = a(1-b), y = b with weight (1-b) absorbed by a Gauss-Jacobi
//    (alpha=1) rule in b; tetrahedron x = a(1-b)(1-c), y = b(1-c), z = c with weights
//    (1-c)^2 and (1-b) absorbed by Gauss-Jacobi (alpha=2, alpha=1) rules; n =
//    ceil((p+1)/2) points per direction integrate total degree p exactly;
//    Gauss-Jacobi nodes by Newton iteration with deflation on the Jacobi
//    three-term recurrence;
//  * the equispaced Lagrange basis is Silvester's product of barycentric factors,
//    phi = prod_m R_{alpha_m}(lambda_m), R_a(l) = prod_{s<a} (k l - s)/(s+1).
// The quadrature sum is then pre-contracted into reference tensors T[k][i*ns+j]
// (section 3.3's outer-product view: every entry of the element matrix is a sum of
// products of an (i)-only and a (j)-only factor, scaled by per-cell constants).

#include <cmath>
#include <vector>
#include <array>
#include "coffee_internal.h"

namespace coffee {

int nnodes(int cell, int k) {
  return cell == 0 ? (k + 1) * (k + 2) / 2 : cell == 1 ? (k + 1) * (k + 2) * (k + 3) / 6
                                                       : (k + 1) * (k + 2) / 2 * (k + 1);  // prism
}

int npairs(int d) { return d * (d + 1) / 2; }

void pair_index(int d, int p, int& a, int& b) {
  int q = 0;
  for (int x = 0; x < d; ++x)
    for (int y = x; y < d; ++y) {
      if (q == p) { a = x; b = y; return; }
      ++q;
    }
  a = b = 0;
}

int quad_degree_for(int form, int k) { return form == FORM_BURGERS ? 3 * k - 1 : 2 * k; }

int form_K(int form, int k, int cell) {
  int d = cell == 0 ? 2 : 3, ns = nnodes(cell, k), P = npairs(d);
  switch (form) {
    case FORM_MASS: return 1;
    case FORM_HELMHOLTZ: return 1 + P;
    case FORM_ADVDIFF: return (d + 1) * P + (d + 1) * d;
    case FORM_BURGERS: return 2 * ns * d + P;
  }
  return 0;
}

namespace {

std::vector<std::array<int, 3>> lattice(int cell, int k) {
  std::vector<std::array<int, 3>> out;
  int cmax = cell == 1 ? k : 0;
  for (int c = 0; c <= cmax; ++c)
    for (int b = 0; b <= k - c; ++b)
      for (int a = 0; a <= k - b - c; ++a) out.push_back({a, b, c});
  return out;
}

// Jacobi polynomial P_n^{(al,be)}(x) and its derivative.
void jacobi(int n, double al, double be, double x, double& p, double& dp) {
  auto eval = [&](int m, double a, double b, double xx) {
    if (m == 0) return 1.0;
    double p0 = 1.0, p1 = 0.5 * ((a + b + 2.0) * xx + (a - b));
    for (int j = 2; j <= m; ++j) {
      double s = 2.0 * j + a + b;
      double a1 = 2.0 * j * (j + a + b) * (s - 2.0);
      double a2 = (s - 1.0) * (a * a - b * b);
      double a3 = (s - 2.0) * (s - 1.0) * s;
      double a4 = 2.0 * (j + a - 1.0) * (j + b - 1.0) * s;
      double p2 = ((a2 + a3 * xx) * p1 - a4 * p0) / a1;
      p0 = p1;
      p1 = p2;
    }
    return p1;
  };
  p = eval(n, al, be, x);
  dp = n == 0 ? 0.0 : 0.5 * (n + al + be + 1.0) * eval(n - 1, al + 1.0, be + 1.0, x);
}

// n-point Gauss-Jacobi rule for int_0^1 f(s) (1-s)^alpha ds.
void gauss_jacobi01(int n, int alpha, std::vector<double>& s, std::vector<double>& w) {
  const double al = alpha, be = 0.0;
  std::vector<double> x(n);
  for (int k = 0; k < n; ++k) {
    double r = -std::cos((2.0 * k + 1.0) * M_PI / (2.0 * n));
    if (k > 0) r = 0.5 * (r + x[k - 1]);
    for (int it = 0; it < 200; ++it) {
      double p, dp;
      jacobi(n, al, be, r, p, dp);
      double sum = 0.0;
      for (int j = 0; j < k; ++j) sum += 1.0 / (r - x[j]);
      double delta = -p / (dp - sum * p);
      r += delta;
      if (std::fabs(delta) < 1e-16) break;
    }
    x[k] = r;
  }
  // weights on [-1,1]: 2^(al+be+1) G(n+al+1) G(n+be+1) / (G(n+al+be+1) n!) / ((1-x^2) P'^2)
  double C = std::pow(2.0, al + be + 1.0) *
             std::exp(std::lgamma(n + al + 1.0) + std::lgamma(n + be + 1.0) -
                      std::lgamma(n + al + be + 1.0) - std::lgamma(n + 1.0));
  s.resize(n);
  w.resize(n);
  for (int k = 0; k < n; ++k) {
    double p, dp;
    jacobi(n, al, be, x[k], p, dp);
    double wk = C / ((1.0 - x[k] * x[k]) * dp * dp);
    s[k] = 0.5 * (1.0 + x[k]);
    w[k] = wk * std::pow(0.5, al + 1.0);  // (1-s)^al = ((1-x)/2)^al, ds = dx/2
  }
}

// Silvester factor R_a(l) = prod_{s<a} (k l - s)/(s+1) and its derivative in l.
void silvester(int a, int k, double l, double& R, double& dR) {
  R = 1.0;
  dR = 0.0;
  for (int s = 0; s < a; ++s) {
    double f = (k * l - s) / (s + 1.0), df = k / (s + 1.0);
    dR = dR * f + R * df;
    R *= f;
  }
}

}  // namespace

void quadrature_rule(int cell, int degree, std::vector<double>& pts, std::vector<double>& wts) {
  int n = (degree + 2) / 2;  // ceil((degree+1)/2)
  if (n < 1) n = 1;
  pts.clear();
  wts.clear();
  std::vector<double> a0, w0, a1, w1, a2, w2;
  gauss_jacobi01(n, 0, a0, w0);
  gauss_jacobi01(n, 1, a1, w1);
  if (cell == 0) {
    for (int j = 0; j < n; ++j)      // b (alpha = 1)
      for (int i = 0; i < n; ++i) {  // a (alpha = 0)
        double b = a1[j], a = a0[i];
        pts.push_back(a * (1.0 - b));
        pts.push_back(b);
        wts.push_back(w1[j] * w0[i]);
      }
  } else {
    gauss_jacobi01(n, 2, a2, w2);
    for (int l = 0; l < n; ++l)        // c (alpha = 2)
      for (int j = 0; j < n; ++j)      // b (alpha = 1)
        for (int i = 0; i < n; ++i) {  // a (alpha = 0)
          double c = a2[l], b = a1[j], a = a0[i];
          pts.push_back(a * (1.0 - b) * (1.0 - c));
          pts.push_back(b * (1.0 - c));
          pts.push_back(c);
          wts.push_back(w2[l] * w1[j] * w0[i]);
        }
  }
}

void lagrange_basis(int cell, int k, int npts, const double* x, double* phi, double* grads) {
  const int d = cell == 0 ? 2 : 3;
  auto L = lattice(cell, k);
  const int n = (int)L.size();
  for (int p = 0; p < npts; ++p) {
    const double* xp = x + (size_t)p * d;
    double lam[4];
    lam[0] = 1.0;
    for (int a = 0; a < d; ++a) {
      lam[a + 1] = xp[a];
      lam[0] -= xp[a];
    }
    for (int i = 0; i < n; ++i) {
      int al[4] = {k - L[i][0] - L[i][1] - L[i][2], L[i][0], L[i][1], L[i][2]};
      double R[4], dR[4];
      for (int m = 0; m <= d; ++m) silvester(al[m], k, lam[m], R[m], dR[m]);
      double v = 1.0;
      for (int m = 0; m <= d; ++m) v *= R[m];
      if (phi) phi[(size_t)p * n + i] = v;
      if (grads) {
        double dl[4];  // d phi / d lambda_m
        for (int m = 0; m <= d; ++m) {
          double g = dR[m];
          for (int o = 0; o <= d; ++o)
            if (o != m) g *= R[o];
          dl[m] = g;
        }
        for (int a = 0; a < d; ++a) grads[((size_t)p * n + i) * d + a] = dl[a + 1] - dl[0];
      }
    }
  }
}

// Reference tensors T[K][ns*ns] of a form (see coffee_reference_tensor).
//  MASS:      T0 = int phi_i phi_j
//  HELMHOLTZ: T0 = mass; T_{1+p} = int d_a phi_i d_b phi_j + [a!=b] d_b phi_i d_a phi_j
//             for the p-th pair a <= b
//  ADVDIFF:   T_{v*P+p} = int lambda_v (d_a phi_i d_b phi_j + [a!=b] d_b phi_i d_a phi_j)
//             T_{(d+1)P + v*d + a} = int lambda_v phi_i d_a phi_j
//  BURGERS:   T_{r*d+a} = int d_a phi_r phi_i phi_j            (r < ns)
//             T_{ns*d + r*d+a} = int phi_r phi_i d_a phi_j
//             T_{2 ns d + p} = stiffness pair tensor as in HELMHOLTZ
void reference_tensor(int form, int k, int cell, std::vector<double>& T) {
  const int d = cell == 0 ? 2 : 3, ns = nnodes(cell, k), N = ns * ns, P = npairs(d);
  const int K = form_K(form, k, cell);
  std::vector<double> pts, wts;
  quadrature_rule(cell, quad_degree_for(form, k), pts, wts);
  const int nq = (int)wts.size();
  std::vector<double> phi((size_t)nq * ns), dphi((size_t)nq * ns * d);
  std::vector<double> lam((size_t)nq * (d + 1));
  lagrange_basis(cell, k, nq, pts.data(), phi.data(), dphi.data());
  lagrange_basis(cell, 1, nq, pts.data(), lam.data(), nullptr);
  T.assign((size_t)K * N, 0.0);
  auto at = [&](int kk, int i, int j) -> double& { return T[(size_t)kk * N + i * ns + j]; };
  for (int q = 0; q < nq; ++q) {
    const double w = wts[q];
    const double* ph = &phi[(size_t)q * ns];
    const double* dp = &dphi[(size_t)q * ns * d];
    const double* lm = &lam[(size_t)q * (d + 1)];
    for (int i = 0; i < ns; ++i)
      for (int j = 0; j < ns; ++j) {
        double m = w * ph[i] * ph[j];
        double st[6];
        for (int p = 0; p < P; ++p) {
          int a, b;
          pair_index(d, p, a, b);
          double s = dp[i * d + a] * dp[j * d + b];
          if (a != b) s += dp[i * d + b] * dp[j * d + a];
          st[p] = w * s;
        }
        if (form == FORM_MASS) {
          at(0, i, j) += m;
        } else if (form == FORM_HELMHOLTZ) {
          at(0, i, j) += m;
          for (int p = 0; p < P; ++p) at(1 + p, i, j) += st[p];
        } else if (form == FORM_ADVDIFF) {
          for (int v = 0; v <= d; ++v) {
            for (int p = 0; p < P; ++p) at(v * P + p, i, j) += lm[v] * st[p];
            for (int a = 0; a < d; ++a)
              at((d + 1) * P + v * d + a, i, j) += w * lm[v] * ph[i] * dp[j * d + a];
          }
        } else {
          for (int r = 0; r < ns; ++r)
            for (int a = 0; a < d; ++a) {
              at(r * d + a, i, j) += w * dp[r * d + a] * ph[i] * ph[j];
              at(ns * d + r * d + a, i, j) += w * ph[r] * ph[i] * dp[j * d + a];
            }
          for (int p = 0; p < P; ++p) at(2 * ns * d + p, i, j) += st[p];
        }
      }
  }
}

}  // namespace coffee

// ---------------------------------------------------------------------------------------
// Prisms (the paper's third element shape, section 5.2): reference triangle x [0,1].
// Degree-k space: triangle Lagrange functions (Silvester) times interval Lagrange functions
// on the nodes c/k; dof (a,b,c) at (a/k, b/k, c/k), zeta level c slowest, triangle lattice
// order inside a level. The prism map is not affine, so the quadrature is not pre-summed:
// the reference tensors keep one block per quadrature point (see prism_tensor).
// Rule: n = k+2 Gauss-Legendre points per direction on [0,1]; triangle points (s, t(1-s)),
// weight w_s w_t (1-s); zeta = r, weight w_r.
// ---------------------------------------------------------------------------------------
namespace coffee {

int prism_nnodes(int k) { return (k + 1) * (k + 2) / 2 * (k + 1); }

void prism_rule_points(int n, std::vector<double>& pts, std::vector<double>& wts) {
  std::vector<double> g, w;
  gauss_jacobi01(n, 0, g, w);  // alpha = 0: Gauss-Legendre
  pts.clear();
  wts.clear();
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      for (int l = 0; l < n; ++l) {
        pts.push_back(g[i]);
        pts.push_back(g[j] * (1.0 - g[i]));
        pts.push_back(g[l]);
        wts.push_back(w[i] * w[j] * (1.0 - g[i]) * w[l]);
      }
}

void prism_rule(int k, std::vector<double>& pts, std::vector<double>& wts) { prism_rule_points(k + 2, pts, wts); }

void prism_basis(int k, int npts, const double* x, double* phi, double* grads) {
  const int nt = (k + 1) * (k + 2) / 2, n = prism_nnodes(k);
  std::vector<double> tp(nt), tg((size_t)nt * 2);
  for (int p = 0; p < npts; ++p) {
    const double* xp = x + (size_t)p * 3;
    lagrange_basis(0, k, 1, xp, tp.data(), tg.data());
    for (int c = 0; c <= k; ++c) {
      // interval Lagrange function on the nodes m/k: prod_{m != c} (k z - m) / (c - m)
      double L = 1.0, dL = 0.0;
      for (int m = 0; m <= k; ++m) {
        if (m == c) continue;
        const double f = (k * xp[2] - m) / (double)(c - m), df = k / (double)(c - m);
        dL = dL * f + L * df;
        L *= f;
      }
      for (int t = 0; t < nt; ++t) {
        const size_t i = (size_t)p * n + (size_t)c * nt + t;
        if (phi) phi[i] = tp[t] * L;
        if (grads) {
          grads[i * 3 + 0] = tg[(size_t)t * 2 + 0] * L;
          grads[i * 3 + 1] = tg[(size_t)t * 2 + 1] * L;
          grads[i * 3 + 2] = tp[t] * dL;
        }
      }
    }
  }
}

// Per-point reference tensors on prisms, A_e = sum_q sum_kq G_e[q][kq] T[q*KQ+kq]:
//  MASS (KQ = 1):      T[q] = phi_i phi_j;                      G = w |det|
//  HELMHOLTZ (KQ = 7): T[q*7] = phi_i phi_j, T[q*7+1+p] = d_a phi_i d_b phi_j + [a!=b] d_b phi_i d_a phi_j
//                      for the p-th pair a <= b;                G = w |det| (1, (K K^T)_ab)
//  ADVDIFF (KQ = 9):   T[q*9+p] = the pair tensors, T[q*9+6+a] = phi_i d_a phi_j;
//                      G = w |det| (eps_q (K K^T)_ab, (K b_q)_a)
void prism_tensor(int form, int k, std::vector<double>& T, std::vector<double>& pts, std::vector<double>& wts) {
  prism_rule(k, pts, wts);
  const int Q = (int)wts.size(), n = prism_nnodes(k), N = n * n;
  const int KQ = form == FORM_HELMHOLTZ ? 7 : form == FORM_ADVDIFF ? 9 : 1;
  std::vector<double> phi((size_t)Q * n), g((size_t)Q * n * 3);
  prism_basis(k, Q, pts.data(), phi.data(), g.data());
  T.assign((size_t)Q * KQ * N, 0.0);
  for (int q = 0; q < Q; ++q) {
    const double* ph = &phi[(size_t)q * n];
    const double* gr = &g[(size_t)q * n * 3];
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        const size_t o = (size_t)i * n + j;
        if (KQ != 9) T[((size_t)q * KQ) * N + o] = ph[i] * ph[j];
        if (KQ >= 7) {
          const int p0 = KQ == 7 ? 1 : 0;  // first pair column of the point
          for (int pp = 0; pp < 6; ++pp) {
            int a, b;
            pair_index(3, pp, a, b);
            double v = gr[(size_t)i * 3 + a] * gr[(size_t)j * 3 + b];
            if (a != b) v += gr[(size_t)i * 3 + b] * gr[(size_t)j * 3 + a];
            T[((size_t)q * KQ + p0 + pp) * N + o] = v;
          }
        }
        if (KQ == 9)
          for (int a = 0; a < 3; ++a) T[((size_t)q * KQ + 6 + a) * N + o] = ph[i] * gr[(size_t)j * 3 + a];
      }
  }
}

// Vector Burgers on prisms: the basis at the points of its rule, (3k+3)/2 Gauss-Legendre points per
// direction (the trilinear term phi_i phi_j grad u has degree 3k-1 in the triangle variables and
// 3k in zeta on prisms with planar faces), as tab [Q][n][4] = (phi, d_s phi, d_t phi, d_z phi),
// then the points [Q][3] and the weights [Q]. The kernel evaluates the quadrature loop directly.
int prism_burgers_points(int k) { return (3 * k + 3) / 2; }

void prism_burgers_table(int k, std::vector<double>& tab, int& Q) {
  std::vector<double> pts, wts;
  prism_rule_points(prism_burgers_points(k), pts, wts);
  Q = (int)wts.size();
  const int n = prism_nnodes(k);
  std::vector<double> phi((size_t)Q * n), g((size_t)Q * n * 3);
  prism_basis(k, Q, pts.data(), phi.data(), g.data());
  tab.assign((size_t)Q * n * 4, 0.0);
  for (size_t i = 0; i < (size_t)Q * n; ++i) {
    tab[i * 4] = phi[i];
    for (int a = 0; a < 3; ++a) tab[i * 4 + 1 + a] = g[i * 3 + a];
  }
  tab.insert(tab.end(), pts.begin(), pts.end());
  tab.insert(tab.end(), wts.begin(), wts.end());
}

}  // namespace coffee
