// FP64 CPU oracle for finite-element local assembly (COFFEE, arXiv:1407.0904).
//
// TEST INFRASTRUCTURE ONLY. This file is the slow, plain reference against which
// the CUDA path is checked. Only the test suite, the smoke check and the timed CPU
// baseline of the benchmark may load it. It shares no code, table or constant with
// the CUDA library: its quadrature rule (collapsed Gauss-Legendre with the Duffy
// Jacobian written out), its Lagrange basis (monomial Vandermonde inversion) and its
// per-cell loop nest are written here independently.
//
// What it computes (paper section 2, "Structure of a local assembly kernel" and
// Listings 1-2): for every cell, (1) the affine Jacobian J, its determinant and its
// inverse K; (2) the basis functions and their reference derivatives at the points
// of a quadrature rule; (3) the element matrix as a loop nest over quadrature
// points i, test functions j and trial functions k, accumulating
// integrand * |det| * W[i].  Listing 1 fixes the gradient convention
// dphi/dx_c = sum_a K[a][c] * dphi/dxi_a (K row-major, x = x0 + J xi).
// The quadrature is exact for the polynomial integrands of affine cells, so the
// result is the plain definition of the element matrix up to rounding.
//
// Conventions (the paper is silent on these; the readings are listed in the design
// notes of the repository): reference simplices with vertices 0, e_1, .., e_d;
// Lagrange nodes are the lattice points (a,b,c)/k, a+b+c <= k, ordered with c
// slowest, then b, then a fastest; element matrix rows are test functions and
// columns trial functions; vector-valued dofs are blocked by component; the
// measure is |det J|.
//
// Build: g++ -O2 -std=c++17 -fopenmp -shared -fPIC oracle.cpp -o liboracle.so

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#include <array>
#include <algorithm>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

enum { CELL_TRI = 0, CELL_TET = 1 };
enum { FORM_MASS = 0, FORM_HELMHOLTZ = 1, FORM_ADVDIFF = 2, FORM_BURGERS = 3 };

int dim_of(int cell) { return cell == CELL_TRI ? 2 : 3; }

// Lattice multi-indices (a,b,c) with a+b+c <= k; c slowest, then b, a fastest.
// The same enumeration lists the monomials x^a y^b z^c of total degree <= k.
std::vector<std::array<int, 3>> lattice(int cell, int k) {
  std::vector<std::array<int, 3>> out;
  int cmax = (cell == CELL_TET) ? k : 0;
  for (int c = 0; c <= cmax; ++c)
    for (int b = 0; b <= k - c; ++b)
      for (int a = 0; a <= k - b - c; ++a) out.push_back({a, b, c});
  return out;
}

// ---------------------------------------------------------------------------
// Quadrature: Gauss-Legendre on [0,1] (nodes by Newton iteration on the
// three-term Legendre recurrence), collapsed onto the simplex by the Duffy map
//   tri: (s,t) -> (s, t(1-s)),                  |Jac| = (1-s)
//   tet: (s,t,r) -> (s, t(1-s), r(1-s)(1-t)),   |Jac| = (1-s)^2 (1-t)
// A monomial of total degree p has degree <= p+d-1 in s after the map, so
// n = ceil((p+3)/2) points per direction integrate it exactly on both shapes.
// ---------------------------------------------------------------------------
void gauss_legendre01(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;  // P_0, P_1
      for (int j = 1; j < n; ++j) {  // P_{j+1} from P_j, P_{j-1}
        double p2 = ((2.0 * j + 1.0) * z * p1 - j * p0) / (j + 1.0);
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);  // P_n'
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    {
      double p0 = 1.0, p1 = z;
      for (int j = 1; j < n; ++j) {
        double p2 = ((2.0 * j + 1.0) * z * p1 - j * p0) / (j + 1.0);
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
    }
    // node on [-1,1] is z with weight 2/((1-z^2) P_n'(z)^2); map to [0,1]
    x[i] = 0.5 * (1.0 + z);
    w[i] = 0.5 * 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

struct Rule {
  int nq = 0;
  std::vector<double> pts;  // [nq][d]
  std::vector<double> wts;  // [nq]
};

Rule collapsed_rule(int cell, int degree) {
  int n = (degree + 3 + 1) / 2;  // ceil((degree+3)/2)
  std::vector<double> x, w;
  gauss_legendre01(n, x, w);
  Rule R;
  if (cell == CELL_TRI) {
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        double s = x[i], t = x[j];
        R.pts.push_back(s);
        R.pts.push_back(t * (1.0 - s));
        R.wts.push_back(w[i] * w[j] * (1.0 - s));
      }
  } else {
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j)
        for (int l = 0; l < n; ++l) {
          double s = x[i], t = x[j], r = x[l];
          R.pts.push_back(s);
          R.pts.push_back(t * (1.0 - s));
          R.pts.push_back(r * (1.0 - s) * (1.0 - t));
          R.wts.push_back(w[i] * w[j] * w[l] * (1.0 - s) * (1.0 - s) * (1.0 - t));
        }
  }
  R.nq = (int)R.wts.size();
  return R;
}

// ---------------------------------------------------------------------------
// Lagrange basis by Vandermonde inversion: V[n][m] = monomial m at node n,
// C = V^{-1} by Gaussian elimination with partial pivoting, and
// phi_i(x) = sum_m C[m][i] * monomial_m(x).
// ---------------------------------------------------------------------------
double ipow(double x, int e) {
  double r = 1.0;
  for (int i = 0; i < e; ++i) r *= x;
  return r;
}

// inverse of the n x n row-major matrix A (overwritten), result in Inv
bool invert(int n, std::vector<double> A, std::vector<double>& Inv) {
  Inv.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) Inv[(size_t)i * n + i] = 1.0;
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (std::fabs(A[(size_t)r * n + col]) > std::fabs(A[(size_t)piv * n + col])) piv = r;
    if (A[(size_t)piv * n + col] == 0.0) return false;
    if (piv != col)
      for (int c = 0; c < n; ++c) {
        std::swap(A[(size_t)piv * n + c], A[(size_t)col * n + c]);
        std::swap(Inv[(size_t)piv * n + c], Inv[(size_t)col * n + c]);
      }
    double d = A[(size_t)col * n + col];
    for (int c = 0; c < n; ++c) {
      A[(size_t)col * n + c] /= d;
      Inv[(size_t)col * n + c] /= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      double f = A[(size_t)r * n + col];
      if (f == 0.0) continue;
      for (int c = 0; c < n; ++c) {
        A[(size_t)r * n + c] -= f * A[(size_t)col * n + c];
        Inv[(size_t)r * n + c] -= f * Inv[(size_t)col * n + c];
      }
    }
  }
  return true;
}

struct Basis {
  int cell = 0, k = 0, d = 0, n = 0;
  std::vector<std::array<int, 3>> mono;  // exponents
  std::vector<double> C;                 // [m][i]
};

Basis lagrange(int cell, int k) {
  Basis B;
  B.cell = cell;
  B.k = k;
  B.d = dim_of(cell);
  B.mono = lattice(cell, k);
  B.n = (int)B.mono.size();
  std::vector<double> V((size_t)B.n * B.n);
  for (int nd = 0; nd < B.n; ++nd) {
    double X[3] = {(double)B.mono[nd][0] / k, (double)B.mono[nd][1] / k, (double)B.mono[nd][2] / k};
    for (int m = 0; m < B.n; ++m) {
      double v = 1.0;
      for (int a = 0; a < B.d; ++a) v *= ipow(X[a], B.mono[m][a]);
      V[(size_t)nd * B.n + m] = v;
    }
  }
  invert(B.n, V, B.C);
  return B;
}

// values phi[i] and reference derivatives dphi[i*d + a] at the point x
void eval_basis(const Basis& B, const double* x, double* phi, double* dphi) {
  int n = B.n, d = B.d;
  std::vector<double> mv(n), md((size_t)n * d);
  for (int m = 0; m < n; ++m) {
    const auto& e = B.mono[m];
    double v = 1.0;
    for (int a = 0; a < d; ++a) v *= ipow(x[a], e[a]);
    mv[m] = v;
    for (int a = 0; a < d; ++a) {
      if (e[a] == 0) { md[(size_t)m * d + a] = 0.0; continue; }
      double g = e[a] * ipow(x[a], e[a] - 1);
      for (int b = 0; b < d; ++b)
        if (b != a) g *= ipow(x[b], e[b]);
      md[(size_t)m * d + a] = g;
    }
  }
  for (int i = 0; i < n; ++i) {
    double v = 0.0;
    for (int m = 0; m < n; ++m) v += B.C[(size_t)m * n + i] * mv[m];
    if (phi) phi[i] = v;
    if (dphi)
      for (int a = 0; a < d; ++a) {
        double g = 0.0;
        for (int m = 0; m < n; ++m) g += B.C[(size_t)m * n + i] * md[(size_t)m * d + a];
        dphi[(size_t)i * d + a] = g;
      }
  }
}

// ---------------------------------------------------------------------------
// Forward-mode dual numbers, used only to differentiate the very same cell
// routine that computes the element matrix (one seed per cell-local input).
// ---------------------------------------------------------------------------
struct Dual {
  double v, d;
  Dual(double a = 0.0, double b = 0.0) : v(a), d(b) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) { return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)); }
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual dabs(Dual a) { return a.v < 0 ? -a : a; }
inline double dabs(double a) { return std::fabs(a); }
inline double value_of(double a) { return a; }
inline double value_of(Dual a) { return a.v; }

// ---------------------------------------------------------------------------
// Per-form context: the rule and the tabulated reference basis.
// ---------------------------------------------------------------------------
struct Ctx {
  int form = 0, cell = 0, k = 0, d = 0;
  int ns = 0;    // scalar nodes per cell of the degree-k space
  int ndof = 0;  // rows of the element matrix (d*ns for the vector form)
  int ncoef = 0; // coefficient nodes per cell (d+1 for P1 fields, ns for Burgers)
  double nu = 0.01;
  Rule rule;
  std::vector<double> phi, dphi;   // [q][ns], [q][ns][d]
  std::vector<double> lam;         // P1 basis at the points [q][d+1]
};

int quad_degree(int form, int k) {
  // exact degree of the integrand on affine cells
  if (form == FORM_BURGERS) return 3 * k - 1;
  return 2 * k;
}

Ctx make_ctx(int form, int k, int cell, double nu) {
  Ctx c;
  c.form = form;
  c.cell = cell;
  c.k = k;
  c.d = dim_of(cell);
  c.nu = nu;
  Basis B = lagrange(cell, k);
  c.ns = B.n;
  c.ndof = (form == FORM_BURGERS) ? c.d * c.ns : c.ns;
  c.ncoef = (form == FORM_ADVDIFF) ? c.d + 1 : (form == FORM_BURGERS ? c.ns : 0);
  c.rule = collapsed_rule(cell, quad_degree(form, k));
  int nq = c.rule.nq;
  c.phi.resize((size_t)nq * c.ns);
  c.dphi.resize((size_t)nq * c.ns * c.d);
  Basis B1 = lagrange(cell, 1);
  c.lam.resize((size_t)nq * (c.d + 1));
  for (int q = 0; q < nq; ++q) {
    eval_basis(B, &c.rule.pts[(size_t)q * c.d], &c.phi[(size_t)q * c.ns], &c.dphi[(size_t)q * c.ns * c.d]);
    eval_basis(B1, &c.rule.pts[(size_t)q * c.d], &c.lam[(size_t)q * (c.d + 1)], nullptr);
  }
  return c;
}

// Geometry (section 2, step 1): J[r][c] = X[c+1][r] - X[0][r]; det; K = J^{-1}
// by the explicit adjugate formula.
template <class S>
void geometry(int d, const S* X, S* K, S& det) {
  S J[3][3];
  for (int r = 0; r < d; ++r)
    for (int c = 0; c < d; ++c) J[r][c] = X[(c + 1) * d + r] - X[r];
  if (d == 2) {
    det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    K[0] = J[1][1] / det;
    K[1] = -J[0][1] / det;
    K[2] = -J[1][0] / det;
    K[3] = J[0][0] / det;
  } else {
    S c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    S c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    S c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    S c10 = J[0][2] * J[2][1] - J[0][1] * J[2][2];
    S c11 = J[0][0] * J[2][2] - J[0][2] * J[2][0];
    S c12 = J[0][1] * J[2][0] - J[0][0] * J[2][1];
    S c20 = J[0][1] * J[1][2] - J[0][2] * J[1][1];
    S c21 = J[0][2] * J[1][0] - J[0][0] * J[1][2];
    S c22 = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
    // K = adj(J)/det, adj[i][j] = cofactor[j][i]
    K[0] = c00 / det; K[1] = c10 / det; K[2] = c20 / det;
    K[3] = c01 / det; K[4] = c11 / det; K[5] = c21 / det;
    K[6] = c02 / det; K[7] = c12 / det; K[8] = c22 / det;
  }
}

// Element matrix of one cell (section 2, step 3; Listings 1 and 2). X holds the
// (d+1) vertex coordinates, cf the cell-local coefficient values:
//   ADVDIFF: [eps_v (d+1) | b_v (d+1)*d]; BURGERS: u[r][c] (ns*d).
template <class S>
void cell_matrix(const Ctx& c, const S* X, const S* cf, S* A) {
  const int d = c.d, ns = c.ns, n = c.ndof, nq = c.rule.nq;
  S K[9], det;
  geometry(d, X, K, det);
  S D = dabs(det);
  for (int i = 0; i < n * n; ++i) A[i] = S(0.0);
  std::vector<S> g((size_t)ns * d);  // physical gradients at the point
  for (int q = 0; q < nq; ++q) {
    const double* ph = &c.phi[(size_t)q * ns];
    const double* dph = &c.dphi[(size_t)q * ns * d];
    for (int i = 0; i < ns; ++i)
      for (int r = 0; r < d; ++r) {
        S s = S(0.0);
        for (int a = 0; a < d; ++a) s += K[a * d + r] * S(dph[i * d + a]);
        g[(size_t)i * d + r] = s;
      }
    S Dw = D * S(c.rule.wts[q]);
    if (c.form == FORM_MASS) {
      for (int i = 0; i < ns; ++i)
        for (int j = 0; j < ns; ++j) A[i * n + j] += S(ph[i] * ph[j]) * Dw;
    } else if (c.form == FORM_HELMHOLTZ) {
      for (int i = 0; i < ns; ++i)
        for (int j = 0; j < ns; ++j) {
          S s = S(ph[i] * ph[j]);
          for (int r = 0; r < d; ++r) s += g[(size_t)i * d + r] * g[(size_t)j * d + r];
          A[i * n + j] += s * Dw;
        }
    } else if (c.form == FORM_ADVDIFF) {
      // eps and b are P1 fields: values at the point from the vertex values
      const double* lam = &c.lam[(size_t)q * (d + 1)];
      S eps = S(0.0), b[3] = {S(0.0), S(0.0), S(0.0)};
      for (int v = 0; v <= d; ++v) {
        eps += cf[v] * S(lam[v]);
        for (int r = 0; r < d; ++r) b[r] += cf[(d + 1) + v * d + r] * S(lam[v]);
      }
      for (int i = 0; i < ns; ++i)
        for (int j = 0; j < ns; ++j) {
          S gg = S(0.0), bg = S(0.0);
          for (int r = 0; r < d; ++r) {
            gg += g[(size_t)i * d + r] * g[(size_t)j * d + r];
            bg += b[r] * g[(size_t)j * d + r];
          }
          A[i * n + j] += (eps * gg + S(ph[i]) * bg) * Dw;
        }
    } else {  // FORM_BURGERS: Jacobian of (u.grad u).v + nu grad u : grad v
      S u[3] = {S(0.0), S(0.0), S(0.0)}, gu[3][3];
      for (int a = 0; a < d; ++a)
        for (int m = 0; m < d; ++m) gu[a][m] = S(0.0);
      for (int r = 0; r < ns; ++r)
        for (int a = 0; a < d; ++a) {
          S ura = cf[r * d + a];
          u[a] += ura * S(ph[r]);
          for (int m = 0; m < d; ++m) gu[a][m] += ura * g[(size_t)r * d + m];
        }
      for (int ci = 0; ci < d; ++ci)
        for (int i = 0; i < ns; ++i)
          for (int cj = 0; cj < d; ++cj)
            for (int j = 0; j < ns; ++j) {
              // (du.grad u).v with du = phi_j e_cj, v = phi_i e_ci
              S s = S(ph[i] * ph[j]) * gu[ci][cj];
              if (ci == cj) {
                S ug = S(0.0), gg = S(0.0);
                for (int m = 0; m < d; ++m) {
                  ug += u[m] * g[(size_t)j * d + m];
                  gg += g[(size_t)i * d + m] * g[(size_t)j * d + m];
                }
                s += S(ph[i]) * ug + S(c.nu) * gg;
              }
              A[(ci * ns + i) * n + cj * ns + j] += s * Dw;
            }
    }
  }
}

// Burgers residual R[(c,i)] = int (u.grad u_c) phi_i + nu grad u_c . grad phi_i
void cell_residual_burgers(const Ctx& c, const double* X, const double* cf, double* R) {
  const int d = c.d, ns = c.ns, nq = c.rule.nq;
  double K[9], det;
  geometry(d, X, K, det);
  double D = std::fabs(det);
  for (int i = 0; i < d * ns; ++i) R[i] = 0.0;
  std::vector<double> g((size_t)ns * d);
  for (int q = 0; q < nq; ++q) {
    const double* ph = &c.phi[(size_t)q * ns];
    const double* dph = &c.dphi[(size_t)q * ns * d];
    for (int i = 0; i < ns; ++i)
      for (int r = 0; r < d; ++r) {
        double s = 0.0;
        for (int a = 0; a < d; ++a) s += K[a * d + r] * dph[i * d + a];
        g[(size_t)i * d + r] = s;
      }
    double u[3] = {0, 0, 0}, gu[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int r = 0; r < ns; ++r)
      for (int a = 0; a < d; ++a) {
        u[a] += cf[r * d + a] * ph[r];
        for (int m = 0; m < d; ++m) gu[a][m] += cf[r * d + a] * g[(size_t)r * d + m];
      }
    double Dw = D * c.rule.wts[q];
    for (int ci = 0; ci < d; ++ci) {
      double adv = 0.0;
      for (int m = 0; m < d; ++m) adv += u[m] * gu[ci][m];
      for (int i = 0; i < ns; ++i) {
        double visc = 0.0;
        for (int m = 0; m < d; ++m) visc += gu[ci][m] * g[(size_t)i * d + m];
        R[ci * ns + i] += (adv * ph[i] + c.nu * visc) * Dw;
      }
    }
  }
}

// gather the cell-local inputs of cell e
void gather(const Ctx& c, const double* coords, const int32_t* c2v, const double* coef,
            const int32_t* c2d, int64_t ncoefnodes, int64_t e, double* X, double* cf) {
  const int d = c.d;
  for (int v = 0; v <= d; ++v) {
    int64_t vid = c2v[e * (d + 1) + v];
    for (int r = 0; r < d; ++r) X[v * d + r] = coords[vid * d + r];
  }
  if (c.form == FORM_ADVDIFF) {
    for (int v = 0; v <= d; ++v) {
      int64_t id = c2d[e * (d + 1) + v];
      cf[v] = coef[id * (d + 1)];
      for (int r = 0; r < d; ++r) cf[(d + 1) + v * d + r] = coef[id * (d + 1) + 1 + r];
    }
  } else if (c.form == FORM_BURGERS) {
    for (int rr = 0; rr < c.ns; ++rr) {
      int64_t id = c2d[e * c.ns + rr];
      for (int a = 0; a < d; ++a) cf[rr * d + a] = coef[id * d + a];
    }
  }
}

int ncf_local(const Ctx& c) {
  if (c.form == FORM_ADVDIFF) return (c.d + 1) * (1 + c.d);
  if (c.form == FORM_BURGERS) return c.ns * c.d;
  return 0;
}

bool valid(int form, int k, int cell) {
  return form >= 0 && form <= 3 && (cell == CELL_TRI || cell == CELL_TET) && k >= 1 && k <= 4;
}

// ---------------------------------------------------------------------------
// Prisms: the paper's third element shape (section 5.2 tests triangles, tetrahedra and
// prisms). Reference prism: the reference triangle (0,0),(1,0),(0,1) times [0,1] in zeta;
// vertices 0,1,2 at zeta = 0 and 3,4,5 above them at zeta = 1. The degree-k Lagrange space is
// the tensor product of the degree-k triangle space and the degree-k interval space; node
// (a,b,c) sits at (a/k, b/k, c/k), ordered with the zeta level c slowest and the triangle's
// lattice order inside a level. The geometry x(xi) = sum_v N_v(xi) X_v uses the degree-1
// prism functions N_v, so J varies over the cell (the cell is not affine) and the element
// matrix is the quadrature sum itself.
// Quadrature (this definition is the one the library implements too): n = k+2 Gauss-Legendre
// points per direction on [0,1]; the triangle factor collapsed by (s,t) -> (s, t(1-s)) with
// weight w_s w_t (1-s); zeta = r with weight w_r. It integrates the mass integrand of any
// prism exactly (degree <= 2k+1 in the triangle variables and <= 2k+2 in zeta).
// ---------------------------------------------------------------------------
Rule prism_rule(int k) {
  const int n = k + 2;
  std::vector<double> x, w;
  gauss_legendre01(n, x, w);
  Rule R;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      for (int l = 0; l < n; ++l) {
        const double s = x[i], t = x[j], r = x[l];
        R.pts.push_back(s);
        R.pts.push_back(t * (1.0 - s));
        R.pts.push_back(r);
        R.wts.push_back(w[i] * w[j] * (1.0 - s) * w[l]);
      }
  R.nq = (int)R.wts.size();
  return R;
}

// interval Lagrange function c of degree k on the nodes m/k, and its derivative
void line_lagrange(int k, int c, double z, double& v, double& dv) {
  v = 1.0;
  dv = 0.0;
  for (int m = 0; m <= k; ++m) {
    if (m == c) continue;
    const double den = (double)(c - m) / k, fac = (z - (double)m / k) / den;
    dv = dv * fac + v / den;  // product rule, one factor at a time
    v *= fac;
  }
}

int prism_ndof(int k) { return (k + 1) * (k + 2) / 2 * (k + 1); }

// values phi[i] and reference derivatives dphi[i*3 + a] of the prism basis at x
void eval_prism_basis(const Basis& T, int k, const double* x, double* phi, double* dphi) {
  const int nt = T.n;
  std::vector<double> pt(nt), dpt((size_t)nt * 2);
  eval_basis(T, x, pt.data(), dpt.data());
  for (int c = 0; c <= k; ++c) {
    double L, dL;
    line_lagrange(k, c, x[2], L, dL);
    for (int t = 0; t < nt; ++t) {
      const int i = c * nt + t;
      if (phi) phi[i] = pt[t] * L;
      if (dphi) {
        dphi[(size_t)i * 3 + 0] = dpt[(size_t)t * 2 + 0] * L;
        dphi[(size_t)i * 3 + 1] = dpt[(size_t)t * 2 + 1] * L;
        dphi[(size_t)i * 3 + 2] = pt[t] * dL;
      }
    }
  }
}

// Jacobian of the prism map at xi: J[r][c] = sum_v X[v][r] dN_v/dxi_c
void prism_jacobian(const double* X, const double* xi, double J[3][3]) {
  const double s = xi[0], t = xi[1], z = xi[2];
  const double lam[3] = {1.0 - s - t, s, t};
  const double dlam[3][2] = {{-1.0, -1.0}, {1.0, 0.0}, {0.0, 1.0}};
  double dN[6][3];
  for (int v = 0; v < 3; ++v) {
    dN[v][0] = dlam[v][0] * (1.0 - z);
    dN[v][1] = dlam[v][1] * (1.0 - z);
    dN[v][2] = -lam[v];
    dN[v + 3][0] = dlam[v][0] * z;
    dN[v + 3][1] = dlam[v][1] * z;
    dN[v + 3][2] = lam[v];
  }
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double acc = 0.0;
      for (int v = 0; v < 6; ++v) acc += X[v * 3 + r] * dN[v][c];
      J[r][c] = acc;
    }
}

// Element matrix of one prism (MASS, HELMHOLTZ or ADVDIFF): the quadrature loop nest of
// section 2, with the Jacobian, its determinant and inverse evaluated at every point. For
// ADVDIFF, cf holds (eps, b_0, b_1, b_2) at the six vertices; eps and b are degree-1 prism
// fields, evaluated at each point with the prism's own vertex functions N_v.
void prism_matrix(int form, int k, const Basis& T, const Rule& R, const double* phiq, const double* dphiq,
                  const double* X, const double* cf, double* A) {
  const int n = prism_ndof(k);
  std::fill(A, A + (size_t)n * n, 0.0);
  std::vector<double> grad((size_t)n * 3);
  for (int q = 0; q < R.nq; ++q) {
    double J[3][3];
    prism_jacobian(X, &R.pts[(size_t)q * 3], J);
    // inverse by the adjugate: K[a][c] = cofactor(c,a) / det
    const double C00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    const double C01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    const double C02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    const double det = J[0][0] * C00 + J[0][1] * C01 + J[0][2] * C02;
    double K[3][3];
    K[0][0] = C00 / det;
    K[1][0] = C01 / det;
    K[2][0] = C02 / det;
    K[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
    K[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
    K[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
    K[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
    K[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
    K[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
    const double* phi = phiq + (size_t)q * n;
    const double* dphi = dphiq + (size_t)q * n * 3;
    for (int i = 0; i < n; ++i)
      for (int c = 0; c < 3; ++c) {
        double g = 0.0;
        for (int a = 0; a < 3; ++a) g += K[a][c] * dphi[(size_t)i * 3 + a];
        grad[(size_t)i * 3 + c] = g;
      }
    const double wd = R.wts[q] * std::fabs(det);
    double eps = 0.0, b[3] = {0.0, 0.0, 0.0};
    if (form == FORM_ADVDIFF) {
      const double* x = &R.pts[(size_t)q * 3];
      const double lam[3] = {1.0 - x[0] - x[1], x[0], x[1]};
      for (int v = 0; v < 6; ++v) {
        const double Nv = v < 3 ? lam[v] * (1.0 - x[2]) : lam[v - 3] * x[2];
        eps += Nv * cf[v * 4];
        for (int r = 0; r < 3; ++r) b[r] += Nv * cf[v * 4 + 1 + r];
      }
    }
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        const double gg = grad[(size_t)i * 3] * grad[(size_t)j * 3] + grad[(size_t)i * 3 + 1] * grad[(size_t)j * 3 + 1] +
                          grad[(size_t)i * 3 + 2] * grad[(size_t)j * 3 + 2];
        double v;
        if (form == FORM_ADVDIFF)
          v = eps * gg + phi[i] * (b[0] * grad[(size_t)j * 3] + b[1] * grad[(size_t)j * 3 + 1] +
                                   b[2] * grad[(size_t)j * 3 + 2]);
        else
          v = phi[i] * phi[j] + (form == FORM_HELMHOLTZ ? gg : 0.0);
        A[(size_t)i * n + j] += wd * v;
      }
  }
}

// Vector Burgers on prisms (section 5.2 runs Burgers on prisms too). The element matrix is the
// Jacobian of the residual R[(c,i)] = int (u.grad u_c) phi_i + nu grad u_c . grad phi_i, taken as
// in cell_matrix's Burgers branch, with the prism's Jacobian, determinant and inverse at every
// quadrature point. u is the degree-k vector field, u[r][c] at the n prism nodes.
// Quadrature: the same construction as prism_rule with n = (3k+3)/2 points per direction, since
// the trilinear term phi_i phi_j d u has degree 3k-1 in the triangle variables (one more under
// the collapsed map) and 3k in zeta on prisms with planar faces.
int prism_burgers_points(int k) { return (3 * k + 3) / 2; }

Rule prism_rule_points(int n) {
  std::vector<double> x, w;
  gauss_legendre01(n, x, w);
  Rule R;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      for (int l = 0; l < n; ++l) {
        R.pts.push_back(x[i]);
        R.pts.push_back(x[j] * (1.0 - x[i]));
        R.pts.push_back(x[l]);
        R.wts.push_back(w[i] * w[j] * (1.0 - x[i]) * w[l]);
      }
  R.nq = (int)R.wts.size();
  return R;
}

// physical gradients g[i][m] = sum_a K[a][m] dphi_i[a] of the n prism functions at a point, and
// w |det J| there (K = J^{-1} by the adjugate)
double prism_point(const double* X, const double* xi, double w, const double* dphi, int n, double* g) {
  double J[3][3];
  prism_jacobian(X, xi, J);
  double adj[3][3];  // adj[a][m] = cofactor(m, a)
  adj[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  adj[1][0] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
  adj[2][0] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  adj[0][1] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
  adj[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
  adj[2][1] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
  adj[0][2] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
  adj[1][2] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
  adj[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
  const double det = J[0][0] * adj[0][0] + J[0][1] * adj[1][0] + J[0][2] * adj[2][0];
  for (int i = 0; i < n; ++i)
    for (int m = 0; m < 3; ++m) {
      double s = 0.0;
      for (int a = 0; a < 3; ++a) s += adj[a][m] / det * dphi[(size_t)i * 3 + a];
      g[(size_t)i * 3 + m] = s;
    }
  return w * std::fabs(det);
}

// u(x_q)[a] and grad u(x_q)[a][m] from the nodal values
void prism_u_at(const double* u, const double* phi, const double* g, int n, double uq[3], double gu[3][3]) {
  for (int a = 0; a < 3; ++a) {
    uq[a] = 0.0;
    for (int m = 0; m < 3; ++m) gu[a][m] = 0.0;
  }
  for (int r = 0; r < n; ++r)
    for (int a = 0; a < 3; ++a) {
      uq[a] += u[r * 3 + a] * phi[r];
      for (int m = 0; m < 3; ++m) gu[a][m] += u[r * 3 + a] * g[(size_t)r * 3 + m];
    }
}

// element matrix [3n][3n] (component-blocked rows and columns (c, i))
void prism_burgers_matrix(int k, const Rule& R, const double* phiq, const double* dphiq, const double* X,
                          const double* u, double nu, double* A) {
  const int n = prism_ndof(k), N = 3 * n;
  std::fill(A, A + (size_t)N * N, 0.0);
  std::vector<double> g((size_t)n * 3);
  for (int q = 0; q < R.nq; ++q) {
    const double* ph = phiq + (size_t)q * n;
    const double Dw = prism_point(X, &R.pts[(size_t)q * 3], R.wts[q], dphiq + (size_t)q * n * 3, n, g.data());
    double uq[3], gu[3][3];
    prism_u_at(u, ph, g.data(), n, uq, gu);
    for (int ci = 0; ci < 3; ++ci)
      for (int i = 0; i < n; ++i)
        for (int cj = 0; cj < 3; ++cj)
          for (int j = 0; j < n; ++j) {
            // (du.grad u).v + (u.grad du).v + nu grad du : grad v, du = phi_j e_cj, v = phi_i e_ci
            double s = ph[i] * ph[j] * gu[ci][cj];
            if (ci == cj) {
              double ug = 0.0, gg = 0.0;
              for (int m = 0; m < 3; ++m) {
                ug += uq[m] * g[(size_t)j * 3 + m];
                gg += g[(size_t)i * 3 + m] * g[(size_t)j * 3 + m];
              }
              s += ph[i] * ug + nu * gg;
            }
            A[(size_t)(ci * n + i) * N + cj * n + j] += s * Dw;
          }
  }
}

// element residual [3n]
void prism_burgers_residual(int k, const Rule& R, const double* phiq, const double* dphiq, const double* X,
                            const double* u, double nu, double* Rv) {
  const int n = prism_ndof(k);
  std::fill(Rv, Rv + 3 * n, 0.0);
  std::vector<double> g((size_t)n * 3);
  for (int q = 0; q < R.nq; ++q) {
    const double* ph = phiq + (size_t)q * n;
    const double Dw = prism_point(X, &R.pts[(size_t)q * 3], R.wts[q], dphiq + (size_t)q * n * 3, n, g.data());
    double uq[3], gu[3][3];
    prism_u_at(u, ph, g.data(), n, uq, gu);
    for (int c = 0; c < 3; ++c) {
      double adv = 0.0;
      for (int m = 0; m < 3; ++m) adv += uq[m] * gu[c][m];
      for (int i = 0; i < n; ++i) {
        double visc = 0.0;
        for (int m = 0; m < 3; ++m) visc += gu[c][m] * g[(size_t)i * 3 + m];
        Rv[c * n + i] += (adv * ph[i] + nu * visc) * Dw;
      }
    }
  }
}

void set_threads(int nthreads) {
#ifdef _OPENMP
  omp_set_num_threads(nthreads > 0 ? nthreads : omp_get_num_procs());
#else
  (void)nthreads;
#endif
}

}  // namespace

extern "C" {

int oracle_ndof(int form, int degree, int cell) {
  if (!valid(form, degree, cell)) return -1;
  int ns = (int)lattice(cell, degree).size();
  return form == FORM_BURGERS ? dim_of(cell) * ns : ns;
}

int oracle_threads_available(void) {
#ifdef _OPENMP
  return omp_get_num_procs();
#else
  return 1;
#endif
}

// Quadrature rule exact to `degree`: returns nq; fills pts [nq*d], wts [nq] when non-NULL.
int oracle_quadrature(int cell, int degree, double* pts, double* wts) {
  if (!(cell == CELL_TRI || cell == CELL_TET) || degree < 0 || degree > 40) return -1;
  Rule R = collapsed_rule(cell, degree);
  if (pts) std::memcpy(pts, R.pts.data(), R.pts.size() * sizeof(double));
  if (wts) std::memcpy(wts, R.wts.data(), R.wts.size() * sizeof(double));
  return R.nq;
}

// Lagrange nodes of degree k on the reference cell: X [n*d]; returns n.
int oracle_nodes(int cell, int k, double* X) {
  if (!(cell == CELL_TRI || cell == CELL_TET) || k < 1 || k > 6) return -1;
  auto L = lattice(cell, k);
  int d = dim_of(cell);
  if (X)
    for (size_t n = 0; n < L.size(); ++n)
      for (int a = 0; a < d; ++a) X[n * d + a] = (double)L[n][a] / k;
  return (int)L.size();
}

// Degree-k Lagrange basis at npts points x [npts*d]: phi [npts*n], dphi [npts*n*d].
int oracle_basis(int cell, int k, int npts, const double* x, double* phi, double* dphi) {
  if (!(cell == CELL_TRI || cell == CELL_TET) || k < 1 || k > 6) return -1;
  Basis B = lagrange(cell, k);
  int d = B.d;
  for (int p = 0; p < npts; ++p)
    eval_basis(B, x + (size_t)p * d, phi ? phi + (size_t)p * B.n : nullptr,
               dphi ? dphi + (size_t)p * B.n * d : nullptr);
  return B.n;
}

// Element matrices out [ncells][ndof][ndof] (float64) for cells [0, ncells).
// coef/c2d: ADVDIFF: coef = [ncoefnodes][1+d] rows (eps, b_0..b_{d-1}), c2d [ncells][d+1];
//           BURGERS: coef = u [ncoefnodes][d], c2d [ncells][ns]; otherwise unused.
int oracle_assemble(int form, int degree, int cell, double nu, const double* coords,
                    const int32_t* c2v, const double* coef, const int32_t* c2d,
                    int64_t ncoefnodes, int64_t ncells, double* out, int nthreads) {
  if (!valid(form, degree, cell) || ncells < 0) return -1;
  Ctx c = make_ctx(form, degree, cell, nu);
  const int n = c.ndof, d = c.d;
  set_threads(nthreads);
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < ncells; ++e) {
    double X[12], cf[128];  // up to d*ns = 105 Burgers coefficients (vector P4 tetrahedron)
    gather(c, coords, c2v, coef, c2d, ncoefnodes, e, X, cf);
    cell_matrix<double>(c, X, cf, out + e * (int64_t)n * n);
  }
  (void)d;
  return 0;
}

// Element matrices of a subset of cells: out [nsel][ndof][ndof] for cells sel[].
int oracle_assemble_cells(int form, int degree, int cell, double nu, const double* coords,
                          const int32_t* c2v, const double* coef, const int32_t* c2d,
                          int64_t ncoefnodes, const int64_t* sel, int64_t nsel, double* out,
                          int nthreads) {
  if (!valid(form, degree, cell) || nsel < 0) return -1;
  Ctx c = make_ctx(form, degree, cell, nu);
  const int n = c.ndof;
  set_threads(nthreads);
#pragma omp parallel for schedule(static)
  for (int64_t s = 0; s < nsel; ++s) {
    double X[12], cf[128];  // up to d*ns = 105 Burgers coefficients (vector P4 tetrahedron)
    gather(c, coords, c2v, coef, c2d, ncoefnodes, sel[s], X, cf);
    cell_matrix<double>(c, X, cf, out + s * (int64_t)n * n);
  }
  return 0;
}

// Burgers element residual vectors out [ncells][d*ns].
int oracle_burgers_residual(int degree, int cell, double nu, const double* coords,
                            const int32_t* c2v, const double* u, const int32_t* c2d,
                            int64_t ncoefnodes, int64_t ncells, double* out) {
  if (!valid(FORM_BURGERS, degree, cell) || ncells < 0) return -1;
  Ctx c = make_ctx(FORM_BURGERS, degree, cell, nu);
  for (int64_t e = 0; e < ncells; ++e) {
    double X[12], cf[128];  // up to d*ns = 105 Burgers coefficients (vector P4 tetrahedron)
    gather(c, coords, c2v, u, c2d, ncoefnodes, e, X, cf);
    cell_residual_burgers(c, X, cf, out + e * (int64_t)c.d * c.ns);
  }
  return 0;
}

// Adjoint of the assembly: given dL/dA (dout [ncells][ndof][ndof]) accumulate
// dL/dcoords (d_coords [nverts][d], +=) and dL/dcoef (d_coef, coef layout, +=).
// Each cell's derivative is the forward-mode (dual number) derivative of the
// same cell routine that computes the element matrix, one seed per local input.
int oracle_assemble_backward(int form, int degree, int cell, double nu, const double* coords,
                             const int32_t* c2v, const double* coef, const int32_t* c2d,
                             int64_t ncoefnodes, int64_t ncells, const double* dout,
                             double* d_coords, double* d_coef, int nthreads) {
  if (!valid(form, degree, cell) || ncells < 0) return -1;
  Ctx c = make_ctx(form, degree, cell, nu);
  const int n = c.ndof, d = c.d, nx = (d + 1) * d, ncf = ncf_local(c);
  const int nseed = nx + ncf;
  std::vector<double> local((size_t)ncells * nseed);
  set_threads(nthreads);
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < ncells; ++e) {
    double X[12], cf[128];  // up to d*ns = 105 Burgers coefficients (vector P4 tetrahedron)
    gather(c, coords, c2v, coef, c2d, ncoefnodes, e, X, cf);
    std::vector<Dual> Xd(nx), cfd(ncf > 0 ? ncf : 1), Ad((size_t)n * n);
    const double* G = dout + e * (int64_t)n * n;
    for (int s = 0; s < nseed; ++s) {
      for (int i = 0; i < nx; ++i) Xd[i] = Dual(X[i], s == i ? 1.0 : 0.0);
      for (int i = 0; i < ncf; ++i) cfd[i] = Dual(cf[i], s == nx + i ? 1.0 : 0.0);
      cell_matrix<Dual>(c, Xd.data(), cfd.data(), Ad.data());
      double acc = 0.0;
      for (int i = 0; i < n * n; ++i) acc += G[i] * Ad[i].d;
      local[(size_t)e * nseed + s] = acc;
    }
  }
  // scatter-add in cell order
  for (int64_t e = 0; e < ncells; ++e) {
    const double* L = &local[(size_t)e * nseed];
    for (int v = 0; v <= d; ++v) {
      int64_t vid = c2v[e * (d + 1) + v];
      for (int r = 0; r < d; ++r) d_coords[vid * d + r] += L[v * d + r];
    }
    if (form == FORM_ADVDIFF) {
      for (int v = 0; v <= d; ++v) {
        int64_t id = c2d[e * (d + 1) + v];
        d_coef[id * (d + 1)] += L[nx + v];
        for (int r = 0; r < d; ++r) d_coef[id * (d + 1) + 1 + r] += L[nx + (d + 1) + v * d + r];
      }
    } else if (form == FORM_BURGERS) {
      for (int rr = 0; rr < c.ns; ++rr) {
        int64_t id = c2d[e * c.ns + rr];
        for (int a = 0; a < d; ++a) d_coef[id * d + a] += L[nx + rr * d + a];
      }
    }
  }
  return 0;
}

// ---- prisms ----
int oracle_prism_ndof(int degree) { return (degree >= 1 && degree <= 4) ? prism_ndof(degree) : -1; }

// the prism quadrature rule: pts [nq][3], wts [nq]; NULL pointers query nq
int oracle_prism_rule(int degree, double* pts, double* wts) {
  if (degree < 1 || degree > 4) return -1;
  Rule R = prism_rule(degree);
  if (pts) std::memcpy(pts, R.pts.data(), R.pts.size() * sizeof(double));
  if (wts) std::memcpy(wts, R.wts.data(), R.wts.size() * sizeof(double));
  return R.nq;
}

// prism basis values [npts][n] and reference derivatives [npts][n][3] at x [npts][3]
int oracle_prism_basis(int degree, int npts, const double* x, double* phi, double* dphi) {
  if (degree < 1 || degree > 4) return -1;
  Basis T = lagrange(CELL_TRI, degree);
  const int n = prism_ndof(degree);
  for (int p = 0; p < npts; ++p)
    eval_prism_basis(T, degree, x + (size_t)p * 3, phi ? phi + (size_t)p * n : nullptr,
                     dphi ? dphi + (size_t)p * n * 3 : nullptr);
  return 0;
}

// element matrices [ncells][n][n] of MASS, HELMHOLTZ or ADVDIFF on prisms: coords [nverts][3],
// cell2vert [ncells][6] (bottom triangle, then the top vertices above it); ADVDIFF: coef rows
// (eps, b_0, b_1, b_2) per coefficient node, cell2dof [ncells][6] (the cell's vertices)
int oracle_prism_assemble(int form, int degree, const double* coords, const int32_t* c2v, const double* coef,
                          const int32_t* c2d, int64_t ncells, double* out, int nthreads) {
  if (!(form == FORM_MASS || form == FORM_HELMHOLTZ || form == FORM_ADVDIFF) || degree < 1 || degree > 4 ||
      ncells < 0)
    return -1;
  if (form == FORM_ADVDIFF && (!coef || !c2d)) return -1;
  Basis T = lagrange(CELL_TRI, degree);
  Rule R = prism_rule(degree);
  const int n = prism_ndof(degree);
  std::vector<double> phiq((size_t)R.nq * n), dphiq((size_t)R.nq * n * 3);
  for (int q = 0; q < R.nq; ++q)
    eval_prism_basis(T, degree, &R.pts[(size_t)q * 3], &phiq[(size_t)q * n], &dphiq[(size_t)q * n * 3]);
  set_threads(nthreads);
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < ncells; ++e) {
    double X[18], cf[24] = {0};
    for (int v = 0; v < 6; ++v)
      for (int r = 0; r < 3; ++r) X[v * 3 + r] = coords[(int64_t)c2v[e * 6 + v] * 3 + r];
    if (form == FORM_ADVDIFF)
      for (int v = 0; v < 6; ++v)
        for (int r = 0; r < 4; ++r) cf[v * 4 + r] = coef[(int64_t)c2d[e * 6 + v] * 4 + r];
    prism_matrix(form, degree, T, R, phiq.data(), dphiq.data(), X, cf, out + e * (int64_t)n * n);
  }
  return 0;
}

// the Burgers prism rule ((3k+3)/2 points per direction): pts [nq][3], wts [nq]; NULL queries nq
int oracle_prism_burgers_rule(int degree, double* pts, double* wts) {
  if (degree < 1 || degree > 4) return -1;
  Rule R = prism_rule_points(prism_burgers_points(degree));
  if (pts) std::memcpy(pts, R.pts.data(), R.pts.size() * sizeof(double));
  if (wts) std::memcpy(wts, R.wts.data(), R.wts.size() * sizeof(double));
  return R.nq;
}

// vector Burgers on prisms: u [ncoefnodes][3], cell2dof [ncells][n] (n = prism_ndof(degree));
// residual 0: Jacobians out [ncells][3n][3n]; residual 1: residual vectors out [ncells][3n]
int oracle_prism_burgers(int degree, int residual, double nu, const double* coords, const int32_t* c2v,
                         const double* u, const int32_t* c2d, int64_t ncells, double* out, int nthreads) {
  if (degree < 1 || degree > 4 || ncells < 0 || !u || !c2d) return -1;
  Basis T = lagrange(CELL_TRI, degree);
  Rule R = prism_rule_points(prism_burgers_points(degree));
  const int n = prism_ndof(degree), N = 3 * n;
  std::vector<double> phiq((size_t)R.nq * n), dphiq((size_t)R.nq * n * 3);
  for (int q = 0; q < R.nq; ++q)
    eval_prism_basis(T, degree, &R.pts[(size_t)q * 3], &phiq[(size_t)q * n], &dphiq[(size_t)q * n * 3]);
  set_threads(nthreads);
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < ncells; ++e) {
    double X[18];
    std::vector<double> ue((size_t)n * 3);
    for (int v = 0; v < 6; ++v)
      for (int r = 0; r < 3; ++r) X[v * 3 + r] = coords[(int64_t)c2v[e * 6 + v] * 3 + r];
    for (int r = 0; r < n; ++r)
      for (int a = 0; a < 3; ++a) ue[(size_t)r * 3 + a] = u[(int64_t)c2d[e * n + r] * 3 + a];
    if (residual)
      prism_burgers_residual(degree, R, phiq.data(), dphiq.data(), X, ue.data(), nu, out + e * (int64_t)N);
    else
      prism_burgers_matrix(degree, R, phiq.data(), dphiq.data(), X, ue.data(), nu, out + e * (int64_t)N * N);
  }
  return 0;
}

}  // extern "C"
