// Host construction of the reference-triangle tables of the CUDA path (Sec. 2):
// Gauss-Jacobi rules (Golub-Welsch with an implicit-shift QL eigen-solver),
// discretization nodes (Blyth-Pozrikidis on interior Gauss-Lobatto points, the
// stand-in for Vioreanu-Rokhlin nodes), V = U^{-1}, ||V||_2, and the conical
// smooth-rule family.  FP64, computed once per context.
#include <math.h>

#include <algorithm>
#include <vector>

#include "lcq_internal.h"

namespace lcq {
namespace {

// Symmetric tridiagonal eigenproblem (diagonal a, off-diagonal b[1..n-1]) by the
// implicit QL method with Wilkinson-type shifts; z returns the first component of
// each normalized eigenvector (needed for Gauss weights).
bool tridiag_eig(std::vector<double>& a, std::vector<double> b, std::vector<double>* z) {
  const int n = (int)a.size();
  std::vector<double> e(n, 0.0);
  for (int i = 1; i < n; ++i) e[i - 1] = b[i];
  z->assign(n, 0.0);
  (*z)[0] = 1.0;
  for (int l = 0; l < n; ++l) {
    int iter = 0;
    int m;
    do {
      for (m = l; m < n - 1; ++m) {
        const double dd = fabs(a[m]) + fabs(a[m + 1]);
        if (fabs(e[m]) <= 1e-17 * dd) break;
      }
      if (m != l) {
        if (++iter > 100) return false;
        double g = (a[l + 1] - a[l]) / (2.0 * e[l]);
        double r = hypot(g, 1.0);
        g = a[m] - a[l] + e[l] / (g + (g >= 0 ? fabs(r) : -fabs(r)));
        double s = 1.0, c = 1.0, p = 0.0;
        int i;
        bool early = false;
        for (i = m - 1; i >= l; --i) {
          double f = s * e[i];
          const double bb = c * e[i];
          r = hypot(f, g);
          e[i + 1] = r;
          if (r == 0.0) {
            a[i + 1] -= p;
            e[m] = 0.0;
            early = true;
            break;
          }
          s = f / r;
          c = g / r;
          g = a[i + 1] - p;
          r = (a[i] - g) * s + 2.0 * c * bb;
          p = s * r;
          a[i + 1] = g + p;
          g = c * r - bb;
          f = (*z)[i + 1];
          (*z)[i + 1] = s * (*z)[i] + c * f;
          (*z)[i] = c * (*z)[i] - s * f;
        }
        if (early) continue;
        a[l] -= p;
        e[l] = g;
        e[m] = 0.0;
      }
    } while (m != l);
  }
  return true;
}

// Gauss-Jacobi rule with weight (1-x)^al (1+x)^be on [-1, 1], ascending nodes.
bool gauss_jacobi(int n, double al, double be, std::vector<double>* x, std::vector<double>* w) {
  std::vector<double> a(n), b(n, 0.0);
  for (int k = 0; k < n; ++k) {
    const double s = 2.0 * k + al + be;
    a[k] = (k == 0) ? (be - al) / (al + be + 2.0) : (be * be - al * al) / (s * (s + 2.0));
    if (k >= 1) {
      const double num = 4.0 * k * (k + al) * (k + be) * (k + al + be);
      const double den = s * s * (s + 1.0) * (s - 1.0);
      b[k] = sqrt(num / den);
    }
  }
  std::vector<double> z;
  if (!tridiag_eig(a, b, &z)) return false;
  const double mu0 = pow(2.0, al + be + 1.0) * tgamma(al + 1.0) * tgamma(be + 1.0) /
                     tgamma(al + be + 2.0);
  std::vector<int> idx(n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  std::sort(idx.begin(), idx.end(), [&](int p, int q) { return a[p] < a[q]; });
  x->resize(n);
  w->resize(n);
  for (int i = 0; i < n; ++i) {
    (*x)[i] = a[idx[i]];
    (*w)[i] = mu0 * z[idx[i]] * z[idx[i]];
  }
  return true;
}

// Gauss-Jordan inverse with partial pivoting (row-major n x n).
bool invert(int n, std::vector<double> A, std::vector<double>* inv) {
  inv->assign(n * n, 0.0);
  for (int i = 0; i < n; ++i) (*inv)[i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabs(A[r * n + c]) > fabs(A[piv * n + c])) piv = r;
    if (A[piv * n + c] == 0.0) return false;
    if (piv != c)
      for (int k = 0; k < n; ++k) {
        std::swap(A[c * n + k], A[piv * n + k]);
        std::swap((*inv)[c * n + k], (*inv)[piv * n + k]);
      }
    const double d = 1.0 / A[c * n + c];
    for (int k = 0; k < n; ++k) {
      A[c * n + k] *= d;
      (*inv)[c * n + k] *= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const double f = A[r * n + c];
      if (f == 0.0) continue;
      for (int k = 0; k < n; ++k) {
        A[r * n + k] -= f * A[c * n + k];
        (*inv)[r * n + k] -= f * (*inv)[c * n + k];
      }
    }
  }
  return true;
}

// Largest eigenvalue of a symmetric matrix by cyclic Jacobi rotations.
double sym_max_eig(int n, std::vector<double> S) {
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += S[p * n + q] * S[p * n + q];
    if (off < 1e-34) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = S[p * n + q];
        if (apq == 0.0) continue;
        const double th = (S[q * n + q] - S[p * n + p]) / (2.0 * apq);
        const double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {
          const double skp = S[k * n + p], skq = S[k * n + q];
          S[k * n + p] = c * skp - s * skq;
          S[k * n + q] = s * skp + c * skq;
        }
        for (int k = 0; k < n; ++k) {
          const double spk = S[p * n + k], sqk = S[q * n + k];
          S[p * n + k] = c * spk - s * sqk;
          S[q * n + k] = s * spk + c * sqk;
        }
      }
  }
  double mx = S[0];
  for (int i = 1; i < n; ++i) mx = std::max(mx, S[i * n + i]);
  return mx;
}

}  // namespace

void ref_nodes_host(int d, std::vector<double>* u, std::vector<double>* v) {
  std::vector<double> x, w;
  gauss_jacobi(d + 1, 1.0, 1.0, &x, &w);
  // exact antisymmetry of the root set, then map to (0,1)
  std::vector<double> t(d + 1);
  for (int i = 0; i <= d; ++i) t[i] = (1.0 + 0.5 * (x[i] - x[d - i])) / 2.0;
  u->clear();
  v->clear();
  for (int i = 0; i <= d; ++i)
    for (int j = 0; j <= d - i; ++j) {
      const int k = d - i - j;
      u->push_back((1.0 + 2.0 * t[i] - t[j] - t[k]) / 3.0);
      v->push_back((1.0 + 2.0 * t[j] - t[i] - t[k]) / 3.0);
    }
}

// K_nm(u,v) = c_nm (1-v)^m P^{(0,2m+1)}_{n-m}(1-2v) P_m((2u+v-1)/(1-v)), order n-major.
void koornwinder_host(int d, double u, double v, double* K) {
  const double s = 2.0 * u + v - 1.0, q2 = (1.0 - v) * (1.0 - v), y = 1.0 - 2.0 * v;
  double Lp = 0.0, L = 1.0;
  for (int m = 0; m <= d; ++m) {
    if (m > 0) {
      const double Ln = ((2.0 * m - 1.0) * s * L - (m - 1.0) * q2 * Lp) / m;
      Lp = L;
      L = Ln;
    }
    const double b = 2.0 * m + 1.0;
    double Pp = 0.0, P = 1.0;
    for (int a = 0; a <= d - m; ++a) {
      const int n = m + a;
      K[n * (n + 1) / 2 + m] = sqrt(2.0 * (2 * m + 1) * (n + 1)) * L * P;
      const double den = 2.0 * (a + 1) * (a + b + 1) * (2 * a + b);
      const double c1 = (2 * a + b + 1) * (2 * a + b + 2) * (2 * a + b) / den;
      const double c0 = -(2 * a + b + 1) * b * b / den;
      const double c2 = 2.0 * a * (a + b) * (2 * a + b + 2) / den;
      const double Pn = (c1 * y + c0) * P - c2 * Pp;
      Pp = P;
      P = Pn;
    }
  }
}

// K_nm and its u, v derivatives at (u, v) (the scaled-Legendre and Jacobi recurrences
// differentiated term by term).
static void koornwinder_host_derivs(int d, double u, double v, double* K, double* Ku, double* Kv) {
  const double s = 2.0 * u + v - 1.0, q = 1.0 - v, q2 = q * q, y = 1.0 - 2.0 * v;
  double Lp = 0.0, L = 1.0, Lup = 0.0, Lu = 0.0, Lvp = 0.0, Lv = 0.0;
  for (int m = 0; m <= d; ++m) {
    if (m > 0) {
      const double f1 = 2.0 * m - 1.0, f2 = m - 1.0;
      const double Ln = (f1 * s * L - f2 * q2 * Lp) / m;
      const double Lun = (f1 * (2.0 * L + s * Lu) - f2 * q2 * Lup) / m;
      const double Lvn = (f1 * (L + s * Lv) - f2 * (-2.0 * q * Lp + q2 * Lvp)) / m;
      Lp = L;
      L = Ln;
      Lup = Lu;
      Lu = Lun;
      Lvp = Lv;
      Lv = Lvn;
    }
    const double b = 2.0 * m + 1.0;
    double Pp = 0.0, P = 1.0, dPp = 0.0, dP = 0.0;
    for (int a = 0; a <= d - m; ++a) {
      const int n = m + a, idx = n * (n + 1) / 2 + m;
      const double cn = sqrt(2.0 * (2 * m + 1) * (n + 1));
      K[idx] = cn * L * P;
      Ku[idx] = cn * Lu * P;
      Kv[idx] = cn * (Lv * P - 2.0 * L * dP);  // d/dv of P(1 - 2v) is -2 P'
      const double den = 2.0 * (a + 1) * (a + b + 1) * (2 * a + b);
      const double c1 = (2 * a + b + 1) * (2 * a + b + 2) * (2 * a + b) / den;
      const double c0 = -(2 * a + b + 1) * b * b / den;
      const double c2 = 2.0 * a * (a + b) * (2 * a + b + 2) / den;
      const double t = c1 * y + c0;
      const double Pn = t * P - c2 * Pp;
      const double dPn = c1 * P + t * dP - c2 * dPp;
      Pp = P;
      P = Pn;
      dPp = dP;
      dP = dPn;
    }
  }
}

// Du[nm][j] = int_T0 dK_nm/du K_j, Dv likewise, j over the degree d-1 basis: the
// derivative of a degree-d series sum_nm x_nm K_nm is sum_j (sum_nm x_nm D[nm][j]) K_j
// (the basis is orthonormal on T0).  Conical-product rule of m = d + 1 points per
// direction, exact to degree 2d + 1.
static bool build_derivative_tables(int d, std::vector<double>* Du, std::vector<double>* Dv) {
  const int n = n_basis(d), nd = n_basis(d - 1);
  Du->assign((size_t)n * nd, 0.0);
  Dv->assign((size_t)n * nd, 0.0);
  std::vector<double> xa, wa, xb, wb, K(n), Ku(n), Kv(n);
  const int m = d + 1;
  if (!gauss_jacobi(m, 1.0, 0.0, &xa, &wa) || !gauss_jacobi(m, 0.0, 0.0, &xb, &wb)) return false;
  for (int i = 0; i < m; ++i) {
    const double a = 0.5 * (1.0 + xa[i]), Wa = wa[i] / 4.0;
    for (int j = 0; j < m; ++j) {
      const double bb = 0.5 * (1.0 + xb[j]), W = Wa * wb[j] / 2.0;
      koornwinder_host_derivs(d, bb * (1.0 - a), a, K.data(), Ku.data(), Kv.data());
      for (int r = 0; r < n; ++r)
        for (int c = 0; c < nd; ++c) {
          (*Du)[(size_t)r * nd + c] += W * Ku[r] * K[c];
          (*Dv)[(size_t)r * nd + c] += W * Kv[r] * K[c];
        }
    }
  }
  return true;
}

bool build_deg_tables(int d, DegTables* t) {
  if (d < 1 || d > kMaxDeg) return false;
  const int n = n_basis(d);
  t->d = d;
  t->n = n;
  ref_nodes_host(d, &t->u, &t->v);
  // A[l][nm] = K_nm(u_l, v_l); V = A^{-1} has rows nm (Eq. v2c)
  std::vector<double> A(n * n), K(n);
  for (int l = 0; l < n; ++l) {
    koornwinder_host(d, t->u[l], t->v[l], K.data());
    for (int i = 0; i < n; ++i) A[l * n + i] = K[i];
  }
  if (!invert(n, A, &t->V)) return false;
  // interpolatory weights w_l = sum_nm V[nm][l] int K_nm, int K_nm = delta/sqrt(2)
  t->w.assign(n, 0.0);
  for (int l = 0; l < n; ++l) t->w[l] = t->V[0 * n + l] / sqrt(2.0);
  std::vector<double> S(n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double acc = 0.0;
      for (int k = 0; k < n; ++k) acc += t->V[k * n + i] * t->V[k * n + j];
      S[i * n + j] = acc;
    }
  t->normV = sqrt(sym_max_eig(n, S));
  return build_derivative_tables(d, &t->Du, &t->Dv);
}

bool build_rule_tables(RuleTables* t) {
  t->off.assign(kMaxRule + 2, 0);
  t->u.clear();
  t->v.clear();
  t->w.clear();
  for (int m = 1; m <= kMaxRule; ++m) {
    t->off[m] = (int)t->u.size();
    std::vector<double> xa, wa, xb, wb;
    if (!gauss_jacobi(m, 1.0, 0.0, &xa, &wa)) return false;   // weight (1-x)
    if (!gauss_jacobi(m, 0.0, 0.0, &xb, &wb)) return false;
    for (int i = 0; i < m; ++i) {
      const double a = 0.5 * (1.0 + xa[i]), Wa = wa[i] / 4.0;
      for (int j = 0; j < m; ++j) {
        const double b = 0.5 * (1.0 + xb[j]), Wb = wb[j] / 2.0;
        t->u.push_back(b * (1.0 - a));
        t->v.push_back(a);
        t->w.push_back(Wa * Wb);
      }
    }
  }
  t->off[kMaxRule + 1] = (int)t->u.size();
  t->gl_off.assign(kMaxGL + 2, 0);
  t->gl_x.clear();
  t->gl_w.clear();
  for (int g = 1; g <= kMaxGL; ++g) {
    t->gl_off[g] = (int)t->gl_x.size();
    std::vector<double> x, w;
    if (!gauss_jacobi(g, 0.0, 0.0, &x, &w)) return false;
    for (int i = 0; i < g; ++i) {
      t->gl_x.push_back(0.5 * (1.0 + 0.5 * (x[i] - x[g - 1 - i])));
      t->gl_w.push_back(0.25 * (w[i] + w[g - 1 - i]));
    }
  }
  t->gl_off[kMaxGL + 1] = (int)t->gl_x.size();
  return true;
}

}  // namespace lcq
