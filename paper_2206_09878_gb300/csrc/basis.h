// Host-side B-spline operators for the inhomogeneous (y) direction.
//
// Paper Appendix C (Eq. disc_f_inhomo and the B* space): every field except m2 is expanded in
// maximum-continuity B-splines of order p (degree p-1); m2 uses order p+1 on the same breakpoints,
// so that d/dy maps the m2 space exactly onto the space of the other fields. Knots are clamped
// with uniform breakpoints on [y0, y1]; Ny order-p functions, Ny+1 order-(p+1) functions.
// Collocation points are Greville abscissae.
#pragma once
#include <vector>

namespace lmvd {

// Row-banded matrix: row i holds entries for columns [c0[i], c0[i] + w).
struct RowBand {
  int rows = 0, cols = 0, w = 0;
  std::vector<int> c0;
  std::vector<double> v;  // rows * w
  double at(int i, int j) const {
    int q = j - c0[i];
    return (q >= 0 && q < w) ? v[(size_t)i * w + q] : 0.0;
  }
};

// Square matrix in diagonal band storage: a[i*(2K+1) + K + (j-i)] = A[i][j] for |j-i| <= K.
struct DiagBand {
  int n = 0, K = 0;
  std::vector<double> a;
  double& el(int i, int j) { return a[(size_t)i * (2 * K + 1) + K + (j - i)]; }
  double get(int i, int j) const {
    int q = j - i;
    return (q < -K || q > K) ? 0.0 : a[(size_t)i * (2 * K + 1) + K + q];
  }
};

struct Knots {
  int order = 0, n = 0;  // n basis functions
  std::vector<double> t;
};

Knots clamped_uniform(int order, int n, double y0, double y1);
std::vector<double> greville(const Knots& k);
// All `order` possibly non-zero basis functions (and their deriv-th derivative) at x:
// returns the first index; vals[r] belongs to function first + r.
int eval_nonzero(const Knots& k, double x, int deriv, double* vals);
RowBand collocation(const Knots& k, const std::vector<double>& pts, int deriv);
DiagBand to_diag(const RowBand& m, int K);
// Transposes (used by the adjoint): the transpose of a banded matrix is banded.
RowBand transpose(const RowBand& m);
DiagBand transpose(const DiagBand& a);

// No-pivoting LU of a band matrix (stable here: the y-systems have growth factor ~1).
// L multipliers lo[i*K + q-1] (q = 1..K, multiplier of row i-q); U: up[i*K + r-1] (r = 1..K),
// invd[i] = 1 / U[i][i]. nl[i], nu[i]: used lengths of the rows of L and U (profile).
struct BandLU {
  int n = 0, K = 0;
  std::vector<double> lo, up, invd;
  std::vector<int> nl, nu;
};
BandLU band_lu(const DiagBand& A);
// Weights w_i with sum_i w_i f(g_i) = integral over [y0, y1] of the order-p spline that interpolates f at
// the Greville points g_i: w = A^{-T} b, A the collocation matrix (B0g), b_j = (t_{j+p} - t_j) / p the
// integral of B_j.
std::vector<double> greville_quadrature(const Knots& k, const RowBand& B0g);
// Structural profile of L and U for the pattern union of A2 and A0 (no numerical values).
void band_profile(const DiagBand& A2, const DiagBand& A0, std::vector<int>& nl, std::vector<int>& nu);

}  // namespace lmvd
