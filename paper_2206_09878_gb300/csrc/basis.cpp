// Host-side B-spline operators (paper Appendix C). See basis.h.
//
// Evaluation uses de Boor's triangular recurrence for the order-(k-d) values in the knot interval
// containing x, and obtains d-th derivatives by differentiating each unit coefficient vector d
// times in coefficient space (d/dy sum c_j B_{j,k} = sum_j (k-1)(c_j - c_{j-1})/(t_{j+k-1}-t_j) B_{j,k-1}).
#include "basis.h"

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <stdexcept>

namespace lmvd {

Knots clamped_uniform(int order, int n, double y0, double y1) {
  Knots k;
  k.order = order;
  k.n = n;
  int nint = n - order + 1;
  if (nint < 1) throw std::invalid_argument("need n >= order");
  for (int i = 0; i < order - 1; ++i) k.t.push_back(y0);
  for (int i = 0; i <= nint; ++i) k.t.push_back(i == nint ? y1 : y0 + (y1 - y0) * (double)i / nint);
  for (int i = 0; i < order - 1; ++i) k.t.push_back(y1);
  return k;
}

std::vector<double> greville(const Knots& k) {
  std::vector<double> g(k.n);
  for (int j = 0; j < k.n; ++j) {
    double s = 0;
    for (int q = 1; q < k.order; ++q) s += k.t[j + q];
    g[j] = s / (k.order - 1);
  }
  return g;
}

// index l with t[l] <= x < t[l+1], t[l] < t[l+1]; x at the right end maps to the last interval
static int find_interval(const Knots& k, double x) {
  int lo = k.order - 1, hi = k.n;  // valid intervals are [t[l], t[l+1]) for l in [order-1, n-1]
  if (x >= k.t[hi]) return hi - 1;
  if (x <= k.t[lo]) return lo;
  int l = lo;
  while (l + 1 < hi && k.t[l + 1] <= x) ++l;
  return l;
}

// values of the `ord` order-`ord` B-splines B_{l-ord+1..l} at x in [t[l], t[l+1])
static void values_in_interval(const std::vector<double>& t, int l, int ord, double x, double* b) {
  std::vector<double> left(ord + 1), right(ord + 1);
  b[0] = 1.0;
  for (int j = 1; j < ord; ++j) {
    left[j] = x - t[l + 1 - j];
    right[j] = t[l + j] - x;
    double saved = 0.0;
    for (int r = 0; r < j; ++r) {
      double temp = b[r] / (right[r + 1] + left[j - r]);
      b[r] = saved + right[r + 1] * temp;
      saved = left[j - r] * temp;
    }
    b[j] = saved;
  }
}

int eval_nonzero(const Knots& k, double x, int deriv, double* vals) {
  const int K = k.order;
  const int l = find_interval(k, x);
  const int first = l - K + 1;
  for (int r = 0; r < K; ++r) vals[r] = 0.0;
  if (deriv >= K) return first;
  const int ko = K - deriv;
  std::vector<double> bl(ko);
  values_in_interval(k.t, l, ko, x, bl.data());  // B_{l-ko+1..l, ko}
  // for each basis function first + r: differentiate its unit coefficient vector deriv times
  std::vector<double> c(K), cn(K);
  for (int r = 0; r < K; ++r) {
    // coefficients on indices first..l (K of them) of the order-K space
    std::fill(c.begin(), c.end(), 0.0);
    c[r] = 1.0;
    for (int s = 0; s < deriv; ++s) {
      const int o = K - s;  // current order
      for (int q = 0; q < K; ++q) {
        const int j = first + q;
        const double h = k.t[j + o - 1] - k.t[j];
        const double prev = q > 0 ? c[q - 1] : 0.0;
        cn[q] = h > 0 ? (o - 1) * (c[q] - prev) / h : 0.0;
      }
      c.swap(cn);
    }
    // evaluate with the order-ko values: B_{j, ko} for j = l-ko+1..l, i.e. q = j - first = deriv..K-1
    double v = 0.0;
    for (int q = deriv; q < K; ++q) v += c[q] * bl[q - deriv];
    vals[r] = v;
  }
  return first;
}

RowBand collocation(const Knots& k, const std::vector<double>& pts, int deriv) {
  RowBand m;
  m.rows = (int)pts.size();
  m.cols = k.n;
  m.w = k.order;
  m.c0.resize(m.rows);
  m.v.assign((size_t)m.rows * m.w, 0.0);
  std::vector<double> vals(k.order);
  for (int i = 0; i < m.rows; ++i) {
    int first = eval_nonzero(k, pts[i], deriv, vals.data());
    // keep the window inside [0, n)
    int c0 = std::max(0, std::min(first, k.n - m.w));
    m.c0[i] = c0;
    for (int r = 0; r < k.order; ++r) {
      int j = first + r;
      if (j < 0 || j >= k.n) continue;
      m.v[(size_t)i * m.w + (j - c0)] = vals[r];
    }
  }
  return m;
}

DiagBand to_diag(const RowBand& m, int K) {
  DiagBand d;
  d.n = m.rows;
  d.K = K;
  d.a.assign((size_t)d.n * (2 * K + 1), 0.0);
  for (int i = 0; i < m.rows; ++i)
    for (int q = 0; q < m.w; ++q) {
      int j = m.c0[i] + q;
      double v = m.v[(size_t)i * m.w + q];
      if (v == 0.0) continue;
      if (std::abs(j - i) > K) throw std::runtime_error("band wider than K");
      d.el(i, j) = v;
    }
  return d;
}

RowBand transpose(const RowBand& m) {
  RowBand t;
  t.rows = m.cols;
  t.cols = m.rows;
  std::vector<int> lo(t.rows, t.cols), hi(t.rows, -1);
  for (int i = 0; i < m.rows; ++i)
    for (int q = 0; q < m.w; ++q) {
      const int j = m.c0[i] + q;
      if (j < 0 || j >= m.cols || m.v[(size_t)i * m.w + q] == 0.0) continue;
      lo[j] = std::min(lo[j], i);
      hi[j] = std::max(hi[j], i);
    }
  t.w = 1;
  for (int j = 0; j < t.rows; ++j)
    if (hi[j] >= lo[j]) t.w = std::max(t.w, hi[j] - lo[j] + 1);
  t.w = std::min(t.w, t.cols);
  t.c0.assign(t.rows, 0);
  t.v.assign((size_t)t.rows * t.w, 0.0);
  for (int j = 0; j < t.rows; ++j) {
    int c = hi[j] >= lo[j] ? lo[j] : 0;
    t.c0[j] = std::max(0, std::min(c, t.cols - t.w));
  }
  for (int i = 0; i < m.rows; ++i)
    for (int q = 0; q < m.w; ++q) {
      const int j = m.c0[i] + q;
      const double v = m.v[(size_t)i * m.w + q];
      if (j < 0 || j >= m.cols || v == 0.0) continue;
      t.v[(size_t)j * t.w + (i - t.c0[j])] = v;
    }
  return t;
}

DiagBand transpose(const DiagBand& a) {
  DiagBand t;
  t.n = a.n;
  t.K = a.K;
  t.a.assign(a.a.size(), 0.0);
  for (int i = 0; i < a.n; ++i)
    for (int q = -a.K; q <= a.K; ++q) {
      const int j = i + q;
      if (j >= 0 && j < a.n) t.el(j, i) = a.get(i, j);
    }
  return t;
}

void band_profile(const DiagBand& A2, const DiagBand& A0, std::vector<int>& nl, std::vector<int>& nu) {
  const int n = A2.n, K = A2.K;
  nl.assign(n, 0);
  nu.assign(n, 0);
  std::vector<int> last(n, 0);
  for (int i = 0; i < n; ++i) {
    int first = i, lst = i;
    for (int q = -K; q <= K; ++q) {
      int j = i + q;
      if (j < 0 || j >= n) continue;
      if (A2.get(i, j) != 0.0 || A0.get(i, j) != 0.0) {
        first = std::min(first, j);
        lst = std::max(lst, j);
      }
    }
    for (int c = first; c < i; ++c) lst = std::max(lst, last[c]);  // fill-in from eliminated rows
    last[i] = lst;
    nl[i] = i - first;
    nu[i] = lst - i;
    if (nl[i] > K || nu[i] > K) throw std::runtime_error("fill-in beyond K");
  }
}

std::vector<double> greville_quadrature(const Knots& k, const RowBand& B0g) {
  const int n = B0g.rows, p = k.order;
  int K = 0;
  for (int i = 0; i < n; ++i) K = std::max({K, std::abs(B0g.c0[i] - i), std::abs(B0g.c0[i] + B0g.w - 1 - i)});
  const BandLU f = band_lu(transpose(to_diag(B0g, K)));
  std::vector<double> w(n);
  for (int j = 0; j < n; ++j) w[j] = (k.t[j + p] - k.t[j]) / p;
  for (int i = 0; i < n; ++i)  // L y = b (unit lower)
    for (int q = 1; q <= f.nl[i]; ++q) w[i] -= f.lo[(size_t)i * K + q - 1] * w[i - q];
  for (int i = n - 1; i >= 0; --i) {  // U x = y
    for (int r = 1; r <= f.nu[i]; ++r) w[i] -= f.up[(size_t)i * K + r - 1] * w[i + r];
    w[i] *= f.invd[i];
  }
  return w;
}

BandLU band_lu(const DiagBand& A) {
  BandLU f;
  const int n = A.n, K = A.K;
  f.n = n;
  f.K = K;
  band_profile(A, A, f.nl, f.nu);
  f.lo.assign((size_t)n * K, 0.0);
  f.up.assign((size_t)n * K, 0.0);
  f.invd.assign(n, 0.0);
  std::vector<double> row(2 * K + 1);
  for (int i = 0; i < n; ++i) {
    for (int q = -K; q <= K; ++q) row[K + q] = A.get(i, i + q);
    for (int q = f.nl[i]; q >= 1; --q) {  // eliminate columns i-q in increasing column order
      const int c = i - q;
      const double l = row[K - q] * f.invd[c];
      f.lo[(size_t)i * K + q - 1] = l;
      row[K - q] = 0.0;
      for (int r = 1; r <= f.nu[c]; ++r) row[K - q + r] -= l * f.up[(size_t)c * K + r - 1];
    }
    if (row[K] == 0.0) throw std::runtime_error("zero pivot");
    f.invd[i] = 1.0 / row[K];
    for (int r = 1; r <= K; ++r) f.up[(size_t)i * K + r - 1] = row[K + r];
  }
  return f;
}

}  // namespace lmvd
