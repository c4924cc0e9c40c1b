// Banded-LU solves and banded evaluations shared by the forward and adjoint y-kernels.
#pragma once
#include "lmvd_internal.h"

namespace lmvd {

// ------------------------------------------------------------------ band LU access
__device__ inline double lu_lo(const DLU& f, int i, int q, int m) {
  return __ldg(f.lo + (f.mstride ? ((size_t)(i * f.K + q - 1) * f.mstride + m) : (size_t)(i * f.K + q - 1)));
}
__device__ inline double lu_up(const DLU& f, int i, int r, int m) {
  return __ldg(f.up + (f.mstride ? ((size_t)(i * f.K + r - 1) * f.mstride + m) : (size_t)(i * f.K + r - 1)));
}
__device__ inline double lu_invd(const DLU& f, int i, int m) {
  return __ldg(f.invd + (f.mstride ? ((size_t)i * f.mstride + m) : (size_t)i));
}

// Forward then backward substitution of L U x = rhs for mode m.
// rhs(i) gives row i of the right-hand side; y is scratch of n rows (stride M) that may alias the
// output; out(i, x_i, x_{i+1}) receives the solution in decreasing i.
template <class Rhs, class Out>
__device__ void band_solve(const DLU& f, int m, cd* y, size_t M, Rhs rhs, Out out) {
  cd win[KMAX];
#pragma unroll
  for (int q = 0; q < KMAX; ++q) win[q] = mk(0, 0);
  for (int i = 0; i < f.n; ++i) {
    cd v = rhs(i);
    const int nl = __ldg(f.nl + i);
#pragma unroll
    for (int q = 1; q <= KMAX; ++q)
      if (q <= nl) v = fma_rc(-lu_lo(f, i, q, m), win[q - 1], v);
#pragma unroll
    for (int q = KMAX - 1; q > 0; --q) win[q] = win[q - 1];
    win[0] = v;
    y[(size_t)i * M + m] = v;
  }
#pragma unroll
  for (int q = 0; q < KMAX; ++q) win[q] = mk(0, 0);
  for (int i = f.n - 1; i >= 0; --i) {
    cd v = y[(size_t)i * M + m];
    const int nu = __ldg(f.nu + i);
#pragma unroll
    for (int r = 1; r <= KMAX; ++r)
      if (r <= nu) v = fma_rc(-lu_up(f, i, r, m), win[r - 1], v);
    v = lu_invd(f, i, m) * v;
    out(i, v, win[0]);
#pragma unroll
    for (int q = KMAX - 1; q > 0; --q) win[q] = win[q - 1];
    win[0] = v;
  }
}

__device__ inline double band_row_real(const DBand& B, int i, const double* x) {
  const int c = B.c0[i];
  const double* v = B.v + (size_t)i * B.w;
  double acc = 0.0;
  for (int q = 0; q < B.w; ++q) acc = fma(__ldg(v + q), x[c + q], acc);
  return acc;
}

// Solve A^T x = rhs with the factors A = L U of A (no pivoting): A^T = U^T L^T, so a forward sweep
// with U^T (lower triangular, diagonal of U) is followed by a backward sweep with L^T (unit upper).
// Entries of the factors outside their profile are stored as zeros, so the sweeps run over K.
template <class Rhs, class Out>
__device__ void band_solve_T(const DLU& f, int m, cd* y, size_t M, Rhs rhs, Out out) {
  cd win[KMAX];
#pragma unroll
  for (int q = 0; q < KMAX; ++q) win[q] = mk(0, 0);
  for (int i = 0; i < f.n; ++i) {
    cd v = rhs(i);
#pragma unroll
    for (int r = 1; r <= KMAX; ++r)
      if (r <= f.K && i - r >= 0) v = fma_rc(-lu_up(f, i - r, r, m), win[r - 1], v);
    v = lu_invd(f, i, m) * v;
#pragma unroll
    for (int q = KMAX - 1; q > 0; --q) win[q] = win[q - 1];
    win[0] = v;
    y[(size_t)i * M + m] = v;
  }
#pragma unroll
  for (int q = 0; q < KMAX; ++q) win[q] = mk(0, 0);
  for (int i = f.n - 1; i >= 0; --i) {
    cd v = y[(size_t)i * M + m];
#pragma unroll
    for (int q = 1; q <= KMAX; ++q)
      if (q <= f.K && i + q < f.n) v = fma_rc(-lu_lo(f, i + q, q, m), win[q - 1], v);
    out(i, v, win[0]);
#pragma unroll
    for (int q = KMAX - 1; q > 0; --q) win[q] = win[q - 1];
    win[0] = v;
  }
}

}  // namespace lmvd
