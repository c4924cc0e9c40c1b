// Banded-LU solves and banded evaluations shared by the forward and adjoint y-kernels.
#pragma once
#include "lmvd_internal.h"

namespace lmvd {

// ------------------------------------------------------------------ band LU access
// element (i, q) of L, (i, r) of U, 1 / U(i, i) for factor mode mf (ignored for shared factors)
__device__ inline double lu_lo(const DLU& f, int i, int q, int mf) {
  return __ldg(f.lo + (f.mstride ? ((size_t)(i * f.K + q - 1) * f.mstride + mf) : (size_t)(i * f.K + q - 1)));
}
__device__ inline double lu_up(const DLU& f, int i, int r, int mf) {
  return __ldg(f.up + (f.mstride ? ((size_t)(i * f.K + r - 1) * f.mstride + mf) : (size_t)(i * f.K + r - 1)));
}
__device__ inline double lu_invd(const DLU& f, int i, int mf) {
  return __ldg(f.invd + (f.mstride ? ((size_t)i * f.mstride + mf) : (size_t)i));
}

// Banded solves with the LU factors, for right-hand sides stored complex [row][mode]. Every y-system
// matrix is real, so the real and imaginary parts of a right-hand side are independent recurrences. A
// thread solves one element type V of one mode: V = cd (both parts; one thread per mode, each factor
// loaded once per mode) or V = double (one part, comp 0 = real, 1 = imaginary; two threads per mode).
// The second halves each thread's chain of dependent FP64 operations, which is what bounds these solves
// when the grid has few Fourier modes (GB300 retires 2 FP64 lanes per clock per SM, so a lone warp's
// dependent FP64 instruction costs ~64 cycles); with many modes the FP64 pipe is saturated either way
// and the first reads half as many factor words. A warp's accesses stay contiguous in both (16 modes x
// 2 parts, or 32 modes, of one row).
__device__ inline double vfma(double s, double x, double acc) { return fma(s, x, acc); }
__device__ inline cd vfma(double s, cd x, cd acc) { return fma_rc(s, x, acc); }
template <class V>
__device__ inline V vzero() {
  return V{};
}

// Element (i, m) of a [row][mode] complex array seen as V: its index in V units
template <class V>
__device__ inline size_t vidx(int i, size_t M, int m, int comp) {
  return sizeof(V) == sizeof(cd) ? (size_t)i * M + m : ((size_t)i * M + m) * 2 + comp;
}

// L U x = in, then out = x (+ add). out may alias in; add may be null.
template <class V>
__device__ void band_solve_v(const DLU& f, int m, int mf, int comp, const V* in, const V* add, V* out, size_t M) {
  if (!LMVD_IN(m, M) || (f.mstride && !LMVD_IN(mf, f.mstride)) || !LMVD_IN(f.K, KMAX + 1)) return;
  V win[KMAX];
#pragma unroll
  for (int q = 0; q < KMAX; ++q) win[q] = vzero<V>();
  for (int i = 0; i < f.n; ++i) {
    V v = in[vidx<V>(i, M, m, comp)];
    const int nl = __ldg(f.nl + i);
#pragma unroll
    for (int q = 1; q <= KMAX; ++q)
      if (q <= nl) v = vfma(-lu_lo(f, i, q, mf), win[q - 1], v);
#pragma unroll
    for (int q = KMAX - 1; q > 0; --q) win[q] = win[q - 1];
    win[0] = v;
    out[vidx<V>(i, M, m, comp)] = v;
  }
#pragma unroll
  for (int q = 0; q < KMAX; ++q) win[q] = vzero<V>();
  for (int i = f.n - 1; i >= 0; --i) {
    const size_t o = vidx<V>(i, M, m, comp);
    V v = out[o];
    const int nu = __ldg(f.nu + i);
#pragma unroll
    for (int r = 1; r <= KMAX; ++r)
      if (r <= nu) v = vfma(-lu_up(f, i, r, mf), win[r - 1], v);
    v = lu_invd(f, i, mf) * v;
#pragma unroll
    for (int q = KMAX - 1; q > 0; --q) win[q] = win[q - 1];
    win[0] = v;
    out[o] = add ? v + add[o] : v;
  }
}

// Solve A^T x = in with the factors A = L U of A (no pivoting): A^T = U^T L^T, so a forward sweep with
// U^T (lower triangular, diagonal of U) is followed by a backward sweep with L^T (unit upper). Entries of
// the factors outside their profile are stored as zeros, so the sweeps run over K. Rows of the result
// outside [zlo, zhi] are stored as zero (the recurrence itself uses the unmodified values). out may
// alias in.
template <class V>
__device__ void band_solve_T_v(const DLU& f, int m, int mf, int comp, const V* in, V* out, size_t M, int zlo,
                               int zhi) {
  if (!LMVD_IN(m, M) || (f.mstride && !LMVD_IN(mf, f.mstride)) || !LMVD_IN(f.K, KMAX + 1)) return;
  V win[KMAX];
#pragma unroll
  for (int q = 0; q < KMAX; ++q) win[q] = vzero<V>();
  for (int i = 0; i < f.n; ++i) {
    V v = in[vidx<V>(i, M, m, comp)];
#pragma unroll
    for (int r = 1; r <= KMAX; ++r)
      if (r <= f.K && i - r >= 0) v = vfma(-lu_up(f, i - r, r, mf), win[r - 1], v);
    v = lu_invd(f, i, mf) * v;
#pragma unroll
    for (int q = KMAX - 1; q > 0; --q) win[q] = win[q - 1];
    win[0] = v;
    out[vidx<V>(i, M, m, comp)] = v;
  }
#pragma unroll
  for (int q = 0; q < KMAX; ++q) win[q] = vzero<V>();
  for (int i = f.n - 1; i >= 0; --i) {
    const size_t o = vidx<V>(i, M, m, comp);
    V v = out[o];
#pragma unroll
    for (int q = 1; q <= KMAX; ++q)
      if (q <= f.K && i + q < f.n) v = vfma(-lu_lo(f, i + q, q, mf), win[q - 1], v);
#pragma unroll
    for (int q = KMAX - 1; q > 0; --q) win[q] = win[q - 1];
    win[0] = v;
    out[o] = (i < zlo || i > zhi) ? vzero<V>() : v;
  }
}

__device__ inline double band_row_real(const DBand& B, int i, const double* x) {
  double acc = 0.0;
  if (!LMVD_IN(i, B.rows)) return acc;
  const int c = B.c0[i];
  const double* v = B.v + (size_t)i * B.w;
  for (int q = 0; q < B.w; ++q)
    if (LMVD_IN(c + q, B.cols)) acc = fma(__ldg(v + q), x[c + q], acc);
  return acc;
}

}  // namespace lmvd
