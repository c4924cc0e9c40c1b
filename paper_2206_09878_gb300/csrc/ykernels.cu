// Kernels along the inhomogeneous direction y: one thread per Fourier mode (kx, kz) walks the
// B-spline rows, so a warp reads 32 consecutive modes of one row (coalesced, [y][kz][kx] layout).
//
// Paper: Sec. 4.1 (m^d, Eq. phi_poisson, md_recon), Sec. 4.2 (m^c, Eq. COM_fourier, CF_fourier,
// mc_recon, mc_mean), Sec. 4.4 (Eq. DNS_system, Algorithm 2), Sec. 3.2-3.3 (Eq. dzdt_guesses,
// midpoint RK2), Appendix C (B-spline spaces and the exact derivative map D*).
#include "band.cuh"
#include "ykernels.h"

namespace lmvd {

LMVD_DEFINE_OOB_TAKE(yk)

// ------------------------------------------------------------------ step 1-2 inputs: values at g
// out[0..7] = z, dz/dx, dz/dz, dz/dy, lap z, m1^d, m2^d, m3^d at the Greville points of the order-p space.
// m1^d, m3^d follow Eq. md_recon with d m2^d / dy evaluated directly from the order-(p+1) space;
// the k = 0 mode carries the plane means (and m2^d = 0).
// Rows are split into gridDim.y chunks (row_range), so that a grid with few modes still has enough
// threads, each with its own loads in flight.
__global__ void k_eval_p1(Grid g, DBand B0g, DBand B1g, DBand B2g, DBand Sg0, DBand Sg1, const cd* z,
                          const cd* om, const cd* m2, const double* mm1, const double* mm3, Fields8 out) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= (int)g.M) return;
  const size_t M = g.M;
  int r0, r1;
  row_range(g.ny, blockIdx.y, gridDim.y, r0, r1);
  if (is_nyquist(g, m)) {
    for (int i = r0; i < r1; ++i)
      for (int f = 0; f < 8; ++f) out.p[f][(size_t)i * M + m] = mk(0, 0);
    return;
  }
  double k1, k3;
  wavenumbers(g, m, k1, k3);
  const double k2 = k1 * k1 + k3 * k3;
  const double ik2 = m == 0 ? 0.0 : 1.0 / k2;
  for (int i = r0; i < r1; ++i) {
    const size_t o = (size_t)i * M + m;
    const cd zg = band_row(B0g, i, z, M, m);
    const cd zy = band_row(B1g, i, z, M, m);
    const cd zyy = band_row(B2g, i, z, M, m);
    out.p[0][o] = zg;
    out.p[1][o] = k1 * times_i(zg);
    out.p[2][o] = k3 * times_i(zg);
    out.p[3][o] = zy;
    out.p[4][o] = (-k2) * zg + zyy;
    if (m == 0) {
      out.p[5][o] = mk(band_row_real(B0g, i, mm1), 0.0);
      out.p[6][o] = mk(0, 0);
      out.p[7][o] = mk(band_row_real(B0g, i, mm3), 0.0);
    } else {
      const cd dm2 = band_row(Sg1, i, m2, M, m);
      const cd omg = band_row(B0g, i, om, M, m);
      out.p[5][o] = ik2 * times_i(k1 * dm2 - k3 * omg);
      out.p[6][o] = band_row(Sg0, i, m2, M, m);
      out.p[7][o] = ik2 * times_i(k3 * dm2 + k1 * omg);
    }
  }
}

// ------------------------------------------------------------------ generic values at points
// job blockIdx.y: out = B in (or out += B in), rows B.rows split into gridDim.z chunks; Nyquist modes
// zero (or unchanged).
__global__ void k_eval(Grid g, EvalJobs jobs) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= (int)g.M) return;
  const EvalJob& jb = jobs.j[blockIdx.y];
  const size_t M = g.M;
  const bool ny = is_nyquist(g, m);
  int r0, r1;
  row_range(jb.B.rows, blockIdx.z, gridDim.z, r0, r1);
  if (jb.acc) {
    if (ny) return;
    for (int i = r0; i < r1; ++i) jb.out[(size_t)i * M + m] = jb.out[(size_t)i * M + m] + band_row(jb.B, i, jb.in, M, m);
    return;
  }
  for (int i = r0; i < r1; ++i)
    jb.out[(size_t)i * M + m] = ny ? mk(0, 0) : band_row(jb.B, i, jb.in, M, m);
}

// ------------------------------------------------------------------ evaluations in double-float
// The precision path (precision = 1) evaluates the B-spline sums that feed the inverse transforms and the
// right-hand sides that follow the forward transforms in double-float on the FP32 pipe: the band entries
// come as pairs (DBand.vf), each complex double input is split with integer operations, the products are
// accumulated without renormalisation (error <= ~w 2^-48 of the sum of |terms|), and the result is
// renormalised and rounded back to a double with integer operations. The per-mode multipliers (i k1,
// 1/k^2, ...) are applied in double-float too, so these kernels issue no FP64 instruction per term.

// acc + b * x without renormalisation: TwoProd by FMA, TwoSum of the high parts, low parts summed
__device__ __forceinline__ df dfma_lazy(df b, df x, df acc) {
  const float p = __fmul_rn(b.hi, x.hi);
  float e = __fmaf_rn(b.hi, x.hi, -p);
  e = __fmaf_rn(b.hi, x.lo, e);
  e = __fmaf_rn(b.lo, x.hi, e);
  float s, t;
  two_sum(acc.hi, p, s, t);
  return df{s, __fadd_rn(__fadd_rn(acc.lo, e), t)};
}
__device__ __forceinline__ df drenorm(df a) {
  float s, e;
  two_sum(a.hi, a.lo, s, e);
  return df{s, e};
}
__device__ __forceinline__ cdf cd_to_cdf(cd x) { return cdf{df_from_double_int(x.re), df_from_double_int(x.im)}; }
__device__ __forceinline__ cd cdf_to_cd(cdf x) {
  return cd{df_to_double_int(drenorm(x.re)), df_to_double_int(drenorm(x.im))};
}
// The values these evaluations produce feed only the precision path's inverse transforms, whose z-pass
// works in double-float: they are stored as renormalised pairs (cdf, the same 16 bytes as a complex
// double) and the z-pass reads them as they are (fft_inverse_df_in), so neither side converts.
__device__ __forceinline__ void put_df(cd* p, size_t o, cdf v) {
  reinterpret_cast<cdf*>(p)[o] = cdf{drenorm(v.re), drenorm(v.im)};
}
__device__ __forceinline__ void put_df(cd* p, size_t o, cd v) { reinterpret_cast<cdf*>(p)[o] = cd_to_cdf(v); }

// A thread walks the rows of one mode, and a band's first column c0[i] never decreases and grows by at
// most one per row (Greville points are at most one knot interval apart), so each input coefficient is
// split into a double-float pair once and kept in a register window of the W columns c .. c + W - 1
// (W = the band width) instead of once per band entry that reads it.
template <int W>
struct DfWin {
  cdf v[W];
  int c = -(1 << 30);
  cd pre;             // the raw coefficient of column pre_col, loaded one row ahead
  int pre_col = -1;
  __device__ __forceinline__ cdf fetch(const cd* x, size_t M, int m, int col, int cols) const {
    if (col == pre_col) return cd_to_cdf(pre);
    return (col < cols && LMVD_IN(col, cols)) ? cd_to_cdf(x[(size_t)col * M + m]) : cdf{};
  }
  __device__ __forceinline__ void load(const cd* x, size_t M, int m, int c0, int cols) {
    c = c0;
#pragma unroll
    for (int q = 0; q < W; ++q) v[q] = fetch(x, M, m, c0 + q, cols);
  }
  // move the window to start at column c0
  __device__ __forceinline__ void seek(const cd* x, size_t M, int m, int c0, int cols) {
    if (c0 < c || c0 > c + 2) {
      load(x, M, m, c0, cols);
      return;
    }
    while (c < c0) {
#pragma unroll
      for (int q = 0; q < W - 1; ++q) v[q] = v[q + 1];
      v[W - 1] = fetch(x, M, m, c + W, cols);
      ++c;
    }
  }
  // issue the load of the column the next row's window adds (its first column is c_next), so that its
  // latency overlaps this row's arithmetic; a thread otherwise has a single load in flight
  __device__ __forceinline__ void prefetch(const cd* x, size_t M, int m, int c_next, int cols) {
    const int col = c_next + W - 1;
    if (c_next > c && col > c + W - 1 && col != pre_col && col < cols && LMVD_IN(col, cols)) {
      pre = x[(size_t)col * M + m];
      pre_col = col;
    }
  }
  // sum over q < w of b[q] v[q] (lazy accumulation)
  __device__ __forceinline__ cdf dot(const DBand& B, int i) const {
    const float2* b = reinterpret_cast<const float2*>(B.vf) + (size_t)i * B.w;
    df ar{0.f, 0.f}, ai{0.f, 0.f};
#pragma unroll
    for (int q = 0; q < W; ++q)
      if (q < B.w) {
        const float2 bq = __ldg(b + q);
        const df bb{bq.x, bq.y};
        ar = dfma_lazy(bb, v[q].re, ar);
        ai = dfma_lazy(bb, v[q].im, ai);
      }
    return cdf{ar, ai};
  }
};
__device__ __forceinline__ cdf cdf_add_lazy(cdf a, cdf b) { return cdf{dadd_lazy(a.re, b.re), dadd_lazy(a.im, b.im)}; }
__device__ __forceinline__ df df_of(double x) { return df_from_double_int(x); }

// k_eval_p1 in double-float (same outputs, same layout, FP64 values); WB: width of the order-p bands (B0g,
// B1g, B2g, one window each for z and Omega2), WS: of the order-(p+1) ones (Sg0, Sg1; one window for m2)
template <int WB, int WS>
__global__ void __launch_bounds__(128) k_eval_p1_df(Grid g, DBand B0g, DBand B1g, DBand B2g, DBand Sg0, DBand Sg1,
                                                    const cd* z, const cd* om, const cd* m2, const double* mm1,
                                                    const double* mm3, Fields8 out) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= (int)g.M) return;
  const size_t M = g.M;
  int r0, r1;
  row_range(g.ny, blockIdx.y, gridDim.y, r0, r1);
  if (is_nyquist(g, m)) {
    for (int i = r0; i < r1; ++i)
      for (int f = 0; f < 8; ++f) put_df(out.p[f], (size_t)i * M + m, mk(0, 0));
    return;
  }
  if (m == 0) {  // the plane means and the k = 0 z values: one mode, kept in FP64
    for (int i = r0; i < r1; ++i) {
      const size_t o = (size_t)i * M;
      put_df(out.p[0], o, band_row(B0g, i, z, M, 0));
      put_df(out.p[1], o, mk(0, 0));
      put_df(out.p[2], o, mk(0, 0));
      put_df(out.p[3], o, band_row(B1g, i, z, M, 0));
      put_df(out.p[4], o, band_row(B2g, i, z, M, 0));
      put_df(out.p[5], o, mk(band_row_real(B0g, i, mm1), 0.0));
      put_df(out.p[6], o, mk(0, 0));
      put_df(out.p[7], o, mk(band_row_real(B0g, i, mm3), 0.0));
    }
    return;
  }
  double k1d, k3d;
  wavenumbers(g, m, k1d, k3d);
  const double k2d = k1d * k1d + k3d * k3d;
  // per-mode multipliers, split once (one FP64 division per mode, none per row)
  const df k1 = df_of(k1d), k3 = df_of(k3d), nk2 = df_of(-k2d), ik2 = df_of(1.0 / k2d);
  const df nk1 = dneg(k1), nk3 = dneg(k3);
  DfWin<WB> wz, wo;
  DfWin<WS> wm;
  for (int i = r0; i < r1; ++i) {
    if (!LMVD_IN(i, B0g.rows) || !LMVD_IN(i, Sg0.rows)) continue;
    const size_t o = (size_t)i * M + m;
    const int cb = __ldg(B0g.c0 + i), cs = __ldg(Sg0.c0 + i);
    wz.seek(z, M, m, cb, B0g.cols);
    wo.seek(om, M, m, cb, B0g.cols);
    wm.seek(m2, M, m, cs, Sg0.cols);
    if (i + 1 < r1) {
      const int nb = __ldg(B0g.c0 + i + 1), ns = __ldg(Sg0.c0 + i + 1);
      wz.prefetch(z, M, m, nb, B0g.cols);
      wo.prefetch(om, M, m, nb, B0g.cols);
      wm.prefetch(m2, M, m, ns, Sg0.cols);
    }
    const cdf zg = wz.dot(B0g, i), zy = wz.dot(B1g, i), zyy = wz.dot(B2g, i);
    const cdf dm2 = wm.dot(Sg1, i), omg = wo.dot(B0g, i);
    const cdf zgr{drenorm(zg.re), drenorm(zg.im)};
    put_df(out.p[0], o, zgr);
    put_df(out.p[1], o, cdf{dmul(nk1, zgr.im), dmul(k1, zgr.re)});   // i k1 z
    put_df(out.p[2], o, cdf{dmul(nk3, zgr.im), dmul(k3, zgr.re)});   // i k3 z
    put_df(out.p[3], o, zy);
    put_df(out.p[4], o, cdf_add_lazy(cdf{dmul(nk2, zgr.re), dmul(nk2, zgr.im)}, zyy));  // -k^2 z + z''
    const cdf dmr{drenorm(dm2.re), drenorm(dm2.im)}, omr{drenorm(omg.re), drenorm(omg.im)};
    // m1^d = (i k1 dm2 - i k3 om) / k^2, m3^d = (i k3 dm2 + i k1 om) / k^2 (Eq. md_recon)
    const df a1 = ddot2(k1, dmr.re, nk3, omr.re), b1 = ddot2(k1, dmr.im, nk3, omr.im);
    const df a3 = ddot2(k3, dmr.re, k1, omr.re), b3 = ddot2(k3, dmr.im, k1, omr.im);
    put_df(out.p[5], o, cdf{dmul(ik2, dneg(b1)), dmul(ik2, a1)});
    put_df(out.p[6], o, wm.dot(Sg0, i));
    put_df(out.p[7], o, cdf{dmul(ik2, dneg(b3)), dmul(ik2, a3)});
  }
}

// k_eval in double-float (jobs without accumulation into out; values as double-float pairs); W: the widest
// band of the jobs
template <int W>
__global__ void __launch_bounds__(128) k_eval_df(Grid g, EvalJobs jobs) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= (int)g.M) return;
  const EvalJob& jb = jobs.j[blockIdx.y];
  const size_t M = g.M;
  const bool ny = is_nyquist(g, m);
  int r0, r1;
  row_range(jb.B.rows, blockIdx.z, gridDim.z, r0, r1);
  DfWin<W> win;
  for (int i = r0; i < r1; ++i) {
    if (ny) {
      put_df(jb.out, (size_t)i * M + m, mk(0, 0));
      continue;
    }
    win.seek(jb.in, M, m, __ldg(jb.B.c0 + i), jb.B.cols);
    if (i + 1 < r1) win.prefetch(jb.in, M, m, __ldg(jb.B.c0 + i + 1), jb.B.cols);
    put_df(jb.out, (size_t)i * M + m, win.dot(jb.B, i));
  }
}

// k_rhs_eval in double-float; the k = 0 mean right-hand sides stay in FP64 (one mode). WB: band width of the
// order-p space (B1g, B2g at g; Bs0..Bs3 at g*). Two sweeps: R_Omega2 (two windows), then R_phi2 (four).
template <int WB>
__global__ void __launch_bounds__(128) k_rhs_eval_df(Grid g, DBand B1g, DBand B2g, DBand Bs0, DBand Bs1, DBand Bs2,
                                                     DBand Bs3, Fields7C st, cd* r_om, cd* r_phi, double* r_m) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= (int)g.M) return;
  const size_t M = g.M;
  const int ny = g.ny;
  int r0, r1;
  row_range(ny + 1, blockIdx.y, gridDim.y, r0, r1);
  if (m == 0 || is_nyquist(g, m)) {
    for (int i = r0; i < r1; ++i) {
      if (i < ny) r_om[(size_t)i * M + m] = mk(0, 0);
      r_phi[(size_t)i * M + m] = mk(0, 0);
      if (m == 0 && i < ny) {
        r_m[i] = (band_row(B1g, i, st.p[1], M, 0) + band_row(B2g, i, st.p[2], M, 0)).re;
        r_m[ny + i] = (band_row(B1g, i, st.p[4], M, 0) + band_row(B2g, i, st.p[5], M, 0)).re;
      }
    }
    return;
  }
  {
    DfWin<WB> w1, w2;
    for (int i = r0; i < min(r1, ny); ++i) {
      const int c = __ldg(B1g.c0 + i);
      w1.seek(st.p[1], M, m, c, B1g.cols);
      w2.seek(st.p[2], M, m, c, B2g.cols);
      if (i + 1 < min(r1, ny)) {
        const int cn = __ldg(B1g.c0 + i + 1);
        w1.prefetch(st.p[1], M, m, cn, B1g.cols);
        w2.prefetch(st.p[2], M, m, cn, B2g.cols);
      }
      const cdf a = cdf_add_lazy(w1.dot(B1g, i), w2.dot(B2g, i));
      r_om[(size_t)i * M + m] = cdf_to_cd(cdf_add_lazy(a, cd_to_cdf(st.p[0][(size_t)i * M + m])));
    }
  }
  DfWin<WB> w3, w4, w5, w6;
  for (int i = r0; i < r1; ++i) {
    const int c = __ldg(Bs0.c0 + i);
    w3.seek(st.p[3], M, m, c, Bs0.cols);
    w4.seek(st.p[4], M, m, c, Bs1.cols);
    w5.seek(st.p[5], M, m, c, Bs2.cols);
    w6.seek(st.p[6], M, m, c, Bs3.cols);
    if (i + 1 < r1) {
      const int cn = __ldg(Bs0.c0 + i + 1);
      w3.prefetch(st.p[3], M, m, cn, Bs0.cols);
      w4.prefetch(st.p[4], M, m, cn, Bs1.cols);
      w5.prefetch(st.p[5], M, m, cn, Bs2.cols);
      w6.prefetch(st.p[6], M, m, cn, Bs3.cols);
    }
    const cdf b = cdf_add_lazy(w3.dot(Bs0, i), w4.dot(Bs1, i));
    const cdf d = cdf_add_lazy(w5.dot(Bs2, i), w6.dot(Bs3, i));
    r_phi[(size_t)i * M + m] = cdf_to_cd(cdf_add_lazy(b, d));
  }
}

// launchers for spline orders 4..8 (band widths 4..9); api.cu brackets them with its launch accounting
void launch_eval_p1_df(int p, dim3 grid, int tpb, cudaStream_t st, const Grid& g, const DBand& B0g, const DBand& B1g,
                       const DBand& B2g, const DBand& Sg0, const DBand& Sg1, const cd* z, const cd* om, const cd* m2,
                       const double* mm1, const double* mm3, const Fields8& out) {
  switch (p) {
#define LMVD_P1(P) \
    case P: k_eval_p1_df<P, P + 1><<<grid, tpb, 0, st>>>(g, B0g, B1g, B2g, Sg0, Sg1, z, om, m2, mm1, mm3, out); break;
    LMVD_P1(4) LMVD_P1(5) LMVD_P1(6) LMVD_P1(7) LMVD_P1(8)
#undef LMVD_P1
  }
}
void launch_eval_df(int w, dim3 grid, int tpb, cudaStream_t st, const Grid& g, const EvalJobs& jobs) {
  switch (w) {
#define LMVD_EV(W) \
    case W: k_eval_df<W><<<grid, tpb, 0, st>>>(g, jobs); break;
    LMVD_EV(4) LMVD_EV(5) LMVD_EV(6) LMVD_EV(7) LMVD_EV(8) LMVD_EV(9)
#undef LMVD_EV
  }
}
void launch_rhs_eval_df(int p, dim3 grid, int tpb, cudaStream_t st, const Grid& g, const DBand& B1g, const DBand& B2g,
                        const DBand* Bs, const Fields7C& stc, cd* r_om, cd* r_phi, double* r_m) {
  switch (p) {
#define LMVD_RE(P) \
    case P: k_rhs_eval_df<P><<<grid, tpb, 0, st>>>(g, B1g, B2g, Bs[0], Bs[1], Bs[2], Bs[3], stc, r_om, r_phi, r_m); break;
    LMVD_RE(4) LMVD_RE(5) LMVD_RE(6) LMVD_RE(7) LMVD_RE(8)
#undef LMVD_RE
  }
}

// ------------------------------------------------------------------ banded solves
// job blockIdx.y: out = A^{-1} in (+ add), factors shared or per mode (DLU.mstride); used for the
// collocation (interpolation) solves and the per-mode systems. out may alias in. Nyquist modes are set to
// zero. k_solve_cd: one thread per mode; k_solve_re: one thread per (mode, real part), see band_solve_v.
template <class V>
__device__ void solve_job(const Grid& g, const DLU& lu, const SolveJob& jb) {
  constexpr int TPM = sizeof(V) == sizeof(cd) ? 1 : 2;
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= TPM * g.M) return;
  const int m = (int)(t / TPM), comp = (int)(t % TPM);
  const size_t M = g.M;
  V* out = reinterpret_cast<V*>(jb.out);
  if (is_nyquist(g, m)) {
    for (int i = 0; i < lu.n; ++i) out[vidx<V>(i, M, m, comp)] = vzero<V>();
    return;
  }
  band_solve_v<V>(lu, m, lu.mstride ? factor_mode(g, m) : 0, comp, reinterpret_cast<const V*>(jb.in),
                  reinterpret_cast<const V*>(jb.add), out, M);
}
__global__ void k_solve_cd(Grid g, DLU lu, SolveJobs jobs) { solve_job<cd>(g, lu, jobs.j[blockIdx.y]); }
__global__ void k_solve_re(Grid g, DLU lu, SolveJobs jobs) { solve_job<double>(g, lu, jobs.j[blockIdx.y]); }

// ------------------------------------------------------------------ m^c from rho_t
// Eq. COM_fourier + CF_fourier with m_par eliminated: rows 1..ny-1 collocate
// (B*'' - k^2 B*) m2^c = -B' rho_t at the interior order-(p+1) Greville points, rows 0 and ny hold the
// boundary rows (walls: m2^c(+-1) = 0; potential matching: the Robin rows), all with zero right-hand side.
// Then m_par = i (rho_t + D* m2^c) / k (exact mass conservation in B-coefficient space) and
// Eq. mc_recon m1^c = k1/k m_par, m3^c = k3/k m_par.
// k = 0 (Eq. mc_mean): D* <m2^c> = -<rho_t> with <m2^c>(+1) = 0; <m1^c> = <m3^c> = 0.
// Three launches: k_mc_rhs (right-hand side into m2c), the banded solve (in place, per-mode factors),
// k_mc_post (m1c, m3c; the k = 0 mean).

// rows 0..ny split over gridDim.y chunks
__global__ void k_mc_rhs(Grid g, DBand Bs1, const cd* rt, cd* m2c) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= (int)g.M) return;
  const size_t M = g.M;
  const int ny = g.ny;
  int r0, r1;
  row_range(ny + 1, blockIdx.y, gridDim.y, r0, r1);
  const bool zero = m == 0 || is_nyquist(g, m);
  for (int i = r0; i < r1; ++i) {
    cd v = mk(0, 0);
    if (!zero && i > 0 && i < ny) {
      const cd d = band_row(Bs1, i, rt, M, m);
      v = mk(-d.re, -d.im);
    }
    m2c[(size_t)i * M + m] = v;
  }
}

// rows 0..ny-1 split over gridDim.y chunks; the k = 0 mode is one serial pass (chunk 0)
__global__ void k_mc_post(Grid g, const double* dstar, const cd* rt, cd* m1c, cd* m2c, cd* m3c) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= (int)g.M) return;
  const size_t M = g.M;
  const int ny = g.ny;
  int r0, r1;
  row_range(ny, blockIdx.y, gridDim.y, r0, r1);
  if (is_nyquist(g, m)) {
    for (int i = r0; i < r1; ++i) m1c[(size_t)i * M + m] = m3c[(size_t)i * M + m] = mk(0, 0);
    return;
  }
  if (m == 0) {
    if (blockIdx.y != 0) return;
    cd c = mk(0, 0);
    m2c[(size_t)ny * M] = c;
    for (int i = ny - 1; i >= 0; --i) {
      c = c + (1.0 / __ldg(dstar + i)) * rt[(size_t)i * M];
      m2c[(size_t)i * M] = c;
      m1c[(size_t)i * M] = m3c[(size_t)i * M] = mk(0, 0);
    }
    return;
  }
  double k1, k3;
  wavenumbers(g, m, k1, k3);
  const double k = sqrt(k1 * k1 + k3 * k3), ik = 1.0 / k;
  for (int i = r0; i < r1; ++i) {
    if (!LMVD_IN(i + 1, ny + 1)) continue;
    const cd x = m2c[(size_t)i * M + m], xn = m2c[(size_t)(i + 1) * M + m];
    const cd dm = __ldg(dstar + i) * (xn - x);
    const cd mpar = ik * times_i(rt[(size_t)i * M + m] + dm);
    m1c[(size_t)i * M + m] = (k1 * ik) * mpar;
    m3c[(size_t)i * M + m] = (k3 * ik) * mpar;
  }
}

// ------------------------------------------------------------------ RHS streams (Eq. DNS_system)
// sv[0..9] = C11, C12, C13, C22, C23, C33, u1, u2, u3, rho at the Greville points (values).
// With H_i = d_j C_ij + mu lap u_i - g rho delta_i2 (the (1/3) grad div u part of the viscous force is
// a gradient and cancels in both curls):
//   RHS_Omega2 = i k3 H1 - i k1 H3 = st0 + d/dy st1 + d2/dy2 st2,
//   RHS_phi2 = -k^2 H2 - d/dy (i k1 H1 + i k3 H3) = st3 + d/dy st4 + d2/dy2 st5 + d3/dy3 st6,
// so only st1..st6 need B-spline coefficients (st0 is already the value at g).
// k = 0: st1 = <C12>, st2 = mu <u1>, st4 = <C23>, st5 = mu <u3> carry the mean equations
// (Eq. mean_m1m3); the k = 0 values of all seven streams vanish otherwise.
__global__ void k_rhs_combine(Grid g, double mu, double grav, Fields10C sv, Fields7 st) {
  const size_t n = (size_t)g.ny * g.M;
  for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
    const int m = (int)(o % g.M);
    cd r[7];
    for (int q = 0; q < 7; ++q) r[q] = mk(0, 0);
    if (!is_nyquist(g, m)) {
      const cd C11 = sv.p[0][o], C12 = sv.p[1][o], C13 = sv.p[2][o], C22 = sv.p[3][o], C23 = sv.p[4][o],
               C33 = sv.p[5][o], u1 = sv.p[6][o], u2 = sv.p[7][o], u3 = sv.p[8][o], rho = sv.p[9][o];
      if (m == 0) {
        r[1] = C12;
        r[2] = mu * u1;
        r[4] = C23;
        r[5] = mu * u3;
      } else {
        double k1, k3;
        wavenumbers(g, m, k1, k3);
        const double k2 = k1 * k1 + k3 * k3;
        const cd w13 = times_i(k3 * u1 - k1 * u3);        // i k3 u1 - i k1 u3
        const cd d13 = times_i(k1 * u1 + k3 * u3);        // i k1 u1 + i k3 u3
        const cd c1223 = times_i(k1 * C12 + k3 * C23);    // i k1 C12 + i k3 C23
        r[0] = (-k1 * k3) * C11 + (k1 * k1 - k3 * k3) * C13 + (k1 * k3) * C33 - (mu * k2) * w13;
        r[1] = times_i(k3 * C12 - k1 * C23);
        r[2] = mu * w13;
        r[3] = (-k2) * (c1223 - grav * rho) + (mu * k2 * k2) * u2;
        r[4] = (-k2) * C22 + (k1 * k1) * C11 + (2.0 * k1 * k3) * C13 + (k3 * k3) * C33 + (mu * k2) * d13;
        r[5] = mk(-c1223.re, -c1223.im) - (mu * k2) * u2;
        r[6] = (-mu) * d13;
      }
    }
    for (int q = 0; q < 7; ++q) st.p[q][o] = r[q];
  }
}

// RHS values from the streams (st1..st6 now B coefficients): R_Omega2 at g (ny rows), R_phi2 at g*
// (ny + 1 rows), and for k = 0 the mean RHS (2 ny reals).
// Rows 0..ny (R_phi2 has ny + 1) are split into gridDim.y chunks.
__global__ void k_rhs_eval(Grid g, DBand B1g, DBand B2g, DBand Bs0, DBand Bs1, DBand Bs2, DBand Bs3, Fields7C st,
                           cd* r_om, cd* r_phi, double* r_m) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= (int)g.M) return;
  const size_t M = g.M;
  const int ny = g.ny;
  int r0, r1;
  row_range(ny + 1, blockIdx.y, gridDim.y, r0, r1);
  if (m == 0 || is_nyquist(g, m)) {
    for (int i = r0; i < r1; ++i) {
      if (i < ny) r_om[(size_t)i * M + m] = mk(0, 0);
      r_phi[(size_t)i * M + m] = mk(0, 0);
      if (m == 0 && i < ny) {
        r_m[i] = (band_row(B1g, i, st.p[1], M, 0) + band_row(B2g, i, st.p[2], M, 0)).re;
        r_m[ny + i] = (band_row(B1g, i, st.p[4], M, 0) + band_row(B2g, i, st.p[5], M, 0)).re;
      }
    }
    return;
  }
  for (int i = r0; i < r1; ++i) {
    if (i < ny)
      r_om[(size_t)i * M + m] = st.p[0][(size_t)i * M + m] + band_row(B1g, i, st.p[1], M, m) +
                                band_row(B2g, i, st.p[2], M, m);
    r_phi[(size_t)i * M + m] = band_row(Bs0, i, st.p[3], M, m) + band_row(Bs1, i, st.p[4], M, m) +
                               band_row(Bs2, i, st.p[5], M, m) + band_row(Bs3, i, st.p[6], M, m);
  }
}

// ------------------------------------------------------------------ RK2 update (step 6)
// Midpoint RK2 in low-storage form at the collocation points, X^{s+1} = X^s + dt (al R^s + be R^{s-1}),
// followed by the boundary-row solves (banded solves in place). Omega2 (blockIdx.z = 0): values at g,
// Dirichlet rows (interpolation LU); z (blockIdx.z = 1): values at g advanced with (dz/dt)^{k_f},
// Neumann rows dz/dy(+-1) = 0 (Neumann LU). This kernel writes the right-hand sides; rows split over
// gridDim.y chunks.
__global__ void k_update_om_z_rhs(Grid g, DBand B0g, UpdateArgs a) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= (int)g.M) return;
  const size_t M = g.M;
  const int ny = g.ny;
  const int job = blockIdx.z;
  cd* out = job == 0 ? a.om_new : a.z_new;
  int r0, r1;
  row_range(ny, blockIdx.y, gridDim.y, r0, r1);
  const bool zero = is_nyquist(g, m) || (job == 0 && m == 0);
  const double dt = a.dt, al = a.al, be = a.be;
  for (int i = r0; i < r1; ++i) {
    cd v = mk(0, 0);
    if (!zero && i > 0 && i < ny - 1) {
      if (job == 0) {
        const size_t o = (size_t)i * M + m;
        v = band_row(B0g, i, a.om, M, m) + dt * (al * a.r_om[o] + be * a.r_om_prev[o]);
      } else {
        const int c = B0g.c0[i];
        const double* w = B0g.v + (size_t)i * B0g.w;
        for (int q = 0; q < B0g.w; ++q) {
          const size_t o = (size_t)(c + q) * M + m;
          const cd zz = a.z[o] + dt * (al * a.zdot[o] + be * a.zdot_prev[o]);
          v = fma_rc(__ldg(w + q), zz, v);
        }
      }
    }
    out[(size_t)i * M + m] = v;
  }
}

// Plane means <m1>, <m3>: values at g advanced, no-slip Dirichlet rows (one thread per component).
__global__ void k_update_means(Grid g, DBand B0g, DLU lu_i, UpdateArgs a) {
  const int c = threadIdx.x;
  if (c > 1) return;
  const int ny = g.ny;
  const double* cur = c == 0 ? a.mm1 : a.mm3;
  double* out = c == 0 ? a.mm1_new : a.mm3_new;
  const double* r = a.r_m + c * ny;
  const double* rp = a.r_m_prev + c * ny;
  // real solve through the complex routine with a 1-mode stride
  double win[KMAX];
  for (int q = 0; q < KMAX; ++q) win[q] = 0.0;
  for (int i = 0; i < ny; ++i) {
    double v = 0.0;
    if (i > 0 && i < ny - 1) v = band_row_real(B0g, i, cur) + a.dt * (a.al * r[i] + a.be * rp[i]);
    const int nl = lu_i.nl[i];
    for (int q = 1; q <= nl; ++q) v -= lu_lo(lu_i, i, q, 0) * win[q - 1];
    for (int q = KMAX - 1; q > 0; --q) win[q] = win[q - 1];
    win[0] = v;
    out[i] = v;
  }
  for (int q = 0; q < KMAX; ++q) win[q] = 0.0;
  for (int i = ny - 1; i >= 0; --i) {
    double v = out[i];
    const int nu = lu_i.nu[i];
    for (int q = 1; q <= nu; ++q) v -= lu_up(lu_i, i, q, 0) * win[q - 1];
    v *= lu_i.invd[i];
    for (int q = KMAX - 1; q > 0; --q) win[q] = win[q - 1];
    win[0] = v;
    out[i] = v;
  }
}

// m2^d (Eq. phi_poisson): phi2 = (B*'' - k^2 B*) m2^d at g*_2 .. g*_{ny-2} advanced with RHS_phi2, four
// boundary rows (no-slip or potential matching) with zero right-hand side; k = 0: m2^d = 0. This kernel
// writes the right-hand side into m2_new (rows split over gridDim.y chunks); the banded solve with the
// per-mode factors then runs in place.
__global__ void k_update_m2_rhs(Grid g, DBand Ss0, DBand Ss2, UpdateArgs a) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= (int)g.M) return;
  const size_t M = g.M;
  const int ny = g.ny;
  int r0, r1;
  row_range(ny + 1, blockIdx.y, gridDim.y, r0, r1);
  cd* out = a.m2_new;
  const bool zero = m == 0 || is_nyquist(g, m);
  double k1 = 0.0, k3 = 0.0;
  if (!zero) wavenumbers(g, m, k1, k3);
  const double k2 = k1 * k1 + k3 * k3;
  const double dt = a.dt, al = a.al, be = a.be;
  for (int i = r0; i < r1; ++i) {
    cd v = mk(0, 0);
    if (!zero && i >= 2 && i <= ny - 2) {
      const size_t o = (size_t)i * M + m;
      const cd phi = band_row(Ss2, i, a.m2, M, m) - k2 * band_row(Ss0, i, a.m2, M, m);
      v = phi + dt * (al * a.r_phi[o] + be * a.r_phi_prev[o]);
    }
    out[(size_t)i * M + m] = v;
  }
}

// ------------------------------------------------------------------ failure detection
// Sets bit 0 of *flag if array blockIdx.y of the job list holds a non-finite double (inf or nan: all
// exponent bits set). Integer tests on the bit pattern keep this off the FP64 pipe; one atomic per warp.
__global__ void k_check_finite(CheckJobs jobs, unsigned* flag) {
  const CheckJob jb = pick(jobs.j, (int)blockIdx.y);
  bool bad = false;
  for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < jb.n; o += (size_t)gridDim.x * blockDim.x)
    bad |= (__double_as_longlong(jb.p[o]) & 0x7FF0000000000000ll) == 0x7FF0000000000000ll;
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1u);
}

// ------------------------------------------------------------------ diagnostics (lmvd_diagnostics)
// Block sums then one atomicAdd per block (the record is not bitwise reproducible; it is diagnostic only).
__device__ inline void block_add(double v, double* out) {
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) atomicAdd(out, v);
  }
}

// out[0] += |a - b|^2, out[1] += |a|^2 over n complex entries
__global__ void k_diff_norms(size_t n, const cd* a, const cd* b, double* out) {
  double d = 0.0, s = 0.0;
  for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
    const cd x = a[o], y = b[o];
    const double dr = x.re - y.re, di = x.im - y.im;
    d += dr * dr + di * di;
    s += x.re * x.re + x.im * x.im;
  }
  block_add(d, out);
  block_add(s, out + 1);
}

// Mass conservation of m^c in B-coefficient space (Sec. 4.2): out[0] += |rho_t + i k1 m1 + i k3 m3 + D* m2|^2,
// out[1] += |rho_t|^2, over all rows and modes (k = 0 included: D* <m2^c> = -<rho_t>)
__global__ void k_mass_norms(Grid g, const double* dstar, const cd* rt, const cd* m1, const cd* m2, const cd* m3,
                             double* out) {
  const size_t n = (size_t)g.ny * g.M;
  double d = 0.0, s = 0.0;
  for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
    const int m = (int)(o % g.M), i = (int)(o / g.M);
    double k1, k3;
    wavenumbers(g, m, k1, k3);
    const cd r = rt[o];
    const cd dm = __ldg(dstar + i) * (m2[o + g.M] - m2[o]);
    const cd res = r + times_i(k1 * m1[o] + k3 * m3[o]) + dm;
    d += res.re * res.re + res.im * res.im;
    s += r.re * r.re + r.im * r.im;
  }
  block_add(d, out);
  block_add(s, out + 1);
}

// Kinetic energy (1/2) integral of |m|^2 / rho over the domain and max |m|^2 over the grid, m = m^d + m^c on the
// padded grid. A plane's mean of a product on the 3/2 grid is the k = 0 coefficient of the dealiased product;
// the y-integral uses the quadrature weights of the Greville interpolant (wq), and the x-z area lx lz is
// applied on the host. df_fields: the physical fields hold double-float pairs (precision 1).
__device__ __forceinline__ double phys_value(const double* p, size_t o, int df_fields) {
  if (!df_fields) return p[o];
  const float2 v = reinterpret_cast<const float2*>(p)[o];
  return (double)v.x + (double)v.y;
}
__global__ void k_energy_norms(Grid g, const double* wq, Fields3C md, Fields3C mc, const double* invrho, int df_fields,
                               double* ke, unsigned long long* m2max) {
  const size_t n = (size_t)g.ny * g.P;
  double e = 0.0, mx = 0.0;
  for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
    double mm = 0.0;
    for (int c = 0; c < 3; ++c) {
      const double m = phys_value(md.p[c], o, df_fields) + phys_value(mc.p[c], o, df_fields);
      mm = fma(m, m, mm);
    }
    e = fma(0.5 * __ldg(wq + o / g.P) * mm, phys_value(invrho, o, df_fields), e);
    mx = fmax(mx, mm);
  }
  block_add(e / (double)g.P, ke);
  for (int q = 16; q > 0; q >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, q));
  if ((threadIdx.x & 31) == 0) atomicMax(m2max, (unsigned long long)__double_as_longlong(mx));
}

// bit 1 of *flag if the last (the kf-th) fixed-point application, recorded at diag[2 kf], diag[2 kf + 1],
// still changed dz/dt by half its size or more
__global__ void k_fp_check(const double* diag, int kf, unsigned* flag) {
  if (kf < 1) return;
  const double d = diag[2 * kf], s = diag[2 * kf + 1];
  if (d >= 0.25 * s && d > 0.0) atomicOr(flag, 2u);
}

// ------------------------------------------------------------------ elementwise helpers
// BDF-like guess (Eq. dzdt_guesses): zdot = (a0 z^s + a1 z^{s-1} + a2 z^{s-2} + a3 z^{s-3}) / dt.
__global__ void k_bdf(size_t n, double a0, double a1, double a2, double a3, double idt, const cd* z, const cd* h0,
                      const cd* h1, const cd* h2, cd* out) {
  for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x)
    out[o] = idt * (a0 * z[o] + a1 * h0[o] + a2 * h1[o] + a3 * h2[o]);
}

// start-up history: zh_q = z - c_q dt zdot
__global__ void k_backfill(size_t n, double c0, double c1, double c2, const cd* z, const cd* zdot, cd* h0, cd* h1,
                           cd* h2) {
  for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
    const cd zz = z[o], d = zdot[o];
    h0[o] = zz - c0 * d;
    h1[o] = zz - c1 * d;
    h2[o] = zz - c2 * d;
  }
}

// zero the Nyquist slots of a spectral field and, if zero_mean, its k = 0 slot
__global__ void k_sanitize(Grid g, int rows, cd* f, int zero_mean) {
  const size_t n = (size_t)rows * g.M;
  for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
    const int m = (int)(o % g.M);
    if (is_nyquist(g, m) || (zero_mean && m == 0)) f[o] = mk(0, 0);
  }
}

// ------------------------------------------------------------------ per-mode factorisation
// LU (no pivoting) of A(k) = A2 - k^2 A0 + k A1 for the factor modes (kx, kz >= 0), mf = jz * nxh + kx,
// jz = 0..nz/2 (stride Mh = (nz/2 + 1) nxh); A2, A0, A1 in diagonal band storage (half-width K, shared),
// profile nl/nu shared; entries outside the profile are stored as zeros. k = 0 and Nyquist modes get
// identity factors.
__global__ void k_factor(Grid g, int n, int K, const double* A2, const double* A0, const double* A1, const int* nl,
                         const int* nu, double* lo, double* up, double* invd) {
  const size_t Mh = (size_t)(g.nz / 2 + 1) * g.nxh;
  const int mf = blockIdx.x * blockDim.x + threadIdx.x;
  if (mf >= (int)Mh) return;
  const int jz = mf / g.nxh, kx = mf - jz * g.nxh;
  const int W = 2 * K + 1;
  if (mf == 0 || kx == g.nx / 2 || jz == g.nz / 2) {
    for (int i = 0; i < n; ++i) {
      for (int q = 0; q < K; ++q) lo[(size_t)(i * K + q) * Mh + mf] = up[(size_t)(i * K + q) * Mh + mf] = 0.0;
      invd[(size_t)i * Mh + mf] = 1.0;
    }
    return;
  }
  const double k1 = 6.283185307179586476925286766559 / g.lx * kx;
  const double k3 = 6.283185307179586476925286766559 / g.lz * jz;
  const double k2 = k1 * k1 + k3 * k3, k = sqrt(k2);
  double row[2 * KMAX + 1];
  for (int i = 0; i < n; ++i) {
    for (int q = 0; q < W; ++q)
      row[q] = A2[(size_t)i * W + q] - k2 * A0[(size_t)i * W + q] + k * A1[(size_t)i * W + q];
    for (int q = nl[i]; q >= 1; --q) {
      const int c = i - q;
      const double l = row[K - q] * invd[(size_t)c * Mh + mf];
      lo[(size_t)(i * K + q - 1) * Mh + mf] = l;
      row[K - q] = 0.0;
      for (int r = 1; r <= nu[c]; ++r) row[K - q + r] -= l * up[(size_t)(c * K + r - 1) * Mh + mf];
    }
    invd[(size_t)i * Mh + mf] = 1.0 / row[K];
    for (int r = 1; r <= K; ++r) up[(size_t)(i * K + r - 1) * Mh + mf] = r <= nu[i] ? row[K + r] : 0.0;
    for (int q = nl[i] + 1; q <= K; ++q) lo[(size_t)(i * K + q - 1) * Mh + mf] = 0.0;
  }
}

}  // namespace lmvd
