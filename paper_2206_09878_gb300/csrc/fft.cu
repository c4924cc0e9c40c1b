// Batched Fourier transforms in the periodic directions with the 3/2 rule (paper Eq. disc_f and
// Sec. 4.4: products are formed in physical space on a grid padded to 3N/2 points, so that
// quadratic products of retained modes do not alias; coefficients are truncated back to
// |kx| < nx/2, |kz| < nz/2 with the Nyquist slots zero).
//
// Each field transform runs in two passes through an intermediate array T[y][z][kx]
// (kx < nx/2 only -- the padded kx range carries zeros and is never stored):
//   inverse: z-pass (complex, length pz, zero-padded in kz) then x-pass (complex-to-real, length px,
//            two real rows packed into one complex transform);
//   forward: x-pass (real-to-complex, two rows per complex transform, split by Hermitian symmetry; the
//            split's factor 1/2 is left to the z-pass) then z-pass (complex, truncated, scaled by
//            1/(2 px pz), which is bit-for-bit the same as halving first: power-of-two scaling commutes
//            with every rounding of the pass).
// Synthesis is unnormalised: f(x, z) = sum_k fhat_k exp(i (k1 x + k3 z)).
// A pass is one CTA per (plane, field, batch of columns / row pairs); every 1D transform is a
// Stockham autosort FFT in shared memory with radix-4/3/2 stages and a precomputed twiddle table. The
// x-passes read and write their contiguous rows with the CTA's threads; the z-passes fetch their columns
// with TMA tile copies (cp.async.bulk.tensor) and write them with the threads.
//
// Arithmetic: complex double (precision 0) or complex double-float (precision 1, df64.h) selected
// by the complex type C. Spectral inputs and outputs are always complex double; the intermediate
// T and the physical fields are stored in the arithmetic's own type (double, or hi/lo float pairs
// of the same size), so the double-float path converts only at the spectral ends.
#include <cuda.h>  // CUtensorMap and its enums (the encoder is reached through the runtime, no libcuda link)

#include <cmath>
#include <cstring>
#include <mutex>
#include <type_traits>

#include "df64.h"
#include "lmvd_internal.h"

namespace lmvd {

LMVD_DEFINE_OOB_TAKE(fft)

struct FieldsC {
  const cd* p[10];
};
struct FieldsW {
  cd* p[10];
};
struct FieldsRC {
  const void* p[10];
};
struct FieldsRW {
  void* p[10];
};

// ------------------------------------------------------------------ arithmetic traits
template <class C>
struct FT;

template <>
struct FT<cd> {
  using R = double;
  __device__ static cd zero() { return mk(0, 0); }
  __device__ static cd add(cd a, cd b) { return a + b; }
  __device__ static cd sub(cd a, cd b) { return a - b; }
  __device__ static cd add_lazy(cd a, cd b) { return a + b; }
  __device__ static cd sub_lazy(cd a, cd b) { return a - b; }
  __device__ static cd ti(cd a) { return times_i(a); }
  __device__ static cd neg(cd a) { return cd{-a.re, -a.im}; }
  __device__ static cd cj(cd a) { return conj(a); }
  __device__ static cd half(cd a) { return 0.5 * a; }
  template <int SIGN>
  __device__ static cd mulw(cd v, const FFTPlan& p, int idx) {
    const double2 w = p.tw[idx];
    return cmul(v, cd{w.x, SIGN * w.y});
  }
  template <int SIGN>
  __device__ static cd mul_s3(cd v, const FFTPlan&) {  // SIGN sin(2 pi / 3) v
    return (SIGN * 0.86602540378443864676372317075294) * v;
  }
  __device__ static cd from_spec(cd x) { return x; }
  __device__ static cd to_spec(cd x, const FFTPlan& p) { return p.scale_d * x; }
  __device__ static cd make(R a, R b) { return cd{a, b}; }
  __device__ static R re(cd a) { return a.re; }
  __device__ static R im(cd a) { return a.im; }
  __device__ static R rzero() { return 0.0; }
  __device__ static R rmul(R a, R b) { return a * b; }
  // -(w1 m1 + w2 m2 + w3 m3), the expression of k_product_L
  __device__ static R dot3neg(R w1, R m1, R w2, R m2, R w3, R m3) { return -(w1 * m1 + w2 * m2 + w3 * m3); }
};

template <>
struct FT<cdf> {
  using R = df;
  __device__ static cdf zero() { return cdf{df{0.f, 0.f}, df{0.f, 0.f}}; }
  __device__ static cdf add(cdf a, cdf b) { return cadd(a, b); }
  __device__ static cdf sub(cdf a, cdf b) { return csub(a, b); }
  // intermediates of a butterfly that feed only add / sub: not renormalised
  __device__ static cdf add_lazy(cdf a, cdf b) { return cadd_lazy(a, b); }
  __device__ static cdf sub_lazy(cdf a, cdf b) { return csub_lazy(a, b); }
  __device__ static cdf ti(cdf a) { return ctimes_i(a); }
  __device__ static cdf neg(cdf a) { return cdf{dneg(a.re), dneg(a.im)}; }
  __device__ static cdf cj(cdf a) { return cconj(a); }
  __device__ static cdf half(cdf a) { return cdf{dscale2(a.re, 0.5f), dscale2(a.im, 0.5f)}; }
  template <int SIGN>
  __device__ static cdf mulw(cdf v, const FFTPlan& p, int idx) {
    const float4 w = p.twf[idx];
    const df wr{w.x, w.y};
    const df wi = SIGN > 0 ? df{w.z, w.w} : df{-w.z, -w.w};
    return cmulw_lazy(v, wr, wi);  // feeds only the butterfly's add / sub
  }
  template <int SIGN>
  __device__ static cdf mul_s3(cdf v, const FFTPlan& p) {
    const df s = SIGN > 0 ? p.s3f : dneg(p.s3f);
    return cdf{dmul(v.re, s), dmul(v.im, s)};
  }
  __device__ static cdf from_spec(cd x) { return cdf{df_from_double_int(x.re), df_from_double_int(x.im)}; }
  __device__ static cd to_spec(cdf x, const FFTPlan& p) {
    return cd{df_to_double_int(dmul(x.re, p.scale_f)), df_to_double_int(dmul(x.im, p.scale_f))};
  }
  __device__ static cdf make(R a, R b) { return cdf{a, b}; }
  __device__ static R re(cdf a) { return a.re; }
  __device__ static R im(cdf a) { return a.im; }
  __device__ static R rzero() { return df{0.f, 0.f}; }
  __device__ static R rmul(R a, R b) { return dmul(a, b); }
  // -(w1 m1 + w2 m2 + w3 m3), the arithmetic of k_product_L_df
  __device__ static R dot3neg(R w1, R m1, R w2, R m2, R w3, R m3) {
    return dneg(dadd(ddot2(w1, m1, w2, m2), dmul(w3, m3)));
  }
};

// One radix-R Stockham stage, in place in shared memory. The transform of length n is shared by
// tpt = n / EPT threads; thread tt owns the butterflies tt, tt + tpt, ... (EPT / R of them), loads all
// their inputs into registers, waits for the whole block, then writes the outputs back to the same
// buffer (the reads of every thread are complete before any write).
// Pruning by the 3/2 rule, in separate instantiations so that the other stages keep their registers:
// ZERO (a first radix-4 stage, L = 1): inputs at positions [lo, hi) are known to be zero (the padding of
// a synthesis), so their loads and the additions with them are skipped. SKIP (a last stage): outputs at
// positions [lo, hi) are not wanted (the truncated modes of an analysis), so their additions and stores
// are skipped.
// S: distance in elements between consecutive points of a transform in shared memory (1: contiguous; the
// z-passes interleave their columns, point i of column c at (i S + c)).
template <class C, int SIGN, int R, int EPT, bool ZERO = false, bool SKIP = false, int S = 1>
__device__ __forceinline__ void fft_stage(C* x, const FFTPlan& pl, int L, int tt, int tpt, int lo = 0, int hi = 0) {
  using F = FT<C>;
  static_assert(!ZERO || R == 4, "zero-input pruning is written for a first radix-4 stage");
  constexpr int NBT = EPT / R;
  const int n = pl.n;
  const int nb = n / R, Ls = L * R, tws = n / Ls;
  const bool pow2 = (L & (L - 1)) == 0;
  C v[NBT][R];
#pragma unroll
  for (int j = 0; j < NBT; ++j) {
    const int b = tt + j * tpt;
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int i = b + q * nb;
      bool ld = LMVD_IN(i, n);
      if constexpr (ZERO) ld = ld && (i < lo || i >= hi);
      v[j][q] = ld ? x[i * S] : FT<C>::zero();
    }
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < NBT; ++j) {
    const int b = tt + j * tpt;
    const int k = pow2 ? (b & (L - 1)) : (b % L);
    const int base = (b - k) * R + k;
    if (!LMVD_IN(base + (R - 1) * L, n)) continue;
    if (!ZERO && k) {
#pragma unroll
      for (int q = 1; q < R; ++q) v[j][q] = F::template mulw<SIGN>(v[j][q], pl, q * k * tws);
    }
    // output q at base + q L is written unless SKIP drops it
    auto want = [&](int q) { return !SKIP || base + q * L < lo || base + q * L >= hi; };
    if (R == 4) {
      C t0, t1, t2, d3;
      // ZERO: v2 = 0 gives t0 = t1 = v0; v1 = 0 gives t2 = v3 and v1 - v3 = -v3
      if (ZERO && b + 2 * nb >= lo && b + 2 * nb < hi) {
        t0 = v[j][0];
        t1 = v[j][0];
      } else {
        t0 = F::add_lazy(v[j][0], v[j][2]);
        t1 = F::sub_lazy(v[j][0], v[j][2]);
      }
      if (ZERO && b + nb >= lo && b + nb < hi) {
        t2 = v[j][3];
        d3 = F::ti(F::neg(v[j][3]));
      } else {
        t2 = F::add_lazy(v[j][1], v[j][3]);
        d3 = F::ti(F::sub_lazy(v[j][1], v[j][3]));
      }
      const C t3 = SIGN > 0 ? d3 : F::neg(d3);  // (SIGN i) (v1 - v3)
      if (want(0)) x[base * S] = F::add(t0, t2);
      if (want(1)) x[(base + L) * S] = F::add(t1, t3);
      if (want(2)) x[(base + 2 * L) * S] = F::sub(t0, t2);
      if (want(3)) x[(base + 3 * L) * S] = F::sub(t1, t3);
    } else if (R == 3) {
      const C t1 = F::add_lazy(v[j][1], v[j][2]);
      const C m = F::sub_lazy(v[j][0], F::half(t1));
      const C u = F::ti(F::template mul_s3<SIGN>(F::sub_lazy(v[j][1], v[j][2]), pl));
      if (want(0)) x[base * S] = F::add(v[j][0], t1);
      if (want(1)) x[(base + L) * S] = F::add(m, u);
      if (want(2)) x[(base + 2 * L) * S] = F::sub(m, u);
    } else {
      if (want(0)) x[base * S] = F::add(v[j][0], v[j][1]);
      if (want(1)) x[(base + L) * S] = F::sub(v[j][0], v[j][1]);
    }
  }
  __syncthreads();
}

template <class C, int SIGN, int EPT, bool SKIP, int S>
__device__ __forceinline__ void fft_stage_r(unsigned r2, C* x, const FFTPlan& pl, int L, int tt, int tpt, int lo,
                                            int hi) {
  if (r2 == 0) fft_stage<C, SIGN, 4, EPT, false, SKIP, S>(x, pl, L, tt, tpt, lo, hi);
  else if (r2 == 2) fft_stage<C, SIGN, 3, EPT, false, SKIP, S>(x, pl, L, tt, tpt, lo, hi);
  else fft_stage<C, SIGN, 2, EPT, false, SKIP, S>(x, pl, L, tt, tpt, lo, hi);
}

// All stages of one transform held at x (the caller has synchronised after filling x).
// SIGN = +1: synthesis (exp(+i)), -1: analysis. The result is in natural order in x. With PZ, positions
// [lo, hi) of the input are zero (pruned in a first radix-4 stage); with PS, positions [lo, hi) of the
// output are not wanted (pruned in the last stage). Compile-time switches, so that a pass without pruning
// compiles to the plain stages. The FP64 passes prune (synthesis 7%, analysis <1% faster at 512^3); the
// double-float ones do not (their x-passes spilled at the 72-register cap and lost 6%).
template <class C, int SIGN, int EPT, bool PZ = false, bool PS = false, int S = 1>
__device__ void fft_inplace(C* x, const FFTPlan& pl, int tt, int tpt, int lo = 0, int hi = 0) {
  int L = 1, s = 0;
  unsigned code = pl.code;
  if (PZ && lo < hi && (code & 3u) == 0 && pl.nst > 1) {
    fft_stage<C, SIGN, 4, EPT, true, false, S>(x, pl, 1, tt, tpt, lo, hi);
    L = 4;
    s = 1;
    code >>= 2;
  }
  const int last = PS && lo < hi ? pl.nst - 1 : pl.nst;
  for (; s < last; ++s, code >>= 2) {
    const unsigned r2 = code & 3u;
    fft_stage_r<C, SIGN, EPT, false, S>(r2, x, pl, L, tt, tpt, 0, 0);
    L *= r2 == 0 ? 4 : (r2 == 2 ? 3 : 2);
  }
  if (PS && s < pl.nst) fft_stage_r<C, SIGN, EPT, true, S>(code & 3u, x, pl, L, tt, tpt, lo, hi);
}

// The passes that prune (see fft_inplace).
template <class C>
constexpr bool kPrune = std::is_same<C, cd>::value;

// Whether fft_inplace with PZ = kPrune<C> skips a zero input band of plan pl: only a first radix-4 stage
// prunes, so a plan without one (n with a single factor 2) reads the band and it must hold zeros.
template <class C>
__device__ __forceinline__ bool prunes_zero_band(const FFTPlan& pl) {
  return kPrune<C> && (pl.code & 3u) == 0 && pl.nst > 1;
}

// Launch bounds: every pass caps its registers (FftMinCtas below); the FP64 kernels would otherwise take ~100
// and fit fewer CTAs, whose warps hide less of the FP64 pipe's latency. The x-passes run small CTAs (2
// transforms of 768 points, 6-7 per SM), so that the load, compute and store phases of different CTAs
// (separated by barriers) overlap: 7-8% faster in double-float at 512^3 than 256-thread CTAs. The z-passes
// take 4 kx columns per CTA (2 when 4 transforms do not fit FFT_CTA_Z threads); with 2 at 768 points the
// double-float inverse z-pass was 13% slower.
constexpr int FFT_CTA_X = 128, FFT_CTA_Z = 256;
// CTAs per SM each pass is compiled for, i.e. its register cap. FP64: 6 x-pass and 3 z-pass CTAs (80
// registers). Double-float: the x-passes fit 7 CTAs at 72 registers without spilling (inverse 1.5%, forward
// 2.8% faster at 512^3 than at 6) and the forward z-pass 4 at 64 (4.4% faster); the inverse z-pass lost 2.3%
// at 64 registers and keeps 3.
template <class C>
struct FftMinCtas {
  static constexpr int x = 6, z_inv = 3, z_fwd = 3;
};
template <>
struct FftMinCtas<cdf> {
  static constexpr int x = 7, z_inv = 3, z_fwd = 4;
};
// Loads a thread issues before it stores any of them, in the forward x-pass's gather and the inverse x-pass's
// loads of f': one load at a time would serialise a memory latency per iteration (ncu: long-scoreboard
// stalls dominated the double-float passes). The z-passes and the inverse x-pass's input come by TMA.
constexpr int FFT_LOAD_CHUNK = 4;

// ---------------------------------------------------------------- tile loads (TMA)
// The z-passes read columns of a row-major plane: batch consecutive kx (16-byte elements) of every z-row. A
// tensor-map tile copy (cp.async.bulk.tensor) fetches such a box (2 batch doubles x rows) into shared
// memory as one asynchronous operation completing on an mbarrier, instead of one 16-byte load per thread
// and element. The box lands row-major, i.e. as the interleaved layout the z-pass transforms work in.
struct ZMaps {
  CUtensorMap m[TBUF_FIELDS];  // one per field of the launch (z_inv: the spectral inputs; z_fwd: m[0] = T)
};

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// box of the 3D map at (x, y, z) (x in doubles) into dst; completes tx bytes on bar
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(smem_addr(dst)), "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
      : "memory");
}

// bytes (a multiple of 16, both addresses 16-byte aligned) from src to dst; completes them on bar
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

// Every thread waits for phase 0 of bar, for at most ~1 s of SM clock; false (and bit 2 of the context's
// status word, when there is one) if the copies did not complete by then.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned* flags) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, 0)) {
    if (clock64() - t0 > 2000000000ll) {
      if (flags && threadIdx.x == 0) atomicOr(flags, 4u);
      return false;
    }
  }
  return true;
}

// ---------------------------------------------------------------- inverse z-pass
// in: spectral value fields [ny][nz][nxh] (complex double); T: [f][ny][pz][nx/2] of C
// IN_DF (double-float arithmetic only): the inputs already hold double-float pairs (the precision path's
// evaluations store them so), read without conversion.
// A CTA transforms COLS kx columns of one plane. Shared layout: point z of column c at a[z COLS + c]; two
// tile loads per row block put the kz >= 0 rows at the top and the kz < 0 rows at the bottom of the padded
// column (the Nyquist row lands inside the zero band, which the FP64 passes never read and the double-float
// ones clear).
template <class C, int EPT, int COLS, bool IN_DF = false>
__global__ void __launch_bounds__(FFT_CTA_Z, FftMinCtas<C>::z_inv)
    k_fft_z_inv(FFTPlan pl, Grid g, const __grid_constant__ ZMaps maps, C* T, size_t tstride, unsigned* flags) {
  using F = FT<C>;
  extern __shared__ __align__(128) unsigned char sm_raw[];
  C* a = reinterpret_cast<C*>(sm_raw);
  const int pz = g.pz, nz = g.nz, h = g.nx / 2, n2 = nz / 2, H = pl.rows_in;
  const int kx0 = blockIdx.x * COLS, j = blockIdx.y, f = blockIdx.z;
  const int c = threadIdx.x % COLS, tt = threadIdx.x / COLS;
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(sm_raw + (size_t)pz * COLS * sizeof(C));
  if (threadIdx.x == 0) mbar_init(bar);
  __syncthreads();
  if (threadIdx.x == 0 && LMVD_IN(f, TBUF_FIELDS)) {
    mbar_expect_tx(bar, (unsigned)(nz * COLS * sizeof(C)));
    for (int r = 0; r < nz; r += H) {
      const int pos = r < n2 ? r : pz - nz + r;
      if (LMVD_IN((pos + H) * COLS - 1, pz * COLS)) tma_load_3d(a + (size_t)pos * COLS, &maps.m[f], 2 * kx0, r, j, bar);
    }
  }
  if (!mbar_wait_bounded(bar, flags)) return;
  constexpr bool convert = !IN_DF && !std::is_same<C, cd>::value;
  const bool zero_band = !prunes_zero_band<C>(pl);
  if (zero_band || convert) {
    // the padding band [n2, pz - n2 + 1) zeroed where the arithmetic reads it; spectral doubles to pairs
    for (int idx = threadIdx.x; idx < pz * COLS; idx += blockDim.x) {
      const int z = idx / COLS;
      if (z >= n2 && z < pz - n2 + 1) {
        if (zero_band) a[idx] = F::zero();
      } else if (convert) {
        a[idx] = F::from_spec(reinterpret_cast<const cd*>(a)[idx]);
      }
    }
    __syncthreads();
  }
  fft_inplace<C, 1, EPT, kPrune<C>, false, COLS>(a + c, pl, tt, pl.tpt, n2, pz - n2 + 1);  // kz padding: zero
  C* dst = T + f * tstride + (size_t)j * pz * h;
  for (int idx = threadIdx.x; idx < pz * COLS; idx += blockDim.x) {
    const int zz = idx / COLS, kx = kx0 + idx % COLS;
    if (kx < h && LMVD_IN((size_t)zz * h + kx, (size_t)pz * h)) dst[(size_t)zz * h + kx] = a[idx];
  }
}

// (row, column) of a flat index idx = row n + column that a thread advances by a fixed step: one division at
// the start instead of one per element (n is a run-time value, and an integer division costs tens of
// instructions in passes that are bound by their instruction issue).
struct RowCol {
  int r, c;
  __device__ __forceinline__ RowCol(int idx, int n) : r(idx / n), c(idx - (idx / n) * n) {}
  __device__ __forceinline__ void advance(int step, int n) {
    c += step;
    while (c >= n) {
      c -= n;
      ++r;
    }
  }
};

// ---------------------------------------------------------------- inverse x-pass (c2r, 2 rows per transform)
// With MUL the epilogue stores w * phys instead of phys (w: a physical field of the same layout, one for all
// fields of the launch): the product f'(z) dz/dt of the fixed point (Sec. 4.3) formed as the transform is
// written, so neither dz/dt on the grid nor a separate product pass is needed.
template <class C, int EPT, bool MUL>
__device__ __forceinline__ void x_inv_body(const FFTPlan& pl, const Grid& g, const C* T, size_t tstride,
                                           const FieldsRW& out, const void* wmul, unsigned* flags) {
  using F = FT<C>;
  using R = typename F::R;
  extern __shared__ __align__(128) unsigned char sm_raw[];
  C* a = reinterpret_cast<C*>(sm_raw);
  const int batch = pl.batch, ld = pl.n + pl.pad, px = g.px, pz = g.pz, h = g.nx / 2;
  const int pr0 = blockIdx.x * batch, j = blockIdx.y, f = blockIdx.z;
  const int bt = threadIdx.x / pl.tpt, tt = threadIdx.x - bt * pl.tpt;
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(sm_raw + (size_t)batch * ld * sizeof(C));
  if (threadIdx.x == 0) mbar_init(bar);
  __syncthreads();
  // A transform's rows za = 2 (pr0 + bb) and za + 1 of T are contiguous (2 h elements): one bulk copy each
  // (TMA, cp.async.bulk) into the upper part [h, 3 h) = [h, px) of its buffer, completing on the mbarrier
  if (threadIdx.x == 0) {
    const C* src = T + f * tstride + (size_t)j * pz * h;
    int nb = 0;
    while (nb < batch && 2 * (pr0 + nb) < pz) ++nb;
    mbar_expect_tx(bar, (unsigned)(nb * 2 * h * sizeof(C)));
    for (int bb = 0; bb < nb; ++bb) {
      const int za = 2 * (pr0 + bb);
      if (LMVD_IN(bb * ld + px - 1, batch * ld) && LMVD_IN((size_t)(za + 2) * h - 1, (size_t)pz * h))
        bulk_load(a + bb * ld + h, src + (size_t)za * h, (unsigned)(2 * h * sizeof(C)), bar);
    }
  }
  if (!mbar_wait_bounded(bar, flags)) return;
  // two real rows into one complex transform: y[k] = Xa[k] + i Xb[k], y[px - k] = conj(Xa[k]) + i conj(Xb[k]).
  // Every thread reads its EPT / 3 pairs (batch h = blockDim.x EPT / 3 of them) before any is written,
  // since the written y[px - k] overlay the copied rows.
  constexpr int NP = EPT / 3;
  C ta[NP], tb[NP];
  int kk[NP], bs[NP];
  RowCol rc(threadIdx.x, h);
#pragma unroll
  for (int u = 0; u < NP; ++u) {
    const int bb = rc.r, k = rc.c;
    rc.advance(blockDim.x, h);
    kk[u] = -1;
    if (bb >= batch || 2 * (pr0 + bb) >= pz || !LMVD_IN(bb * ld + 3 * h - 1, batch * ld)) continue;
    kk[u] = k;
    bs[u] = bb;
    ta[u] = a[bb * ld + h + k];
    tb[u] = a[bb * ld + 2 * h + k];
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < NP; ++u) {
    if (kk[u] < 0) continue;
    const int k = kk[u];
    C* y = a + bs[u] * ld;
    if (k == 0) {
      y[0] = F::make(F::re(ta[u]), F::re(tb[u]));  // the kx = 0 coefficient of a real row is real
    } else {
      y[k] = F::add(ta[u], F::ti(tb[u]));                        // Xa[k] + i Xb[k]
      y[px - k] = F::add(F::cj(ta[u]), F::ti(F::cj(tb[u])));  // conj(Xa[k]) + i conj(Xb[k])
    }
  }
  // the padding band [h, px - h + 1) = [h, 2 h]: zero where the arithmetic reads it (it held copied rows)
  if (!prunes_zero_band<C>(pl)) {
    RowCol rz(threadIdx.x, h + 1);
    for (int idx = threadIdx.x; idx < batch * (h + 1); idx += blockDim.x) {
      const int bb = rz.r, q = rz.c;
      rz.advance(blockDim.x, h + 1);
      if (LMVD_IN(bb * ld + h + q, batch * ld)) a[bb * ld + h + q] = F::zero();
    }
  }
  __syncthreads();
  fft_inplace<C, 1, EPT, kPrune<C>, false>(a + bt * ld, pl, tt, pl.tpt, h, px - h + 1);  // kx padding: zero
  const C* res = a;
  R* dst = reinterpret_cast<R*>(pick(out.p, f)) + (size_t)j * g.P;
  if (MUL) {
    const R* w = reinterpret_cast<const R*>(wmul) + (size_t)j * g.P;
    RowCol rw(threadIdx.x, px);
    for (int base = threadIdx.x; base < batch * px; base += FFT_LOAD_CHUNK * blockDim.x) {
      R wa[FFT_LOAD_CHUNK], wb[FFT_LOAD_CHUNK];
      int xs[FFT_LOAD_CHUNK], bs[FFT_LOAD_CHUNK];
#pragma unroll
      for (int u = 0; u < FFT_LOAD_CHUNK; ++u) {
        const int idx = base + u * blockDim.x;
        const int bb = rw.r, x = rw.c;
        rw.advance(blockDim.x, px);
        xs[u] = -1;
        if (idx >= batch * px) continue;
        const int za = 2 * (pr0 + bb), zb = za + 1;
        if (za >= pz) continue;
        if (!LMVD_IN((size_t)za * px + x, g.P) || !LMVD_IN(bb * ld + x, batch * ld)) continue;
        xs[u] = x;
        bs[u] = bb;
        wa[u] = w[(size_t)za * px + x];
        wb[u] = zb < pz ? w[(size_t)zb * px + x] : F::rzero();
      }
#pragma unroll
      for (int u = 0; u < FFT_LOAD_CHUNK; ++u) {
        if (xs[u] < 0) continue;
        const int x = xs[u], za = 2 * (pr0 + bs[u]), zb = za + 1;
        const C v = res[bs[u] * ld + x];
        dst[(size_t)za * px + x] = F::rmul(wa[u], F::re(v));
        if (zb < pz) dst[(size_t)zb * px + x] = F::rmul(wb[u], F::im(v));
      }
    }
    return;
  }
  RowCol ro(threadIdx.x, px);
  for (int idx = threadIdx.x; idx < batch * px; idx += blockDim.x) {
    const int bb = ro.r, x = ro.c;
    ro.advance(blockDim.x, px);
    const int za = 2 * (pr0 + bb), zb = za + 1;
    if (za >= pz) continue;
    if (!LMVD_IN((size_t)za * px + x, g.P) || !LMVD_IN(bb * ld + x, batch * ld)) continue;
    const C v = res[bb * ld + x];
    dst[(size_t)za * px + x] = F::re(v);
    if (zb < pz) dst[(size_t)zb * px + x] = F::im(v);
  }
}
template <class C, int EPT>
__global__ void __launch_bounds__(FFT_CTA_X, FftMinCtas<C>::x) k_fft_x_inv(FFTPlan pl, Grid g, const C* T, size_t tstride, FieldsRW out,
                                                                         unsigned* flags) {
  x_inv_body<C, EPT, false>(pl, g, T, tstride, out, nullptr, flags);
}
template <class C, int EPT>
__global__ void __launch_bounds__(FFT_CTA_X, FftMinCtas<C>::x) k_fft_x_inv_mul(FFTPlan pl, Grid g, const C* T, size_t tstride, FieldsRW out,
                                                                             const void* wmul, unsigned* flags) {
  x_inv_body<C, EPT, true>(pl, g, T, tstride, out, wmul, flags);
}

// ---------------------------------------------------------------- forward x-pass (r2c, 2 rows per transform)
// With DOT3 the load prologue forms -(w1 m1 + w2 m2 + w3 m3) from six physical fields instead of reading
// one (d: w[0..2], m[0..2]; one launch, one field): the tail -(1/rho) grad z . m^c of L (Sec. 4.3) formed as
// the transform reads it, so no product pass and no product field are needed.
struct Dot3 {
  const void* w[3];
  const void* m[3];
};
template <class C, int EPT, bool DOT3>
__device__ __forceinline__ void x_fwd_body(const FFTPlan& pl, const Grid& g, const FieldsRC& in, C* T, size_t tstride,
                                           const Dot3& d) {
  using F = FT<C>;
  using R = typename F::R;
  extern __shared__ __align__(128) unsigned char sm_raw[];
  C* a = reinterpret_cast<C*>(sm_raw);
  const int batch = pl.batch, ld = pl.n + pl.pad, px = g.px, pz = g.pz, h = g.nx / 2;
  const int pr0 = blockIdx.x * batch, j = blockIdx.y, f = blockIdx.z;
  const int bt = threadIdx.x / pl.tpt, tt = threadIdx.x - bt * pl.tpt;
  const R* src = reinterpret_cast<const R*>(pick(in.p, f)) + (size_t)j * g.P;
  // DOT3 reads six fields per point: fewer points per chunk keep the registers in check
  constexpr int CH = DOT3 ? 2 : FFT_LOAD_CHUNK;
  RowCol rc(threadIdx.x, px);
  for (int base = threadIdx.x; base < batch * px; base += CH * blockDim.x) {
    R va[CH], vb[CH];
    int ds[CH];
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      const int idx = base + u * blockDim.x;
      const int bb = rc.r, x = rc.c;
      rc.advance(blockDim.x, px);
      ds[u] = -1;
      va[u] = vb[u] = F::rzero();
      if (idx >= batch * px) continue;
      const int za = 2 * (pr0 + bb), zb = za + 1;
      if (!LMVD_IN(bb * ld + x, batch * ld)) continue;
      ds[u] = bb * ld + x;
      if (za < pz && LMVD_IN((size_t)za * px + x, g.P)) {
        if (DOT3) {
          const size_t plane = (size_t)j * g.P;
          const R* w0 = reinterpret_cast<const R*>(d.w[0]) + plane;
          const R* w1 = reinterpret_cast<const R*>(d.w[1]) + plane;
          const R* w2 = reinterpret_cast<const R*>(d.w[2]) + plane;
          const R* m0 = reinterpret_cast<const R*>(d.m[0]) + plane;
          const R* m1 = reinterpret_cast<const R*>(d.m[1]) + plane;
          const R* m2 = reinterpret_cast<const R*>(d.m[2]) + plane;
          size_t o = (size_t)za * px + x;
          va[u] = F::dot3neg(w0[o], m0[o], w1[o], m1[o], w2[o], m2[o]);
          if (zb < pz) {
            o += px;
            vb[u] = F::dot3neg(w0[o], m0[o], w1[o], m1[o], w2[o], m2[o]);
          }
        } else {
          va[u] = src[(size_t)za * px + x];
          if (zb < pz) vb[u] = src[(size_t)zb * px + x];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < CH; ++u)
      if (ds[u] >= 0) a[ds[u]] = F::make(va[u], vb[u]);
  }
  __syncthreads();
  fft_inplace<C, -1, EPT, false, kPrune<C>>(a + bt * ld, pl, tt, pl.tpt, h, px - h + 1);  // truncated kx
  const C* res = a;
  C* dst = T + f * tstride + (size_t)j * pz * h;
  RowCol ro(threadIdx.x, h);
  for (int idx = threadIdx.x; idx < batch * h; idx += blockDim.x) {
    const int bb = ro.r, k = ro.c;
    ro.advance(blockDim.x, h);
    const int za = 2 * (pr0 + bb), zb = za + 1;
    if (za >= pz) continue;
    if (!LMVD_IN((size_t)za * h + k, (size_t)pz * h) || !LMVD_IN(bb * ld + px - 1, batch * ld)) continue;
    const C yk = res[bb * ld + k];
    const C ym = F::cj(res[bb * ld + (k == 0 ? 0 : px - k)]);
    // twice the two rows' spectra (the 1/2 is in the z-pass's scale): yk + ym and (yk - ym) / i
    dst[(size_t)za * h + k] = F::add(yk, ym);
    if (zb < pz) dst[(size_t)zb * h + k] = F::neg(F::ti(F::sub(yk, ym)));
  }
}
template <class C, int EPT>
__global__ void __launch_bounds__(FFT_CTA_X, FftMinCtas<C>::x) k_fft_x_fwd(FFTPlan pl, Grid g, FieldsRC in, C* T, size_t tstride) {
  x_fwd_body<C, EPT, false>(pl, g, in, T, tstride, Dot3{});
}
template <class C, int EPT>
__global__ void __launch_bounds__(FFT_CTA_X, FftMinCtas<C>::x) k_fft_x_fwd_dot3(FFTPlan pl, Grid g, C* T, size_t tstride, Dot3 d) {
  x_fwd_body<C, EPT, true>(pl, g, FieldsRC{}, T, tstride, d);
}

// ---------------------------------------------------------------- forward z-pass (truncate, scale)
// T: [f][ny][pz][nx/2] of C, read through maps.m[0] (all fields of the launch: planes f ny + j); out:
// spectral fields [ny][nz][nxh]. Same interleaved layout as the inverse z-pass; kx = nx/2 and the kz
// Nyquist row are written as zero.
template <class C, int EPT, int COLS>
__global__ void __launch_bounds__(FFT_CTA_Z, FftMinCtas<C>::z_fwd)
    k_fft_z_fwd(FFTPlan pl, Grid g, const __grid_constant__ ZMaps maps, FieldsW out, unsigned* flags) {
  using F = FT<C>;
  extern __shared__ __align__(128) unsigned char sm_raw[];
  C* a = reinterpret_cast<C*>(sm_raw);
  const int pz = g.pz, nz = g.nz, h = g.nx / 2, n2 = nz / 2, H = pl.rows_t;
  const int kx0 = blockIdx.x * COLS, j = blockIdx.y, f = blockIdx.z;
  const int c = threadIdx.x % COLS, tt = threadIdx.x / COLS;
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(sm_raw + (size_t)pz * COLS * sizeof(C));
  if (threadIdx.x == 0) mbar_init(bar);
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_expect_tx(bar, (unsigned)(pz * COLS * sizeof(C)));
    for (int r = 0; r < pz; r += H)
      if (LMVD_IN((r + H) * COLS - 1, pz * COLS)) tma_load_3d(a + (size_t)r * COLS, &maps.m[0], 2 * kx0, r, f * g.ny + j, bar);
  }
  if (!mbar_wait_bounded(bar, flags)) return;
  fft_inplace<C, -1, EPT, false, kPrune<C>, COLS>(a + c, pl, tt, pl.tpt, n2, pz - n2 + 1);  // truncated kz
  cd* dst = pick(out.p, f) + (size_t)j * g.M;
  for (int idx = threadIdx.x; idx < nz * COLS; idx += blockDim.x) {
    const int jz = idx / COLS, cc = idx % COLS, kx = kx0 + cc;
    if (kx > h) continue;
    const int pos = jz < n2 ? jz : pz - nz + jz;
    cd v = mk(0, 0);
    if (kx < h && jz != n2 && LMVD_IN(pos * COLS + cc, pz * COLS)) v = F::to_spec(a[pos * COLS + cc], pl);
    if (LMVD_IN((size_t)jz * g.nxh + kx, g.M)) dst[(size_t)jz * g.nxh + kx] = v;
  }
}

// ---------------------------------------------------------------- host side
// Radix order 4s, 2s, 3s: the sub-length L is a power of two in every radix-4/2 stage (mask arithmetic).
// 12 elements per thread (6 when n has a single factor 2, hence no radix-4 stage); at most cta threads per
// CTA (so n <= 12 cta); one shared buffer of batch transforms with leading dimension n + pad.
static bool make_plan(int n, int cta, FFTPlan& p) {
  p.n = n;
  p.nst = 0;
  int m = n;
  while (m % 4 == 0) { p.radix[p.nst++] = 4; m /= 4; }
  while (m % 2 == 0) { p.radix[p.nst++] = 2; m /= 2; }
  while (m % 3 == 0) { p.radix[p.nst++] = 3; m /= 3; }
  if (m != 1 || p.nst > 16) return false;
  p.code = 0;
  for (int s2 = 0; s2 < p.nst; ++s2)
    p.code |= (unsigned)(p.radix[s2] == 4 ? 0 : (p.radix[s2] == 2 ? 1 : 2)) << (2 * s2);
  p.ept = (n % 12 == 0) ? 12 : ((n % 6 == 0) ? 6 : 0);
  if (!p.ept) return false;
  p.tpt = n / p.ept;
  if (p.tpt > cta) return false;
  p.batch = cta / p.tpt;
  p.pad = 1;  // the x-passes: leading dimension n + 1 keeps the transforms of a batch in different banks
  if (cta == FFT_CTA_Z) {
    // the z-passes: 4 interleaved columns per CTA (2 when 4 transforms of n do not fit in cta threads; the
    // 6-element plans exist only for 4), and tile copies whose rows divide their range and start on 128-byte
    // boundaries in shared memory (rows x batch x 16 bytes a multiple of 128)
    p.batch = 4 * p.tpt <= cta ? 4 : (p.ept == 12 && 2 * p.tpt <= cta ? 2 : 0);
    if (!p.batch || n % 3) return false;
    p.pad = 0;
    auto rows = [&](int total) {
      for (int r = total < 256 ? total : 256; r > 0; --r)
        if (total % r == 0 && (r * p.batch) % 8 == 0) return r;
      return 0;
    };
    p.rows_in = rows(n / 3);  // nz / 2 = pz / 3
    p.rows_t = rows(n);
    if (!p.rows_in || !p.rows_t) return false;
  }
  return true;
}

// a pass's buffer is followed by its mbarrier (the z-passes' and the inverse x-pass's copies)
static size_t smem_bytes(const FFTPlan& p) { return (size_t)p.batch * (p.n + p.pad) * sizeof(cd) + 16; }

// Tensor maps for the z-passes' tile copies. cuTensorMapEncodeTiled is a driver function; the runtime hands
// out its address, so the library needs no link to the driver library.
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

// A map over planes x rows x cols 16-byte elements at base (row-major, contiguous), addressed in doubles:
// boxes of (2 bcols doubles, brows rows, 1 plane); out-of-range parts of a box read as zero.
static bool tile_map(CUtensorMap* m, const void* base, size_t cols, size_t rows, size_t planes, int bcols, int brows) {
  const EncodeTiledFn fn = encode_tiled();
  if (!fn || !base || ((uintptr_t)base & 15)) return false;
  const cuuint64_t dims[3] = {2 * (cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)planes};
  const cuuint64_t strides[2] = {16 * (cuuint64_t)cols, 16 * (cuuint64_t)cols * rows};
  const cuuint32_t box[3] = {(cuuint32_t)(2 * bcols), (cuuint32_t)brows, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
static unsigned threads(const FFTPlan& p) { return (unsigned)(p.batch * p.tpt); }

static df host_split(long double x) {
  const float h = (float)x;
  return df{h, (float)(x - (long double)h)};
}

// Every pass may take up to kFftSmemMax bytes of dynamic shared memory. The limit is a property of the
// kernel, shared by all contexts and the allocation-free path in the process: setting it to one grid's size
// would break the launches of another context with a larger grid, so it is set once, to the maximum a plan
// may ask for (fft_prepare rejects larger plans).
constexpr int kFftSmemMax = 200 * 1024;

template <class C, int EPT, int COLS>
static int set_smem_z(int sz) {
  if (cudaFuncSetAttribute(k_fft_z_inv<C, EPT, COLS>, cudaFuncAttributeMaxDynamicSharedMemorySize, sz) != cudaSuccess ||
      cudaFuncSetAttribute(k_fft_z_fwd<C, EPT, COLS>, cudaFuncAttributeMaxDynamicSharedMemorySize, sz) != cudaSuccess)
    return LMVD_ERR_CUDA;
  if constexpr (std::is_same<C, cdf>::value) {
    if (cudaFuncSetAttribute(k_fft_z_inv<C, EPT, COLS, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sz) !=
        cudaSuccess)
      return LMVD_ERR_CUDA;
  }
  return LMVD_OK;
}

template <class C, int EPT>
static int set_smem_e(int sx, int sz) {
  if constexpr (EPT == 12) {
    if (set_smem_z<C, EPT, 2>(sz)) return LMVD_ERR_CUDA;
  }
  if (set_smem_z<C, EPT, 4>(sz) ||
      cudaFuncSetAttribute(k_fft_x_inv<C, EPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, sx) != cudaSuccess ||
      cudaFuncSetAttribute(k_fft_x_fwd<C, EPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, sx) != cudaSuccess ||
      cudaFuncSetAttribute(k_fft_x_inv_mul<C, EPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, sx) != cudaSuccess ||
      cudaFuncSetAttribute(k_fft_x_fwd_dot3<C, EPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, sx) != cudaSuccess)
    return LMVD_ERR_CUDA;
  return LMVD_OK;
}

template <class C>
static int set_smem() {
  int e = set_smem_e<C, 12>(kFftSmemMax, kFftSmemMax);
  if (!e) e = set_smem_e<C, 6>(kFftSmemMax, kFftSmemMax);
  return e;
}

int fft_prepare(Ctx& c) {
  if (!make_plan(c.g.px, FFT_CTA_X, c.fx) || !make_plan(c.g.pz, FFT_CTA_Z, c.fz)) return LMVD_ERR_UNSUPPORTED;
  const long double scale = 1.0L / ((long double)c.g.px * (long double)c.g.pz);
  const long double pi = 3.141592653589793238462643383279502884L;
  for (FFTPlan* p : {&c.fx, &c.fz}) {
    if (smem_bytes(*p) > kFftSmemMax) return LMVD_ERR_UNSUPPORTED;
    std::vector<double2> tw(p->n);
    std::vector<float4> twf(p->n);
    for (int m = 0; m < p->n; ++m) {
      const long double ang = 2.0L * pi * (long double)m / (long double)p->n;
      const long double cs = cosl(ang), sn = sinl(ang);
      tw[m] = make_double2((double)cs, (double)sn);
      const df hc = host_split(cs), hs = host_split(sn);
      twf[m] = make_float4(hc.hi, hc.lo, hs.hi, hs.lo);
    }
    if (cudaMalloc(&p->tw, sizeof(double2) * p->n) != cudaSuccess) return LMVD_ERR_OOM;
    c.small_allocs.push_back(p->tw);
    if (cudaMalloc(&p->twf, sizeof(float4) * p->n) != cudaSuccess) return LMVD_ERR_OOM;
    c.small_allocs.push_back(p->twf);
    c.small_bytes += (sizeof(double2) + sizeof(float4)) * p->n;
    if (cudaMemcpy(p->tw, tw.data(), sizeof(double2) * p->n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(p->twf, twf.data(), sizeof(float4) * p->n, cudaMemcpyHostToDevice) != cudaSuccess)
      return LMVD_ERR_CUDA;
    p->scale_d = (double)(scale / 2);  // used by the forward z-pass (see the file head)
    p->scale_f = host_split(scale / 2);
    p->s3f = host_split(sqrtl(3.0L) / 2.0L);
  }
  int e = set_smem<cd>();
  if (!e) e = set_smem<cdf>();
  return e;
}

static inline unsigned cdiv(unsigned a, unsigned b) { return (a + b - 1) / b; }
// conventional algorithmic flop count of one complex transform of length n: 5 n log2 n
static inline double fft_flops(double n) { return 5.0 * n * std::log2(n); }

// A tensor map that could not be encoded: the context's status becomes LMVD_ERR_CUDA (unless one is set).
static void map_failed(Ctx& c) {
  if (c.status == LMVD_OK) c.status = LMVD_ERR_CUDA;
}

// The inverse z-pass of n fields (spectral inputs fi) into T, and the forward z-pass of n fields of T into
// fo: tensor maps for their tile copies, then one launch of the instantiation the plan selects.
template <class C, bool IN_DF>
static void z_inv_launch(Ctx& c, const FieldsC& fi, int n, C* T, size_t tstride, double fl, double by) {
  const Grid& g = c.g;
  const FFTPlan& p = c.fz;
  ZMaps maps;
  for (int f = 0; f < n; ++f)
    if (!tile_map(&maps.m[f], fi.p[f], g.nxh, g.nz, g.ny, p.batch, p.rows_in)) {
      map_failed(c);
      return;
    }
  const dim3 gz(cdiv(g.nx / 2, p.batch), g.ny, n);
  if (p.ept == 12 && p.batch == 4)
    LMVD_LAUNCH(c, KC_FFT_Z_INV, fl, by, (k_fft_z_inv<C, 12, 4, IN_DF>), gz, threads(p), smem_bytes(p), p, g, maps, T,
                tstride, c.dflags);
  else if (p.ept == 12)
    LMVD_LAUNCH(c, KC_FFT_Z_INV, fl, by, (k_fft_z_inv<C, 12, 2, IN_DF>), gz, threads(p), smem_bytes(p), p, g, maps, T,
                tstride, c.dflags);
  else
    LMVD_LAUNCH(c, KC_FFT_Z_INV, fl, by, (k_fft_z_inv<C, 6, 4, IN_DF>), gz, threads(p), smem_bytes(p), p, g, maps, T,
                tstride, c.dflags);
}

template <class C>
static void z_fwd_launch(Ctx& c, const C* T, int n, const FieldsW& fo, double fl, double by) {
  const Grid& g = c.g;
  const FFTPlan& p = c.fz;
  ZMaps maps;
  if (!tile_map(&maps.m[0], T, g.nx / 2, g.pz, (size_t)n * g.ny, p.batch, p.rows_t)) {
    map_failed(c);
    return;
  }
  const dim3 gz(cdiv(g.nx / 2 + 1, p.batch), g.ny, n);
  if (p.ept == 12 && p.batch == 4)
    LMVD_LAUNCH(c, KC_FFT_Z_FWD, fl, by, (k_fft_z_fwd<C, 12, 4>), gz, threads(p), smem_bytes(p), p, g, maps, fo,
                c.dflags);
  else if (p.ept == 12)
    LMVD_LAUNCH(c, KC_FFT_Z_FWD, fl, by, (k_fft_z_fwd<C, 12, 2>), gz, threads(p), smem_bytes(p), p, g, maps, fo,
                c.dflags);
  else
    LMVD_LAUNCH(c, KC_FFT_Z_FWD, fl, by, (k_fft_z_fwd<C, 6, 4>), gz, threads(p), smem_bytes(p), p, g, maps, fo,
                c.dflags);
}

template <class C>
static void inverse_t(Ctx& c, cd* const* in, void* const* out, int nf, const void* wmul = nullptr, bool in_df = false) {
  const Grid& g = c.g;
  const size_t tstride = (size_t)g.ny * g.pz * (g.nx / 2);
  C* T = reinterpret_cast<C*>(c.tbuf);
  for (int f0 = 0; f0 < nf; f0 += c.tbuf_n) {
    const int n = nf - f0 < c.tbuf_n ? nf - f0 : c.tbuf_n;
    FieldsC fi{};
    FieldsRW fo{};
    for (int f = 0; f < n; ++f) {
      fi.p[f] = in[f0 + f];
      fo.p[f] = out[f0 + f];
    }
    const double h = g.nx / 2, ny = g.ny, pz = g.pz, px = g.px;
    const double zfl = n * ny * h * fft_flops(pz), zby = n * ny * h * 16.0 * ((g.nz - 1) + pz);
    // double-float inputs only exist for the double-float arithmetic
    if (in_df && std::is_same<C, cdf>::value) z_inv_launch<C, std::is_same<C, cdf>::value>(c, fi, n, T, tstride, zfl, zby);
    else z_inv_launch<C, false>(c, fi, n, T, tstride, zfl, zby);
    dim3 gx(cdiv(cdiv(g.pz, 2), c.fx.batch), g.ny, n);
    const double xfl = n * ny * ((g.pz + 1) / 2) * fft_flops(px), xby = n * ny * pz * (16.0 * h + 8.0 * px);
    if (wmul) {  // the product with w in the epilogue: one more physical field read, one multiply per point
      if (c.fx.ept == 12)
        LMVD_LAUNCH(c, KC_FFT_X_INV, xfl + n * ny * pz * px, xby + n * ny * pz * 8.0 * px, (k_fft_x_inv_mul<C, 12>),
                    gx, threads(c.fx), smem_bytes(c.fx), c.fx, g, T, tstride, fo, wmul, c.dflags);
      else
        LMVD_LAUNCH(c, KC_FFT_X_INV, xfl + n * ny * pz * px, xby + n * ny * pz * 8.0 * px, (k_fft_x_inv_mul<C, 6>),
                    gx, threads(c.fx), smem_bytes(c.fx), c.fx, g, T, tstride, fo, wmul, c.dflags);
    } else if (c.fx.ept == 12) {
      LMVD_LAUNCH(c, KC_FFT_X_INV, xfl, xby, (k_fft_x_inv<C, 12>), gx, threads(c.fx), smem_bytes(c.fx), c.fx, g, T,
                  tstride, fo, c.dflags);
    } else {
      LMVD_LAUNCH(c, KC_FFT_X_INV, xfl, xby, (k_fft_x_inv<C, 6>), gx, threads(c.fx), smem_bytes(c.fx), c.fx, g, T,
                  tstride, fo, c.dflags);
    }
  }
}

template <class C>
static void forward_t(Ctx& c, void* const* in, cd* const* out, int nf) {
  const Grid& g = c.g;
  const size_t tstride = (size_t)g.ny * g.pz * (g.nx / 2);
  C* T = reinterpret_cast<C*>(c.tbuf);
  for (int f0 = 0; f0 < nf; f0 += c.tbuf_n) {
    const int n = nf - f0 < c.tbuf_n ? nf - f0 : c.tbuf_n;
    FieldsRC fi{};
    FieldsW fo{};
    for (int f = 0; f < n; ++f) {
      fi.p[f] = in[f0 + f];
      fo.p[f] = out[f0 + f];
    }
    const double h = g.nx / 2, ny = g.ny, pz = g.pz, px = g.px;
    dim3 gx(cdiv(cdiv(g.pz, 2), c.fx.batch), g.ny, n);
    if (c.fx.ept == 12)
      LMVD_LAUNCH(c, KC_FFT_X_FWD, n * ny * ((g.pz + 1) / 2) * fft_flops(px), n * ny * pz * (16.0 * h + 8.0 * px),
                  (k_fft_x_fwd<C, 12>), gx, threads(c.fx), smem_bytes(c.fx), c.fx, g, fi, T, tstride);
    else
      LMVD_LAUNCH(c, KC_FFT_X_FWD, n * ny * ((g.pz + 1) / 2) * fft_flops(px), n * ny * pz * (16.0 * h + 8.0 * px),
                  (k_fft_x_fwd<C, 6>), gx, threads(c.fx), smem_bytes(c.fx), c.fx, g, fi, T, tstride);
    z_fwd_launch<C>(c, T, n, fo, n * ny * h * fft_flops(pz), n * ny * 16.0 * (pz * h + (double)g.nz * g.nxh));
  }
}

// forward transform of -(w1 m1 + w2 m2 + w3 m3), formed in the x-pass prologue, into one spectral field
template <class C>
static void forward_dot3_t(Ctx& c, const double* const* w, const double* const* m, cd* out) {
  const Grid& g = c.g;
  const size_t tstride = (size_t)g.ny * g.pz * (g.nx / 2);
  C* T = reinterpret_cast<C*>(c.tbuf);
  Dot3 d{};
  for (int f = 0; f < 3; ++f) {
    d.w[f] = w[f];
    d.m[f] = m[f];
  }
  FieldsW fo{};
  fo.p[0] = out;
  const double h = g.nx / 2, ny = g.ny, pz = g.pz, px = g.px;
  dim3 gx(cdiv(cdiv(g.pz, 2), c.fx.batch), g.ny, 1);
  const double xfl = ny * ((g.pz + 1) / 2) * fft_flops(px) + 6.0 * ny * pz * px, xby = ny * pz * (16.0 * h + 48.0 * px);
  if (c.fx.ept == 12)
    LMVD_LAUNCH(c, KC_FFT_X_FWD, xfl, xby, (k_fft_x_fwd_dot3<C, 12>), gx, threads(c.fx), smem_bytes(c.fx), c.fx, g, T,
                tstride, d);
  else
    LMVD_LAUNCH(c, KC_FFT_X_FWD, xfl, xby, (k_fft_x_fwd_dot3<C, 6>), gx, threads(c.fx), smem_bytes(c.fx), c.fx, g, T,
                tstride, d);
  z_fwd_launch<C>(c, T, 1, fo, ny * h * fft_flops(pz), ny * 16.0 * (pz * h + (double)g.nz * g.nxh));
}

void fft_inverse_mul(Ctx& c, cd* in, double* out, const double* w) {
  cd* i[1] = {in};
  void* o[1] = {out};
  if (c.cfg.precision == 1) inverse_t<cdf>(c, i, o, 1, w, true);
  else inverse_t<cd>(c, i, o, 1, w);
}

void fft_forward_dot3(Ctx& c, const double* const* w, const double* const* m, cd* out) {
  if (c.cfg.precision == 1) forward_dot3_t<cdf>(c, w, m, out);
  else forward_dot3_t<cd>(c, w, m, out);
}

// The bounded wait of the z-passes, on its own (lmvd_tile_wait_probe): one CTA expects 128 + extra bytes on
// an mbarrier and copies 128 of them; with extra > 0 the phase never completes and the wait gives up.
__global__ void k_tile_wait_probe(const double* src, int extra, unsigned* status) {
  __shared__ __align__(128) double buf[16];
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x == 0) mbar_init(&bar);
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_expect_tx(&bar, 128u + (unsigned)extra);
    bulk_load(buf, src, 128u, &bar);
  }
  if (!mbar_wait_bounded(&bar, status)) return;
  if (threadIdx.x < 16 && buf[threadIdx.x] != src[threadIdx.x]) atomicOr(status, 8u);
}

void fft_inverse_as(Ctx& c, cd* const* in, double* const* out, int nf, int precision) {
  void* o[64];
  for (int f = 0; f < nf; ++f) o[f] = out[f];
  if (precision == 1) inverse_t<cdf>(c, in, o, nf);
  else inverse_t<cd>(c, in, o, nf);
}

void fft_forward_as(Ctx& c, double* const* in, cd* const* out, int nf, int precision) {
  void* i[64];
  for (int f = 0; f < nf; ++f) i[f] = in[f];
  if (precision == 1) forward_t<cdf>(c, i, out, nf);
  else forward_t<cd>(c, i, out, nf);
}

void fft_inverse(Ctx& c, cd* const* in, double* const* out, int nf) {
  if (c.cfg.precision == 1) {  // the substage's inputs come from the double-float evaluations
    void* o[64];
    for (int f = 0; f < nf; ++f) o[f] = out[f];
    inverse_t<cdf>(c, in, o, nf, nullptr, true);
  } else {
    fft_inverse_as(c, in, out, nf, 0);
  }
}

void fft_forward(Ctx& c, double* const* in, cd* const* out, int nf) { fft_forward_as(c, in, out, nf, c.cfg.precision); }

}  // namespace lmvd

// ====================================================================== allocation-free inverse transform
// lmvd_inverse_transform_noalloc: the same synthesis as lmvd_inverse_transform, for callers that cannot
// allocate device memory (no context exists, so nothing of lmvd_create is needed). Its only working
// memory is the file-scope array below, which the CUDA module reserves on every device that loads the
// library and keeps until the process exits. All calls on a device share it: the twiddle tables and
// the intermediate array are rewritten by each call before they are read (nothing has to start at
// zero), and calls whose work overlaps on the GPU (other streams, other host threads) race on it.
namespace lmvd {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;  // 32 MiB per device
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kNoAllocMaxDevices] = {};

// twiddle table tw[m] = (cos 2 pi m / n, sin 2 pi m / n) computed on the device
__global__ void k_twiddles(double2* tw, int n) {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n; m += gridDim.x * blockDim.x) {
    double s, c;
    sincospi(2.0 * (double)m / (double)n, &s, &c);
    tw[m] = make_double2(c, s);
  }
}

// Once per device, with that device current: the device address of the scratch array (in host code
// the array's name is only a stand-in) and the shared-memory limits of the two kernels.
int noalloc_setup(int dev, void** ptr) {
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (g_noalloc_ptr[dev]) {
    *ptr = g_noalloc_ptr[dev];
    return LMVD_OK;
  }
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return LMVD_ERR_CUDA;
  if (set_smem<cd>())
    return LMVD_ERR_CUDA;
  g_noalloc_ptr[dev] = p;
  *ptr = p;
  return LMVD_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

}  // namespace lmvd

extern "C" int lmvd_inverse_transform_noalloc(int nx, int ny, int nz, const void* spec, double* phys, int nfields,
                                              void* cuda_stream) {
  using namespace lmvd;
  if (!spec || !phys || nfields < 0 || ny < 1 || nx < 4 || nz < 4 || (nx % 2) || (nz % 2) || ((uintptr_t)spec & 15))
    return LMVD_ERR_INVALID_ARG;
  if (ny > 65535) return LMVD_ERR_INVALID_ARG;  // ny is the grid's y-dimension (at most 65535 CTAs)
  Grid g{};
  g.nx = nx;
  g.ny = ny;
  g.nz = nz;
  g.nxh = nx / 2 + 1;
  g.px = 3 * nx / 2;
  g.pz = 3 * nz / 2;
  g.M = (size_t)nz * g.nxh;
  g.P = (size_t)g.px * g.pz;
  FFTPlan fx, fz;
  if (!make_plan(g.px, FFT_CTA_X, fx) || !make_plan(g.pz, FFT_CTA_Z, fz)) return LMVD_ERR_UNSUPPORTED;
  for (FFTPlan* p : {&fx, &fz})
    if (smem_bytes(*p) > kFftSmemMax) return LMVD_ERR_UNSUPPORTED;
  // scratch layout: x twiddles | z twiddles | one field's intermediate T[ny][pz][nx/2]
  const size_t off_tz = align256(sizeof(double2) * g.px);
  const size_t off_tb = off_tz + align256(sizeof(double2) * g.pz);
  const size_t tbytes = sizeof(cd) * (size_t)ny * g.pz * (nx / 2);
  if (off_tb + tbytes > kNoAllocScratchBytes) return LMVD_ERR_INVALID_ARG;  // grid too large for the scratch
  // a launch error left pending on this host thread by earlier work is not this call's to report
  (void)cudaGetLastError();
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) return LMVD_ERR_CUDA;
  void* base = nullptr;
  int err = noalloc_setup(dev, &base);
  if (err) return err;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  char* sb = (char*)base;
  fx.tw = (double2*)sb;
  fz.tw = (double2*)(sb + off_tz);
  cd* T = (cd*)(sb + off_tb);
  k_twiddles<<<(g.px + 255) / 256, 256, 0, st>>>(fx.tw, g.px);
  if (cudaGetLastError() != cudaSuccess) return LMVD_ERR_CUDA;
  k_twiddles<<<(g.pz + 255) / 256, 256, 0, st>>>(fz.tw, g.pz);
  if (cudaGetLastError() != cudaSuccess) return LMVD_ERR_CUDA;
  const size_t S = (size_t)ny * g.M, P = (size_t)ny * g.P;
  for (int f = 0; f < nfields; ++f) {
    FieldsC fi{};
    FieldsRW fo{};
    fi.p[0] = (const cd*)spec + (size_t)f * S;
    fo.p[0] = phys + (size_t)f * P;
    ZMaps maps;
    if (!tile_map(&maps.m[0], fi.p[0], g.nxh, nz, ny, fz.batch, fz.rows_in)) return LMVD_ERR_CUDA;
    dim3 gz(cdiv(nx / 2, fz.batch), ny, 1);
    if (fz.ept == 12 && fz.batch == 4) k_fft_z_inv<cd, 12, 4><<<gz, threads(fz), smem_bytes(fz), st>>>(fz, g, maps, T, 0, nullptr);
    else if (fz.ept == 12) k_fft_z_inv<cd, 12, 2><<<gz, threads(fz), smem_bytes(fz), st>>>(fz, g, maps, T, 0, nullptr);
    else k_fft_z_inv<cd, 6, 4><<<gz, threads(fz), smem_bytes(fz), st>>>(fz, g, maps, T, 0, nullptr);
    if (cudaGetLastError() != cudaSuccess) return LMVD_ERR_CUDA;
    dim3 gx(cdiv(cdiv(g.pz, 2), fx.batch), ny, 1);
    if (fx.ept == 12) k_fft_x_inv<cd, 12><<<gx, threads(fx), smem_bytes(fx), st>>>(fx, g, T, 0, fo, nullptr);
    else k_fft_x_inv<cd, 6><<<gx, threads(fx), smem_bytes(fx), st>>>(fx, g, T, 0, fo, nullptr);
    if (cudaGetLastError() != cudaSuccess) return LMVD_ERR_CUDA;
  }
  return LMVD_OK;
}

extern "C" int lmvd_tile_wait_probe(const double* src, int extra_bytes, unsigned* status, void* cuda_stream) {
  using namespace lmvd;
  if (!src || !status || ((uintptr_t)src & 15) || extra_bytes < 0 || extra_bytes > 1024 || (extra_bytes & 15))
    return LMVD_ERR_INVALID_ARG;
  (void)cudaGetLastError();
  k_tile_wait_probe<<<1, 32, 0, (cudaStream_t)cuda_stream>>>(src, extra_bytes, status);
  return cudaGetLastError() == cudaSuccess ? LMVD_OK : LMVD_ERR_CUDA;
}
