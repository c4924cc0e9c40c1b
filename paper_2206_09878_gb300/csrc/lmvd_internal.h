// Internal definitions shared by the CUDA translation units of liblmvd.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/lmvd.h"
#include "df64.h"

namespace lmvd {

// ---------------------------------------------------------------- index checks (checked build)
// Built with -DLMVD_CHECK (liblmvd_check.so), LMVD_IN(i, n) tests 0 <= i < n before an access: a failed
// test sets bit 0 of this translation unit's device word and the access is skipped (no trap, the kernel
// runs on). lmvd_synchronize reads and clears the words of every translation unit (oob_take_*) and latches
// LMVD_ERR_OUT_OF_BOUNDS. In the normal build LMVD_IN is the constant true and costs nothing.
#ifdef LMVD_CHECK
static __device__ unsigned lmvd_oob_word;
__device__ __forceinline__ bool lmvd_in(long long i, long long n) {
  if (i >= 0 && i < n) return true;
  atomicOr(&lmvd_oob_word, 1u);
  return false;
}
#define LMVD_IN(i, n) ::lmvd::lmvd_in((long long)(i), (long long)(n))
#define LMVD_DEFINE_OOB_TAKE(NAME)                                                                  \
  unsigned oob_take_##NAME() {                                                                     \
    unsigned v = 0, z = 0;                                                                          \
    if (cudaMemcpyFromSymbol(&v, ::lmvd::lmvd_oob_word, sizeof v) != cudaSuccess) return 2u;        \
    cudaMemcpyToSymbol(::lmvd::lmvd_oob_word, &z, sizeof z);                                        \
    return v;                                                                                       \
  }
constexpr bool kCheckedBuild = true;
#else
#define LMVD_IN(i, n) true
#define LMVD_DEFINE_OOB_TAKE(NAME) \
  unsigned oob_take_##NAME() { return 0u; }
constexpr bool kCheckedBuild = false;
#endif
// the index-check words of the translation units (0 in the normal build)
unsigned oob_take_api();
unsigned oob_take_fft();
unsigned oob_take_yk();
unsigned oob_take_pw();
unsigned oob_take_adj();

constexpr int KMAX = 8;   // widest band (each side) of any y-system LU supported
// Device-memory budget of one context: the transform intermediate holds up to TBUF_FIELDS fields
// (transforms of more fields run in chunks), there are up to PW_FIELDS physical work fields, and the RHS
// streams overwrite the first seven spectral value fields. When that layout would not leave room on the
// device (768 x 769 x 768), lmvd_create uses the lean one: TBUF_LEAN and PW_LEAN fields.
constexpr int TBUF_FIELDS = 4;
constexpr int PW_FIELDS = 10;
constexpr int TBUF_LEAN = 2;
constexpr int PW_LEAN = 6;
constexpr int WMAX = 9;   // widest row of a collocation matrix (spline order <= 9)

// ---------------------------------------------------------------- complex helpers (FP64)
struct cd {
  double re, im;
};
__host__ __device__ inline cd mk(double r, double i) { return cd{r, i}; }
__host__ __device__ inline cd operator+(cd a, cd b) { return cd{a.re + b.re, a.im + b.im}; }
__host__ __device__ inline cd operator-(cd a, cd b) { return cd{a.re - b.re, a.im - b.im}; }
__host__ __device__ inline cd operator*(double s, cd a) { return cd{s * a.re, s * a.im}; }
__host__ __device__ inline cd cmul(cd a, cd b) { return cd{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__host__ __device__ inline cd conj(cd a) { return cd{a.re, -a.im}; }
__host__ __device__ inline cd times_i(cd a) { return cd{-a.im, a.re}; }         // i * a
__host__ __device__ inline cd fma_rc(double s, cd x, cd acc) { return cd{fma(s, x.re, acc.re), fma(s, x.im, acc.im)}; }

// ---------------------------------------------------------------- y-operators in device memory
// Row-banded collocation matrix: row i covers columns c0[i] .. c0[i] + w - 1. vf holds the same entries
// as double-float pairs (hi = v rounded to a float, lo = the remainder rounded to a float) for the
// evaluations of the precision path.
struct DBand {
  const int* c0;
  const double* v;
  int rows, w;
  const df* vf;
  int cols;  // rows of the array a row of the band reads (index checks of the checked build)
};
// LU factors of band systems, K entries per row (zeros outside the profile nl / nu). Shared factors:
// mstride = 0, element (i, q) at [i * K + q]; per-mode factors: element (i, q) of factor mode mf at
// [(i * K + q) * mstride + mf], where A(k) depends on kz only through kz^2, so only the modes with
// kz >= 0 are stored (factor_mode): mstride = (nz/2 + 1) * nxh.
struct DLU {
  const double* lo;
  const double* up;
  const double* invd;
  const int* nl;
  const int* nu;
  int n, K;
  size_t mstride;
  double flops_per_mode;  // host-side: flops of one complex solve (sum over rows of 4 (nl + nu) + 2)
};

// Spectral field: complex [rows][nz][nxh], mode index m = jz * nxh + kx, M = nz * nxh.
struct Grid {
  int nx, ny, nz, nxh, px, pz;
  size_t M;      // modes per y-row
  size_t P;      // physical points per plane = px * pz
  double lx, lz;
};

// Entry f of a table passed by value as a kernel parameter. A runtime index into the parameter space makes
// every thread copy the whole table to its local memory first; a chain of selects over the entries (each a
// constant-bank operand) does not.
template <class T, int N>
__device__ __forceinline__ T pick(const T (&tab)[N], int f) {
  T r = tab[0];
#pragma unroll
  for (int q = 1; q < N; ++q) r = (f == q) ? tab[q] : r;
  return r;
}

__device__ inline bool is_nyquist(const Grid& g, int m) {
  int kx = m % g.nxh, jz = m / g.nxh;
  return kx == g.nx / 2 || jz == g.nz / 2;
}
__device__ inline void wavenumbers(const Grid& g, int m, double& k1, double& k3) {
  int kx = m % g.nxh, jz = m / g.nxh;
  int kz = jz < g.nz / 2 ? jz : jz - g.nz;
  k1 = 6.283185307179586476925286766559 / g.lx * kx;
  k3 = 6.283185307179586476925286766559 / g.lz * kz;
}

// Index of mode m's per-mode factors: the mode with the same kx and |kz| (kz >= 0 half-plane).
__device__ inline int factor_mode(const Grid& g, int m) {
  int jz = m / g.nxh;
  const int kx = m - jz * g.nxh;
  if (jz > g.nz / 2) jz = g.nz - jz;
  return jz * g.nxh + kx;
}

// Rows [r0, r1) of chunk c out of nc over `rows` rows (contiguous, sizes differing by at most one).
__host__ __device__ inline void row_range(int rows, int c, int nc, int& r0, int& r1) {
  r0 = (int)((long long)rows * c / nc);
  r1 = (int)((long long)rows * (c + 1) / nc);
}

// Row chunks for the evaluation kernels: enough threads for about 1024 per SM when the grid has few
// Fourier modes, at least 8 rows per thread.
inline unsigned row_chunks(const Grid& g, int rows) {
  const size_t want = ((size_t)152 * 1024 + g.M - 1) / g.M;
  const size_t cap = (size_t)(rows / 8 > 1 ? rows / 8 : 1);
  const size_t ch = want < cap ? want : cap;
  return (unsigned)(ch > 1 ? ch : 1);
}

// Threads per mode of the banded-solve kernels: 2 (one per real part) when the grid has fewer than 65536
// Fourier modes per row, else 1 (see band_solve_v).
inline int solve_split(const Grid& g) { return g.M < 65536 ? 2 : 1; }

__device__ inline cd band_row(const DBand& B, int i, const cd* x, size_t M, int m) {
  cd acc = mk(0, 0);
  if (!LMVD_IN(i, B.rows) || !LMVD_IN(m, M)) return acc;
  const int c = B.c0[i];
  const double* v = B.v + (size_t)i * B.w;
  for (int q = 0; q < B.w; ++q)
    if (LMVD_IN(c + q, B.cols)) acc = fma_rc(__ldg(v + q), x[(size_t)(c + q) * M + m], acc);
  return acc;
}

// ---------------------------------------------------------------- FFT plan
struct FFTPlan {
  int n = 0;
  int nst = 0;
  int radix[24];
  unsigned code = 0;       // the radix sequence, 2 bits per stage (0: 4, 1: 2, 2: 3), first stage lowest
  double2* tw = nullptr;   // tw[m] = (cos 2 pi m / n, sin 2 pi m / n), device
  float4* twf = nullptr;   // the same as double-float pairs (cos.hi, cos.lo, sin.hi, sin.lo), device
  int batch = 1;           // transforms per CTA
  int ept = 12;            // elements per thread (a multiple of every radix of the plan)
  int tpt = 1;             // threads per transform = n / ept; a CTA has tpt * batch threads
  int pad = 1;             // shared-memory leading dimension of a transform: n + pad (x-passes; the z-passes
                           // interleave their batch columns, pad 0)
  int rows_in = 0;         // z-passes: rows per tile copy of the spectral input (divides nz / 2) ...
  int rows_t = 0;          // ... and of the intermediate T (divides pz); 0 for the x-passes
  double scale_d = 1.0;    // 1 / (2 px pz) for the forward z-pass (with the x-pass's 1/2)
  df scale_f{1.f, 0.f};
  df s3f{0.f, 0.f};        // sin(2 pi / 3) as a double-float
};

// ---------------------------------------------------------------- tracing
// NVTX range (visible to ncu / nsys; a no-op without an attached tool) around host-side enqueueing of a
// step of Algorithm 2. advance_impl opens one inner range and, at each step boundary, pops it and pushes
// the next step's, so the inner object's destructor closes the last one (also on an early return).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// ---------------------------------------------------------------- per-class launch accounting
// Kernel classes, in the order of lmvd_kernel_class_name().
enum KClass {
  KC_FFT_Z_INV, KC_FFT_X_INV, KC_FFT_X_FWD, KC_FFT_Z_FWD, KC_EVAL_P1, KC_EVAL, KC_SOLVE, KC_MC_SOLVE,
  KC_RHS_COMBINE, KC_RHS_EVAL, KC_UPDATE, KC_PRODUCTS, KC_MISC, KC_COUNT
};
struct Prof {
  bool on = false;
  long long launches = 0;       // every kernel enqueued since creation
  long long n[KC_COUNT] = {};   // launches per class since profiling was enabled
  double flops[KC_COUNT] = {};  // algorithmic flops per class
  double bytes[KC_COUNT] = {};  // algorithmic DRAM bytes per class
  double ms[KC_COUNT] = {};
  struct Pending { int cls; cudaEvent_t a, b; };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
};

// ---------------------------------------------------------------- adjoint support
constexpr int KF_MAX_ADJ = 15;
constexpr int DIAG_KE = 2 * KF_MAX_ADJ + 4, DIAG_MMAX = DIAG_KE + 1, DIAG_MC2 = DIAG_KE + 2;
constexpr int DIAG_N = DIAG_KE + 4;  // doubles in the diagnostics record
// Physical fields of one forward substage that the adjoint of the products needs.
struct Tape {
  double* zp[5];                   // z, dz/dx, dz/dz, dz/dy, lap z (pass 1)
  double* a[KF_MAX_ADJ + 1];       // dz/dt^{k-1} on the grid, k = 1 .. kf + 1 (the last for the final m^c)
  double* b[KF_MAX_ADJ + 1][3];    // m^c(dz/dt^{k-1}) on the grid
};
struct AdjWork;

// ---------------------------------------------------------------- context
struct Ctx {
  lmvd_config cfg;
  Grid g;
  cudaStream_t stream = nullptr;
  int s = 0;               // substage counter (even: stage n, odd: stage ')
  int status = 0;

  // operators
  DBand B0g, B1g, B2g, Bs[4], Sg0, Sg1, Ss0, Ss2;
  double* dstar = nullptr;  // ny entries: (D* c)_i = dstar[i] (c_{i+1} - c_i)
  DLU lu_interp, lu_neumann, lu_mc, lu_md;
  DLU lu_means;  // lu_interp (walls) or lu_neumann (potential matching): not owned
  FFTPlan fx, fz;

  // memory arena
  void* arena = nullptr;
  size_t arena_bytes = 0;
  std::vector<void*> small_allocs;
  size_t small_bytes = 0;  // bytes of small_allocs

  // state and history (spectral, B coefficients)
  cd *z, *om, *m2;
  double *mm1, *mm3;
  cd* zh[3];
  cd *zdot_prev, *r_om_prev, *r_phi_prev;
  double* r_m_prev;  // 2 * ny
  // substage work (spectral)
  cd *z_new, *om_new, *m2_new;
  double *mm1_new, *mm3_new;
  cd *Rz, *zdot, *rt, *m1c, *m2c, *m3c, *r_om, *r_phi;
  double* r_m;        // 2 * ny
  cd* sv[10];         // spectral value fields at g (FFT outputs / inputs)
  cd* st[7];          // RHS streams: the same memory as sv[0..6] (formed in place from sv)
  cd* tbuf;           // FFT intermediate: tbuf_n fields of ny * pz * (nx/2)
  // physical
  double *md[3], *rho, *invrho, *fprime, *w[3];
  double* pw[PW_FIELDS];  // physical work fields (pw_n of them allocated)
  int pw_n = PW_FIELDS, tbuf_n = TBUF_FIELDS;

  Prof prof;
  AdjWork* adj = nullptr;
  unsigned* dflags = nullptr;  // device status word: bit 0 = a non-finite value in the state (k_check_finite),
                               // bit 1 = the fixed point did not converge (diagnostics on), bit 2 = a z-pass
                               // tile copy (TMA) did not complete within its ~1 s wait (the CTA skipped its work)
  // diagnostics record of the last substage (lmvd_diagnostics): [0, 1] = |mass residual|^2, |rho_t|^2,
  // [2 + 2k, 3 + 2k] = |dz/dt^{k+1} - dz/dt^k|^2, |dz/dt^{k+1}|^2 for k < kf; [DIAG_KE] = kinetic energy,
  // [DIAG_MMAX] = max |m|^2 over the grid (the bits of a non-negative double, ordered as an integer),
  // [DIAG_MC2] = <m2^c> at y0
  bool diag_on = false;
  double* ddiag = nullptr;
  double* wq = nullptr;  // ny quadrature weights at the Greville points (integral of the interpolant)

  // CUDA graphs of one substage (lmvd_graphs_enable), one per launch pattern (see graph_key in api.cu)
  static constexpr int GRAPH_KEY = 23;
  struct SubstageGraph {
    const void* key[GRAPH_KEY];
    cudaGraphExec_t exec;
    long long launches;  // kernels in the graph, and their per-class accounting
    long long n[KC_COUNT];
    double flops[KC_COUNT], bytes[KC_COUNT];
  };
  bool graphs_on = true;
  std::vector<SubstageGraph> graphs;
};

// one substage (api.cu); with a tape the physical fields the adjoint needs are kept
int advance(Ctx& c, const Tape* tape);
// the start-up of lmvd_set_state without history (api.cu), recording the physical z fields of pass 1 in
// tape->zp and dz/dt before each fixed-point application in iterates (n_startup spectral fields)
int startup_record(Ctx& c, const Tape* tape, cd* iterates);
// one fixed-point application from zdot_in (api.cu), recording its physical fields a and b[3]
int fp_record(Ctx& c, const cd* zdot_in, double* a, double* const* b);
// device bytes held by the adjoint workspace (adjoint.cu; 0 before its first use)
size_t adj_device_bytes(const Ctx& c);
// adjoint of one substage (adjoint.cu); blobs as documented for lmvd_adjoint_substage
int adjoint_substage(Ctx& c, const void* sbar_out, const void* hbar_out, void* sbar_in, void* hbar_in);
// adjoint of the start-up (adjoint.cu); blobs as documented for lmvd_adjoint_startup
int adjoint_startup(Ctx& c, const void* sbar_out, const void* hbar_out, void* sbar_in);
void adj_destroy(Ctx& c);

// Bracket a launch: counts it, and with profiling on records CUDA events around it on the stream.
cudaEvent_t prof_begin(Ctx& c);
void prof_end(Ctx& c, int cls, cudaEvent_t a, double flops, double bytes);
#define LMVD_LAUNCH(C, CLS, FLOPS, BYTES, KERN, GRID, BLOCK, SMEM, ...)       \
  do {                                                                      \
    cudaEvent_t ev_a_ = ::lmvd::prof_begin(C);                              \
    KERN<<<GRID, BLOCK, SMEM, (C).stream>>>(__VA_ARGS__);                   \
    ::lmvd::prof_end(C, CLS, ev_a_, (double)(FLOPS), (double)(BYTES));      \
  } while (0)

// The same accounting around a call that launches exactly one kernel on (C).stream.
#define LMVD_LAUNCH_CALL(C, CLS, FLOPS, BYTES, CALL)                     \
  do {                                                                  \
    cudaEvent_t ev_a_ = ::lmvd::prof_begin(C);                          \
    CALL;                                                               \
    ::lmvd::prof_end(C, CLS, ev_a_, (double)(FLOPS), (double)(BYTES));  \
  } while (0)

// ---------------------------------------------------------------- launchers (defined in .cu files)
int fft_prepare(Ctx& c);                       // plans, twiddles, smem attributes
// inverse: nf spectral value fields (in[f]) -> physical (out[f]); in the precision path (precision 1) the
// inputs are the double-float pairs the evaluation kernels store
void fft_inverse(Ctx& c, cd* const* in, double* const* out, int nf);
// forward: nf physical fields -> spectral value fields, truncated and scaled
void fft_forward(Ctx& c, double* const* in, cd* const* out, int nf);
// the same with an explicit arithmetic (0: complex double, 1: double-float), nf <= 64
void fft_inverse_as(Ctx& c, cd* const* in, double* const* out, int nf, int precision);
void fft_forward_as(Ctx& c, double* const* in, cd* const* out, int nf, int precision);
// the fixed point's products formed inside the x-passes (Sec. 4.3): inverse transform of one field whose
// x-pass stores w * phys (rho_t = f'(z) dz/dt), and forward transform of -(w1 m1 + w2 m2 + w3 m3) formed
// in the x-pass prologue (the tail of L); w, m: physical fields in the arithmetic of the precision
void fft_inverse_mul(Ctx& c, cd* in, double* out, const double* w);  // input as for fft_inverse
void fft_forward_dot3(Ctx& c, const double* const* w, const double* const* m, cd* out);

}  // namespace lmvd
