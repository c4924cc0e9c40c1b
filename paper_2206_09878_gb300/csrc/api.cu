// C-ABI of liblmvd (include/lmvd.h) and the host orchestration of one substage (Algorithm 2).
// The host only enqueues kernels on the context's stream; no call synchronises except
// lmvd_create, lmvd_synchronize and lmvd_set_state when it must read a history counter.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <stdexcept>

#include "basis.h"
#include "ykernels.h"

using namespace lmvd;

struct lmvd_ctx {
  Ctx c;
  long long s_blob = 0;
};

namespace lmvd {

LMVD_DEFINE_OOB_TAKE(api)

cudaEvent_t prof_begin(Ctx& c) {
  c.prof.launches++;
  if (!c.prof.on) return nullptr;
  cudaEvent_t a;
  if (!c.prof.pool.empty()) {
    a = c.prof.pool.back();
    c.prof.pool.pop_back();
  } else if (cudaEventCreate(&a) != cudaSuccess) {
    return nullptr;
  }
  cudaEventRecord(a, c.stream);
  return a;
}

void prof_end(Ctx& c, int cls, cudaEvent_t a, double flops, double bytes) {
  c.prof.n[cls]++;
  c.prof.flops[cls] += flops;
  c.prof.bytes[cls] += bytes;
  if (!a) return;
  cudaEvent_t b;
  if (!c.prof.pool.empty()) {
    b = c.prof.pool.back();
    c.prof.pool.pop_back();
  } else if (cudaEventCreate(&b) != cudaSuccess) {
    c.prof.pool.push_back(a);
    return;
  }
  cudaEventRecord(b, c.stream);
  c.prof.pending.push_back(Prof::Pending{cls, a, b});
}

}  // namespace lmvd

namespace {

// fold recorded event pairs into per-class milliseconds (the stream must be synchronised)
void prof_collect(Ctx& c) {
  for (auto& p : c.prof.pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) c.prof.ms[p.cls] += ms;
    c.prof.pool.push_back(p.a);
    c.prof.pool.push_back(p.b);
  }
  c.prof.pending.clear();
}

constexpr int TPB_MODE = 128;

unsigned mode_blocks(const Grid& g) { return (unsigned)((g.M + TPB_MODE - 1) / TPB_MODE); }

unsigned elem_blocks(size_t n) {
  size_t b = (n + 255) / 256;
  return (unsigned)std::min<size_t>(b, 152 * 32);
}

int latch(Ctx& c, int err) {
  if (err != LMVD_OK && c.status == LMVD_OK) c.status = err;
  return err;
}
int cuda_check(Ctx& c) {
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) return LMVD_OK;
  return latch(c, e == cudaErrorMemoryAllocation ? LMVD_ERR_OOM : LMVD_ERR_CUDA);
}

// A device allocation owned by the context (freed by lmvd_destroy, counted by lmvd_device_bytes).
int device_alloc(Ctx& c, void** p, size_t bytes) {
  if (cudaMalloc(p, bytes) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return LMVD_ERR_OOM;
  }
  c.small_allocs.push_back(*p);
  c.small_bytes += bytes;
  return LMVD_OK;
}

template <class T>
int upload(Ctx& c, const std::vector<T>& h, T** d) {
  int e = device_alloc(c, (void**)d, sizeof(T) * std::max<size_t>(1, h.size()));
  if (e) return e;
  if (!h.empty() && cudaMemcpy(*d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return LMVD_ERR_CUDA;
  return LMVD_OK;
}

int upload_band(Ctx& c, const RowBand& m, DBand& d) {
  int* c0;
  double* v;
  df* vf;
  int e = upload(c, m.c0, &c0);
  if (e) return e;
  e = upload(c, m.v, &v);
  if (e) return e;
  std::vector<df> split(m.v.size());
  for (size_t q = 0; q < m.v.size(); ++q) {
    const float hi = (float)m.v[q];
    split[q] = df{hi, (float)(m.v[q] - (double)hi)};
  }
  e = upload(c, split, &vf);
  if (e) return e;
  d.c0 = c0;
  d.v = v;
  d.vf = vf;
  d.cols = m.cols;
  d.rows = m.rows;
  d.w = m.w;
  return LMVD_OK;
}

int half_width(const RowBand& m) {
  int K = 0;
  for (int i = 0; i < m.rows; ++i)
    for (int q = 0; q < m.w; ++q)
      if (m.v[(size_t)i * m.w + q] != 0.0) K = std::max(K, std::abs(m.c0[i] + q - i));
  return K;
}

int upload_lu(Ctx& c, const BandLU& f, DLU& d) {
  double *lo, *up, *invd;
  int *nl, *nu;
  int e = upload(c, f.lo, &lo);
  if (!e) e = upload(c, f.up, &up);
  if (!e) e = upload(c, f.invd, &invd);
  if (!e) e = upload(c, f.nl, &nl);
  if (!e) e = upload(c, f.nu, &nu);
  if (e) return e;
  d = DLU{lo, up, invd, nl, nu, f.n, f.K, 0, 0.0};
  for (int i = 0; i < f.n; ++i) d.flops_per_mode += 4.0 * (f.nl[i] + f.nu[i]) + 2.0;
  return LMVD_OK;
}

// Band matrices of the per-mode systems A(k) = A2 - k^2 A0 + k A1: A2 is the k-independent part,
// A0 the coefficient of -k^2, A1 the coefficient of k (non-zero only in the potential-matching rows).
struct PerMode {
  DiagBand A2, A0, A1;
};

PerMode per_mode_base(const RowBand& Ss0, const RowBand& Ss2, int K) {
  PerMode p;
  p.A2 = to_diag(Ss2, K);
  p.A0 = to_diag(Ss0, K);
  p.A1 = p.A0;
  std::fill(p.A1.a.begin(), p.A1.a.end(), 0.0);
  return p;
}

// Sets row r of the system to the row vectors (a2, a0, a1) of the order-(p+1) space.
void set_row(PerMode& p, int r, int K, const RowBand* a2, int r2, const RowBand* a0, int r0, const RowBand* a1,
             int r1, double s2 = 1.0) {
  const int n = p.A2.n;
  for (int q = -K; q <= K; ++q) {
    const int j = r + q;
    if (j < 0 || j >= n) continue;
    p.A2.el(r, j) = a2 ? s2 * a2->at(r2, j) : 0.0;
    p.A0.el(r, j) = a0 ? a0->at(r0, j) : 0.0;
    p.A1.el(r, j) = a1 ? a1->at(r1, j) : 0.0;
  }
}

// Potential matching (Eq. bc_both times k): row 0: k m2(y0) - dm2/dy(y0) = 0; row n-1: k m2(y1) + dm2/dy(y1)
// = 0. The clamped order-(p+1) Greville points g*_0 and g*_ny are y0 and y1.
void robin_rows(PerMode& p, int K, const RowBand& Ss0, const RowBand& Ss1) {
  const int n = p.A2.n;
  set_row(p, 0, K, &Ss1, 0, nullptr, 0, &Ss0, 0, -1.0);
  set_row(p, n - 1, K, &Ss1, n - 1, nullptr, 0, &Ss0, n - 1, 1.0);
}

// m^c system: rows 1..ny-1: (B*'' - k^2 B*) at g*_i; rows 0 and ny: m2^c(y0) = m2^c(y1) = 0 (walls) or the
// Robin rows (potential matching).
PerMode mc_system(const RowBand& Ss0, const RowBand& Ss1, const RowBand& Ss2, int K, int bc_mode) {
  const int n = Ss0.rows;
  PerMode p = per_mode_base(Ss0, Ss2, K);
  if (bc_mode == 1) {
    robin_rows(p, K, Ss0, Ss1);
  } else {
    for (int r : {0, n - 1}) {
      set_row(p, r, K, nullptr, 0, nullptr, 0, nullptr, 0);
      p.A2.el(r, r) = 1.0;
    }
  }
  return p;
}

// m2^d update: rows 2..ny-2: (B*'' - k^2 B*) at g*_i. Walls: rows 0, ny: m2 = 0; rows 1, ny-1: dm2/dy = 0 at
// y0, y1. Potential matching: rows 0, ny: Robin; row 1: phi2(y0) = 0; row ny-1: phi2(y1) = 0 (Eq. md_bc).
PerMode md_system(const RowBand& Ss0, const RowBand& Ss1, const RowBand& Ss2, int K, int bc_mode) {
  const int n = Ss0.rows;
  PerMode p = per_mode_base(Ss0, Ss2, K);
  if (bc_mode == 1) {
    robin_rows(p, K, Ss0, Ss1);
    set_row(p, 1, K, &Ss2, 0, &Ss0, 0, nullptr, 0);
    set_row(p, n - 2, K, &Ss2, n - 1, &Ss0, n - 1, nullptr, 0);
  } else {
    for (int r : {0, n - 1}) {
      set_row(p, r, K, nullptr, 0, nullptr, 0, nullptr, 0);
      p.A2.el(r, r) = 1.0;
    }
    set_row(p, 1, K, &Ss1, 0, nullptr, 0, nullptr, 0);
    set_row(p, n - 2, K, &Ss1, n - 1, nullptr, 0, nullptr, 0);
  }
  return p;
}

int factor_per_mode(Ctx& c, const PerMode& pm, int K, DLU& out) {
  std::vector<int> nl, nu;
  DiagBand pattern = pm.A0;  // union of the non-zero patterns of A0 and A1 (A2 is the other argument)
  for (size_t i = 0; i < pattern.a.size(); ++i)
    if (pm.A1.a[i] != 0.0) pattern.a[i] = 1.0;
  try {
    band_profile(pm.A2, pattern, nl, nu);
  } catch (const std::exception&) {
    return LMVD_ERR_UNSUPPORTED;
  }
  const int n = pm.A2.n;
  double *A2, *A0, *A1, *lo, *up, *invd;
  int *dnl, *dnu;
  int e = upload(c, pm.A2.a, &A2);
  if (!e) e = upload(c, pm.A0.a, &A0);
  if (!e) e = upload(c, pm.A1.a, &A1);
  if (!e) e = upload(c, nl, &dnl);
  if (!e) e = upload(c, nu, &dnu);
  if (e) return e;
  // factors of the kz >= 0 half-plane (A(k) depends on kz^2): Mh = (nz/2 + 1) nxh factor modes
  const size_t Mh = (size_t)(c.g.nz / 2 + 1) * c.g.nxh;
  if (!(e = device_alloc(c, (void**)&lo, sizeof(double) * (size_t)n * K * Mh)) &&
      !(e = device_alloc(c, (void**)&up, sizeof(double) * (size_t)n * K * Mh)))
    e = device_alloc(c, (void**)&invd, sizeof(double) * (size_t)n * Mh);
  if (e) return e;
  LMVD_LAUNCH(c, KC_MISC, 0, 8.0 * n * (2 * K + 1) * Mh, k_factor, (unsigned)((Mh + TPB_MODE - 1) / TPB_MODE),
              TPB_MODE, 0, c.g, n, K, A2, A0, A1, dnl, dnu, lo, up, invd);
  out = DLU{lo, up, invd, dnl, dnu, n, K, Mh, 0.0};
  for (int i = 0; i < n; ++i) out.flops_per_mode += 4.0 * (nl[i] + nu[i]) + 2.0;
  return cuda_check(c);
}

// ------------------------------------------------------------------ workspace arena
struct Carver {
  char* base;
  size_t off = 0;
  template <class T>
  T* take(size_t count) {
    off = (off + 255) & ~(size_t)255;
    T* p = (T*)(base ? base + off : nullptr);
    off += sizeof(T) * count;
    return p;
  }
};

void carve(Ctx& c, Carver& cv) {
  const Grid& g = c.g;
  const size_t S = (size_t)g.ny * g.M, Sp = (size_t)(g.ny + 1) * g.M, P = (size_t)g.ny * g.P;
  const int ny = g.ny;
  c.z = cv.take<cd>(S);
  c.om = cv.take<cd>(S);
  c.m2 = cv.take<cd>(Sp);
  c.z_new = cv.take<cd>(S);
  c.om_new = cv.take<cd>(S);
  c.m2_new = cv.take<cd>(Sp);
  for (auto& h : c.zh) h = cv.take<cd>(S);
  c.zdot_prev = cv.take<cd>(S);
  c.r_om_prev = cv.take<cd>(S);
  c.r_phi_prev = cv.take<cd>(Sp);
  c.Rz = cv.take<cd>(S);
  c.zdot = cv.take<cd>(S);
  c.rt = cv.take<cd>(S);
  c.m1c = cv.take<cd>(S);
  c.m2c = cv.take<cd>(Sp);
  c.m3c = cv.take<cd>(S);
  c.r_om = cv.take<cd>(S);
  c.r_phi = cv.take<cd>(Sp);
  for (auto& p : c.sv) p = cv.take<cd>(S);
  for (int q = 0; q < 7; ++q) c.st[q] = c.sv[q];
  c.mm1 = cv.take<double>(ny);
  c.mm3 = cv.take<double>(ny);
  c.mm1_new = cv.take<double>(ny);
  c.mm3_new = cv.take<double>(ny);
  c.r_m = cv.take<double>(2 * ny);
  c.r_m_prev = cv.take<double>(2 * ny);
  for (auto& p : c.md) p = cv.take<double>(P);
  c.rho = cv.take<double>(P);
  c.invrho = cv.take<double>(P);
  c.fprime = cv.take<double>(P);
  for (auto& p : c.w) p = cv.take<double>(P);
  for (int f = 0; f < PW_FIELDS; ++f) c.pw[f] = f < c.pw_n ? cv.take<double>(P) : nullptr;
  c.tbuf = cv.take<cd>((size_t)c.tbuf_n * ny * g.pz * (g.nx / 2));
}

// ------------------------------------------------------------------ substage pieces
void eval_jobs(Ctx& c, std::initializer_list<EvalJob> jobs) {
  EvalJobs ej{};
  int n = 0;
  double rows = 0, fl = 0;
  for (const EvalJob& j : jobs) {
    ej.j[n++] = j;
    rows += 2.0 * j.B.rows;
    fl += 4.0 * j.B.rows * j.B.w;
  }
  int maxrows = 0, maxw = 0;
  for (int q = 0; q < n; ++q) {
    maxrows = std::max(maxrows, ej.j[q].B.rows);
    maxw = std::max(maxw, ej.j[q].B.w);
  }
  // the precision path evaluates the values that feed its transforms in double-float, stored as pairs for
  // its inverse transforms (fft_inverse); its jobs never accumulate
  if (c.cfg.precision == 1) {
    const dim3 grid(mode_blocks(c.g), n, row_chunks(c.g, maxrows));
    LMVD_LAUNCH_CALL(c, KC_EVAL, fl * c.g.M, 16.0 * rows * c.g.M,
                     launch_eval_df(maxw, grid, TPB_MODE, c.stream, c.g, ej));
  } else
    LMVD_LAUNCH(c, KC_EVAL, fl * c.g.M, 16.0 * rows * c.g.M, k_eval,
                dim3(mode_blocks(c.g), n, row_chunks(c.g, maxrows)), TPB_MODE, 0, c.g, ej);
}

// out = A^{-1} in (+ add) for each job; shared or per-mode factors; one or two threads per mode
// (solve_split)
void solve_modes(Ctx& c, KClass cls, std::initializer_list<SolveJob> jobs, const DLU& lu) {
  SolveJobs sj{};
  int n = 0;
  double arrays = 0;
  for (const SolveJob& j : jobs) {
    sj.j[n++] = j;
    arrays += j.add ? 3 : 2;
  }
  const double rowsM = (double)lu.n * c.g.M;
  const double factors = lu.mstride ? 8.0 * (2 * lu.K + 1) * rowsM * n : 0.0;
  const int tpm = solve_split(c.g);
  const unsigned blocks = (unsigned)((tpm * c.g.M + TPB_MODE - 1) / TPB_MODE);
  if (tpm == 2)
    LMVD_LAUNCH(c, cls, n * lu.flops_per_mode * c.g.M, 16.0 * arrays * rowsM + factors, k_solve_re, dim3(blocks, n),
                TPB_MODE, 0, c.g, lu, sj);
  else
    LMVD_LAUNCH(c, cls, n * lu.flops_per_mode * c.g.M, 16.0 * arrays * rowsM + factors, k_solve_cd, dim3(blocks, n),
                TPB_MODE, 0, c.g, lu, sj);
}
void solve_interp(Ctx& c, std::initializer_list<SolveJob> jobs, const DLU& lu) { solve_modes(c, KC_SOLVE, jobs, lu); }

// steps 1-2: m^d and z-derived fields in physical space; rho, 1/rho, f', grad z / rho; R_z.
// zp: where z, dz/dx, dz/dz, dz/dy, lap z land on the physical grid (work fields by default; the adjoint
// keeps them).
void physical_pass_1(Ctx& c, double* const* zp = nullptr) {
  double* zf[5] = {c.pw[0], c.pw[1], c.pw[2], c.pw[3], c.pw[4]};
  if (zp)
    for (int f = 0; f < 5; ++f) zf[f] = zp[f];
  Fields8 o{};
  for (int f = 0; f < 8; ++f) o.p[f] = c.sv[f];
  const double SM = (double)c.g.ny * c.g.M;
  if (c.cfg.precision == 1) {
    const dim3 grid(mode_blocks(c.g), row_chunks(c.g, c.g.ny));
    LMVD_LAUNCH_CALL(c, KC_EVAL_P1, SM * (4.0 * 6 * c.B0g.w + 20.0), 16.0 * SM * 11 + 16.0 * c.g.M,
                     launch_eval_p1_df(c.cfg.spline_order, grid, TPB_MODE, c.stream, c.g, c.B0g, c.B1g, c.B2g, c.Sg0,
                                       c.Sg1, c.z, c.om, c.m2, c.mm1, c.mm3, o));
  } else
    LMVD_LAUNCH(c, KC_EVAL_P1, SM * (4.0 * 6 * c.B0g.w + 20.0), 16.0 * SM * 11 + 16.0 * c.g.M, k_eval_p1,
                dim3(mode_blocks(c.g), row_chunks(c.g, c.g.ny)), TPB_MODE, 0, c.g, c.B0g, c.B1g, c.B2g, c.Sg0,
                c.Sg1, c.z, c.om, c.m2, c.mm1, c.mm3, o);
  // physical: z, zx, zz, zy, lapz -> pw[0..4]; m^d -> md[0..2]
  cd* in[8] = {c.sv[0], c.sv[1], c.sv[2], c.sv[3], c.sv[4], c.sv[5], c.sv[6], c.sv[7]};
  double* out[8] = {zf[0], zf[1], zf[2], zf[3], zf[4], c.md[0], c.md[1], c.md[2]};
  fft_inverse(c, in, out, 8);
  const size_t n = (size_t)c.g.ny * c.g.P;
  EosArgs e{c.cfg.rho_heavy, c.cfg.rho_light, 1.0 / (c.cfg.re * c.cfg.sc)};
  if (c.cfg.precision == 1)
    LMVD_LAUNCH(c, KC_PRODUCTS, 25.0 * n, 8.0 * 15 * n, k_products_p1_df, elem_blocks(n), 256, 0, n, e, zf[0],
                zf[1], zf[2], zf[3], zf[4], c.md[0], c.md[1], c.md[2], c.rho, c.invrho, c.fprime, c.w[0],
                c.w[1], c.w[2], c.pw[5]);
  else
    LMVD_LAUNCH(c, KC_PRODUCTS, 25.0 * n, 8.0 * 15 * n, k_products_p1, elem_blocks(n), 256, 0, n, e, zf[0],
                zf[1], zf[2], zf[3], zf[4], c.md[0], c.md[1], c.md[2], c.rho, c.invrho, c.fprime, c.w[0],
                c.w[1], c.w[2], c.pw[5]);
  double* fin[1] = {c.pw[5]};
  cd* fout[1] = {c.sv[0]};
  fft_forward(c, fin, fout, 1);
  solve_interp(c, {SolveJob{c.sv[0], nullptr, c.Rz}}, c.lu_interp);
}

// rho_t = P[f'(z) zdot] and m^c = C(rho_t) (B coefficients), then m^c on the physical grid.
// a: where zdot lands on the physical grid; b: where m^c lands (work fields by default).
void mc_from_zdot(Ctx& c, double* a = nullptr, double* const* b = nullptr) {
  const size_t n = (size_t)c.g.ny * c.g.P;
  const bool keep_a = a != nullptr;  // the adjoint's tape keeps dz/dt on the grid: separate product pass
  if (!a) a = c.pw[0];
  double* bb[3] = {c.pw[0], c.pw[1], c.pw[2]};
  if (b)
    for (int f = 0; f < 3; ++f) bb[f] = b[f];
  eval_jobs(c, {EvalJob{c.B0g, c.zdot, c.sv[0], 0}});
  if (!keep_a) {
    // rho_t = f' dz/dt formed in the epilogue of the inverse x-pass (dz/dt on the grid is not stored)
    fft_inverse_mul(c, c.sv[0], c.pw[1], c.fprime);
  } else {
    {
      cd* in[1] = {c.sv[0]};
      double* out[1] = {a};
      fft_inverse(c, in, out, 1);
    }
    if (c.cfg.precision == 1)
      LMVD_LAUNCH(c, KC_PRODUCTS, 1.0 * n, 24.0 * n, k_product_rt_df, elem_blocks(n), 256, 0, n, c.fprime, a,
                  c.pw[1]);
    else
      LMVD_LAUNCH(c, KC_PRODUCTS, 1.0 * n, 24.0 * n, k_product_rt, elem_blocks(n), 256, 0, n, c.fprime, a, c.pw[1]);
  }
  {
    double* in[1] = {c.pw[1]};
    cd* out[1] = {c.sv[1]};
    fft_forward(c, in, out, 1);
  }
  solve_interp(c, {SolveJob{c.sv[1], nullptr, c.rt}}, c.lu_interp);
  {
    const double rowsM = (double)(c.g.ny + 1) * c.g.M;
    LMVD_LAUNCH(c, KC_MC_SOLVE, rowsM * 4.0 * c.Bs[1].w, rowsM * 16.0 * 2, k_mc_rhs,
                dim3(mode_blocks(c.g), row_chunks(c.g, c.g.ny + 1)), TPB_MODE, 0, c.g, c.Bs[1], c.rt, c.m2c);
    solve_modes(c, KC_MC_SOLVE, {SolveJob{c.m2c, nullptr, c.m2c}}, c.lu_mc);
    LMVD_LAUNCH(c, KC_MC_SOLVE, rowsM * 20.0, rowsM * 16.0 * 5, k_mc_post,
                dim3(mode_blocks(c.g), row_chunks(c.g, c.g.ny)), TPB_MODE, 0, c.g, c.dstar, c.rt, c.m1c, c.m2c,
                c.m3c);
  }
  eval_jobs(c, {EvalJob{c.B0g, c.m1c, c.sv[0], 0}, EvalJob{c.Sg0, c.m2c, c.sv[1], 0}, EvalJob{c.B0g, c.m3c, c.sv[2], 0}});
  cd* in[3] = {c.sv[0], c.sv[1], c.sv[2]};
  fft_inverse(c, in, bb, 3);
}

// one application of the fixed point (Eq. y_k): zdot <- L(z) zdot + R_z
void fp_apply(Ctx& c, double* a = nullptr, double* const* b = nullptr) {
  mc_from_zdot(c, a, b);
  double* bb[3] = {c.pw[0], c.pw[1], c.pw[2]};
  if (b)
    for (int f = 0; f < 3; ++f) bb[f] = b[f];
  // the tail -(grad z / rho) . m^c formed in the prologue of the forward x-pass
  const double* w[3] = {c.w[0], c.w[1], c.w[2]};
  const double* m[3] = {bb[0], bb[1], bb[2]};
  fft_forward_dot3(c, w, m, c.sv[3]);
  solve_interp(c, {SolveJob{c.sv[3], c.Rz, c.zdot}}, c.lu_interp);
}

// Reading R6: n_startup fixed-point applications from dz/dt = 0, then the Taylor back-fill of the history.
// tape (optional): records the physical z fields of pass 1; iterates (optional): receives dz/dt before each
// application, n_startup consecutive spectral fields (the adjoint re-records each application from these).
void startup(Ctx& c, const Tape* tape = nullptr, cd* iterates = nullptr) {
  NvtxRange range("lmvd start-up");
  const size_t S = (size_t)c.g.ny * c.g.M;
  physical_pass_1(c, tape ? tape->zp : nullptr);
  cudaMemsetAsync(c.zdot, 0, sizeof(cd) * S, c.stream);
  for (int it = 0; it < c.cfg.n_startup; ++it) {
    if (iterates)
      cudaMemcpyAsync(iterates + (size_t)it * S, c.zdot, sizeof(cd) * S, cudaMemcpyDeviceToDevice, c.stream);
    fp_apply(c);
  }
  const double dt = c.cfg.dt;
  LMVD_LAUNCH(c, KC_MISC, 12.0 * S, 80.0 * S, k_backfill, elem_blocks(S), 256, 0, S, 0.5 * dt, dt, 1.5 * dt, c.z,
              c.zdot, c.zh[0], c.zh[1], c.zh[2]);
  cudaMemcpyAsync(c.zdot_prev, c.zdot, sizeof(cd) * S, cudaMemcpyDeviceToDevice, c.stream);
  cudaMemsetAsync(c.r_om_prev, 0, sizeof(cd) * S, c.stream);
  cudaMemsetAsync(c.r_phi_prev, 0, sizeof(cd) * (S + c.g.M), c.stream);
  cudaMemsetAsync(c.r_m_prev, 0, sizeof(double) * 2 * c.g.ny, c.stream);
  c.s = 0;
}

// Enqueues the kernels of one substage on c.stream (no host synchronisation, no allocation: the sequence
// can be captured into a CUDA graph); rotate_history() then advances the host-side buffer assignment.
void enqueue_substage(Ctx& c, const Tape* tape) {
  const Grid& g = c.g;
  const lmvd_config& cf = c.cfg;
  const size_t S = (size_t)g.ny * g.M;
  const size_t n = (size_t)g.ny * g.P;
  const bool stage_n = (c.s % 2) == 0;
  NvtxRange substage_range("lmvd substage (Algorithm 2)");
  // steps 1-2
  NvtxRange pass1_range("steps 1-2: m^d, pass 1, R_z, BDF guess");
  physical_pass_1(c, tape ? tape->zp : nullptr);
  double a[4];
  if (stage_n) {
    const double b = cf.beta_n;
    a[0] = 2.0; a[1] = -(2.0 + 0.5 * b); a[2] = b; a[3] = -0.5 * b;
  } else {
    const double b = cf.beta_p;
    a[0] = 4.0 + b; a[1] = -(5.0 + 2.0 * b); a[2] = b; a[3] = 1.0;
  }
  LMVD_LAUNCH(c, KC_MISC, 16.0 * S, 80.0 * S, k_bdf, elem_blocks(S), 256, 0, S, a[0], a[1], a[2], a[3], 1.0 / cf.dt,
              c.z, c.zh[0], c.zh[1], c.zh[2], c.zdot);
  // step 3
  nvtxRangePop();
  nvtxRangePushA("step 3: fixed point, m^c");
  if (c.diag_on) cudaMemsetAsync(c.ddiag, 0, sizeof(double) * DIAG_N, c.stream);
  for (int k = 0; k < cf.kf; ++k) {
    // diagnostics: the change of this application (the previous iterate kept in sv[9], unused until pass 2)
    if (c.diag_on && k < KF_MAX_ADJ + 1)
      cudaMemcpyAsync(c.sv[9], c.zdot, sizeof(cd) * S, cudaMemcpyDeviceToDevice, c.stream);
    fp_apply(c, tape ? tape->a[k] : nullptr, tape ? tape->b[k] : nullptr);
    if (c.diag_on && k < KF_MAX_ADJ + 1)
      LMVD_LAUNCH(c, KC_MISC, 6.0 * S, 32.0 * S, k_diff_norms, elem_blocks(S), 256, 0, S, c.zdot, c.sv[9],
                  c.ddiag + 2 + 2 * k);
  }
  mc_from_zdot(c, tape ? tape->a[cf.kf] : nullptr, tape ? tape->b[cf.kf] : nullptr);
  if (c.diag_on) {
    LMVD_LAUNCH(c, KC_MISC, 20.0 * S, 16.0 * 5 * S, k_mass_norms, elem_blocks(S), 256, 0, g, c.dstar, c.rt, c.m1c,
                c.m2c, c.m3c, c.ddiag);
    if (cf.kf <= KF_MAX_ADJ + 1)
      LMVD_LAUNCH(c, KC_MISC, 0, 0, k_fp_check, 1, 1, 0, c.ddiag, cf.kf, c.dflags);
  }
  const double* mcp[3] = {c.pw[0], c.pw[1], c.pw[2]};
  if (tape)
    for (int f = 0; f < 3; ++f) mcp[f] = tape->b[cf.kf][f];
  nvtxRangePop();
  nvtxRangePushA("steps 4-5: pass 2, RHS");
  // steps 4-5: products with m = m^d + m^c, forward transforms, RHS streams, collocation solves, RHS.
  // The ten products overwrite m^c where it sits in pw[0..2] (each point's inputs are read before its
  // outputs are written): one batch into pw[0..9] in the full layout; in the lean one (6 work fields)
  // C11-C13 and C22-C33 through pw[3..5], then u and rho into pw[0..3].
  struct Batch { int first, count, slot; };
  const Batch full[1] = {{0, 10, 0}}, lean[3] = {{0, 3, 3}, {3, 3, 3}, {6, 4, 0}};
  if (c.diag_on) {
    // kinetic energy and max |m| of m = m^d + m^c (before the products overwrite m^c), <m2^c> at y0
    Fields3C mdf{{c.md[0], c.md[1], c.md[2]}}, mcf{{mcp[0], mcp[1], mcp[2]}};
    LMVD_LAUNCH(c, KC_MISC, 10.0 * n, 8.0 * 7 * n, k_energy_norms, elem_blocks(n), 256, 0, g, c.wq, mdf, mcf,
                c.invrho, cf.precision == 1 ? 1 : 0, c.ddiag + DIAG_KE,
                reinterpret_cast<unsigned long long*>(c.ddiag + DIAG_MMAX));
    cudaMemcpyAsync(c.ddiag + DIAG_MC2, c.m2c, sizeof(double), cudaMemcpyDeviceToDevice, c.stream);
  }
  const Batch* batches = c.pw_n >= 10 ? full : lean;
  const int nb = c.pw_n >= 10 ? 1 : 3;
  for (int b = 0; b < nb; ++b) {
    const Batch& bt = batches[b];
    P2Out q{};
    for (int f = 0; f < bt.count; ++f) q.p[bt.first + f] = c.pw[bt.slot + f];
    const double fl = 1.8 * bt.count * n, by = 8.0 * (8 + bt.count) * n;
    if (cf.precision == 1)
      LMVD_LAUNCH(c, KC_PRODUCTS, fl, by, k_products_p2_df, elem_blocks(n), 256, 0, n, c.md[0], c.md[1], c.md[2],
                  mcp[0], mcp[1], mcp[2], c.rho, c.invrho, q);
    else
      LMVD_LAUNCH(c, KC_PRODUCTS, fl, by, k_products_p2, elem_blocks(n), 256, 0, n, c.md[0], c.md[1], c.md[2],
                  mcp[0], mcp[1], mcp[2], c.rho, c.invrho, q);
    fft_forward(c, c.pw + bt.slot, c.sv + bt.first, bt.count);
  }
  Fields10C svc{};
  for (int f = 0; f < 10; ++f) svc.p[f] = c.sv[f];
  Fields7 stw{};
  for (int f = 0; f < 7; ++f) stw.p[f] = c.st[f];
  LMVD_LAUNCH(c, KC_RHS_COMBINE, 90.0 * S, 16.0 * 17 * S, k_rhs_combine, elem_blocks(S), 256, 0, g, 1.0 / cf.re,
              1.0 / (cf.fr * cf.fr), svc, stw);
  solve_interp(c,
               {SolveJob{c.st[1], nullptr, c.st[1]}, SolveJob{c.st[2], nullptr, c.st[2]},
                SolveJob{c.st[3], nullptr, c.st[3]}, SolveJob{c.st[4], nullptr, c.st[4]},
                SolveJob{c.st[5], nullptr, c.st[5]}, SolveJob{c.st[6], nullptr, c.st[6]}},
               c.lu_interp);
  Fields7C stc{};
  for (int f = 0; f < 7; ++f) stc.p[f] = c.st[f];
  if (cf.precision == 1) {
    const dim3 grid(mode_blocks(g), row_chunks(g, g.ny + 1));
    LMVD_LAUNCH_CALL(c, KC_RHS_EVAL, S * (4.0 * 6 * c.B1g.w + 4.0), 16.0 * 9 * S,
                     launch_rhs_eval_df(cf.spline_order, grid, TPB_MODE, c.stream, g, c.B1g, c.B2g, c.Bs, stc, c.r_om,
                                        c.r_phi, c.r_m));
  } else
    LMVD_LAUNCH(c, KC_RHS_EVAL, S * (4.0 * 6 * c.B1g.w + 4.0), 16.0 * 9 * S, k_rhs_eval,
                dim3(mode_blocks(g), row_chunks(g, g.ny + 1)), TPB_MODE, 0,
                g, c.B1g, c.B2g, c.Bs[0], c.Bs[1], c.Bs[2], c.Bs[3], stc, c.r_om, c.r_phi, c.r_m);
  nvtxRangePop();
  nvtxRangePushA("step 6: RK2 update");
  // step 6: midpoint RK2, low-storage: (al, be) = (1/2, 0) at stage n, (1, -1/2) at stage '
  UpdateArgs u{};
  u.dt = cf.dt;
  u.al = stage_n ? 0.5 : 1.0;
  u.be = stage_n ? 0.0 : -0.5;
  u.om = c.om; u.r_om = c.r_om; u.r_om_prev = c.r_om_prev;
  u.z = c.z; u.zdot = c.zdot; u.zdot_prev = c.zdot_prev;
  u.m2 = c.m2; u.r_phi = c.r_phi; u.r_phi_prev = c.r_phi_prev;
  u.mm1 = c.mm1; u.mm3 = c.mm3; u.r_m = c.r_m; u.r_m_prev = c.r_m_prev;
  u.om_new = c.om_new; u.z_new = c.z_new; u.m2_new = c.m2_new; u.mm1_new = c.mm1_new; u.mm3_new = c.mm3_new;
  LMVD_LAUNCH(c, KC_UPDATE, S * (12.0 * c.B0g.w + 20.0), 16.0 * 7 * S, k_update_om_z_rhs,
              dim3(mode_blocks(g), row_chunks(g, g.ny), 2), TPB_MODE, 0, g, c.B0g, u);
  solve_modes(c, KC_UPDATE, {SolveJob{c.om_new, nullptr, c.om_new}}, c.lu_interp);
  solve_modes(c, KC_UPDATE, {SolveJob{c.z_new, nullptr, c.z_new}}, c.lu_neumann);
  LMVD_LAUNCH(c, KC_UPDATE, 0, 0, k_update_means, 1, 32, 0, g, c.B0g, c.lu_means, u);
  {
    const double Sp = (double)(g.ny + 1) * g.M;
    LMVD_LAUNCH(c, KC_UPDATE, Sp * (8.0 * c.Ss0.w + 10.0), 16.0 * 4 * Sp, k_update_m2_rhs,
                dim3(mode_blocks(g), row_chunks(g, g.ny + 1)), TPB_MODE, 0, g, c.Ss0, c.Ss2, u);
    solve_modes(c, KC_UPDATE, {SolveJob{c.m2_new, nullptr, c.m2_new}}, c.lu_md);
  }
  // failure detection: any non-finite value in the new state sets the device status word
  {
    CheckJobs cj{};
    cj.j[0] = CheckJob{reinterpret_cast<const double*>(c.z_new), 2 * S};
    cj.j[1] = CheckJob{reinterpret_cast<const double*>(c.om_new), 2 * S};
    cj.j[2] = CheckJob{reinterpret_cast<const double*>(c.m2_new), 2 * (S + g.M)};
    cj.j[3] = CheckJob{c.mm1_new, (size_t)g.ny};
    cj.j[4] = CheckJob{c.mm3_new, (size_t)g.ny};
    LMVD_LAUNCH(c, KC_MISC, 0, 8.0 * (6 * S + 2 * g.M + 2 * g.ny), k_check_finite, dim3(elem_blocks(2 * S), 5), 256,
                0, cj, c.dflags);
  }
}

// history rotation (pointer swaps): z cycles through five buffers, the other pairs swap
void rotate_history(Ctx& c) {
  cd* oldest = c.zh[2];
  c.zh[2] = c.zh[1];
  c.zh[1] = c.zh[0];
  c.zh[0] = c.z;
  c.z = c.z_new;
  c.z_new = oldest;
  std::swap(c.om, c.om_new);
  std::swap(c.m2, c.m2_new);
  std::swap(c.mm1, c.mm1_new);
  std::swap(c.mm3, c.mm3_new);
  std::swap(c.zdot_prev, c.zdot);
  std::swap(c.r_om_prev, c.r_om);
  std::swap(c.r_phi_prev, c.r_phi);
  std::swap(c.r_m_prev, c.r_m);
  c.s += 1;
}

// What decides the launch sequence of a substage besides the configuration: the stage, the diagnostics
// flag and which buffer plays which role. z rotates with period 5 and the pairs with period 2, so a run
// meets 10 keys.
void graph_key(const Ctx& c, const void** k) {
  const void* p[Ctx::GRAPH_KEY] = {c.z, c.z_new, c.zh[0], c.zh[1], c.zh[2], c.om, c.om_new, c.m2, c.m2_new,
                                   c.mm1, c.mm1_new, c.mm3, c.mm3_new, c.zdot, c.zdot_prev, c.r_om, c.r_om_prev,
                                   c.r_phi, c.r_phi_prev, c.r_m, c.r_m_prev,
                                   reinterpret_cast<const void*>((uintptr_t)(c.s & 1)),
                                   reinterpret_cast<const void*>((uintptr_t)c.diag_on)};
  for (int i = 0; i < Ctx::GRAPH_KEY; ++i) k[i] = p[i];
}

void graphs_clear(Ctx& c) {
  for (auto& G : c.graphs) cudaGraphExecDestroy(G.exec);
  c.graphs.clear();
}

// Capture the substage's launches into a graph (nothing runs during the capture) and instantiate it;
// the launch accounting it enqueued is kept with the graph and added at every replay.
Ctx::SubstageGraph* graph_capture(Ctx& c) {
  if (c.graphs.size() >= 32) graphs_clear(c);
  Ctx::SubstageGraph G{};
  graph_key(c, G.key);
  const Prof before = c.prof;
  if (cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  enqueue_substage(c, nullptr);
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(c.stream, &graph);
  G.launches = c.prof.launches - before.launches;
  for (int k = 0; k < KC_COUNT; ++k) {
    G.n[k] = c.prof.n[k] - before.n[k];
    G.flops[k] = c.prof.flops[k] - before.flops[k];
    G.bytes[k] = c.prof.bytes[k] - before.bytes[k];
  }
  c.prof.launches = before.launches;
  for (int k = 0; k < KC_COUNT; ++k) {
    c.prof.n[k] = before.n[k];
    c.prof.flops[k] = before.flops[k];
    c.prof.bytes[k] = before.bytes[k];
  }
  if (e != cudaSuccess || !graph) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return nullptr;
  }
  const cudaError_t ei = cudaGraphInstantiate(&G.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  c.graphs.push_back(G);
  return &c.graphs.back();
}

Ctx::SubstageGraph* graph_find(Ctx& c) {
  const void* k[Ctx::GRAPH_KEY];
  graph_key(c, k);
  for (auto& G : c.graphs)
    if (std::equal(k, k + Ctx::GRAPH_KEY, G.key)) return &G;
  return nullptr;
}

int advance_impl(Ctx& c, const Tape* tape) {
  // the graph path: not with a tape (adjoint recording), not while profiling (its events time each
  // launch), not on the legacy default stream (it cannot be captured)
  // nor while the caller is capturing the stream into a graph of its own (the launches then go into it)
  cudaStreamCaptureStatus capturing = cudaStreamCaptureStatusNone;
  if (c.graphs_on && !tape && !c.prof.on && c.stream &&
      cudaStreamIsCapturing(c.stream, &capturing) == cudaSuccess && capturing == cudaStreamCaptureStatusNone) {
    Ctx::SubstageGraph* G = graph_find(c);
    if (!G) G = graph_capture(c);
    if (G) {
      NvtxRange range("lmvd substage (graph)");
      if (cudaGraphLaunch(G->exec, c.stream) != cudaSuccess) return latch(c, LMVD_ERR_CUDA);
      c.prof.launches += G->launches;
      for (int k = 0; k < KC_COUNT; ++k) {
        c.prof.n[k] += G->n[k];
        c.prof.flops[k] += G->flops[k];
        c.prof.bytes[k] += G->bytes[k];
      }
      rotate_history(c);
      return cuda_check(c);
    }
    c.graphs_on = false;  // capture refused: eager launches from here on
  }
  enqueue_substage(c, tape);
  rotate_history(c);
  return cuda_check(c);
}

}  // namespace

namespace lmvd {
int advance(Ctx& c, const Tape* tape) { return advance_impl(c, tape); }
int startup_record(Ctx& c, const Tape* tape, cd* iterates) {
  startup(c, tape, iterates);
  return cudaGetLastError() == cudaSuccess ? LMVD_OK : LMVD_ERR_CUDA;
}
int fp_record(Ctx& c, const cd* zdot_in, double* a, double* const* b) {
  cudaMemcpyAsync(c.zdot, zdot_in, sizeof(cd) * c.g.ny * c.g.M, cudaMemcpyDeviceToDevice, c.stream);
  fp_apply(c, a, b);
  return cudaGetLastError() == cudaSuccess ? LMVD_OK : LMVD_ERR_CUDA;
}
}  // namespace lmvd

namespace {

bool valid_cfg(const lmvd_config& f) {
  if (f.nx < 4 || f.nz < 4 || (f.nx % 2) || (f.nz % 2)) return false;
  if (f.spline_order < 4 || f.spline_order > 8 || f.ny < f.spline_order + 4) return false;
  if (!(f.lx > 0) || !(f.lz > 0) || !(f.y1 > f.y0)) return false;
  if (!(f.re > 0) || !(f.sc > 0) || !(f.fr > 0) || !(f.rho_heavy > 0) || !(f.rho_light > 0)) return false;
  if (!(f.dt > 0) || f.kf < 0 || f.n_startup < 0) return false;
  if (f.precision != 0 && f.precision != 1) return false;
  if (f.bc_mode != 0 && f.bc_mode != 1) return false;
  if (f.memory_layout < 0 || f.memory_layout > 2) return false;
  return true;
}

int copy_in(Ctx& c, void* dst, const void* src, size_t bytes) {
  return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, c.stream) == cudaSuccess ? LMVD_OK : LMVD_ERR_CUDA;
}

}  // namespace

// ====================================================================== C-ABI
extern "C" {

int lmvd_default_config(lmvd_config* f, int nx, int ny, int nz) {
  if (!f) return LMVD_ERR_INVALID_ARG;
  std::memset(f, 0, sizeof(*f));
  f->nx = nx;
  f->ny = ny;
  f->nz = nz;
  f->spline_order = 6;
  f->lx = f->lz = 6.283185307179586476925286766559;
  f->y0 = -1.0;
  f->y1 = 1.0;
  f->re = 1000.0;
  f->sc = 1.0;
  f->fr = 1.0;
  f->rho_heavy = 1.0;
  f->rho_light = 1.0 / 3.0;
  f->dt = 1e-3;
  f->kf = 4;
  f->beta_n = 0.0;
  f->beta_p = -4.0;
  f->n_startup = 20;
  return LMVD_OK;
}

int lmvd_create(const lmvd_config* cfg, void* stream, lmvd_ctx** out) {
  if (!cfg || !out) return LMVD_ERR_INVALID_ARG;
  *out = nullptr;
  if (!valid_cfg(*cfg)) return LMVD_ERR_INVALID_ARG;
  lmvd_ctx* h = new (std::nothrow) lmvd_ctx();
  if (!h) return LMVD_ERR_OOM;
  Ctx& c = h->c;
  c.cfg = *cfg;
  c.stream = (cudaStream_t)stream;
  Grid& g = c.g;
  g.nx = cfg->nx;
  g.ny = cfg->ny;
  g.nz = cfg->nz;
  g.nxh = cfg->nx / 2 + 1;
  g.px = 3 * cfg->nx / 2;
  g.pz = 3 * cfg->nz / 2;
  g.M = (size_t)cfg->nz * g.nxh;
  g.P = (size_t)g.px * g.pz;
  g.lx = cfg->lx;
  g.lz = cfg->lz;
  int err = LMVD_OK;
  try {
    const int p = cfg->spline_order, ny = cfg->ny;
    Knots kb = clamped_uniform(p, ny, cfg->y0, cfg->y1);
    Knots ks = clamped_uniform(p + 1, ny + 1, cfg->y0, cfg->y1);
    std::vector<double> gb = greville(kb), gs = greville(ks);
    RowBand B0g = collocation(kb, gb, 0), B1g = collocation(kb, gb, 1), B2g = collocation(kb, gb, 2);
    RowBand Bs[4];
    for (int d = 0; d < 4; ++d) Bs[d] = collocation(kb, gs, d);
    RowBand Sg0 = collocation(ks, gb, 0), Sg1 = collocation(ks, gb, 1);
    RowBand Ss0 = collocation(ks, gs, 0), Ss1 = collocation(ks, gs, 1), Ss2 = collocation(ks, gs, 2);
    // exact derivative map D*: (D* c)_i = (order-1) (c_{i+1} - c_i) / (t*_{i+order} - t*_{i+1})
    std::vector<double> ds(ny);
    for (int i = 0; i < ny; ++i) ds[i] = (double)p / (ks.t[i + p + 1] - ks.t[i + 1]);
    if (!err) err = upload_band(c, B0g, c.B0g);
    if (!err) err = upload_band(c, B1g, c.B1g);
    if (!err) err = upload_band(c, B2g, c.B2g);
    for (int d = 0; d < 4 && !err; ++d) err = upload_band(c, Bs[d], c.Bs[d]);
    if (!err) err = upload_band(c, Sg0, c.Sg0);
    if (!err) err = upload_band(c, Sg1, c.Sg1);
    if (!err) err = upload_band(c, Ss0, c.Ss0);
    if (!err) err = upload_band(c, Ss2, c.Ss2);
    if (!err) err = upload(c, ds, &c.dstar);
    if (!err) err = upload(c, greville_quadrature(kb, B0g), &c.wq);
    // shared LUs: interpolation / Dirichlet (values at g) and Neumann (dz/dy rows at the walls)
    const int Kb = std::max(half_width(B0g), half_width(B1g));
    if (Kb > KMAX) throw std::runtime_error("band");
    DiagBand Ai = to_diag(B0g, Kb), An = to_diag(B0g, Kb);
    for (int r : {0, ny - 1})
      for (int q = -Kb; q <= Kb; ++q) {
        int j = r + q;
        if (j >= 0 && j < ny) An.el(r, j) = B1g.at(r, j);
      }
    if (!err) err = upload_lu(c, band_lu(Ai), c.lu_interp);
    if (!err) err = upload_lu(c, band_lu(An), c.lu_neumann);
    // per-mode LUs of the m^c and m2^d systems
    const int Ks = std::max({half_width(Ss0), half_width(Ss1), half_width(Ss2)});
    if (Ks > KMAX) throw std::runtime_error("band");
    if (!err) err = factor_per_mode(c, mc_system(Ss0, Ss1, Ss2, Ks, cfg->bc_mode), Ks, c.lu_mc);
    if (!err) err = factor_per_mode(c, md_system(Ss0, Ss1, Ss2, Ks, cfg->bc_mode), Ks, c.lu_md);
    // plane means <m1>, <m3>: Dirichlet rows (walls) or Neumann rows (potential matching)
    c.lu_means = cfg->bc_mode == 1 ? c.lu_neumann : c.lu_interp;
  } catch (const std::exception&) {
    err = err ? err : LMVD_ERR_UNSUPPORTED;
  }
  if (!err) err = fft_prepare(c);
  if (!err) {
    // full layout if it takes at most 85% of the free device memory, else the lean one
    Carver probe{nullptr};
    carve(c, probe);
    size_t free_b = 0, total_b = 0;
    bool lean = cfg->memory_layout == 2;
    if (cfg->memory_layout == 0)
      lean = cudaMemGetInfo(&free_b, &total_b) == cudaSuccess && (double)probe.off > 0.85 * (double)free_b;
    if (lean) {
      c.pw_n = PW_LEAN;
      c.tbuf_n = TBUF_LEAN;
      probe = Carver{nullptr};
      carve(c, probe);
    }
    c.arena_bytes = probe.off;
    if (cudaMalloc(&c.arena, c.arena_bytes) != cudaSuccess) {
      cudaGetLastError();
      err = LMVD_ERR_OOM;
    } else {
      cudaMemsetAsync(c.arena, 0, c.arena_bytes, c.stream);
      Carver real{(char*)c.arena};
      carve(c, real);
    }
  }
  if (!err && !(err = device_alloc(c, (void**)&c.dflags, sizeof(unsigned))))
    cudaMemsetAsync(c.dflags, 0, sizeof(unsigned), c.stream);
  if (!err && cudaStreamSynchronize(c.stream) != cudaSuccess) err = LMVD_ERR_CUDA;
  if (err) {
    lmvd_destroy(h);
    return err;
  }
  *out = h;
  return LMVD_OK;
}

void lmvd_destroy(lmvd_ctx* h) {
  if (!h) return;
  Ctx& c = h->c;
  if (c.stream) cudaStreamSynchronize(c.stream);
  else cudaDeviceSynchronize();
  adj_destroy(c);
  graphs_clear(c);
  for (auto& p : c.prof.pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (cudaEvent_t e : c.prof.pool) cudaEventDestroy(e);
  for (void* p : c.small_allocs) cudaFree(p);
  if (c.arena) cudaFree(c.arena);
  delete h;
}

size_t lmvd_history_bytes(const lmvd_ctx* h) {
  if (!h) return 0;
  const Grid& g = h->c.g;
  return 16 + sizeof(cd) * g.M * ((size_t)6 * g.ny + 1) + sizeof(double) * 2 * g.ny;
}

int lmvd_set_state(lmvd_ctx* h, const void* z, const void* om, const void* m2, const double* mm1, const double* mm3,
                   const void* history) {
  if (!h || !z || !om || !m2 || !mm1 || !mm3) return LMVD_ERR_INVALID_ARG;
  Ctx& c = h->c;
  const Grid& g = c.g;
  const size_t S = sizeof(cd) * g.ny * g.M, Sp = sizeof(cd) * (g.ny + 1) * g.M, R = sizeof(double) * g.ny;
  int e = copy_in(c, c.z, z, S);
  if (!e) e = copy_in(c, c.om, om, S);
  if (!e) e = copy_in(c, c.m2, m2, Sp);
  if (!e) e = copy_in(c, c.mm1, mm1, R);
  if (!e) e = copy_in(c, c.mm3, mm3, R);
  if (e) return latch(c, e);
  LMVD_LAUNCH(c, KC_MISC, 0, S, k_sanitize, elem_blocks(g.ny * g.M), 256, 0, g, g.ny, c.z, 0);
  LMVD_LAUNCH(c, KC_MISC, 0, S, k_sanitize, elem_blocks(g.ny * g.M), 256, 0, g, g.ny, c.om, 1);
  LMVD_LAUNCH(c, KC_MISC, 0, Sp, k_sanitize, elem_blocks((g.ny + 1) * g.M), 256, 0, g, g.ny + 1, c.m2, 1);
  if (!history) {
    startup(c);
    return cuda_check(c);
  }
  const char* hb = (const char*)history;
  long long s = 0;
  // the counter is read in the context's stream order (the caller may have written the blob on that
  // stream an instant ago; a plain cudaMemcpy runs on the legacy stream, which does not wait for it)
  if (cudaMemcpyAsync(&s, hb, sizeof(s), cudaMemcpyDefault, c.stream) != cudaSuccess ||
      cudaStreamSynchronize(c.stream) != cudaSuccess)
    return latch(c, LMVD_ERR_CUDA);
  if (s < 0) return LMVD_ERR_INVALID_ARG;
  size_t off = 16;
  for (int q = 0; q < 3 && !e; ++q, off += S) e = copy_in(c, c.zh[q], hb + off, S);
  if (!e) { e = copy_in(c, c.zdot_prev, hb + off, S); off += S; }
  if (!e) { e = copy_in(c, c.r_om_prev, hb + off, S); off += S; }
  if (!e) { e = copy_in(c, c.r_phi_prev, hb + off, Sp); off += Sp; }
  if (!e) e = copy_in(c, c.r_m_prev, hb + off, 2 * R);
  if (e) return latch(c, e);
  c.s = (int)s;
  return cuda_check(c);
}

int lmvd_get_state(lmvd_ctx* h, void* z, void* om, void* m2, double* mm1, double* mm3, void* history) {
  if (!h) return LMVD_ERR_INVALID_ARG;
  Ctx& c = h->c;
  const Grid& g = c.g;
  const size_t S = sizeof(cd) * g.ny * g.M, Sp = sizeof(cd) * (g.ny + 1) * g.M, R = sizeof(double) * g.ny;
  int e = LMVD_OK;
  if (z && !e) e = copy_in(c, z, c.z, S);
  if (om && !e) e = copy_in(c, om, c.om, S);
  if (m2 && !e) e = copy_in(c, m2, c.m2, Sp);
  if (mm1 && !e) e = copy_in(c, mm1, c.mm1, R);
  if (mm3 && !e) e = copy_in(c, mm3, c.mm3, R);
  if (history && !e) {
    char* hb = (char*)history;
    h->s_blob = c.s;
    e = copy_in(c, hb, &h->s_blob, sizeof(long long));
    size_t off = 16;
    for (int q = 0; q < 3 && !e; ++q, off += S) e = copy_in(c, hb + off, c.zh[q], S);
    if (!e) { e = copy_in(c, hb + off, c.zdot_prev, S); off += S; }
    if (!e) { e = copy_in(c, hb + off, c.r_om_prev, S); off += S; }
    if (!e) { e = copy_in(c, hb + off, c.r_phi_prev, Sp); off += Sp; }
    if (!e) e = copy_in(c, hb + off, c.r_m_prev, 2 * R);
  }
  return e ? latch(c, e) : LMVD_OK;
}

int lmvd_advance_substage(lmvd_ctx* h) {
  if (!h) return LMVD_ERR_INVALID_ARG;
  return advance_impl(h->c, nullptr);
}

int lmvd_step(lmvd_ctx* h, int nsteps) {
  if (!h || nsteps < 0) return LMVD_ERR_INVALID_ARG;
  for (int i = 0; i < 2 * nsteps; ++i) {
    int e = advance_impl(h->c, nullptr);
    if (e) return e;
  }
  return LMVD_OK;
}

int lmvd_graphs_enable(lmvd_ctx* h, int on) {
  if (!h) return LMVD_ERR_INVALID_ARG;
  Ctx& c = h->c;
  c.graphs_on = on != 0;
  if (!c.graphs_on) graphs_clear(c);
  return LMVD_OK;
}

int lmvd_graph_count(const lmvd_ctx* h) { return h ? (int)h->c.graphs.size() : -1; }

size_t lmvd_field_bytes(const lmvd_ctx* h, int which) {
  if (!h) return 0;
  const Grid& g = h->c.g;
  switch (which) {
    case LMVD_FIELD_MC2:
    case LMVD_FIELD_R_PHI2: return sizeof(cd) * (g.ny + 1) * g.M;
    case LMVD_FIELD_R_MEANS: return sizeof(double) * 2 * g.ny;
    case LMVD_FIELD_RZ:
    case LMVD_FIELD_ZDOT:
    case LMVD_FIELD_RHO_T:
    case LMVD_FIELD_MC1:
    case LMVD_FIELD_MC3:
    case LMVD_FIELD_R_OMEGA2: return sizeof(cd) * g.ny * g.M;
    default: return 0;
  }
}

int lmvd_get_field(lmvd_ctx* h, int which, void* out) {
  if (!h || !out) return LMVD_ERR_INVALID_ARG;
  Ctx& c = h->c;
  const void* src = nullptr;
  switch (which) {
    case LMVD_FIELD_RZ: src = c.Rz; break;
    case LMVD_FIELD_ZDOT: src = c.s > 0 ? c.zdot_prev : c.zdot; break;
    case LMVD_FIELD_RHO_T: src = c.rt; break;
    case LMVD_FIELD_MC1: src = c.m1c; break;
    case LMVD_FIELD_MC2: src = c.m2c; break;
    case LMVD_FIELD_MC3: src = c.m3c; break;
    case LMVD_FIELD_R_OMEGA2: src = c.r_om_prev; break;
    case LMVD_FIELD_R_PHI2: src = c.r_phi_prev; break;
    case LMVD_FIELD_R_MEANS: src = c.r_m_prev; break;
    default: return LMVD_ERR_INVALID_ARG;
  }
  int e = copy_in(c, out, src, lmvd_field_bytes(h, which));
  return e ? latch(c, e) : LMVD_OK;
}

int lmvd_inverse_transform(lmvd_ctx* h, const void* spec, double* phys, int nfields) {
  // spec is read by TMA tile copies, which need 16-byte alignment (any complex128 element boundary)
  if (!h || !spec || !phys || nfields < 0 || ((uintptr_t)spec & 15)) return LMVD_ERR_INVALID_ARG;
  Ctx& c = h->c;
  const size_t S = (size_t)c.g.ny * c.g.M, P = (size_t)c.g.ny * c.g.P;
  for (int f0 = 0; f0 < nfields; f0 += 10) {
    const int n = std::min(10, nfields - f0);
    cd* in[10];
    double* out[10];
    for (int f = 0; f < n; ++f) {
      in[f] = (cd*)spec + (size_t)(f0 + f) * S;
      out[f] = phys + (size_t)(f0 + f) * P;
    }
    fft_inverse_as(c, in, out, n, 0);
  }
  return cuda_check(c);
}

int lmvd_forward_transform(lmvd_ctx* h, const double* phys, void* spec, int nfields) {
  if (!h || !spec || !phys || nfields < 0) return LMVD_ERR_INVALID_ARG;
  Ctx& c = h->c;
  const size_t S = (size_t)c.g.ny * c.g.M, P = (size_t)c.g.ny * c.g.P;
  for (int f0 = 0; f0 < nfields; f0 += 10) {
    const int n = std::min(10, nfields - f0);
    double* in[10];
    cd* out[10];
    for (int f = 0; f < n; ++f) {
      in[f] = (double*)phys + (size_t)(f0 + f) * P;
      out[f] = (cd*)spec + (size_t)(f0 + f) * S;
    }
    fft_forward_as(c, in, out, n, 0);
  }
  return cuda_check(c);
}

size_t lmvd_state_bytes(const lmvd_ctx* h) {
  if (!h) return 0;
  const Grid& g = h->c.g;
  return sizeof(cd) * g.M * ((size_t)3 * g.ny + 1) + sizeof(double) * 2 * g.ny;
}

int lmvd_adjoint_substage(lmvd_ctx* h, const void* sbar_out, const void* hbar_out, void* sbar_in, void* hbar_in) {
  if (!h || !sbar_out || !hbar_out || !sbar_in || !hbar_in) return LMVD_ERR_INVALID_ARG;
  const int e = adjoint_substage(h->c, sbar_out, hbar_out, sbar_in, hbar_in);
  return e ? latch(h->c, e) : LMVD_OK;
}

int lmvd_adjoint_startup(lmvd_ctx* h, const void* sbar_out, const void* hbar_out, void* sbar_in) {
  if (!h || !sbar_out || !hbar_out || !sbar_in) return LMVD_ERR_INVALID_ARG;
  const int e = adjoint_startup(h->c, sbar_out, hbar_out, sbar_in);
  return e ? latch(h->c, e) : LMVD_OK;
}

size_t lmvd_device_bytes(const lmvd_ctx* h) {
  if (!h) return 0;
  const Ctx& c = h->c;
  return c.arena_bytes + c.small_bytes + adj_device_bytes(c);
}

int lmvd_substage_index(const lmvd_ctx* h) { return h ? h->c.s : -1; }

int lmvd_synchronize(lmvd_ctx* h) {
  if (!h) return LMVD_ERR_INVALID_ARG;
  Ctx& c = h->c;
  if (cudaStreamSynchronize(c.stream) != cudaSuccess) return latch(c, LMVD_ERR_CUDA);
  cuda_check(c);
  unsigned flags = 0;
  if (c.dflags && cudaMemcpy(&flags, c.dflags, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess)
    return latch(c, LMVD_ERR_CUDA);
  if (flags & 1u) latch(c, LMVD_ERR_NONFINITE);
  if (flags & 2u) latch(c, LMVD_ERR_FP_DIVERGED);
  if (flags & 4u) latch(c, LMVD_ERR_CUDA);  // a z-pass tile copy did not complete within its time limit
  if (kCheckedBuild && (oob_take_api() | oob_take_fft() | oob_take_yk() | oob_take_pw() | oob_take_adj()))
    latch(c, LMVD_ERR_OUT_OF_BOUNDS);
  return c.status;
}

int lmvd_checked_build(void) { return kCheckedBuild ? 1 : 0; }

int lmvd_diagnostics_enable(lmvd_ctx* h, int on) {
  if (!h) return LMVD_ERR_INVALID_ARG;
  Ctx& c = h->c;
  if (on && !c.ddiag) {
    const int e = device_alloc(c, (void**)&c.ddiag, sizeof(double) * DIAG_N);
    if (e) return latch(c, e);
    cudaMemsetAsync(c.ddiag, 0, sizeof(double) * DIAG_N, c.stream);
  }
  c.diag_on = on != 0;
  return LMVD_OK;
}

int lmvd_diagnostics(lmvd_ctx* h, double* out, int n) {
  if (!h || !out || n < 0) return LMVD_ERR_INVALID_ARG;
  Ctx& c = h->c;
  if (!c.ddiag) return LMVD_ERR_INVALID_ARG;
  double rec[DIAG_N];
  if (cudaStreamSynchronize(c.stream) != cudaSuccess ||
      cudaMemcpy(rec, c.ddiag, sizeof(rec), cudaMemcpyDeviceToHost) != cudaSuccess)
    return latch(c, LMVD_ERR_CUDA);
  const int kf = std::min(c.cfg.kf, KF_MAX_ADJ + 1);
  const int total = 5 + kf;
  double vals[5 + KF_MAX_ADJ + 1];
  vals[0] = c.s - 1;
  vals[1] = rec[1] > 0 ? std::sqrt(rec[0] / rec[1]) : 0.0;
  for (int k = 0; k < kf; ++k) vals[2 + k] = rec[3 + 2 * k] > 0 ? std::sqrt(rec[2 + 2 * k] / rec[3 + 2 * k]) : 0.0;
  vals[2 + kf] = rec[DIAG_KE] * c.cfg.lx * c.cfg.lz;
  vals[3 + kf] = std::sqrt(rec[DIAG_MMAX]);
  vals[4 + kf] = rec[DIAG_MC2];
  for (int q = 0; q < std::min(n, total); ++q) out[q] = vals[q];
  return total;
}

int lmvd_status(const lmvd_ctx* h) { return h ? h->c.status : LMVD_ERR_INVALID_ARG; }

int lmvd_profile_enable(lmvd_ctx* h, int on) {
  if (!h) return LMVD_ERR_INVALID_ARG;
  Ctx& c = h->c;
  if (cudaStreamSynchronize(c.stream) != cudaSuccess) return latch(c, LMVD_ERR_CUDA);
  prof_collect(c);
  for (int k = 0; k < KC_COUNT; ++k) c.prof.n[k] = 0, c.prof.flops[k] = c.prof.bytes[k] = c.prof.ms[k] = 0.0;
  c.prof.on = on != 0;
  return LMVD_OK;
}

int lmvd_profile_read(lmvd_ctx* h, int cls, double* out4) {
  if (!h || !out4 || cls < 0 || cls >= KC_COUNT) return LMVD_ERR_INVALID_ARG;
  Ctx& c = h->c;
  if (cudaStreamSynchronize(c.stream) != cudaSuccess) return latch(c, LMVD_ERR_CUDA);
  prof_collect(c);
  out4[0] = c.prof.ms[cls];
  out4[1] = (double)c.prof.n[cls];
  out4[2] = c.prof.flops[cls];
  out4[3] = c.prof.bytes[cls];
  return LMVD_OK;
}

const char* lmvd_kernel_class_name(int cls) {
  static const char* names[KC_COUNT] = {"fft_z_inverse", "fft_x_inverse", "fft_x_forward", "fft_z_forward",
                                        "eval_pass1",    "eval",          "solve_collocation", "solve_mc",
                                        "rhs_combine",   "rhs_eval",      "rk_update",     "products",
                                        "misc"};
  return (cls >= 0 && cls < KC_COUNT) ? names[cls] : "unknown";
}

long long lmvd_kernel_launches(const lmvd_ctx* h) { return h ? h->c.prof.launches : -1; }

const char* lmvd_strerror(int code) {
  switch (code) {
    case LMVD_OK: return "ok";
    case LMVD_ERR_INVALID_ARG: return "invalid argument";
    case LMVD_ERR_CUDA: return "CUDA error";
    case LMVD_ERR_OOM: return "device out of memory";
    case LMVD_ERR_NONFINITE: return "non-finite value in the state";
    case LMVD_ERR_FP_DIVERGED: return "fixed-point iteration did not converge";
    case LMVD_ERR_OUT_OF_BOUNDS: return "index out of bounds (checked build)";
    case LMVD_ERR_UNSUPPORTED: return "unsupported configuration";
    default: return "unknown error";
  }
}

}  // extern "C"
