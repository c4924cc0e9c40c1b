// Adjoint (vector-Jacobian product) of one substage of Algorithm 2, FP64.
//
// The substage maps x = (state, history) to y = (state', history'). Given ybar, the adjoint computes
// xbar = J(x)^T ybar with respect to the real inner products sum Re(conj(a) b) over every stored
// spectral entry and sum a b over real arrays. Every linear step is transposed exactly:
//  * synthesis G (3/2-padded inverse transform) and analysis F have G^T = (px pz) W F and
//    F^T = G W^{-1} / (px pz), W = 1 on kx = 0 and 2 on kx > 0 (the half-spectrum carries each
//    kx > 0 mode for itself and its conjugate partner);
//  * banded evaluations B are applied as B^T with transposed band matrices;
//  * band solves A^{-1} are applied as A^{-T} with A's own LU factors (A^T = U^T L^T);
//  * per-mode complex multipliers c become conj(c).
// The pointwise products (Sec. 2.1, 4.3, Eq. om / phi, the EOS of Sec. 5) are differentiated
// analytically at the physical fields the forward substage recorded on its tape.
// Paper passages of each step: see the forward kernels (ykernels.cu, pointwise.cu, api.cu).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <stdexcept>

#include "band.cuh"
#include "basis.h"
#include "ykernels.h"

namespace lmvd {

LMVD_DEFINE_OOB_TAKE(adj)

struct AdjWork {
  void* arena = nullptr;
  size_t bytes = 0;
  std::vector<void*> small;
  DBand B0gT, B1gT, B2gT, BsT[4], Sg0T, Sg1T, Ss0T, Ss2T;
  Tape tape;
  // adjoints of the substage outputs (inputs of the reverse pass)
  cd *oz, *oom, *om2, *ozh[3], *ozdp, *orom, *orphi;
  double *omm1, *omm3, *orm;
  // adjoints of the substage inputs (results)
  cd *z, *om, *m2, *zh[3], *zdp, *romp, *rphip;
  double *mm1, *mm3, *rmp;
  // work
  cd *zd, *rz, *rt, *mc[3], *rom, *rphi, *sv[10], *st[7], *tS, *tSp;
  double* rm;
  double *fp, *w[3], *ir, *rho, *md[3], *pb[10];
  // dz/dt before each start-up application (allocated on the first lmvd_adjoint_startup)
  cd* iterates = nullptr;
  int n_iterates = 0;
  size_t small_bytes = 0;  // bytes of small
};

namespace {

constexpr int TPB = 128;
unsigned mblocks(const Grid& g) { return (unsigned)((g.M + TPB - 1) / TPB); }
unsigned eblocks(size_t n) { return (unsigned)std::min<size_t>((n + 255) / 256, 152 * 32); }

struct FieldsW10 {
  cd* p[10];
};
struct Fields3R {
  double* p[3];
};
struct Fields3RC {
  const double* p[3];
};
struct Fields5RC {
  const double* p[5];
};
struct Fields10R {
  double* p[10];
};

// ------------------------------------------------------------------ elementwise helpers
// f[o] *= (kx == 0 ? s0 : s1); Nyquist slots set to zero. blockIdx.y selects the field.
__global__ void k_wscale(Grid g, FieldsW10 f, double s0, double s1) {
  cd* x = pick(f.p, (int)blockIdx.y);
  const size_t n = (size_t)g.ny * g.M;
  for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
    const int m = (int)(o % g.M);
    x[o] = is_nyquist(g, m) ? mk(0, 0) : ((m % g.nxh) == 0 ? s0 : s1) * x[o];
  }
}

// out = A^{-T} in for job blockIdx.y, shared or per-mode factors; rows of the result outside [zlo, zhi]
// are zero (boundary rows whose forward right-hand side is a constant). out may alias in. Nyquist modes
// are set to zero. k_solve_T_cd: one thread per mode; k_solve_T_re: one thread per (mode, real part).
struct SolveTJob {
  const cd* in;
  cd* out;
  int zlo, zhi;
};
struct SolveTJobs {
  SolveTJob j[8];
};
template <class V>
__device__ void solve_T_job(const Grid& g, const DLU& lu, const SolveTJob& jb) {
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
  band_solve_T_v<V>(lu, m, lu.mstride ? factor_mode(g, m) : 0, comp, reinterpret_cast<const V*>(jb.in), out, M,
                    jb.zlo, jb.zhi);
}
__global__ void k_solve_T_cd(Grid g, DLU lu, SolveTJobs jobs) { solve_T_job<cd>(g, lu, jobs.j[blockIdx.y]); }
__global__ void k_solve_T_re(Grid g, DLU lu, SolveTJobs jobs) { solve_T_job<double>(g, lu, jobs.j[blockIdx.y]); }

// ------------------------------------------------------------------ update (step 6) adjoint
struct AdjUpd {
  double dt, al, be;
  const cd *oom, *oz, *om2;
  const double *omm1, *omm3;
  cd *om, *rom, *romp, *z, *zd, *zdp, *m2, *rphi, *rphip;
  double *mm1, *mm3, *rm, *rmp;
  cd *scr0, *scr1;  // ny rows each
  cd* scrp;         // ny + 1 rows
};

// After the transposed solves v = A^{-T} ybar (boundary rows zero; scr0 for Omega2 with the interpolation
// LU, scr1 for z with the Neumann LU): transposed evaluation and the RK coefficients. Rows split over
// gridDim.y chunks, job blockIdx.z (0: Omega2, 1: z).
__global__ void k_adj_update_om_z_post(Grid g, DBand B0gT, AdjUpd a) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= (int)g.M || is_nyquist(g, m)) return;
  const size_t M = g.M;
  const int job = blockIdx.z;
  if (job == 0 && m == 0) return;  // Omega2 has no k = 0 mode
  const cd* v = job == 0 ? a.scr0 : a.scr1;
  int r0, r1;
  row_range(g.ny, blockIdx.y, gridDim.y, r0, r1);
  for (int j = r0; j < r1; ++j) {
    const size_t o = (size_t)j * M + m;
    const cd t = band_row(B0gT, j, v, M, m);
    if (job == 0) {
      a.om[o] = a.om[o] + t;
      a.rom[o] = a.rom[o] + (a.dt * a.al) * v[o];
      a.romp[o] = a.romp[o] + (a.dt * a.be) * v[o];
    } else {
      a.z[o] = a.z[o] + t;
      a.zd[o] = a.zd[o] + (a.dt * a.al) * t;
      a.zdp[o] = a.zdp[o] + (a.dt * a.be) * t;
    }
  }
}
__global__ void k_adj_update_means(Grid g, DBand B0gT, DLU lu, AdjUpd a) {
  const int c = threadIdx.x;
  if (c > 1) return;
  const int ny = g.ny;
  const double* yb = c == 0 ? a.omm1 : a.omm3;
  double* mmb = c == 0 ? a.mm1 : a.mm3;
  double* v = reinterpret_cast<double*>(c == 0 ? a.scr0 : a.scr1);  // ny doubles of scratch
  double win[KMAX];
  for (int q = 0; q < KMAX; ++q) win[q] = 0.0;
  for (int i = 0; i < ny; ++i) {  // U^T sweep
    double x = yb[i];
    for (int r = 1; r <= lu.K; ++r)
      if (i - r >= 0) x -= lu_up(lu, i - r, r, 0) * win[r - 1];
    x *= lu.invd[i];
    for (int q = KMAX - 1; q > 0; --q) win[q] = win[q - 1];
    win[0] = x;
    v[i] = x;
  }
  for (int q = 0; q < KMAX; ++q) win[q] = 0.0;
  for (int i = ny - 1; i >= 0; --i) {  // L^T sweep
    double x = v[i];
    for (int q = 1; q <= lu.K; ++q)
      if (i + q < ny) x -= lu_lo(lu, i + q, q, 0) * win[q - 1];
    for (int q = KMAX - 1; q > 0; --q) win[q] = win[q - 1];
    win[0] = x;
    v[i] = x;
  }
  v[0] = 0.0;
  v[ny - 1] = 0.0;
  for (int j = 0; j < ny; ++j) {
    double t = 0.0;
    for (int q = 0; q < B0gT.w; ++q) t += B0gT.v[(size_t)j * B0gT.w + q] * v[B0gT.c0[j] + q];
    mmb[j] += t;
    a.rm[c * ny + j] += a.dt * a.al * v[j];
    a.rmp[c * ny + j] += a.dt * a.be * v[j];
  }
}

// After v = A^{-T} m2^d-bar (per-mode factors, rows < 2 and > ny - 2 zero) in scrp: transposed phi2
// evaluation and the RK coefficients. Rows 0..ny split over gridDim.y chunks.
__global__ void k_adj_update_m2_post(Grid g, DBand Ss0T, DBand Ss2T, AdjUpd a) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= (int)g.M || m == 0 || is_nyquist(g, m)) return;
  const size_t M = g.M;
  double k1, k3;
  wavenumbers(g, m, k1, k3);
  const double k2 = k1 * k1 + k3 * k3;
  const cd* v = a.scrp;
  int r0, r1;
  row_range(g.ny + 1, blockIdx.y, gridDim.y, r0, r1);
  for (int j = r0; j < r1; ++j) {
    const size_t o = (size_t)j * M + m;
    a.m2[o] = a.m2[o] + band_row(Ss2T, j, v, M, m) - k2 * band_row(Ss0T, j, v, M, m);
    a.rphi[o] = a.rphi[o] + (a.dt * a.al) * v[o];
    a.rphip[o] = a.rphip[o] + (a.dt * a.be) * v[o];
  }
}

// ------------------------------------------------------------------ RHS (step 5) adjoint
struct St7 {
  cd* p[7];
};
struct Sv10C {
  const cd* p[10];
};

__global__ void k_adj_rhs_eval(Grid g, DBand B1gT, DBand B2gT, DBand Bs0T, DBand Bs1T, DBand Bs2T, DBand Bs3T,
                               const cd* rom, const cd* rphi, const double* rm, St7 st) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= (int)g.M) return;
  const size_t M = g.M;
  const int ny = g.ny;
  for (int q = 0; q < 7; ++q)
    for (int i = 0; i < ny; ++i) st.p[q][(size_t)i * M + m] = mk(0, 0);
  if (is_nyquist(g, m)) return;
  if (m == 0) {
    const double* r1 = rm;
    const double* r3 = rm + ny;
    for (int j = 0; j < ny; ++j) {
      const size_t o = (size_t)j * M;
      st.p[1][o] = mk(band_row_real(B1gT, j, r1), 0.0);
      st.p[2][o] = mk(band_row_real(B2gT, j, r1), 0.0);
      st.p[4][o] = mk(band_row_real(B1gT, j, r3), 0.0);
      st.p[5][o] = mk(band_row_real(B2gT, j, r3), 0.0);
    }
    return;
  }
  for (int j = 0; j < ny; ++j) {
    const size_t o = (size_t)j * M + m;
    st.p[0][o] = rom[o];
    st.p[1][o] = band_row(B1gT, j, rom, M, m);
    st.p[2][o] = band_row(B2gT, j, rom, M, m);
    st.p[3][o] = band_row(Bs0T, j, rphi, M, m);
    st.p[4][o] = band_row(Bs1T, j, rphi, M, m);
    st.p[5][o] = band_row(Bs2T, j, rphi, M, m);
    st.p[6][o] = band_row(Bs3T, j, rphi, M, m);
  }
}

// conj-transpose of the per-mode stream combination of k_rhs_combine
__global__ void k_adj_rhs_combine(Grid g, double mu, double grav, St7 stb, FieldsW10 svb) {
  const size_t n = (size_t)g.ny * g.M;
  for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
    const int m = (int)(o % g.M);
    cd r[10];
    for (int q = 0; q < 10; ++q) r[q] = mk(0, 0);
    if (!is_nyquist(g, m)) {
      const cd s0 = stb.p[0][o], s1 = stb.p[1][o], s2 = stb.p[2][o], s3 = stb.p[3][o], s4 = stb.p[4][o],
               s5 = stb.p[5][o], s6 = stb.p[6][o];
      if (m == 0) {
        r[1] = s1;
        r[6] = mu * s2;
        r[4] = s4;
        r[8] = mu * s5;
      } else {
        double k1, k3;
        wavenumbers(g, m, k1, k3);
        const double k2 = k1 * k1 + k3 * k3;
        r[0] = (-k1 * k3) * s0 + (k1 * k1) * s4;                                          // C11
        r[1] = times_i(k2 * k1 * s3 - k3 * s1 + k1 * s5);                                 // C12
        r[2] = (k1 * k1 - k3 * k3) * s0 + (2.0 * k1 * k3) * s4;                           // C13
        r[3] = (-k2) * s4;                                                                // C22
        r[4] = times_i(k1 * s1 + k2 * k3 * s3 + k3 * s5);                                 // C23
        r[5] = (k1 * k3) * s0 + (k3 * k3) * s4;                                           // C33
        r[6] = times_i((mu * k2 * k3) * s0 - (mu * k3) * s2 - (mu * k2 * k1) * s4 + (mu * k1) * s6);   // u1
        r[7] = (mu * k2 * k2) * s3 - (mu * k2) * s5;                                      // u2
        r[8] = times_i((-mu * k2 * k1) * s0 + (mu * k1) * s2 - (mu * k2 * k3) * s4 + (mu * k3) * s6);  // u3
        r[9] = (k2 * grav) * s3;                                                          // rho
      }
    }
    for (int q = 0; q < 10; ++q) svb.p[q][o] = r[q];
  }
}

// ------------------------------------------------------------------ product adjoints (physical space)
// pass 2: C_ij = -m_i m_j / rho, u_i = m_i / rho (1/rho = ir), rho copied; m = m^d + m^c.
// In: pb[0..9] = adjoints of C11, C12, C13, C22, C23, C33, u1, u2, u3, rho. Out: pb[0..2] = adjoint of m
// (that is, of m^c); accumulates the adjoints of m^d, 1/rho, rho.
__global__ void k_adj_p2(size_t n, Fields10R pb, Fields3RC md, Fields3RC b, const double* ir, Fields3R mdb, double* irb,
                         double* rhob) {
  for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
    const double c11 = pb.p[0][o], c12 = pb.p[1][o], c13 = pb.p[2][o], c22 = pb.p[3][o], c23 = pb.p[4][o],
                 c33 = pb.p[5][o], u1 = pb.p[6][o], u2 = pb.p[7][o], u3 = pb.p[8][o], rb = pb.p[9][o];
    const double r = ir[o];
    const double m1 = md.p[0][o] + b.p[0][o], m2 = md.p[1][o] + b.p[1][o], m3 = md.p[2][o] + b.p[2][o];
    const double g1 = r * (u1 - (2.0 * m1 * c11 + m2 * c12 + m3 * c13));
    const double g2 = r * (u2 - (m1 * c12 + 2.0 * m2 * c22 + m3 * c23));
    const double g3 = r * (u3 - (m1 * c13 + m2 * c23 + 2.0 * m3 * c33));
    irb[o] += (m1 * u1 + m2 * u2 + m3 * u3) -
              (m1 * m1 * c11 + m1 * m2 * c12 + m1 * m3 * c13 + m2 * m2 * c22 + m2 * m3 * c23 + m3 * m3 * c33);
    rhob[o] += rb;
    mdb.p[0][o] += g1;
    mdb.p[1][o] += g2;
    mdb.p[2][o] += g3;
    pb.p[0][o] = g1;
    pb.p[1][o] = g2;
    pb.p[2][o] = g3;
  }
}

// rho_t = f' a: abar = f' rtbar, f'bar += a rtbar
__global__ void k_adj_rt(size_t n, const double* fp, const double* a, const double* rtb, double* ab, double* fpb) {
  for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
    const double t = rtb[o];
    fpb[o] += a[o] * t;
    ab[o] = fp[o] * t;
  }
}

// l = -(w . b): bbar_i = -w_i lbar, wbar_i += -b_i lbar
__global__ void k_adj_L(size_t n, Fields3RC w, Fields3RC b, const double* lb, Fields3R bb, Fields3R wb) {
  for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
    const double t = lb[o];
    for (int i = 0; i < 3; ++i) {
      wb.p[i][o] -= b.p[i][o] * t;
      bb.p[i][o] = -w.p[i][o] * t;
    }
  }
}

// pass 1: ir = (rh - drho z) irlrh, rho = 1/ir, f' = rho^2 drho irlrh, w = (zx, zy, zz) ir,
// R_z = (kappa lap - m^d . (zx, zy, zz)) ir. Out pb[0..7] = adjoints of z, zx, zz, zy, lap, m1d, m2d, m3d.
__global__ void k_adj_p1(size_t n, EosArgs e, Fields5RC zp, Fields3RC md, const double* rho, const double* ir,
                         const double* rhob, const double* irb, const double* fpb, Fields3RC wb, const double* rzb,
                         Fields3RC mdb, Fields10R pb) {
  const double irlrh = 1.0 / (e.rl * e.rh);
  const double drho = e.rh - e.rl;
  for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
    const double zx = zp.p[1][o], zz = zp.p[2][o], zy = zp.p[3][o], lap = zp.p[4][o];
    const double m1 = md.p[0][o], m2 = md.p[1][o], m3 = md.p[2][o];
    const double r = ir[o], rh = rho[o], R = rzb[o];
    const double adv = m1 * zx + m2 * zy + m3 * zz;
    const double irt = irb[o] + wb.p[0][o] * zx + wb.p[1][o] * zy + wb.p[2][o] * zz + R * (e.kappa * lap - adv) -
                       rhob[o] * rh * rh - fpb[o] * 2.0 * rh * rh * rh * drho * irlrh;
    pb.p[0][o] = -irt * drho * irlrh;                    // z
    pb.p[1][o] = (wb.p[0][o] - R * m1) * r;              // dz/dx
    pb.p[2][o] = (wb.p[2][o] - R * m3) * r;              // dz/dz
    pb.p[3][o] = (wb.p[1][o] - R * m2) * r;              // dz/dy
    pb.p[4][o] = R * r * e.kappa;                        // lap z
    pb.p[5][o] = mdb.p[0][o] - R * r * zx;               // m1^d
    pb.p[6][o] = mdb.p[1][o] - R * r * zy;               // m2^d
    pb.p[7][o] = mdb.p[2][o] - R * r * zz;               // m3^d
  }
}

// ------------------------------------------------------------------ spectral adjoints of pass 1 and m^c
struct Sv8C {
  const cd* p[8];
};

// transpose of k_eval_p1: accumulates into zbar, ombar, m2bar and the means
__global__ void k_adj_eval_p1(Grid g, DBand B0gT, DBand B1gT, DBand B2gT, DBand Sg0T, DBand Sg1T, Sv8C v, cd* zb,
                              cd* omb, cd* m2b, double* mm1b, double* mm3b) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= (int)g.M || is_nyquist(g, m)) return;
  const size_t M = g.M;
  const int ny = g.ny;
  double k1, k3;
  wavenumbers(g, m, k1, k3);
  const double k2 = k1 * k1 + k3 * k3;
  const double ik2 = m == 0 ? 0.0 : 1.0 / k2;
  auto at = [&](int f, int i) { return v.p[f][(size_t)i * M + m]; };
  for (int j = 0; j < ny; ++j) {
    cd acc = mk(0, 0);
    for (int q = 0; q < B0gT.w; ++q) {
      const int i = B0gT.c0[j] + q;
      const cd t0 = at(0, i) - times_i(k1 * at(1, i) + k3 * at(2, i)) - k2 * at(4, i);
      acc = acc + __ldg(B0gT.v + (size_t)j * B0gT.w + q) * t0;
    }
    acc = acc + band_row(B1gT, j, v.p[3], M, m) + band_row(B2gT, j, v.p[4], M, m);
    zb[(size_t)j * M + m] = zb[(size_t)j * M + m] + acc;
    if (m == 0) {
      double a1 = 0.0, a3 = 0.0;
      for (int q = 0; q < B0gT.w; ++q) {
        const int i = B0gT.c0[j] + q;
        const double bv = __ldg(B0gT.v + (size_t)j * B0gT.w + q);
        a1 += bv * at(5, i).re;
        a3 += bv * at(7, i).re;
      }
      mm1b[j] += a1;
      mm3b[j] += a3;
    } else {
      cd ao = mk(0, 0);
      for (int q = 0; q < B0gT.w; ++q) {
        const int i = B0gT.c0[j] + q;
        const cd oi = ik2 * times_i(k3 * at(5, i) - k1 * at(7, i));
        ao = ao + __ldg(B0gT.v + (size_t)j * B0gT.w + q) * oi;
      }
      omb[(size_t)j * M + m] = omb[(size_t)j * M + m] + ao;
    }
  }
  if (m == 0) return;
  for (int j = 0; j <= ny; ++j) {
    cd acc = band_row(Sg0T, j, v.p[6], M, m);
    for (int q = 0; q < Sg1T.w; ++q) {
      const int i = Sg1T.c0[j] + q;
      const cd di = (-ik2) * times_i(k1 * at(5, i) + k3 * at(7, i));
      acc = acc + __ldg(Sg1T.v + (size_t)j * Sg1T.w + q) * di;
    }
    m2b[(size_t)j * M + m] = m2b[(size_t)j * M + m] + acc;
  }
}

// transpose of the m^c computation (k_mc_rhs, banded solve, k_mc_post): (m1^c, m2^c, m3^c) bar -> rho_t bar
// Three launches: k_adj_mc_rhs (right-hand side of the transposed m2^c solve into scr),
// the transposed banded solve (in place, per-mode factors, rows 0 and ny zero), k_adj_mc_post (rtbar).
// q_i = conj(i / k) (k1/k m1bar_i + k3/k m3bar_i) is the adjoint of m_par_i.
__device__ inline cd adj_mc_q(const cd* m1b, const cd* m3b, size_t o, double k1, double k3, double ik) {
  const cd t = (k1 * ik) * m1b[o] + (k3 * ik) * m3b[o];
  return ik * mk(t.im, -t.re);
}

// rows 0..ny split over gridDim.y chunks
__global__ void k_adj_mc_rhs(Grid g, const double* dstar, const cd* m1b, const cd* m2b, const cd* m3b, cd* scr) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= (int)g.M) return;
  const size_t M = g.M;
  const int ny = g.ny;
  int r0, r1;
  row_range(ny + 1, blockIdx.y, gridDim.y, r0, r1);
  if (m == 0 || is_nyquist(g, m)) {
    for (int j = r0; j < r1; ++j) scr[(size_t)j * M + m] = mk(0, 0);
    return;
  }
  double k1, k3;
  wavenumbers(g, m, k1, k3);
  const double ik = 1.0 / sqrt(k1 * k1 + k3 * k3);
  for (int j = r0; j < r1; ++j) {
    cd r = m2b[(size_t)j * M + m];
    if (j >= 1) r = r + __ldg(dstar + j - 1) * adj_mc_q(m1b, m3b, (size_t)(j - 1) * M + m, k1, k3, ik);
    if (j < ny) r = r - __ldg(dstar + j) * adj_mc_q(m1b, m3b, (size_t)j * M + m, k1, k3, ik);
    scr[(size_t)j * M + m] = r;
  }
}

// rows 0..ny-1 split over gridDim.y chunks; the k = 0 mode is one serial pass (chunk 0)
__global__ void k_adj_mc_post(Grid g, DBand Bs1T, const double* dstar, const cd* m1b, const cd* m2b, const cd* m3b,
                              const cd* scr, cd* rtb) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= (int)g.M) return;
  const size_t M = g.M;
  const int ny = g.ny;
  int r0, r1;
  row_range(ny, blockIdx.y, gridDim.y, r0, r1);
  if (is_nyquist(g, m)) {
    for (int i = r0; i < r1; ++i) rtb[(size_t)i * M + m] = mk(0, 0);
    return;
  }
  if (m == 0) {  // m2c_i = sum_{j >= i, j < ny} rt_j / alpha_j
    if (blockIdx.y != 0) return;
    cd s = mk(0, 0);
    for (int j = 0; j < ny; ++j) {
      s = s + m2b[(size_t)j * M];
      rtb[(size_t)j * M] = (1.0 / __ldg(dstar + j)) * s;
    }
    return;
  }
  double k1, k3;
  wavenumbers(g, m, k1, k3);
  const double ik = 1.0 / sqrt(k1 * k1 + k3 * k3);
  for (int i = r0; i < r1; ++i)
    rtb[(size_t)i * M + m] = adj_mc_q(m1b, m3b, (size_t)i * M + m, k1, k3, ik) - band_row(Bs1T, i, scr, M, m);
}

// BDF guess adjoint: zbar += a0/dt zdbar, zh_k bar += a_{k+1}/dt zdbar
__global__ void k_adj_bdf(size_t n, double c0, double c1, double c2, double c3, const cd* zd, cd* z, cd* h0, cd* h1,
                          cd* h2) {
  for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
    const cd t = zd[o];
    z[o] = z[o] + c0 * t;
    h0[o] = h0[o] + c1 * t;
    h1[o] = h1[o] + c2 * t;
    h2[o] = h2[o] + c3 * t;
  }
}

// start-up back-fill zh_q = z - c_q zdot (q = 0, 1, 2), zdot_prev = zdot: z += sum zh_q bar, zdot = zdot_prev bar -
// sum c_q zh_q bar
__global__ void k_adj_backfill(size_t n, double c0, double c1, double c2, const cd* h0, const cd* h1, const cd* h2,
                               const cd* zdp, cd* z, cd* zd) {
  for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
    const cd a = h0[o], b = h1[o], d = h2[o];
    z[o] = z[o] + (a + b + d);
    zd[o] = zdp[o] - (c0 * a + c1 * b + c2 * d);
  }
}

__global__ void k_add(size_t n, cd* y, const cd* x) {
  for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x)
    y[o] = y[o] + x[o];
}

// ------------------------------------------------------------------ host helpers
int adj_upload_band(AdjWork& A, const RowBand& m, DBand& d) {
  int* c0 = nullptr;
  double* v = nullptr;
  if (cudaMalloc(&c0, sizeof(int) * m.c0.size()) != cudaSuccess) return LMVD_ERR_OOM;
  A.small.push_back(c0);
  if (cudaMalloc(&v, sizeof(double) * m.v.size()) != cudaSuccess) return LMVD_ERR_OOM;
  A.small.push_back(v);
  A.small_bytes += sizeof(int) * m.c0.size() + sizeof(double) * m.v.size();
  if (cudaMemcpy(c0, m.c0.data(), sizeof(int) * m.c0.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(v, m.v.data(), sizeof(double) * m.v.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return LMVD_ERR_CUDA;
  d = DBand{c0, v, m.rows, m.w, nullptr, m.cols};
  return LMVD_OK;
}

struct Carve {
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

void adj_carve(const Ctx& c, AdjWork& A, Carve& cv) {
  const Grid& g = c.g;
  const size_t S = (size_t)g.ny * g.M, Sp = (size_t)(g.ny + 1) * g.M, P = (size_t)g.ny * g.P;
  const int ny = g.ny, kf = c.cfg.kf;
  for (auto& p : A.tape.zp) p = cv.take<double>(P);
  for (int k = 0; k <= kf; ++k) {
    A.tape.a[k] = cv.take<double>(P);
    for (auto& p : A.tape.b[k]) p = cv.take<double>(P);
  }
  A.oz = cv.take<cd>(S);
  A.oom = cv.take<cd>(S);
  A.om2 = cv.take<cd>(Sp);
  for (auto& p : A.ozh) p = cv.take<cd>(S);
  A.ozdp = cv.take<cd>(S);
  A.orom = cv.take<cd>(S);
  A.orphi = cv.take<cd>(Sp);
  A.omm1 = cv.take<double>(ny);
  A.omm3 = cv.take<double>(ny);
  A.orm = cv.take<double>(2 * ny);
  A.z = cv.take<cd>(S);
  A.om = cv.take<cd>(S);
  A.m2 = cv.take<cd>(Sp);
  for (auto& p : A.zh) p = cv.take<cd>(S);
  A.zdp = cv.take<cd>(S);
  A.romp = cv.take<cd>(S);
  A.rphip = cv.take<cd>(Sp);
  A.mm1 = cv.take<double>(ny);
  A.mm3 = cv.take<double>(ny);
  A.rmp = cv.take<double>(2 * ny);
  A.zd = cv.take<cd>(S);
  A.rz = cv.take<cd>(S);
  A.rt = cv.take<cd>(S);
  A.mc[0] = cv.take<cd>(S);
  A.mc[1] = cv.take<cd>(Sp);
  A.mc[2] = cv.take<cd>(S);
  A.rom = cv.take<cd>(S);
  A.rphi = cv.take<cd>(Sp);
  for (auto& p : A.sv) p = cv.take<cd>(S);
  for (auto& p : A.st) p = cv.take<cd>(S);
  A.tS = cv.take<cd>(2 * S);
  A.tSp = cv.take<cd>(Sp);
  A.rm = cv.take<double>(2 * ny);
  A.fp = cv.take<double>(P);
  for (auto& p : A.w) p = cv.take<double>(P);
  A.ir = cv.take<double>(P);
  A.rho = cv.take<double>(P);
  for (auto& p : A.md) p = cv.take<double>(P);
  for (auto& p : A.pb) p = cv.take<double>(P);
}

int adj_setup(Ctx& c) {
  if (c.adj) return LMVD_OK;
  AdjWork* A = new (std::nothrow) AdjWork();
  if (!A) return LMVD_ERR_OOM;
  c.adj = A;
  const lmvd_config& f = c.cfg;
  const int p = f.spline_order, ny = f.ny;
  int err = LMVD_OK;
  try {
    Knots kb = clamped_uniform(p, ny, f.y0, f.y1), ks = clamped_uniform(p + 1, ny + 1, f.y0, f.y1);
    std::vector<double> gb = greville(kb), gs = greville(ks);
    err = adj_upload_band(*A, transpose(collocation(kb, gb, 0)), A->B0gT);
    if (!err) err = adj_upload_band(*A, transpose(collocation(kb, gb, 1)), A->B1gT);
    if (!err) err = adj_upload_band(*A, transpose(collocation(kb, gb, 2)), A->B2gT);
    for (int d = 0; d < 4 && !err; ++d) err = adj_upload_band(*A, transpose(collocation(kb, gs, d)), A->BsT[d]);
    if (!err) err = adj_upload_band(*A, transpose(collocation(ks, gb, 0)), A->Sg0T);
    if (!err) err = adj_upload_band(*A, transpose(collocation(ks, gb, 1)), A->Sg1T);
    if (!err) err = adj_upload_band(*A, transpose(collocation(ks, gs, 0)), A->Ss0T);
    if (!err) err = adj_upload_band(*A, transpose(collocation(ks, gs, 2)), A->Ss2T);
  } catch (const std::exception&) {
    err = LMVD_ERR_UNSUPPORTED;
  }
  if (!err) {
    Carve probe{nullptr};
    adj_carve(c, *A, probe);
    A->bytes = probe.off;
    if (cudaMalloc(&A->arena, A->bytes) != cudaSuccess) {
      cudaGetLastError();
      err = LMVD_ERR_OOM;
    } else {
      Carve real{(char*)A->arena};
      adj_carve(c, *A, real);
    }
  }
  return err;
}

// ---- transposes of the transforms: G^T = (px pz) W F, F^T = G W^{-1} / (px pz)
void wscale(Ctx& c, cd* const* f, int nf, double s0, double s1) {
  FieldsW10 w{};
  for (int i = 0; i < nf; ++i) w.p[i] = f[i];
  const size_t n = (size_t)c.g.ny * c.g.M;
  LMVD_LAUNCH(c, KC_MISC, 2.0 * n * nf, 32.0 * n * nf, k_wscale, dim3(eblocks(n), nf), 256, 0, c.g, w, s0, s1);
}
void g_transpose(Ctx& c, double* const* phys, cd* const* spec, int nf) {
  fft_forward_as(c, const_cast<double* const*>(phys), spec, nf, 0);
  const double pp = (double)c.g.px * (double)c.g.pz;
  wscale(c, spec, nf, pp, 2.0 * pp);
}
void f_transpose(Ctx& c, cd* const* spec, double* const* phys, int nf) {  // overwrites spec
  const double pp = (double)c.g.px * (double)c.g.pz;
  wscale(c, spec, nf, 1.0 / pp, 0.5 / pp);
  fft_inverse_as(c, spec, phys, nf, 0);
}
// out = A^{-T} in per job (one launch), boundary rows outside [zlo, zhi] zero
void solve_T_jobs(Ctx& c, KClass cls, const DLU& lu, std::initializer_list<SolveTJob> jobs) {
  SolveTJobs sj{};
  int n = 0;
  for (const SolveTJob& j : jobs) sj.j[n++] = j;
  const double rowsM = (double)lu.n * c.g.M;
  const int tpm = solve_split(c.g);
  const dim3 grid((unsigned)((tpm * c.g.M + TPB - 1) / TPB), n);
  if (tpm == 2)
    LMVD_LAUNCH(c, cls, n * lu.flops_per_mode * c.g.M, 32.0 * rowsM * n, k_solve_T_re, grid, TPB, 0, c.g, lu, sj);
  else
    LMVD_LAUNCH(c, cls, n * lu.flops_per_mode * c.g.M, 32.0 * rowsM * n, k_solve_T_cd, grid, TPB, 0, c.g, lu, sj);
}
void solve_T(Ctx& c, const DLU& lu, const cd* in, cd* out) {
  solve_T_jobs(c, KC_SOLVE, lu, {SolveTJob{in, out, 0, lu.n - 1}});
}
void eval_T(Ctx& c, std::initializer_list<EvalJob> jobs) {
  EvalJobs ej{};
  int n = 0;
  for (const EvalJob& j : jobs) ej.j[n++] = j;
  int maxrows = 0;
  for (int q = 0; q < n; ++q) maxrows = std::max(maxrows, ej.j[q].B.rows);
  LMVD_LAUNCH(c, KC_EVAL, 0, 0, k_eval, dim3(mblocks(c.g), n, row_chunks(c.g, maxrows)), TPB, 0, c.g, ej);
}

// adjoint of: a = G(B0 zdot); rt = A^{-1} F(f' a); m^c = C(rt); b = G(E m^c), given bbar (3 physical
// fields, overwritten) and the tape a of this application; adds the result to zdbar (acc) or sets it.
void chain_mc_T(Ctx& c, AdjWork& A, double* const* bb, const double* a_tape, int acc) {
  const size_t n = (size_t)c.g.ny * c.g.P;
  cd* sv3[3] = {A.sv[0], A.sv[1], A.sv[2]};
  g_transpose(c, bb, sv3, 3);
  eval_T(c, {EvalJob{A.B0gT, A.sv[0], A.mc[0], 0}, EvalJob{A.Sg0T, A.sv[1], A.mc[1], 0},
             EvalJob{A.B0gT, A.sv[2], A.mc[2], 0}});
  const int ny = c.g.ny;
  LMVD_LAUNCH(c, KC_MC_SOLVE, 0, 0, k_adj_mc_rhs, dim3(mblocks(c.g), row_chunks(c.g, ny + 1)), TPB, 0, c.g, c.dstar,
              A.mc[0], A.mc[1], A.mc[2], A.tSp);
  solve_T_jobs(c, KC_MC_SOLVE, c.lu_mc, {SolveTJob{A.tSp, A.tSp, 1, ny - 1}});
  LMVD_LAUNCH(c, KC_MC_SOLVE, 0, 0, k_adj_mc_post, dim3(mblocks(c.g), row_chunks(c.g, ny)), TPB, 0, c.g, A.BsT[1],
              c.dstar, A.mc[0], A.mc[1], A.mc[2], A.tSp, A.rt);
  solve_T(c, c.lu_interp, A.rt, A.tS);
  cd* t1[1] = {A.tS};
  double* rtp[1] = {A.pb[3]};
  f_transpose(c, t1, rtp, 1);
  LMVD_LAUNCH(c, KC_PRODUCTS, 2.0 * n, 40.0 * n, k_adj_rt, eblocks(n), 256, 0, n, c.fprime, a_tape, A.pb[3], A.pb[4],
              A.fp);
  double* ab[1] = {A.pb[4]};
  cd* s3[1] = {A.sv[3]};
  g_transpose(c, ab, s3, 1);
  eval_T(c, {EvalJob{A.B0gT, A.sv[3], A.zd, acc}});
}

void fp_step_T(Ctx& c, AdjWork& A, const double* a_tape, double* const* b_tape);
int pass1_T(Ctx& c, AdjWork& A);

int adjoint_impl(Ctx& c) {
  NvtxRange range("lmvd adjoint substage");
  AdjWork& A = *c.adj;
  const Grid& g = c.g;
  const lmvd_config& cf = c.cfg;
  const size_t S = (size_t)g.ny * g.M, Sp = (size_t)(g.ny + 1) * g.M, P = (size_t)g.ny * g.P, n = P;
  const int ny = g.ny, kf = cf.kf;
  const bool stage_n = (c.s % 2) == 0;
  double a[4];
  if (stage_n) {
    a[0] = 2.0; a[1] = -(2.0 + 0.5 * cf.beta_n); a[2] = cf.beta_n; a[3] = -0.5 * cf.beta_n;
  } else {
    a[0] = 4.0 + cf.beta_p; a[1] = -(5.0 + 2.0 * cf.beta_p); a[2] = cf.beta_p; a[3] = 1.0;
  }
  const double al = stage_n ? 0.5 : 1.0, be = stage_n ? 0.0 : -0.5;
  // forward substage from the current state, recording the tape
  int err = advance(c, &A.tape);
  if (err) return err;
  cudaStream_t st = c.stream;
  // accumulators
  for (cd* p : {A.z, A.om, A.zh[2], A.zdp, A.romp, A.rz}) cudaMemsetAsync(p, 0, sizeof(cd) * S, st);
  for (cd* p : {A.m2, A.rphip}) cudaMemsetAsync(p, 0, sizeof(cd) * Sp, st);
  for (double* p : {A.mm1, A.mm3}) cudaMemsetAsync(p, 0, sizeof(double) * ny, st);
  cudaMemsetAsync(A.rmp, 0, sizeof(double) * 2 * ny, st);
  for (double* p : {A.fp, A.w[0], A.w[1], A.w[2], A.ir, A.rho, A.md[0], A.md[1], A.md[2]})
    cudaMemsetAsync(p, 0, sizeof(double) * P, st);
  // history rotation: zh0' = z, zh1' = zh0, zh2' = zh1, zdot_prev' = zdot^{kf}, RHS_prev' = RHS
  cudaMemcpyAsync(A.z, A.ozh[0], sizeof(cd) * S, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(A.zh[0], A.ozh[1], sizeof(cd) * S, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(A.zh[1], A.ozh[2], sizeof(cd) * S, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(A.zd, A.ozdp, sizeof(cd) * S, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(A.rom, A.orom, sizeof(cd) * S, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(A.rphi, A.orphi, sizeof(cd) * Sp, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(A.rm, A.orm, sizeof(double) * 2 * ny, cudaMemcpyDeviceToDevice, st);
  // step 6: RK update
  AdjUpd u{};
  u.dt = cf.dt;
  u.al = al;
  u.be = be;
  u.oom = A.oom; u.oz = A.oz; u.om2 = A.om2; u.omm1 = A.omm1; u.omm3 = A.omm3;
  u.om = A.om; u.rom = A.rom; u.romp = A.romp; u.z = A.z; u.zd = A.zd; u.zdp = A.zdp;
  u.m2 = A.m2; u.rphi = A.rphi; u.rphip = A.rphip; u.mm1 = A.mm1; u.mm3 = A.mm3; u.rm = A.rm; u.rmp = A.rmp;
  u.scr0 = A.tS; u.scr1 = A.tS + S; u.scrp = A.tSp;
  solve_T_jobs(c, KC_UPDATE, c.lu_interp, {SolveTJob{A.oom, u.scr0, 1, ny - 2}});
  solve_T_jobs(c, KC_UPDATE, c.lu_neumann, {SolveTJob{A.oz, u.scr1, 1, ny - 2}});
  LMVD_LAUNCH(c, KC_UPDATE, 0, 0, k_adj_update_om_z_post, dim3(mblocks(g), row_chunks(g, ny), 2), TPB, 0, g, A.B0gT,
              u);
  LMVD_LAUNCH(c, KC_UPDATE, 0, 0, k_adj_update_means, 1, 32, 0, g, A.B0gT, c.lu_means, u);
  solve_T_jobs(c, KC_UPDATE, c.lu_md, {SolveTJob{A.om2, u.scrp, 2, ny - 2}});
  LMVD_LAUNCH(c, KC_UPDATE, 0, 0, k_adj_update_m2_post, dim3(mblocks(g), row_chunks(g, ny + 1)), TPB, 0, g, A.Ss0T,
              A.Ss2T, u);
  // step 5: RHS streams, collocation solves, transforms, products of pass 2
  St7 stw{};
  for (int q = 0; q < 7; ++q) stw.p[q] = A.st[q];
  LMVD_LAUNCH(c, KC_RHS_EVAL, 0, 0, k_adj_rhs_eval, mblocks(g), TPB, 0, g, A.B1gT, A.B2gT, A.BsT[0], A.BsT[1],
              A.BsT[2], A.BsT[3], A.rom, A.rphi, A.rm, stw);
  solve_T_jobs(c, KC_SOLVE, c.lu_interp,
               {SolveTJob{A.st[1], A.st[1], 0, ny - 1}, SolveTJob{A.st[2], A.st[2], 0, ny - 1},
                SolveTJob{A.st[3], A.st[3], 0, ny - 1}, SolveTJob{A.st[4], A.st[4], 0, ny - 1},
                SolveTJob{A.st[5], A.st[5], 0, ny - 1}, SolveTJob{A.st[6], A.st[6], 0, ny - 1}});
  FieldsW10 svw{};
  for (int q = 0; q < 10; ++q) svw.p[q] = A.sv[q];
  LMVD_LAUNCH(c, KC_RHS_COMBINE, 0, 0, k_adj_rhs_combine, eblocks(S), 256, 0, g, 1.0 / cf.re, 1.0 / (cf.fr * cf.fr),
              stw, svw);
  f_transpose(c, A.sv, A.pb, 10);
  Fields10R pbw{};
  for (int q = 0; q < 10; ++q) pbw.p[q] = A.pb[q];
  Fields3RC mdc{{c.md[0], c.md[1], c.md[2]}};
  Fields3RC bfin{{A.tape.b[kf][0], A.tape.b[kf][1], A.tape.b[kf][2]}};
  Fields3R mdb{{A.md[0], A.md[1], A.md[2]}};
  LMVD_LAUNCH(c, KC_PRODUCTS, 0, 0, k_adj_p2, eblocks(n), 256, 0, n, pbw, mdc, bfin, c.invrho, mdb, A.ir, A.rho);
  // final m^c from dz/dt^{kf}: adds to the adjoint of dz/dt^{kf}
  chain_mc_T(c, A, A.pb, A.tape.a[kf], 1);
  // step 3 in reverse: k = kf-1 .. 0, dz/dt^{k+1} = A^{-1} F(-w . b_k) + R_z
  for (int k = kf - 1; k >= 0; --k) fp_step_T(c, A, A.tape.a[k], A.tape.b[k]);
  // BDF-like guess: zdot^0 = (a0 z + a1 zh0 + a2 zh1 + a3 zh2) / dt
  LMVD_LAUNCH(c, KC_MISC, 0, 0, k_adj_bdf, eblocks(S), 256, 0, S, a[0] / cf.dt, a[1] / cf.dt, a[2] / cf.dt,
              a[3] / cf.dt, A.zd, A.z, A.zh[0], A.zh[1], A.zh[2]);
  return pass1_T(c, A);
}

// adjoint of one fixed-point application dz/dt^{k+1} = A^{-1} F(-w . b_k) + R_z, given the adjoint of
// dz/dt^{k+1} in A.zd (replaced by the adjoint of dz/dt^k) and the application's tape (a_k, b_k)
void fp_step_T(Ctx& c, AdjWork& A, const double* a_tape, double* const* b_tape) {
  const size_t S = (size_t)c.g.ny * c.g.M, n = (size_t)c.g.ny * c.g.P;
  Fields3RC wc{{c.w[0], c.w[1], c.w[2]}};
  Fields3R wb{{A.w[0], A.w[1], A.w[2]}};
  LMVD_LAUNCH(c, KC_MISC, 0, 0, k_add, eblocks(S), 256, 0, S, A.rz, A.zd);
  solve_T(c, c.lu_interp, A.zd, A.tS);
  cd* t1[1] = {A.tS};
  double* lp[1] = {A.pb[5]};
  f_transpose(c, t1, lp, 1);
  Fields3RC bk{{b_tape[0], b_tape[1], b_tape[2]}};
  Fields3R bbw{{A.pb[0], A.pb[1], A.pb[2]}};
  LMVD_LAUNCH(c, KC_PRODUCTS, 0, 0, k_adj_L, eblocks(n), 256, 0, n, wc, bk, A.pb[5], bbw, wb);
  chain_mc_T(c, A, A.pb, a_tape, 0);
}

// adjoint of pass 1 (R_z, rho, f', grad z / rho and m^d on the grid from the state), given the adjoints of
// R_z (A.rz), f' (A.fp), w (A.w), rho (A.rho), 1/rho (A.ir), m^d on the grid (A.md); accumulates into the
// state adjoints A.z, A.om, A.m2, A.mm1, A.mm3
int pass1_T(Ctx& c, AdjWork& A) {
  const Grid& g = c.g;
  const lmvd_config& cf = c.cfg;
  const size_t S = (size_t)g.ny * g.M, Sp = (size_t)(g.ny + 1) * g.M, n = (size_t)g.ny * g.P;
  Fields3RC mdc{{c.md[0], c.md[1], c.md[2]}};
  Fields10R pbw{};
  for (int q = 0; q < 10; ++q) pbw.p[q] = A.pb[q];
  // R_z = A^{-1} F(R_z on the grid)
  solve_T(c, c.lu_interp, A.rz, A.tS);
  {
    cd* t1[1] = {A.tS};
    double* rzp[1] = {A.pb[8]};
    f_transpose(c, t1, rzp, 1);
  }
  // products of pass 1, then the transposed synthesis and evaluation of pass 1
  EosArgs e{cf.rho_heavy, cf.rho_light, 1.0 / (cf.re * cf.sc)};
  Fields5RC zpc{{A.tape.zp[0], A.tape.zp[1], A.tape.zp[2], A.tape.zp[3], A.tape.zp[4]}};
  Fields3RC mdbc{{A.md[0], A.md[1], A.md[2]}};
  Fields3RC wbc{{A.w[0], A.w[1], A.w[2]}};
  LMVD_LAUNCH(c, KC_PRODUCTS, 0, 0, k_adj_p1, eblocks(n), 256, 0, n, e, zpc, mdc, c.rho, c.invrho, A.rho, A.ir, A.fp,
              wbc, A.pb[8], mdbc, pbw);
  g_transpose(c, A.pb, A.sv, 8);
  Sv8C v8{};
  for (int q = 0; q < 8; ++q) v8.p[q] = A.sv[q];
  LMVD_LAUNCH(c, KC_EVAL_P1, 0, 0, k_adj_eval_p1, mblocks(g), TPB, 0, g, A.B0gT, A.B1gT, A.B2gT, A.Sg0T, A.Sg1T, v8,
              A.z, A.om, A.m2, A.mm1, A.mm3);
  // lmvd_set_state zeroes these entries of the state, so the substage does not depend on them
  LMVD_LAUNCH(c, KC_MISC, 0, 0, k_sanitize, eblocks(S), 256, 0, g, g.ny, A.z, 0);
  LMVD_LAUNCH(c, KC_MISC, 0, 0, k_sanitize, eblocks(S), 256, 0, g, g.ny, A.om, 1);
  LMVD_LAUNCH(c, KC_MISC, 0, 0, k_sanitize, eblocks(Sp), 256, 0, g, g.ny + 1, A.m2, 1);
  cudaError_t ce = cudaGetLastError();
  return ce == cudaSuccess ? LMVD_OK : LMVD_ERR_CUDA;
}

// Adjoint of the start-up (reading R6) from the current state x: the state passes through; the history is
// zh_q = z - c_q dt zdot, zdot_prev = zdot (c_q = 1/2, 1, 3/2), RHS_prev = 0, with zdot after n_startup
// applications from 0. Each application's physical fields are re-recorded from its stored iterate.
int adjoint_startup_impl(Ctx& c) {
  NvtxRange range("lmvd adjoint start-up");
  AdjWork& A = *c.adj;
  const Grid& g = c.g;
  const lmvd_config& cf = c.cfg;
  const size_t S = (size_t)g.ny * g.M, Sp = (size_t)(g.ny + 1) * g.M, P = (size_t)g.ny * g.P;
  const int ny = g.ny, ns = cf.n_startup;
  cudaStream_t st = c.stream;
  int err = startup_record(c, &A.tape, A.iterates);
  if (err) return err;
  cudaMemcpyAsync(A.z, A.oz, sizeof(cd) * S, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(A.om, A.oom, sizeof(cd) * S, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(A.m2, A.om2, sizeof(cd) * Sp, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(A.mm1, A.omm1, sizeof(double) * ny, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(A.mm3, A.omm3, sizeof(double) * ny, cudaMemcpyDeviceToDevice, st);
  cudaMemsetAsync(A.rz, 0, sizeof(cd) * S, st);
  for (double* p : {A.fp, A.w[0], A.w[1], A.w[2], A.ir, A.rho, A.md[0], A.md[1], A.md[2]})
    cudaMemsetAsync(p, 0, sizeof(double) * P, st);
  const double dt = cf.dt;
  LMVD_LAUNCH(c, KC_MISC, 0, 0, k_adj_backfill, eblocks(S), 256, 0, S, 0.5 * dt, dt, 1.5 * dt, A.ozh[0], A.ozh[1],
              A.ozh[2], A.ozdp, A.z, A.zd);
  for (int j = ns - 1; j >= 0; --j) {
    err = fp_record(c, A.iterates + (size_t)j * S, A.tape.a[0], A.tape.b[0]);
    if (err) return err;
    fp_step_T(c, A, A.tape.a[0], A.tape.b[0]);
  }
  return pass1_T(c, A);
}

int copy_dflt(cudaStream_t st, void* dst, const void* src, size_t bytes) {
  return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, st) == cudaSuccess ? LMVD_OK : LMVD_ERR_CUDA;
}

}  // namespace

size_t adj_device_bytes(const Ctx& c) {
  if (!c.adj) return 0;
  const AdjWork& A = *c.adj;
  return A.bytes + A.small_bytes + sizeof(cd) * c.g.ny * c.g.M * (size_t)A.n_iterates;
}

void adj_destroy(Ctx& c) {
  if (!c.adj) return;
  if (c.adj->iterates) cudaFree(c.adj->iterates);
  for (void* p : c.adj->small) cudaFree(p);
  if (c.adj->arena) cudaFree(c.adj->arena);
  delete c.adj;
  c.adj = nullptr;
}

// state blob: z | Omega2 | m2^d | <m1> | <m3>; history blob as lmvd_get_state
int adjoint_substage(Ctx& c, const void* sbar_out, const void* hbar_out, void* sbar_in, void* hbar_in) {
  if (c.cfg.precision != 0 || c.cfg.kf > KF_MAX_ADJ) return LMVD_ERR_UNSUPPORTED;
  int err = adj_setup(c);
  if (err) return err;
  AdjWork& A = *c.adj;
  const Grid& g = c.g;
  const size_t S = sizeof(cd) * g.ny * g.M, Sp = sizeof(cd) * (g.ny + 1) * g.M, R = sizeof(double) * g.ny;
  cudaStream_t st = c.stream;
  const char* so = (const char*)sbar_out;
  const char* ho = (const char*)hbar_out;
  err = copy_dflt(st, A.oz, so, S);
  if (!err) err = copy_dflt(st, A.oom, so + S, S);
  if (!err) err = copy_dflt(st, A.om2, so + 2 * S, Sp);
  if (!err) err = copy_dflt(st, A.omm1, so + 2 * S + Sp, R);
  if (!err) err = copy_dflt(st, A.omm3, so + 2 * S + Sp + R, R);
  size_t off = 16;
  for (int q = 0; q < 3 && !err; ++q, off += S) err = copy_dflt(st, A.ozh[q], ho + off, S);
  if (!err) { err = copy_dflt(st, A.ozdp, ho + off, S); off += S; }
  if (!err) { err = copy_dflt(st, A.orom, ho + off, S); off += S; }
  if (!err) { err = copy_dflt(st, A.orphi, ho + off, Sp); off += Sp; }
  if (!err) err = copy_dflt(st, A.orm, ho + off, 2 * R);
  if (err) return err;
  static thread_local long long s_before;
  s_before = c.s;
  err = adjoint_impl(c);
  if (err) return err;
  char* si = (char*)sbar_in;
  char* hi = (char*)hbar_in;
  err = copy_dflt(st, si, A.z, S);
  if (!err) err = copy_dflt(st, si + S, A.om, S);
  if (!err) err = copy_dflt(st, si + 2 * S, A.m2, Sp);
  if (!err) err = copy_dflt(st, si + 2 * S + Sp, A.mm1, R);
  if (!err) err = copy_dflt(st, si + 2 * S + Sp + R, A.mm3, R);
  if (!err) err = copy_dflt(st, hi, &s_before, sizeof(long long));
  off = 16;
  for (int q = 0; q < 3 && !err; ++q, off += S) err = copy_dflt(st, hi + off, A.zh[q], S);
  if (!err) { err = copy_dflt(st, hi + off, A.zdp, S); off += S; }
  if (!err) { err = copy_dflt(st, hi + off, A.romp, S); off += S; }
  if (!err) { err = copy_dflt(st, hi + off, A.rphip, Sp); off += Sp; }
  if (!err) err = copy_dflt(st, hi + off, A.rmp, 2 * R);
  if (!err && cudaStreamSynchronize(st) != cudaSuccess) err = LMVD_ERR_CUDA;
  return err;
}

// state blob in and out as lmvd_adjoint_substage; history blob: the adjoint of the start-up's history
// (its RHS_prev part is ignored: the start-up sets RHS_prev = 0)
int adjoint_startup(Ctx& c, const void* sbar_out, const void* hbar_out, void* sbar_in) {
  if (c.cfg.precision != 0 || c.cfg.kf > KF_MAX_ADJ) return LMVD_ERR_UNSUPPORTED;
  int err = adj_setup(c);
  if (err) return err;
  AdjWork& A = *c.adj;
  const Grid& g = c.g;
  const size_t S = sizeof(cd) * g.ny * g.M, Sp = sizeof(cd) * (g.ny + 1) * g.M, R = sizeof(double) * g.ny;
  const int ns = c.cfg.n_startup;
  if (ns > A.n_iterates) {
    if (A.iterates) cudaFree(A.iterates);
    A.iterates = nullptr;
    A.n_iterates = 0;
    if (cudaMalloc(&A.iterates, S * (size_t)ns) != cudaSuccess) {
      cudaGetLastError();
      A.iterates = nullptr;
      return LMVD_ERR_OOM;
    }
    A.n_iterates = ns;
  }
  cudaStream_t st = c.stream;
  const char* so = (const char*)sbar_out;
  const char* ho = (const char*)hbar_out;
  err = copy_dflt(st, A.oz, so, S);
  if (!err) err = copy_dflt(st, A.oom, so + S, S);
  if (!err) err = copy_dflt(st, A.om2, so + 2 * S, Sp);
  if (!err) err = copy_dflt(st, A.omm1, so + 2 * S + Sp, R);
  if (!err) err = copy_dflt(st, A.omm3, so + 2 * S + Sp + R, R);
  size_t off = 16;
  for (int q = 0; q < 3 && !err; ++q, off += S) err = copy_dflt(st, A.ozh[q], ho + off, S);
  if (!err) err = copy_dflt(st, A.ozdp, ho + off, S);
  if (err) return err;
  err = adjoint_startup_impl(c);
  if (err) return err;
  char* si = (char*)sbar_in;
  err = copy_dflt(st, si, A.z, S);
  if (!err) err = copy_dflt(st, si + S, A.om, S);
  if (!err) err = copy_dflt(st, si + 2 * S, A.m2, Sp);
  if (!err) err = copy_dflt(st, si + 2 * S + Sp, A.mm1, R);
  if (!err) err = copy_dflt(st, si + 2 * S + Sp + R, A.mm3, R);
  if (!err && cudaStreamSynchronize(st) != cudaSuccess) err = LMVD_ERR_CUDA;
  return err;
}

}  // namespace lmvd
