// Physical-space products on the 3/2-padded grid (one thread per grid point, grid-stride).
//
// Paper Sec. 2.1 (R_z, L), Sec. 4.3 (applying L: rho_t = f'(z) dz/dt, then -(1/rho) grad z . m^c),
// Eq. om / phi (C_ij = -rho u_i u_j), Sec. 5 (binary-mixing EOS rho = rl rh / (rh - (rh - rl) z)).
// 1/rho is linear in z, so the EOS needs one division per point (rho itself, used by gravity).
#include <algorithm>

#include "ykernels.h"

namespace lmvd {

LMVD_DEFINE_OOB_TAKE(pw)

// rho, 1/rho, f'(z) = rho^2 (rh - rl) / (rl rh), w = grad z / rho, and
// R_z = (-m^d . grad z + (rho D_z) lap z) / rho with rho D_z = kappa constant (Sc = 1 setting).
__global__ void k_products_p1(size_t n, EosArgs e, const double* zp, const double* zx, const double* zz,
                              const double* zy, const double* lapz, const double* m1, const double* m2,
                              const double* m3, double* rho, double* invrho, double* fprime, double* w1, double* w2,
                              double* w3, double* rz) {
  const double irlrh = 1.0 / (e.rl * e.rh);
  const double drho = e.rh - e.rl;
  for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
    const double ir = (e.rh - drho * zp[o]) * irlrh;
    const double r = 1.0 / ir;
    const double gx = zx[o], gy = zy[o], gz = zz[o];
    rho[o] = r;
    invrho[o] = ir;
    fprime[o] = r * r * drho * irlrh;
    w1[o] = gx * ir;
    w2[o] = gy * ir;
    w3[o] = gz * ir;
    rz[o] = (e.kappa * lapz[o] - (m1[o] * gx + m2[o] * gy + m3[o] * gz)) * ir;
  }
}

// rho_t = f'(z) dz/dt
__global__ void k_product_rt(size_t n, const double* fprime, const double* zdot, double* out) {
  for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x)
    out[o] = fprime[o] * zdot[o];
}

// L tail: -(1/rho) grad z . m^c
__global__ void k_product_L(size_t n, const double* w1, const double* w2, const double* w3, const double* m1,
                            const double* m2, const double* m3, double* out) {
  for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x)
    out[o] = -(w1[o] * m1[o] + w2[o] * m2[o] + w3[o] * m3[o]);
}

// m = m^d + m^c; outputs C11, C12, C13, C22, C23, C33 (C_ij = -m_i m_j / rho), u1, u2, u3 (u = m / rho), rho;
// a null output pointer is skipped (the outputs are formed in batches)
__global__ void k_products_p2(size_t n, const double* md1, const double* md2, const double* md3, const double* mc1,
                              const double* mc2, const double* mc3, const double* rho, const double* invrho, P2Out q) {
  for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
    const double ir = invrho[o];
    const double a = md1[o] + mc1[o], b = md2[o] + mc2[o], c = md3[o] + mc3[o];
    const double ua = a * ir, ub = b * ir, uc = c * ir;
    if (q.p[0]) q.p[0][o] = -a * ua;
    if (q.p[1]) q.p[1][o] = -a * ub;
    if (q.p[2]) q.p[2][o] = -a * uc;
    if (q.p[3]) q.p[3][o] = -b * ub;
    if (q.p[4]) q.p[4][o] = -b * uc;
    if (q.p[5]) q.p[5][o] = -c * uc;
    if (q.p[6]) q.p[6][o] = ua;
    if (q.p[7]) q.p[7][o] = ub;
    if (q.p[8]) q.p[8][o] = uc;
    if (q.p[9]) q.p[9][o] = rho[o];
  }
}

}  // namespace lmvd

// ------------------------------------------------------------------ double-float variants (precision 1)
namespace lmvd {

__device__ __forceinline__ df ld(const double* p, size_t o) { return reinterpret_cast<const df*>(p)[o]; }
__device__ __forceinline__ void st(double* p, size_t o, df v) { reinterpret_cast<df*>(p)[o] = v; }

__global__ void k_products_p1_df(size_t n, EosArgs e, const double* zp, const double* zx, const double* zz,
                                 const double* zy, const double* lapz, const double* m1, const double* m2,
                                 const double* m3, double* rho, double* invrho, double* fprime, double* w1,
                                 double* w2, double* w3, double* rz) {
  const double irlrh = 1.0 / (e.rl * e.rh);
  const double drho = e.rh - e.rl;
  const df kap = df_from_double(e.kappa);
  for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
    // the EOS itself (1/rho, rho, f') in FP64 from z rounded to a double; the results are split back into
    // double-float pairs for the products (both conversions on the integer pipe)
    const double zd = df_to_double_int(ld(zp, o));
    const double ird = (e.rh - drho * zd) * irlrh;
    const double rd = 1.0 / ird;
    const df ir = df_from_double_int(ird);
    const df gx = ld(zx, o), gy = ld(zy, o), gz = ld(zz, o);
    st(rho, o, df_from_double_int(rd));
    st(invrho, o, ir);
    st(fprime, o, df_from_double_int(rd * rd * drho * irlrh));
    st(w1, o, dmul(gx, ir));
    st(w2, o, dmul(gy, ir));
    st(w3, o, dmul(gz, ir));
    const df adv = dadd(ddot2(ld(m1, o), gx, ld(m2, o), gy), dmul(ld(m3, o), gz));
    st(rz, o, dmul(dsub(dmul(kap, ld(lapz, o)), adv), ir));
  }
}

__global__ void k_product_rt_df(size_t n, const double* fprime, const double* zdot, double* out) {
  for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x)
    st(out, o, dmul(ld(fprime, o), ld(zdot, o)));
}

__global__ void k_product_L_df(size_t n, const double* w1, const double* w2, const double* w3, const double* m1,
                               const double* m2, const double* m3, double* out) {
  for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
    const df s = dadd(ddot2(ld(w1, o), ld(m1, o), ld(w2, o), ld(m2, o)), dmul(ld(w3, o), ld(m3, o)));
    st(out, o, dneg(s));
  }
}

__global__ void k_products_p2_df(size_t n, const double* md1, const double* md2, const double* md3,
                                 const double* mc1, const double* mc2, const double* mc3, const double* rho,
                                 const double* invrho, P2Out q) {
  for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
    const df ir = ld(invrho, o);
    const df a = dadd(ld(md1, o), ld(mc1, o)), b = dadd(ld(md2, o), ld(mc2, o)), c = dadd(ld(md3, o), ld(mc3, o));
    const df ua = dmul(a, ir), ub = dmul(b, ir), uc = dmul(c, ir);
    if (q.p[0]) st(q.p[0], o, dneg(dmul(a, ua)));
    if (q.p[1]) st(q.p[1], o, dneg(dmul(a, ub)));
    if (q.p[2]) st(q.p[2], o, dneg(dmul(a, uc)));
    if (q.p[3]) st(q.p[3], o, dneg(dmul(b, ub)));
    if (q.p[4]) st(q.p[4], o, dneg(dmul(b, uc)));
    if (q.p[5]) st(q.p[5], o, dneg(dmul(c, uc)));
    if (q.p[6]) st(q.p[6], o, ua);
    if (q.p[7]) st(q.p[7], o, ub);
    if (q.p[8]) st(q.p[8], o, uc);
    if (q.p[9]) st(q.p[9], o, ld(rho, o));
  }
}

}  // namespace lmvd

// ------------------------------------------------------------------ conversion self-test
namespace lmvd {
__global__ void k_df64_convert(size_t n, const double* x, float* hi, float* lo, const float* pair_hi,
                               const float* pair_lo, double* sum) {
  for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
    const df d = df_from_double_int(x[o]);
    hi[o] = d.hi;
    lo[o] = d.lo;
    sum[o] = df_to_double_int(df{pair_hi[o], pair_lo[o]});
  }
}
}  // namespace lmvd

extern "C" int lmvd_df64_convert(const double* x, float* hi, float* lo, const float* pair_hi, const float* pair_lo,
                                 double* sum, size_t n, void* cuda_stream) {
  using namespace lmvd;
  if (n == 0) return LMVD_OK;
  if (!x || !hi || !lo || !pair_hi || !pair_lo || !sum) return LMVD_ERR_INVALID_ARG;
  const size_t blocks = std::min<size_t>((n + 255) / 256, 4096);
  k_df64_convert<<<(unsigned)blocks, 256, 0, (cudaStream_t)cuda_stream>>>(n, x, hi, lo, pair_hi, pair_lo, sum);
  return cudaGetLastError() == cudaSuccess ? LMVD_OK : LMVD_ERR_CUDA;
}
