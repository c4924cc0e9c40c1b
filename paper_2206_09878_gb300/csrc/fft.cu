// Batched Fourier transforms in the periodic directions with the 3/2 rule (paper Eq. disc_f and
// Sec. 4.4: products are formed in physical space on a grid padded to 3N/2 points, so that
// quadratic products of retained modes do not alias; coefficients are truncated back to
// |kx| < nx/2, |kz| < nz/2 with the Nyquist slots zero).
//
// Each field transform runs in two passes through an intermediate array T[y][z][kx]
// (kx < nx/2 only -- the padded kx range carries zeros and is never stored):
//   inverse: z-pass (complex, length pz, zero-padded in kz) then x-pass (complex-to-real, length px,
//            two real rows packed into one complex transform);
//   forward: x-pass (real-to-complex, two rows per complex transform, split by Hermitian symmetry)
//            then z-pass (complex, truncated, scaled by 1/(px pz)).
// Synthesis is unnormalised: f(x, z) = sum_k fhat_k exp(i (k1 x + k3 z)).
// A pass is one CTA per (plane, field, batch of columns / row pairs); every 1D transform is a
// Stockham autosort FFT in shared memory with radix-4/3/2 stages and a double-precision twiddle
// table.
#include <cmath>
#include <cstring>

#include "lmvd_internal.h"

namespace lmvd {

struct FieldsC {
  const cd* p[10];
};
struct FieldsW {
  cd* p[10];
};
struct FieldsRC {
  const double* p[10];
};
struct FieldsRW {
  double* p[10];
};

// One Stockham stage set on a batch of transforms of length n stored with leading dimension ld.
// sign = +1: synthesis (exp(+i)), -1: analysis. Returns the buffer holding the result.
template <int SIGN>
__device__ cd* fft_batch(cd* a, cd* b, const FFTPlan& pl, int batch, int ld) {
  const int n = pl.n;
  cd* in = a;
  cd* out = b;
  int L = 1;
  for (int s = 0; s < pl.nst; ++s) {
    const int r = pl.radix[s];
    const int Ls = L * r;
    const int nb = n / r;
    const int tws = n / Ls;
    for (int t = threadIdx.x; t < batch * nb; t += blockDim.x) {
      const int bt = t / nb;
      const int i = t - bt * nb;
      const int k = i % L;
      const cd* src = in + bt * ld;
      cd* dst = out + bt * ld;
      cd v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (q < r) v[q] = src[i + q * nb];
#pragma unroll
      for (int q = 1; q < 4; ++q)
        if (q < r) {
          const double2 w = pl.tw[q * k * tws];
          v[q] = cmul(v[q], cd{w.x, SIGN * w.y});
        }
      const int base = (i - k) * r + k;
      if (r == 4) {
        const cd t0 = v[0] + v[2], t1 = v[0] - v[2], t2 = v[1] + v[3];
        const cd d3 = times_i(v[1] - v[3]);
        const cd t3 = SIGN > 0 ? d3 : cd{-d3.re, -d3.im};  // (SIGN i) (v1 - v3)
        dst[base] = t0 + t2;
        dst[base + L] = t1 + t3;
        dst[base + 2 * L] = t0 - t2;
        dst[base + 3 * L] = t1 - t3;
      } else if (r == 3) {
        const double sn = SIGN * 0.86602540378443864676372317075294;  // sin(2 pi / 3)
        const cd t1 = v[1] + v[2], t2 = v[1] - v[2];
        const cd m = v[0] - 0.5 * t1;
        const cd u = sn * times_i(t2);
        dst[base] = v[0] + t1;
        dst[base + L] = m + u;
        dst[base + 2 * L] = m - u;
      } else {
        dst[base] = v[0] + v[1];
        dst[base + L] = v[0] - v[1];
      }
    }
    __syncthreads();
    cd* tmp = in;
    in = out;
    out = tmp;
    L = Ls;
  }
  return in;
}

// ---------------------------------------------------------------- inverse z-pass
// in: spectral value fields [ny][nz][nxh]; T: [f][ny][pz][nx/2]
__global__ void k_fft_z_inv(FFTPlan pl, Grid g, FieldsC in, cd* T, size_t tstride) {
  extern __shared__ cd sm[];
  const int batch = pl.batch, ld = pl.n + 1, pz = g.pz, nz = g.nz, h = g.nx / 2;
  const int kx0 = blockIdx.x * batch, j = blockIdx.y, f = blockIdx.z;
  cd* a = sm;
  cd* b = sm + batch * ld;
  for (int idx = threadIdx.x; idx < batch * ld; idx += blockDim.x) a[idx] = mk(0, 0);
  __syncthreads();
  const cd* src = in.p[f] + (size_t)j * g.M;
  for (int idx = threadIdx.x; idx < nz * batch; idx += blockDim.x) {
    const int jz = idx / batch, bb = idx - jz * batch, kx = kx0 + bb;
    if (kx < h && jz != nz / 2) {
      const int pos = jz < nz / 2 ? jz : pz - nz + jz;
      a[bb * ld + pos] = src[(size_t)jz * g.nxh + kx];
    }
  }
  __syncthreads();
  const cd* res = fft_batch<1>(a, b, pl, batch, ld);
  cd* dst = T + f * tstride + (size_t)j * pz * h;
  for (int idx = threadIdx.x; idx < pz * batch; idx += blockDim.x) {
    const int zz = idx / batch, bb = idx - zz * batch, kx = kx0 + bb;
    if (kx < h) dst[(size_t)zz * h + kx] = res[bb * ld + zz];
  }
}

// ---------------------------------------------------------------- inverse x-pass (c2r, 2 rows per transform)
__global__ void k_fft_x_inv(FFTPlan pl, Grid g, const cd* T, size_t tstride, FieldsRW out) {
  extern __shared__ cd sm[];
  const int batch = pl.batch, ld = pl.n + 1, px = g.px, pz = g.pz, h = g.nx / 2;
  const int pr0 = blockIdx.x * batch, j = blockIdx.y, f = blockIdx.z;
  cd* a = sm;
  cd* b = sm + batch * ld;
  for (int idx = threadIdx.x; idx < batch * ld; idx += blockDim.x) a[idx] = mk(0, 0);
  __syncthreads();
  const cd* src = T + f * tstride + (size_t)j * pz * h;
  for (int idx = threadIdx.x; idx < batch * h; idx += blockDim.x) {
    const int bb = idx / h, k = idx - bb * h;
    const int za = 2 * (pr0 + bb), zb = za + 1;
    if (za >= pz) continue;
    const cd ta = src[(size_t)za * h + k];
    const cd tb = zb < pz ? src[(size_t)zb * h + k] : mk(0, 0);
    cd* y = a + bb * ld;
    if (k == 0) {
      y[0] = mk(ta.re, tb.re);  // the kx = 0 coefficient of a real row is real
    } else {
      y[k] = mk(ta.re - tb.im, ta.im + tb.re);       // Xa[k] + i Xb[k]
      y[px - k] = mk(ta.re + tb.im, tb.re - ta.im);  // conj(Xa[k]) + i conj(Xb[k])
    }
  }
  __syncthreads();
  const cd* res = fft_batch<1>(a, b, pl, batch, ld);
  double* dst = out.p[f] + (size_t)j * g.P;
  for (int idx = threadIdx.x; idx < batch * px; idx += blockDim.x) {
    const int bb = idx / px, x = idx - bb * px;
    const int za = 2 * (pr0 + bb), zb = za + 1;
    if (za >= pz) continue;
    const cd v = res[bb * ld + x];
    dst[(size_t)za * px + x] = v.re;
    if (zb < pz) dst[(size_t)zb * px + x] = v.im;
  }
}

// ---------------------------------------------------------------- forward x-pass (r2c, 2 rows per transform)
__global__ void k_fft_x_fwd(FFTPlan pl, Grid g, FieldsRC in, cd* T, size_t tstride) {
  extern __shared__ cd sm[];
  const int batch = pl.batch, ld = pl.n + 1, px = g.px, pz = g.pz, h = g.nx / 2;
  const int pr0 = blockIdx.x * batch, j = blockIdx.y, f = blockIdx.z;
  cd* a = sm;
  cd* b = sm + batch * ld;
  const double* src = in.p[f] + (size_t)j * g.P;
  for (int idx = threadIdx.x; idx < batch * px; idx += blockDim.x) {
    const int bb = idx / px, x = idx - bb * px;
    const int za = 2 * (pr0 + bb), zb = za + 1;
    double va = 0.0, vb = 0.0;
    if (za < pz) {
      va = src[(size_t)za * px + x];
      if (zb < pz) vb = src[(size_t)zb * px + x];
    }
    a[bb * ld + x] = mk(va, vb);
  }
  __syncthreads();
  const cd* res = fft_batch<-1>(a, b, pl, batch, ld);
  cd* dst = T + f * tstride + (size_t)j * pz * h;
  for (int idx = threadIdx.x; idx < batch * h; idx += blockDim.x) {
    const int bb = idx / h, k = idx - bb * h;
    const int za = 2 * (pr0 + bb), zb = za + 1;
    if (za >= pz) continue;
    const cd yk = res[bb * ld + k];
    const cd ym = conj(res[bb * ld + (k == 0 ? 0 : px - k)]);
    const cd fa = 0.5 * (yk + ym);
    const cd d = yk - ym;
    dst[(size_t)za * h + k] = fa;
    if (zb < pz) dst[(size_t)zb * h + k] = mk(0.5 * d.im, -0.5 * d.re);  // (yk - ym) / (2 i)
  }
}

// ---------------------------------------------------------------- forward z-pass (truncate, scale)
__global__ void k_fft_z_fwd(FFTPlan pl, Grid g, const cd* T, size_t tstride, FieldsW out, double scale) {
  extern __shared__ cd sm[];
  const int batch = pl.batch, ld = pl.n + 1, pz = g.pz, nz = g.nz, h = g.nx / 2;
  const int kx0 = blockIdx.x * batch, j = blockIdx.y, f = blockIdx.z;
  cd* a = sm;
  cd* b = sm + batch * ld;
  const cd* src = T + f * tstride + (size_t)j * pz * h;
  for (int idx = threadIdx.x; idx < pz * batch; idx += blockDim.x) {
    const int zz = idx / batch, bb = idx - zz * batch, kx = kx0 + bb;
    a[bb * ld + zz] = kx < h ? src[(size_t)zz * h + kx] : mk(0, 0);
  }
  __syncthreads();
  const cd* res = fft_batch<-1>(a, b, pl, batch, ld);
  cd* dst = out.p[f] + (size_t)j * g.M;
  for (int idx = threadIdx.x; idx < nz * batch; idx += blockDim.x) {
    const int jz = idx / batch, bb = idx - jz * batch, kx = kx0 + bb;
    if (kx > h) continue;
    cd v = mk(0, 0);
    if (kx < h && jz != nz / 2) v = scale * res[bb * ld + (jz < nz / 2 ? jz : pz - nz + jz)];
    dst[(size_t)jz * g.nxh + kx] = v;
  }
}

// ---------------------------------------------------------------- host side
static bool make_plan(int n, FFTPlan& p) {
  p.n = n;
  p.nst = 0;
  int m = n;
  while (m % 4 == 0) { p.radix[p.nst++] = 4; m /= 4; }
  while (m % 2 == 0) { p.radix[p.nst++] = 2; m /= 2; }
  while (m % 3 == 0) { p.radix[p.nst++] = 3; m /= 3; }
  return m == 1 && p.nst < 24;
}

static size_t smem_bytes(const FFTPlan& p) { return (size_t)2 * p.batch * (p.n + 1) * sizeof(cd); }

int fft_prepare(Ctx& c) {
  if (!make_plan(c.g.px, c.fx) || !make_plan(c.g.pz, c.fz)) return LMVD_ERR_UNSUPPORTED;
  for (FFTPlan* p : {&c.fx, &c.fz}) {
    const size_t per = (size_t)2 * (p->n + 1) * sizeof(cd);
    int b = (int)(98304 / per);
    if (b < 1) b = 1;
    if (b > 32) b = 32;
    p->batch = b;
    if (smem_bytes(*p) > 200 * 1024) return LMVD_ERR_UNSUPPORTED;
    std::vector<double2> tw(p->n);
    for (int m = 0; m < p->n; ++m) {
      const long double ang = 2.0L * 3.141592653589793238462643383279502884L * (long double)m / (long double)p->n;
      tw[m] = make_double2((double)cosl(ang), (double)sinl(ang));
    }
    if (cudaMalloc(&p->tw, sizeof(double2) * p->n) != cudaSuccess) return LMVD_ERR_OOM;
    c.small_allocs.push_back(p->tw);
    if (cudaMemcpy(p->tw, tw.data(), sizeof(double2) * p->n, cudaMemcpyHostToDevice) != cudaSuccess)
      return LMVD_ERR_CUDA;
  }
  const int sx = (int)smem_bytes(c.fx), sz = (int)smem_bytes(c.fz);
  if (cudaFuncSetAttribute(k_fft_z_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, sz) != cudaSuccess ||
      cudaFuncSetAttribute(k_fft_z_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, sz) != cudaSuccess ||
      cudaFuncSetAttribute(k_fft_x_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, sx) != cudaSuccess ||
      cudaFuncSetAttribute(k_fft_x_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, sx) != cudaSuccess)
    return LMVD_ERR_CUDA;
  return LMVD_OK;
}

static inline unsigned cdiv(unsigned a, unsigned b) { return (a + b - 1) / b; }
// conventional algorithmic flop count of one complex transform of length n: 5 n log2 n
static inline double fft_flops(double n) { return 5.0 * n * std::log2(n); }

void fft_inverse(Ctx& c, cd* const* in, double* const* out, int nf) {
  const Grid& g = c.g;
  const size_t tstride = (size_t)g.ny * g.pz * (g.nx / 2);
  for (int f0 = 0; f0 < nf; f0 += 10) {
    const int n = nf - f0 < 10 ? nf - f0 : 10;
    FieldsC fi{};
    FieldsRW fo{};
    for (int f = 0; f < n; ++f) {
      fi.p[f] = in[f0 + f];
      fo.p[f] = out[f0 + f];
    }
    const double h = g.nx / 2, ny = g.ny, pz = g.pz, px = g.px;
    dim3 gz(cdiv(g.nx / 2, c.fz.batch), g.ny, n);
    LMVD_LAUNCH(c, KC_FFT_Z_INV, n * ny * h * fft_flops(pz), n * ny * h * 16.0 * ((g.nz - 1) + pz), k_fft_z_inv, gz,
                256, smem_bytes(c.fz), c.fz, g, fi, c.tbuf, tstride);
    dim3 gx(cdiv(cdiv(g.pz, 2), c.fx.batch), g.ny, n);
    LMVD_LAUNCH(c, KC_FFT_X_INV, n * ny * ((g.pz + 1) / 2) * fft_flops(px), n * ny * pz * (16.0 * h + 8.0 * px),
                k_fft_x_inv, gx, 256, smem_bytes(c.fx), c.fx, g, c.tbuf, tstride, fo);
  }
}

void fft_forward(Ctx& c, double* const* in, cd* const* out, int nf) {
  const Grid& g = c.g;
  const size_t tstride = (size_t)g.ny * g.pz * (g.nx / 2);
  const double scale = 1.0 / ((double)g.px * (double)g.pz);
  for (int f0 = 0; f0 < nf; f0 += 10) {
    const int n = nf - f0 < 10 ? nf - f0 : 10;
    FieldsRC fi{};
    FieldsW fo{};
    for (int f = 0; f < n; ++f) {
      fi.p[f] = in[f0 + f];
      fo.p[f] = out[f0 + f];
    }
    const double h = g.nx / 2, ny = g.ny, pz = g.pz, px = g.px;
    dim3 gx(cdiv(cdiv(g.pz, 2), c.fx.batch), g.ny, n);
    LMVD_LAUNCH(c, KC_FFT_X_FWD, n * ny * ((g.pz + 1) / 2) * fft_flops(px), n * ny * pz * (16.0 * h + 8.0 * px),
                k_fft_x_fwd, gx, 256, smem_bytes(c.fx), c.fx, g, fi, c.tbuf, tstride);
    dim3 gz(cdiv(g.nx / 2 + 1, c.fz.batch), g.ny, n);
    LMVD_LAUNCH(c, KC_FFT_Z_FWD, n * ny * h * fft_flops(pz), n * ny * 16.0 * (pz * h + (double)g.nz * g.nxh),
                k_fft_z_fwd, gz, 256, smem_bytes(c.fz), c.fz, g, c.tbuf, tstride, fo, scale);
  }
}

}  // namespace lmvd
