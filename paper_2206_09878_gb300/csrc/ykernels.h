// Declarations of the y-direction and elementwise kernels (see ykernels.cu, pointwise.cu).
#pragma once
#include "lmvd_internal.h"

namespace lmvd {

struct Fields8 {
  cd* p[8];
};
struct Fields7 {
  cd* p[7];
};
struct Fields7C {
  const cd* p[7];
};
struct Fields10C {
  const cd* p[10];
};
struct EvalJob {
  DBand B;
  const cd* in;
  cd* out;
  int acc;  // 1: out += B in
};
struct EvalJobs {
  EvalJob j[4];
};
struct SolveJob {
  const cd* in;
  const cd* add;  // may be null
  cd* out;
};
struct SolveJobs {
  SolveJob j[8];
};
struct UpdateArgs {
  double dt, al, be;
  const cd *om, *r_om, *r_om_prev, *z, *zdot, *zdot_prev, *m2, *r_phi, *r_phi_prev;
  const double *mm1, *mm3, *r_m, *r_m_prev;
  cd *om_new, *z_new, *m2_new;
  double *mm1_new, *mm3_new;
};

struct CheckJob {
  const double* p;
  size_t n;  // doubles
};
struct CheckJobs {
  CheckJob j[5];
};
__global__ void k_check_finite(CheckJobs jobs, unsigned* flag);
__global__ void k_diff_norms(size_t n, const cd* a, const cd* b, double* out);
__global__ void k_mass_norms(Grid g, const double* dstar, const cd* rt, const cd* m1, const cd* m2, const cd* m3,
                             double* out);
__global__ void k_fp_check(const double* diag, int kf, unsigned* flag);
struct Fields3C {
  const double* p[3];
};
__global__ void k_energy_norms(Grid g, const double* wq, Fields3C md, Fields3C mc, const double* invrho, int df_fields,
                               double* ke, unsigned long long* m2max);

__global__ void k_eval_p1(Grid g, DBand B0g, DBand B1g, DBand B2g, DBand Sg0, DBand Sg1, const cd* z,
                          const cd* om, const cd* m2, const double* mm1, const double* mm3, Fields8 out);
__global__ void k_eval(Grid g, EvalJobs jobs);
// double-float evaluations of the precision path (same outputs as k_eval_p1, k_eval without accumulation and
// k_rhs_eval), launched on st for spline orders p = 4..8 (band widths w = 4..9). The first two store their
// values as double-float pairs (for fft_inverse_df_in), the third FP64 values (for the FP64 RK update).
void launch_eval_p1_df(int p, dim3 grid, int tpb, cudaStream_t st, const Grid& g, const DBand& B0g, const DBand& B1g,
                       const DBand& B2g, const DBand& Sg0, const DBand& Sg1, const cd* z, const cd* om, const cd* m2,
                       const double* mm1, const double* mm3, const Fields8& out);
void launch_eval_df(int w, dim3 grid, int tpb, cudaStream_t st, const Grid& g, const EvalJobs& jobs);
void launch_rhs_eval_df(int p, dim3 grid, int tpb, cudaStream_t st, const Grid& g, const DBand& B1g, const DBand& B2g,
                        const DBand* Bs, const Fields7C& stc, cd* r_om, cd* r_phi, double* r_m);
__global__ void k_solve_cd(Grid g, DLU lu, SolveJobs jobs);
__global__ void k_solve_re(Grid g, DLU lu, SolveJobs jobs);
__global__ void k_mc_rhs(Grid g, DBand Bs1, const cd* rt, cd* m2c);
__global__ void k_mc_post(Grid g, const double* dstar, const cd* rt, cd* m1c, cd* m2c, cd* m3c);
__global__ void k_rhs_combine(Grid g, double mu, double grav, Fields10C sv, Fields7 st);
__global__ void k_rhs_eval(Grid g, DBand B1g, DBand B2g, DBand Bs0, DBand Bs1, DBand Bs2, DBand Bs3, Fields7C st,
                           cd* r_om, cd* r_phi, double* r_m);
__global__ void k_update_om_z_rhs(Grid g, DBand B0g, UpdateArgs a);
__global__ void k_update_means(Grid g, DBand B0g, DLU lu_i, UpdateArgs a);
__global__ void k_update_m2_rhs(Grid g, DBand Ss0, DBand Ss2, UpdateArgs a);
__global__ void k_bdf(size_t n, double a0, double a1, double a2, double a3, double idt, const cd* z, const cd* h0,
                      const cd* h1, const cd* h2, cd* out);
__global__ void k_backfill(size_t n, double c0, double c1, double c2, const cd* z, const cd* zdot, cd* h0, cd* h1,
                           cd* h2);
__global__ void k_sanitize(Grid g, int rows, cd* f, int zero_mean);
__global__ void k_factor(Grid g, int n, int K, const double* A2, const double* A0, const double* A1, const int* nl,
                         const int* nu, double* lo, double* up, double* invd);

// pointwise.cu: physical-space products (Sec. 2.1, 4.3, 5)
struct EosArgs {
  double rh, rl, kappa;
};
__global__ void k_products_p1(size_t n, EosArgs e, const double* zp, const double* zx, const double* zz,
                              const double* zy, const double* lapz, const double* m1, const double* m2,
                              const double* m3, double* rho, double* invrho, double* fprime, double* w1, double* w2,
                              double* w3, double* rz);
__global__ void k_product_rt(size_t n, const double* fprime, const double* zdot, double* out);
__global__ void k_product_L(size_t n, const double* w1, const double* w2, const double* w3, const double* m1,
                            const double* m2, const double* m3, double* out);
struct P2Out {
  double* p[10];
};
__global__ void k_products_p2(size_t n, const double* md1, const double* md2, const double* md3, const double* mc1,
                              const double* mc2, const double* mc3, const double* rho, const double* invrho, P2Out o);

// double-float variants (physical fields hold hi/lo float pairs in the same storage)
__global__ void k_products_p1_df(size_t n, EosArgs e, const double* zp, const double* zx, const double* zz,
                                 const double* zy, const double* lapz, const double* m1, const double* m2,
                                 const double* m3, double* rho, double* invrho, double* fprime, double* w1,
                                 double* w2, double* w3, double* rz);
__global__ void k_product_rt_df(size_t n, const double* fprime, const double* zdot, double* out);
__global__ void k_product_L_df(size_t n, const double* w1, const double* w2, const double* w3, const double* m1,
                               const double* m2, const double* m3, double* out);
__global__ void k_products_p2_df(size_t n, const double* md1, const double* md2, const double* md3,
                                 const double* mc1, const double* mc2, const double* mc3, const double* rho,
                                 const double* invrho, P2Out o);

}  // namespace lmvd
