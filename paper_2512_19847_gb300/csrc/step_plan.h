// The launch sequence of one IMEX step (Algorithm 1, CK/ARS tableau with
// stage 1 = X^n, GSA close), shared by the handle path and the
// no-allocation entry point.
#pragma once
#include "../../include/ap_dvm.h"
#include "common.cuh"
#include "dispatch.h"

namespace apd {

enum KernelKind { KK_EXPLICIT, KK_RHS, KK_ROWS_FWD, KK_COLS, KK_ROWS_INV, KK_UPDATE, KK_FINISH, KK_UNPACK };

struct StepKernels {
  StencilSet ks;
  MiscSet km;
  int g_explicit, g_rhs, g_update, g_finish, g_fft;
  size_t fft_smem;
};

// launch(fn, grid, block, smem, args, kind) -> int status (0 = success)
template <class Launch>
int enqueue_imex_step(const ap_dvm_params& t, const StepKernels& K, BatchDev* bp, int f32, Launch&& launch) {
  const int s = t.s;
  const dim3 blk(K.ks.tx, K.ks.ty);
  double weno_eps = t.weno_eps;
  int st;
  auto AEX = [&](int i, int j) { return t.A_ex[(i - 1) * AP_DVM_MAX_STAGES + (j - 1)]; };
  auto AIM = [&](int i, int j) { return t.A_im[(i - 1) * AP_DVM_MAX_STAGES + (j - 1)]; };
  if (f32) {
    void* a[] = {&bp};
    if ((st = launch(K.km.k_unpack, K.g_finish, blk, 0, a, KK_UNPACK))) return st;
  }
  for (int i = 2; i <= s; ++i) {
    int j = i - 1;
    unsigned need = 32u;                                   // v^(i), step 1 of stage i
    for (int k = j + 1; k <= s; ++k) {
      if (AEX(k, j) != 0.0) need |= 1u;                    // E^(j)
      if (AIM(k, j) != 0.0) need |= 2u | 4u | 8u | 16u;    // D0.u, D_Delta theta, D0 theta, D_LF.B(v) of stage j
    }
    if (j == 1) need |= 2u;                                // D0 . u^n enters every right-hand side
    {
      void* a[] = {&bp, &j, &need, &weno_eps};
      if ((st = launch(K.ks.k_explicit, K.g_explicit, blk, K.ks.smem_explicit, a, KK_EXPLICIT))) return st;
    }
    double sign = -1.0;                                    // reading G4
    int first = (i == 2) ? 1 : 0;
    {
      void* a[] = {&bp, &i, &sign, &first};
      if ((st = launch(K.ks.k_rhs, K.g_rhs, blk, K.ks.smem_rhs, a, KK_RHS))) return st;
    }
    {
      void* a[] = {&bp};
      if ((st = launch(K.km.k_rows_fwd, K.g_fft, dim3(256), K.fft_smem, a, KK_ROWS_FWD))) return st;
      void* b[] = {&bp, &i};
      if ((st = launch(K.km.k_cols, K.g_fft, dim3(256), K.fft_smem, b, KK_COLS))) return st;
      if ((st = launch(K.km.k_rows_inv, K.g_fft, dim3(256), K.fft_smem, b, KK_ROWS_INV))) return st;
    }
    {
      void* a[] = {&bp, &i, &weno_eps};
      if ((st = launch(K.ks.k_update, K.g_update, blk, K.ks.smem_update, a, KK_UPDATE))) return st;
    }
  }
  void* a[] = {&bp, &f32};
  return launch(K.km.k_finish, K.g_finish, blk, 0, a, KK_FINISH);
}

// Fill the derived per-instance constants of a descriptor from its parameters.
inline void fill_constants(const ap_dvm_params& p, InstDev& d) {
  d.dx = p.Lx / p.nx;
  d.dy = p.Ly / p.ny;
  d.dt = p.dt;
  d.eps = p.eps;
  d.tau = p.tau < 0 ? 4.0 * p.eps / p.mach : p.tau;
  d.te2 = d.tau * p.eps * p.eps;
  d.rho0 = p.rho0;
  d.amp = p.mach;
  for (int i = 2; i <= p.s; ++i) {
    const double a = p.A_im[(i - 1) * AP_DVM_MAX_STAGES + (i - 1)];
    d.kappa[i] = 2.0 * p.eps * p.eps / (p.dt * p.dt * a * a);
    d.den[i] = d.te2 + p.dt * a;
    d.inv_den[i] = 1.0 / d.den[i];
  }
  d.inv_dx = 1.0 / d.dx;
  d.inv_dy = 1.0 / d.dy;
  for (int i = 2; i <= p.s; ++i) {
    const double aii = p.A_im[(i - 1) * AP_DVM_MAX_STAGES + (i - 1)];
    d.c_dun[i] = 1.0 / (p.dt * aii);
    d.inv_aii[i] = 1.0 / aii;
    for (int j = 1; j <= i; ++j) {
      const double a = p.A_im[(i - 1) * AP_DVM_MAX_STAGES + (j - 1)];
      d.c_du[i][j] = a / (p.dt * aii * aii);
      d.c_db[i][j] = a / aii;
      d.c_lth[i][j] = -1.0 * (a / aii);
    }
  }
  const double ra = 1.0 / (p.rho0 * p.mach);
  d.sc_u = ra;
  d.sc_th = p.eps > 0 ? ra / (2.0 * p.eps) : 0.0;
  d.sc_v = p.eps > 0 ? ra / p.eps : 0.0;
  d.sc_q = p.eps > 0 ? ra / (p.eps * p.eps) : 0.0;
}

}  // namespace apd
