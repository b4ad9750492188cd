// The launch sequence of one IMEX step (Algorithm 1, CK/ARS tableau with
// stage 1 = X^n, GSA close), shared by the handle path and the
// no-allocation entry point.
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cstdlib>

#include "../../include/ap_dvm.h"
#include "common.cuh"
#include "dispatch.h"

namespace apd {

enum KernelKind { KK_EXPLICIT, KK_RHS, KK_ROWS_FWD, KK_COLS, KK_ROWS_INV, KK_UPDATE, KK_FINISH, KK_STAGE1 };

// Kinds of Helmholtz transform work a batch holds (bits of StepKernels::fft_kinds).
enum FftKinds { FFT_X_POW2 = 1, FFT_X_BS = 2, FFT_Y_POW2 = 4, FFT_Y_BS = 8 };

// Transform launches of one implicit stage for the given kinds.
inline int fft_launches(unsigned kinds) {
  return 2 * (((kinds & FFT_X_POW2) ? 1 : 0) + ((kinds & FFT_X_BS) ? 1 : 0)) + ((kinds & FFT_Y_POW2) ? 1 : 0) +
         ((kinds & FFT_Y_BS) ? 1 : 0);
}

struct StepKernels {
  StencilSet ks;
  MiscSet km;
  int g_explicit, g_rhs, g_update, g_finish, g_fft, g_cols, cols_threads;
  size_t fft_smem, cols_smem;   // the power-of-two column pass has its own (wider) work items
  size_t smem_update;
  unsigned fft_kinds;   // FftKinds present among the attached solves
  int g_rows;           // grid of the power-of-two row passes (km.rows_threads threads per block)
};

// Planes k_update stages at its largest stage: theta, v1, v2 and u1, u2 of every
// earlier stage entering the dissipation partner (the explicit-weight predictor
// (1/a_ii) sum_{j<i} (atilde_ij - a_ij) u^(j)).
inline int update_planes_max(const ap_dvm_params& t) {
  int best = 0;
  for (int i = 1; i <= t.s; ++i) {
    int np = 3;
    for (int j = 1; j < i; ++j)
      if (t.A_ex[(i - 1) * AP_DVM_MAX_STAGES + (j - 1)] - t.A_im[(i - 1) * AP_DVM_MAX_STAGES + (j - 1)] != 0.0) np += 2;
    if (np > best) best = np;
  }
  return best;
}

// Shared memory of the transform kernels: every pass of a batch takes work items of
// at most eblk complex values (eblk_cols for the power-of-two column pass), padded in
// the power-of-two kernels (one spare value per 16 FP32 or 8 FP64 complex values).
inline size_t fft_block_bytes(int elems, bool f32) {
  const int ps = f32 ? 4 : 3;
  return (size_t)(elems + (elems >> ps) + 1) * (f32 ? 8 : 16);
}
// Complex values per work item: rows and the other-length kernels eblk (at least
// one transform of the longest length), the power-of-two column pass a few
// adjacent columns (coalesced loads): 8192 values (64 KB) in FP32, 4096 in FP64.
inline int fft_eblk(int nmax) { return nmax > 2048 ? nmax : 2048; }
inline int fft_eblk_cols(int nmax, bool f32) {
  const int e = f32 ? 8192 : 4096;
  return nmax > e ? nmax : e;
}

inline size_t update_smem(const StencilSet& ks, const ap_dvm_params& t) {
  return ks.update_fixed + (size_t)ks.nbuf * update_planes_max(t) * ks.plane_bytes;
}

// Tensor maps of the stage buffers of one instance for TMA staging: map j
// (j = 1: the state X, j >= 2: X^(j)) describes 6 planes of nx x ny values as a
// 3D tensor (x, y, plane) with a box of bw x bh x 1.  Writes s+1 maps to out
// (64-byte aligned) and returns 1, or 0 when TMA is not used for this
// instance (grid smaller than the box, no driver entry point, or the
// environment variable AP_DVM_NO_TMA set).
inline int encode_stage_maps(const ap_dvm_params& p, const InstDev& d, int bw, int bh, CUtensorMap* out) {
  if (std::getenv("AP_DVM_NO_TMA")) return 0;
  if (p.nx < bw || p.ny < bh) return 0;
  // a tensor map's row stride must be a multiple of 16 bytes: other widths stage with plain loads
  if ((size_t)p.nx * (p.precision == AP_DVM_FP64 ? 8 : 4) % 16 != 0) return 0;
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return 0;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const bool f64 = p.precision == AP_DVM_FP64;
  const size_t es = f64 ? 8 : 4;
  const cuuint64_t dims[3] = {(cuuint64_t)p.nx, (cuuint64_t)p.ny, 6};
  const cuuint64_t strides[2] = {(cuuint64_t)p.nx * es, (cuuint64_t)p.nx * p.ny * es};
  const cuuint32_t box[3] = {(cuuint32_t)bw, (cuuint32_t)bh, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  for (int j = 1; j <= p.s; ++j) {
    void* base = d.Xs[j];
    const CUresult r = encode(&out[j], f64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims,
                              strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return 0;
  }
  return 1;
}

// launch(fn, grid, block, smem, args, kind) -> int status (0 = success); form = the precision form
// (AP_DVM_FP64, AP_DVM_FP32_DEV, AP_DVM_FP32_DEV_TH), passed to the finish kernel
// fused: the last stage's update closes the step into the other state buffer
// (I.Xnext; the handle path's double-buffered state), else a finish kernel
// closes it in place.
template <class Launch>
int enqueue_imex_step(const ap_dvm_params& t, const StepKernels& K, BatchDev* bp, int form, Launch&& launch,
                      bool fused = false) {
  const int s = t.s;
  const dim3 blk(K.ks.tx, K.ks.ty);
  double weno_eps = t.weno_eps;
  int st;
  auto AEX = [&](int i, int j) { return t.A_ex[(i - 1) * AP_DVM_MAX_STAGES + (j - 1)]; };
  auto AIM = [&](int i, int j) { return t.A_im[(i - 1) * AP_DVM_MAX_STAGES + (j - 1)]; };
  // type-A tableaux (a_11 != 0) compute stage 1 with the four steps; CK/ARS take X^(1) = X^n
  const bool type_a = AIM(1, 1) != 0.0;
  if (type_a) {
    int c4 = t.space_scheme != AP_DVM_LF1_C2;
    void* a[] = {&bp, &c4};
    if ((st = launch(K.km.k_stage1, K.g_finish, blk, 0, a, KK_STAGE1))) return st;
  }
  for (int i = type_a ? 1 : 2; i <= s; ++i) {
    int j = i - 1;
    unsigned need = 32u;                                   // v^(i), step 1 of stage i
    for (int k = j + 1; k <= s; ++k) {
      if (AEX(k, j) != 0.0) need |= 1u;                    // E^(j)
      if (AIM(k, j) != 0.0) need |= 2u | 4u | 16u;        // D0.u, D_Delta theta, D_LF.B(v) + D0 theta of stage j
    }
    if (j == 1 && !type_a) need |= 2u;                     // D0 . u^n (= D0 . u^(1)) enters every right-hand side
    if (j >= 1) {
      void* a[] = {&bp, &j, &need, &weno_eps};
      if ((st = launch(K.ks.k_explicit, K.g_explicit, blk, K.ks.smem_explicit, a, KK_EXPLICIT))) return st;
    }
    double sign = -1.0;   // theta-history term with a minus sign (the stage equations of Sec. 3.1)
    int first = (i == (type_a ? 1 : 2)) ? 1 : 0;           // the first right-hand side also sums theta^n
    {
      void* a[] = {&bp, &i, &sign, &first};
      if ((st = launch(K.ks.k_rhs, K.g_rhs, dim3(K.ks.rhs_threads), 0, a, KK_RHS))) return st;
    }
    {
      // each pass: the power-of-two kernel and/or the Bluestein kernel, as the batch needs
      void* a[] = {&bp};
      void* b[] = {&bp, &i};
      const unsigned kk = K.fft_kinds;
      if ((kk & FFT_X_POW2) && (st = launch(K.km.k_rows_fwd, K.g_rows, dim3(K.km.rows_threads), K.fft_smem, a, KK_ROWS_FWD))) return st;
      if ((kk & FFT_X_BS) && (st = launch(K.km.k_rows_fwd_bs, K.g_fft, dim3(256), K.fft_smem, a, KK_ROWS_FWD))) return st;
      if ((kk & FFT_Y_POW2) && (st = launch(K.km.k_cols, K.g_cols, dim3(K.cols_threads), K.cols_smem, b, KK_COLS))) return st;
      if ((kk & FFT_Y_BS) && (st = launch(K.km.k_cols_bs, K.g_fft, dim3(256), K.fft_smem, b, KK_COLS))) return st;
      if ((kk & FFT_X_POW2) && (st = launch(K.km.k_rows_inv, K.g_rows, dim3(K.km.rows_threads), K.fft_smem, b, KK_ROWS_INV))) return st;
      if ((kk & FFT_X_BS) && (st = launch(K.km.k_rows_inv_bs, K.g_fft, dim3(256), K.fft_smem, b, KK_ROWS_INV))) return st;
    }
    {
      int close = (fused && i == s) ? 1 : 0;
      void* a[] = {&bp, &i, &weno_eps, &close, &form};
      if ((st = launch(K.ks.k_update, K.g_update, blk, K.smem_update, a, KK_UPDATE))) return st;
    }
  }
  if (fused) return 0;
  void* a[] = {&bp, &form};
  return launch(K.km.k_finish, K.g_finish, blk, 0, a, KK_FINISH);
}

// Fill the derived per-instance constants of a descriptor from its parameters.
// Stage coefficients of one instance, computed in FP64 and rounded once to T.
template <typename T>
inline void fill_coef(const ap_dvm_params& p, const InstDev& d, Coef<T>& k) {
  k = Coef<T>{};
  k.dt = T(d.dt);
  k.te2 = T(d.te2);
  k.qtau = T(0.25) * T(d.tau);
  k.htau = T(0.5 * d.tau);
  k.inv_dx = T(d.inv_dx);
  k.inv_dy = T(d.inv_dy);
  for (int i = 1; i <= p.s; ++i)
    for (int j = 1; j <= p.s; ++j) {
      k.aex[i][j] = T(p.A_ex[(i - 1) * AP_DVM_MAX_STAGES + (j - 1)]);
      k.aim[i][j] = T(p.A_im[(i - 1) * AP_DVM_MAX_STAGES + (j - 1)]);
    }
  for (int i = 1; i <= p.s; ++i) {
    const double aii = p.A_im[(i - 1) * AP_DVM_MAX_STAGES + (i - 1)];
    if (aii == 0.0) continue;                     // stage 1 of a CK/ARS tableau is X^n
    k.kappa[i] = T(d.kappa[i]);
    k.r_n[i] = T(d.te2 * d.inv_den[i]);
    k.c_dun[i] = T(1.0 / (p.dt * aii));
    for (int j = 1; j <= i; ++j) {
      const double a = p.A_im[(i - 1) * AP_DVM_MAX_STAGES + (j - 1)];
      const double ae = p.A_ex[(i - 1) * AP_DVM_MAX_STAGES + (j - 1)];
      k.c_du[i][j] = T(a / (p.dt * aii * aii));
      k.c_db[i][j] = T(a / aii);
      k.c_lth[i][j] = T(-1.0 * (a / aii));
      k.wp[i][j] = T((ae - a) * d.inv_aii[i]);
      k.rv_e[i][j] = T(-p.dt * ae * d.inv_den[i]);
      k.rv_v[i][j] = T(-p.dt * a * d.inv_den[i]);
      k.rq_d[i][j] = T(-p.dt * a * (0.5 * d.tau) * d.inv_den[i]);
    }
  }
}

// Tableau of a batch and the nonzero patterns of its rows.
inline void fill_tableau(const ap_dvm_params& p, BatchDev& b) {
  for (int k = 0; k < APD_MAXS * APD_MAXS; ++k) {
    b.A_ex[k] = p.A_ex[k];
    b.A_im[k] = p.A_im[k];
  }
  for (int i = 1; i <= APD_MAXS; ++i) {
    b.m_ex[i] = b.m_im[i] = b.m_wp[i] = 0u;
    for (int j = 1; j <= APD_MAXS; ++j) {
      const double ae = p.A_ex[(i - 1) * AP_DVM_MAX_STAGES + (j - 1)];
      const double ai = p.A_im[(i - 1) * AP_DVM_MAX_STAGES + (j - 1)];
      if (ae != 0.0) b.m_ex[i] |= 1u << j;
      if (ai != 0.0 && j <= i) b.m_im[i] |= 1u << j;
      if (ae - ai != 0.0 && j < i) b.m_wp[i] |= 1u << j;
    }
  }
  b.m_ex[0] = b.m_im[0] = b.m_wp[0] = 0u;
}

inline void fill_constants(const ap_dvm_params& p, InstDev& d) {
  d.dx = p.Lx / p.nx;
  d.dy = p.Ly / p.ny;
  d.dt = p.dt;
  d.eps = p.eps;
  d.tau = p.tau < 0 ? 4.0 * p.eps / p.mach : p.tau;
  d.te2 = d.tau * p.eps * p.eps;
  d.rho0 = p.rho0;
  d.amp = p.mach;
  d.eps32 = (float)p.eps;
  d.rho032 = (float)p.rho0;
  d.amp32 = (float)p.mach;
  for (int i = 1; i <= p.s; ++i) {
    const double a = p.A_im[(i - 1) * AP_DVM_MAX_STAGES + (i - 1)];
    if (a == 0.0) continue;
    d.kappa[i] = 2.0 * p.eps * p.eps / (p.dt * p.dt * a * a);
    d.den[i] = d.te2 + p.dt * a;
    d.inv_den[i] = 1.0 / d.den[i];
  }
  d.inv_dx = 1.0 / d.dx;
  d.inv_dy = 1.0 / d.dy;
  d.hscale32 = (float)(1.0 / ((double)p.nx * (double)p.ny));
  for (int i = 1; i <= p.s; ++i) {
    const double a = p.A_im[(i - 1) * AP_DVM_MAX_STAGES + (i - 1)];
    d.inv_aii[i] = a != 0.0 ? 1.0 / a : 0.0;
  }
  fill_coef(p, d, d.k64);
  fill_coef(p, d, d.k32);
  const double ra = 1.0 / (p.rho0 * p.mach);
  d.sc_u = ra;
  d.sc_th = p.eps > 0 ? ra / (2.0 * p.eps) : 0.0;
  d.sc_v = p.eps > 0 ? ra / p.eps : 0.0;
  d.sc_q = p.eps > 0 ? ra / (p.eps * p.eps) : 0.0;
  const double sq3 = 1.7320508075688772935;
  d.pmc[0] = d.sc_u;
  d.pmc[1] = 0.5 * d.sc_u;
  d.pmc[2] = 0.5 * sq3 * d.sc_u;
  d.pmc[3] = d.sc_th;
  d.pmc[4] = -0.5 * d.sc_v;
  d.pmc[5] = 0.25 * d.sc_v;
  d.pmc[6] = 0.25 * sq3 * d.sc_v;
  d.pmc[7] = 0.25 * d.sc_q;
}

}  // namespace apd
