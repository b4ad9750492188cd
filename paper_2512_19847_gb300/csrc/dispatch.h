// Kernel tables shared between the instantiation units and the host API.
#pragma once
#include <cstddef>
#include <cuda_runtime.h>

namespace apd {

// Tile shapes of the stencil kernels (index = ap_dvm_set_tile argument).
constexpr int kNumTiles = 6;
constexpr int kTileX[kNumTiles] = {32, 32, 16, 8, 64, 32};
constexpr int kTileY[kNumTiles] = {8, 4, 8, 8, 4, 16};

struct StencilSet {
  const void* k_explicit;
  const void* k_rhs;
  const void* k_update;
  size_t smem_explicit;
  int rhs_threads;                     // k_rhs: threads per block (no dynamic shared memory)
  size_t plane_bytes, update_fixed;   // k_update: update_fixed + nbuf * (planes staged) * plane_bytes
  int nbuf;                            // staged plane buffers of k_update (1 or 2)
  int tx, ty;
  int bw, bh;                          // staged box: (tx + 8) x (ty + 2 * halo)
};

struct MiscSet {
  const void* k_finish;    // per tile shape
  const void* k_stage1;    // per tile shape; type-A tableaux only
  const void* k_rows_fwd;    // Helmholtz transforms, power-of-two axes ...
  const void* k_cols;
  int cols_threads;        // threads per block of k_cols
  int rows_threads;        // threads per block of k_rows_fwd and k_rows_inv
  const void* k_rows_inv;
  const void* k_rows_fwd_bs; // ... and axes of other lengths (Bluestein)
  const void* k_cols_bs;
  const void* k_rows_inv_bs;
  const void* k_set_state;
  const void* k_get_state;
  const void* k_diagnostics;
};

StencilSet stencil_f64_lf1(int tile);
StencilSet stencil_f64_w3(int tile);
StencilSet stencil_f64_w5(int tile);
StencilSet stencil_f32_lf1(int tile);
StencilSet stencil_f32_w3(int tile);
StencilSet stencil_f32_w5(int tile);
MiscSet misc_set(int f32form, int tile);
// One kernel whose bounded wait expires after limit_ns (sets the timeout bit of err).
cudaError_t launch_wait_timeout(unsigned* err, unsigned long long limit_ns, cudaStream_t stream);
// The integer-pipe FP32 <-> FP64 conversions against the instructions (ap_dvm_check_conversions).
cudaError_t launch_check_conversions(const double* in, int n, unsigned* bad, cudaStream_t stream);

}  // namespace apd
