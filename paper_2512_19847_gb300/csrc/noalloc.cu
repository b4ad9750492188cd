// ap_dvm_step_noalloc: IMEX steps of one small FP64 solve with all scratch
// in a file-scope device array, for callers that cannot allocate device
// memory (see include/ap_dvm.h).  It reuses the library's kernels, the launch
// sequence of one step (step_plan.h) and the workspace carving of the handle
// path (workspace.h) unchanged; only the placement of the scratch lives here.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "../../include/ap_dvm.h"
#include "common.cuh"
#include "dispatch.h"
#include "step_plan.h"
#include "workspace.h"

using namespace apd;

namespace {

constexpr int kMaxCells = 128 * 128;                 // largest grid accepted (nx * ny)
constexpr size_t kScratchBytes = size_t(8) << 20;   // 8 MiB
constexpr int kMaxDevices = 64;

// The scratch every call uses.  In host code its name is only a stand-in;
// the device address comes from cudaGetSymbolAddress at set-up.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

void* g_scratch_ptr[kMaxDevices] = {nullptr};

// Layout of the scratch: batch tables, then the instance's planes.
struct Layout {
  size_t batch, inst, tile_start, row_start, col_start, rhs_start, counts, tw, err, ws;
  size_t total;
};

Layout layout(const ap_dvm_params& p, int nmax) {
  Layout L{};
  size_t off = 0;
  auto take = [&](size_t b) { off = align_up(off, 256); size_t r = off; off += b; return r; };
  L.batch = take(sizeof(BatchDev));
  L.inst = take(sizeof(InstDev));
  L.tile_start = take(2 * sizeof(int));
  L.row_start = take(2 * sizeof(int));
  L.col_start = take(2 * sizeof(int));
  L.rhs_start = take(2 * sizeof(int));
  L.counts = take(5 * sizeof(int));
  L.tw = take(sizeof(double2) * (nmax / 2));
  L.err = take(4 * sizeof(unsigned));
  L.ws = take(carve_instance(p, nullptr, nullptr));
  L.total = align_up(off, 256);
  return L;
}

cudaError_t grid_of(const void* fn, int threads, size_t smem, int sms, int* grid) {
  cudaError_t e = cudaSuccess;
  if (smem > 48 * 1024) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads, smem);
  if (e != cudaSuccess) return e;
  *grid = std::max(1, per) * sms;
  return cudaSuccess;
}

}  // namespace

#define NA_TRY(call)                                   \
  do {                                                 \
    if ((call) != cudaSuccess) return AP_DVM_ERR_CUDA; \
  } while (0)

extern "C" ap_dvm_status ap_dvm_step_noalloc(const ap_dvm_params* p, double* d_state6, int nsteps, void* cuda_stream) {
  if (!p || !d_state6 || nsteps < 0) return AP_DVM_ERR_ARG;
  if (ap_dvm_instance_workspace_size(p) == 0) return AP_DVM_ERR_ARG;           // invalid parameters or tableau
  if (p->precision != AP_DVM_FP64) return AP_DVM_ERR_UNSUPPORTED;
  if (p->nx > 128 || p->ny > 128 || (long)p->nx * p->ny > kMaxCells) return AP_DVM_ERR_ARG;  // beyond the static scratch
  if ((p->nx & (p->nx - 1)) || (p->ny & (p->ny - 1))) return AP_DVM_ERR_UNSUPPORTED;         // powers of two only
  const int nmax = std::max(p->nx, p->ny);
  const Layout L = layout(*p, nmax);
  if (L.total > kScratchBytes) return AP_DVM_ERR_ARG;
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(cuda_stream);

  // set-up, once per device, with that device current
  int dev = 0;
  NA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return AP_DVM_ERR_UNSUPPORTED;
  if (!g_scratch_ptr[dev]) {
    void* ptr = nullptr;
    NA_TRY(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
    g_scratch_ptr[dev] = ptr;
  }
  char* base = reinterpret_cast<char*>(g_scratch_ptr[dev]);
  int sms = 0;
  NA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));

  // kernels: the tile rule of the handle path (largest of 32x8, 32x4, 16x8, 8x8 that fits)
  int tile = 3;
  for (int t : {0, 1, 2, 3})
    if (kTileX[t] <= p->nx && kTileY[t] <= p->ny) { tile = t; break; }
  StencilSet ks = p->space_scheme == AP_DVM_LF1_C2 ? stencil_f64_lf1(tile)
                : p->space_scheme == AP_DVM_WENO3_C4 ? stencil_f64_w3(tile) : stencil_f64_w5(tile);
  MiscSet km = misc_set(0, tile);
  const int eblk = fft_eblk(nmax), eblk_cols = fft_eblk_cols(nmax, false);
  const size_t fft_smem = fft_block_bytes(eblk, false), cols_smem = fft_block_bytes(eblk_cols, false);
  const int thr = ks.tx * ks.ty;
  int g_exp = 0, g_rhs = 0, g_upd = 0, g_fin = 0, g1 = 0, g2 = 0, g3 = 0;
  NA_TRY(grid_of(ks.k_explicit, thr, ks.smem_explicit, sms, &g_exp));
  NA_TRY(grid_of(ks.k_rhs, ks.rhs_threads, 0, sms, &g_rhs));
  const size_t smem_upd = update_smem(ks, *p);
  NA_TRY(grid_of(ks.k_update, thr, smem_upd, sms, &g_upd));
  NA_TRY(grid_of(km.k_finish, thr, 0, sms, &g_fin));
  NA_TRY(grid_of(km.k_rows_fwd, km.rows_threads, fft_smem, sms, &g1));
  NA_TRY(grid_of(km.k_cols, km.cols_threads, cols_smem, sms, &g2));
  NA_TRY(grid_of(km.k_rows_inv, km.rows_threads, fft_smem, sms, &g3));
  const int g_fft = std::min(g1, g3);

  // descriptors, built on the host stack and copied into the scratch
  InstDev I{};
  carve_instance(*p, base + L.ws, &I);
  I.nx = p->nx; I.ny = p->ny; I.lnx = ilog2(p->nx); I.lny = ilog2(p->ny);
  I.tiles_x = p->nx / ks.tx; I.tiles_y = p->ny / ks.ty;
  I.row_pairs = std::max(1, std::min(eblk / p->nx, p->ny / 2));
  I.col_group = std::min(2, std::max(1, eblk_cols / p->ny));   // the handle path's rule (FP64)
  I.relax64 = 0;
  fill_constants(*p, I);
  CUtensorMap maps[APD_MAXS + 1];
  I.tma = encode_stage_maps(*p, I, ks.bw, ks.bh, maps);
  BatchDev B{};
  B.inst = reinterpret_cast<InstDev*>(base + L.inst);
  B.tile_start = reinterpret_cast<int*>(base + L.tile_start);
  B.row_start = reinterpret_cast<int*>(base + L.row_start);
  B.col_start = reinterpret_cast<int*>(base + L.col_start);
  B.rhs_start = reinterpret_cast<int*>(base + L.rhs_start);
  B.counts = reinterpret_cast<int*>(base + L.counts);
  B.tw = reinterpret_cast<double2*>(base + L.tw);
  B.lnmax = ilog2(nmax);
  B.s = p->s;
  fill_tableau(*p, B);
  B.err = reinterpret_cast<unsigned*>(base + L.err);
  const int ntiles = I.tiles_x * I.tiles_y;
  const int nrows = (p->ny / 2 + I.row_pairs - 1) / I.row_pairs;
  const int ncols = (p->nx / 2 + 1 + I.col_group - 1) / I.col_group;
  const int nrhs = rhs_items(p->nx, p->ny, false);
  const int ts[2] = {0, ntiles}, rs[2] = {0, nrows}, cs[2] = {0, ncols}, hs[2] = {0, nrhs};
  const int counts[5] = {ntiles, nrows, ncols, 1, nrhs};
  double2 tw[64];                                   // nmax/2 <= 64 for grids of at most 128 cells a side
  double lx[65], ly[128];
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int k = 0; k < nmax / 2; ++k) {
    const long double a = -2.0L * pi * (long double)k / (long double)nmax;
    tw[k].x = (double)std::cos(a);
    tw[k].y = (double)std::sin(a);
  }
  laplacian_symbol(p->nx, I.dx, p->space_scheme, lx, p->nx / 2 + 1);
  laplacian_symbol(p->ny, I.dy, p->space_scheme, ly, p->ny);
  NA_TRY(cudaMemcpyAsync(base + L.batch, &B, sizeof(B), cudaMemcpyHostToDevice, stream));
  NA_TRY(cudaMemcpyAsync(base + L.inst, &I, sizeof(I), cudaMemcpyHostToDevice, stream));
  NA_TRY(cudaMemcpyAsync(B.tile_start, ts, sizeof(ts), cudaMemcpyHostToDevice, stream));
  NA_TRY(cudaMemcpyAsync(B.row_start, rs, sizeof(rs), cudaMemcpyHostToDevice, stream));
  NA_TRY(cudaMemcpyAsync(B.col_start, cs, sizeof(cs), cudaMemcpyHostToDevice, stream));
  NA_TRY(cudaMemcpyAsync(B.rhs_start, hs, sizeof(hs), cudaMemcpyHostToDevice, stream));
  NA_TRY(cudaMemcpyAsync(B.counts, counts, sizeof(counts), cudaMemcpyHostToDevice, stream));
  NA_TRY(cudaMemcpyAsync(B.tw, tw, sizeof(double2) * (nmax / 2), cudaMemcpyHostToDevice, stream));
  NA_TRY(cudaMemcpyAsync(I.lamx, lx, sizeof(double) * (p->nx / 2 + 1), cudaMemcpyHostToDevice, stream));
  NA_TRY(cudaMemcpyAsync(I.lamy, ly, sizeof(double) * p->ny, cudaMemcpyHostToDevice, stream));
  NA_TRY(cudaMemsetAsync(B.err, 0, 4 * sizeof(unsigned), stream));
  if (I.tma)
    NA_TRY(cudaMemcpyAsync(const_cast<void*>(I.tmap), maps, sizeof(maps), cudaMemcpyHostToDevice, stream));
  NA_TRY(cudaMemcpyAsync(I.X, d_state6, 6 * sizeof(double) * p->nx * p->ny, cudaMemcpyDeviceToDevice, stream));
  NA_TRY(cudaStreamSynchronize(stream));            // the host-stack sources above go out of scope

  // the steps: the launch sequence of one IMEX step shared with the handle path
  BatchDev* bp = reinterpret_cast<BatchDev*>(base + L.batch);
  StepKernels K{ks, km, g_exp, g_rhs, g_upd, g_fin, g_fft, g2, km.cols_threads, fft_smem, cols_smem, smem_upd, FFT_X_POW2 | FFT_Y_POW2,
                g_fft};
  auto ln = [&](const void* fn, int grid, dim3 block, size_t smem, void** args, int) -> int {
    return cudaLaunchKernel(fn, dim3(grid), block, args, smem, stream) == cudaSuccess ? 0 : (int)AP_DVM_ERR_CUDA;
  };
  for (int step = 0; step < nsteps; ++step) {
    const int st = enqueue_imex_step(*p, K, bp, 0, ln);
    if (st) return (ap_dvm_status)st;
  }
  NA_TRY(cudaMemcpyAsync(d_state6, I.X, 6 * sizeof(double) * p->nx * p->ny, cudaMemcpyDeviceToDevice, stream));

  // the device error flags of these steps (bit 1: a bounded tile-copy wait expired, bit 0:
  // a non-finite state), read before the next call clears them
  unsigned flags = 0;
  NA_TRY(cudaMemcpyAsync(&flags, B.err, sizeof(unsigned), cudaMemcpyDeviceToHost, stream));
  NA_TRY(cudaStreamSynchronize(stream));
  if (flags & 2u) return AP_DVM_ERR_TIMEOUT;
  if (flags & 1u) return AP_DVM_ERR_NONFINITE;
  return AP_DVM_OK;
}
