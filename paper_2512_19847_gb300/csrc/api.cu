// Host side of the C ABI declared in include/ap_dvm.h.
//
// A handle is a batch: a fixed tableau, scheme and precision, and up to
// `capacity` attached solves, each with its own caller-owned workspace.  The
// per-instance descriptors and the prefix sums of the work decomposition
// live in the batch workspace; every kernel of a step is launched once for
// all attached solves.  One IMEX step (Algorithm 1) enqueues, for a type-A
// tableau first k_stage1 (v^(1), D_0 . u^n), then for each computed stage i
// (i = 1..s for type A; i = 2..s for CK/ARS, whose stage 1 is X^n):
//   k_explicit(i-1)  explicit terms and reusable operators of stage i-1, and step 1 (v^(i))
//   k_rhs(i)         the Helmholtz right-hand side of step 2
//   k_fft_rows_fwd, k_fft_cols(i), k_fft_rows_inv(i)   step 2 (theta^(i)); the _bs kernels
//                    of the same passes for axes whose length is not a power of two
//   k_update(i)      steps 3 and 4 (u^(i), q^(i)); the last stage's update also closes
//                    the step (GSA: X^{n+1} = X^(s); FP32 forms: pack the populations and
//                    sum the next step's moments), written to the other state buffer
// (k_finish closes the step instead only where no update of the last stage can: the
// no-allocation entry point, whose state is single-buffered).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/ap_dvm.h"
#include "common.cuh"
#include "dispatch.h"
#include "step_plan.h"
#include "workspace.h"

using namespace apd;

struct Slot {
  bool attached = false;
  ap_dvm_params p{};
  char* ws = nullptr;
  size_t bytes = 0;
  InstDev dev{};                        // as carved: X = state buffer 0, Xnext = buffer 1
  CUtensorMap maps[2][APD_MAXS + 1];    // host copies of the stage-buffer tensor maps, per parity
  int flip = 0;                         // the state is in buffer (handle parity) ^ flip
  bool paused = false;                  // left out of the steps (ap_dvm_step_slots)
};

// The instance as the kernels of a step of the given parity see it: the state
// is double-buffered (a step reads buffer q = parity ^ flip and closes into
// buffer q ^ 1; flip changes only while the slot sits out steps of
// ap_dvm_step_slots); stage 1 of a CK/ARS tableau is the state itself.
InstDev view(const Slot& s, int parity) {
  InstDev d = s.dev;
  const int q = parity ^ s.flip;
  void* buf[2] = {s.dev.X, s.dev.Xnext};
  d.X = buf[q];
  d.Xnext = buf[q ^ 1];
  if (s.p.A_im[0] == 0.0) {
    d.Xs[1] = d.X;
    d.Dun = d.Du[1];
  }
  d.tmap = reinterpret_cast<const char*>(s.dev.tmap) + (size_t)q * sizeof(CUtensorMap) * (APD_MAXS + 1);
  return d;
}

struct ap_dvm_handle {
  ap_dvm_params tmpl{};
  int capacity = 0;
  int f32 = 0;
  cudaStream_t stream = nullptr;
  int device = 0;
  int num_sms = 0;
  int tile = 0;
  bool tile_auto = true;
  int nmax = 0, lnmax = 0, eblk = 0, eblk_cols = 0;
  // batch workspace
  BatchDev* d_batch[2] = {nullptr, nullptr};   // per step parity (double-buffered state)
  InstDev* d_inst[2] = {nullptr, nullptr};
  int* d_tile_start = nullptr;
  int* d_row_start = nullptr;
  int* d_rhs_start = nullptr;
  int* d_col_start = nullptr;
  int* d_counts = nullptr;
  double2* d_tw = nullptr;
  float2* d_tw32 = nullptr;
  unsigned* d_err = nullptr;
  BatchDev hb[2]{};
  int parity = 0;                    // parity of the next step: which state buffer it reads
  std::vector<Slot> slots;
  bool dirty = true;
  int n_active = 0;
  // upload staging (kept alive across async copies)
  std::vector<InstDev> up_inst[2];
  std::vector<int> up_tiles, up_rows, up_cols, up_rhs;
  int up_counts[5] = {0, 0, 0, 0, 0};
  // kernels
  StencilSet ks{};
  MiscSet km{};
  int grid_explicit = 0, grid_rhs = 0, grid_update = 0, grid_fft = 0, grid_cols = 0, grid_finish = 0, grid_rows = 0;
  unsigned fft_kinds = 0;   // FftKinds of the attached solves (the launches a step enqueues)
  size_t smem_update = 0;
  bool kernels_ready = false;
  // graph
  int graph_steps = 0;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};   // per starting parity
  cudaStream_t cap_stream = nullptr;
  bool graph_valid[2] = {false, false};
  // per-kernel CUDA-event profile (direct launches only)
  bool profile = false;
  std::vector<cudaEvent_t> ev;
  std::vector<int> ev_kind;
  int ev_used = 0;
  double prof_ms[8] = {0};
  long prof_count[8] = {0};
  char err[512] = "";
};

namespace {

ap_dvm_status fail(ap_dvm_handle* h, ap_dvm_status st, const char* fmt, ...) {
  if (h) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(h->err, sizeof(h->err), fmt, ap);
    va_end(ap);
  }
  return st;
}

#define CUDA_TRY(h, call)                                                                                 \
  do {                                                                                                    \
    cudaError_t e_ = (call);                                                                              \
    if (e_ != cudaSuccess) return fail(h, AP_DVM_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));       \
  } while (0)

// Bluestein tables of an axis of n cells (n not a power of two) with
// convolution length m: the chirp exp(-i pi k^2 / n), k < n (k^2 reduced
// modulo 2n before the angle is formed), and the DFT of length m of the filter
// b_j = exp(i pi j^2 / n) for |j| < n (index j mod m), by radix-2 decimation in
// frequency, so in bit-reversed order, scaled by 1/m.
void bluestein_tables(int n, int m, std::vector<std::complex<long double>>& chirp,
                      std::vector<std::complex<long double>>& filt) {
  using CL = std::complex<long double>;
  const long double pi = 3.141592653589793238462643383279502884L;
  chirp.assign(n, CL(0, 0));
  for (int k = 0; k < n; ++k) {
    const long long r = ((long long)k * k) % (2LL * n);
    const long double a = pi * (long double)r / (long double)n;
    chirp[k] = CL(std::cos(a), -std::sin(a));
  }
  filt.assign(m, CL(0, 0));
  for (int j = 0; j < n; ++j) {
    filt[j] = std::conj(chirp[j]);
    if (j > 0) filt[m - j] = std::conj(chirp[j]);
  }
  std::vector<CL> tw(m / 2);
  for (int k = 0; k < m / 2; ++k) {
    const long double a = -2.0L * pi * (long double)k / (long double)m;
    tw[k] = CL(std::cos(a), std::sin(a));
  }
  for (int len = m; len >= 2; len >>= 1) {
    const int half = len >> 1, step = m / len;
    for (int s0 = 0; s0 < m; s0 += len)
      for (int j = 0; j < half; ++j) {
        const CL a = filt[s0 + j], b = filt[s0 + j + half];
        filt[s0 + j] = a + b;
        filt[s0 + j + half] = (a - b) * tw[(size_t)j * step];
      }
  }
  for (CL& z : filt) z /= (long double)m;
}

// Validates one solve's parameters; writes a message into buf.
ap_dvm_status validate(const ap_dvm_params* p, char* buf, size_t n) {
  if (!p) { snprintf(buf, n, "null parameters"); return AP_DVM_ERR_ARG; }
  if (p->nx < 8 || p->ny < 8 || p->nx > 4096 || p->ny > 4096) {
    snprintf(buf, n, "nx, ny must be in [8, 4096] (got %d, %d)", p->nx, p->ny);
    return AP_DVM_ERR_ARG;
  }
  if (!(p->Lx > 0) || !(p->Ly > 0)) { snprintf(buf, n, "Lx, Ly must be > 0"); return AP_DVM_ERR_ARG; }
  if (p->velocity_set != AP_DVM_D2V6) { snprintf(buf, n, "only the D2V6 velocity set exists (Sec. 2.1)"); return AP_DVM_ERR_ARG; }
  if (!(p->eps >= 0) || !std::isfinite(p->eps)) { snprintf(buf, n, "eps must be >= 0"); return AP_DVM_ERR_ARG; }
  if (!(p->mach > 0)) { snprintf(buf, n, "mach must be > 0"); return AP_DVM_ERR_ARG; }
  if (!(p->rho0 > 0)) { snprintf(buf, n, "rho0 must be > 0"); return AP_DVM_ERR_ARG; }
  if (!(p->dt > 0) || !std::isfinite(p->dt)) { snprintf(buf, n, "dt must be > 0"); return AP_DVM_ERR_ARG; }
  if (!std::isfinite(p->tau)) { snprintf(buf, n, "tau must be finite"); return AP_DVM_ERR_ARG; }
  if (p->space_scheme < AP_DVM_LF1_C2 || p->space_scheme > AP_DVM_WENO5_C4) { snprintf(buf, n, "unknown space_scheme"); return AP_DVM_ERR_ARG; }
  if (p->precision != AP_DVM_FP64 && p->precision != AP_DVM_FP32_DEV && p->precision != AP_DVM_FP32_DEV_TH) {
    snprintf(buf, n, "unknown precision");
    return AP_DVM_ERR_ARG;
  }
  const bool f32 = p->precision != AP_DVM_FP64;
  if (f32 && !(p->eps > 0)) { snprintf(buf, n, "the FP32 deviation form needs eps > 0 (population view)"); return AP_DVM_ERR_ARG; }
  if (!(p->weno_eps >= (f32 ? 1e-9 : 1e-30))) {
    snprintf(buf, n, "weno_eps must be >= 1e-30 (FP64) or >= 1e-9 (FP32 form)");
    return AP_DVM_ERR_ARG;
  }
  const int s = p->s;
  if (s < 2 || s > AP_DVM_MAX_STAGES) { snprintf(buf, n, "s must be in [2, %d]", AP_DVM_MAX_STAGES); return AP_DVM_ERR_TABLEAU; }
  auto ae = [&](int i, int j) { return p->A_ex[i * AP_DVM_MAX_STAGES + j]; };
  auto ai = [&](int i, int j) { return p->A_im[i * AP_DVM_MAX_STAGES + j]; };
  for (int i = 0; i < s; ++i)
    for (int j = 0; j < s; ++j) {
      if (!std::isfinite(ae(i, j)) || !std::isfinite(ai(i, j))) { snprintf(buf, n, "non-finite tableau entry"); return AP_DVM_ERR_TABLEAU; }
      if (j >= i && ae(i, j) != 0.0) { snprintf(buf, n, "explicit tableau must be strictly lower triangular"); return AP_DVM_ERR_TABLEAU; }
      if (j > i && ai(i, j) != 0.0) { snprintf(buf, n, "implicit tableau must be lower triangular (DIRK)"); return AP_DVM_ERR_TABLEAU; }
    }
  if (ai(0, 0) < 0.0) { snprintf(buf, n, "a_11 must be 0 (CK/ARS) or > 0 (type A)"); return AP_DVM_ERR_TABLEAU; }
  for (int i = 1; i < s; ++i)
    if (!(ai(i, i) > 0)) { snprintf(buf, n, "a_ii must be > 0 for i >= 2"); return AP_DVM_ERR_TABLEAU; }
  return AP_DVM_OK;
}

bool same_method(const ap_dvm_params& a, const ap_dvm_params& b) {
  if (a.s != b.s || a.space_scheme != b.space_scheme || a.precision != b.precision) return false;
  for (int k = 0; k < AP_DVM_MAX_STAGES * AP_DVM_MAX_STAGES; ++k)
    if (a.A_ex[k] != b.A_ex[k] || a.A_im[k] != b.A_im[k]) return false;
  return true;
}

size_t batch_bytes(int capacity, int nmax) {
  size_t off = 0;
  auto take = [&](size_t b) { off = align_up(off, 256); off += b; };
  take(sizeof(BatchDev) * 2);
  take(sizeof(InstDev) * capacity * 2);
  take(sizeof(int) * (capacity + 1));
  take(sizeof(int) * (capacity + 1));
  take(sizeof(int) * (capacity + 1));
  take(sizeof(int) * (capacity + 1));
  take(sizeof(int) * 5);
  take(sizeof(double2) * (nmax / 2));
  take(sizeof(float2) * (nmax / 2));
  take(sizeof(unsigned) * 4);
  return align_up(off, 256);
}

// FftKinds of the attached solves (of the template while none is attached).
unsigned fft_kinds_of(const ap_dvm_handle* h) {
  unsigned k = 0;
  auto add = [&](const ap_dvm_params& p) {
    k |= is_pow2(p.nx) ? FFT_X_POW2 : FFT_X_BS;
    k |= is_pow2(p.ny) ? FFT_Y_POW2 : FFT_Y_BS;
  };
  for (const Slot& s : h->slots)
    if (s.attached) add(s.p);
  if (!k) add(h->tmpl);
  return k;
}

int auto_tile(const ap_dvm_handle* h) {
  int minx = 1 << 30, miny = 1 << 30;
  for (const Slot& s : h->slots)
    if (s.attached) { minx = std::min(minx, s.p.nx); miny = std::min(miny, s.p.ny); }
  if (minx == (1 << 30)) { minx = h->tmpl.nx; miny = h->tmpl.ny; }
  for (int t : {0, 1, 2, 3})
    if (kTileX[t] <= minx && kTileY[t] <= miny) return t;
  return 3;
}

StencilSet stencil_for(int f32, int scheme, int tile) {
  if (!f32) {
    if (scheme == AP_DVM_LF1_C2) return stencil_f64_lf1(tile);
    if (scheme == AP_DVM_WENO3_C4) return stencil_f64_w3(tile);
    return stencil_f64_w5(tile);
  }
  if (scheme == AP_DVM_LF1_C2) return stencil_f32_lf1(tile);
  if (scheme == AP_DVM_WENO3_C4) return stencil_f32_w3(tile);
  return stencil_f32_w5(tile);
}

ap_dvm_status occupancy_grid(ap_dvm_handle* h, const void* fn, int threads, size_t smem, int* grid) {
  if (smem > 48 * 1024) CUDA_TRY(h, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  CUDA_TRY(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem));
  if (per_sm < 1) return fail(h, AP_DVM_ERR_UNSUPPORTED, "kernel does not fit on an SM (smem %zu)", smem);
  *grid = per_sm * h->num_sms;
  return AP_DVM_OK;
}

size_t fft_smem(const ap_dvm_handle* h) { return fft_block_bytes(h->eblk, h->f32); }
size_t cols_smem(const ap_dvm_handle* h) { return fft_block_bytes(h->eblk_cols, h->f32); }

ap_dvm_status prepare_kernels(ap_dvm_handle* h) {
  if (h->kernels_ready) return AP_DVM_OK;
  if (h->tile_auto) h->tile = auto_tile(h);
  h->ks = stencil_for(h->f32, h->tmpl.space_scheme, h->tile);
  h->km = misc_set(h->f32, h->tile);
  const int thr = h->ks.tx * h->ks.ty;
  ap_dvm_status st;
  if ((st = occupancy_grid(h, h->ks.k_explicit, thr, h->ks.smem_explicit, &h->grid_explicit))) return st;
  if ((st = occupancy_grid(h, h->ks.k_rhs, h->ks.rhs_threads, 0, &h->grid_rhs))) return st;
  h->smem_update = update_smem(h->ks, h->tmpl);
  if ((st = occupancy_grid(h, h->ks.k_update, thr, h->smem_update, &h->grid_update))) return st;
  if ((st = occupancy_grid(h, h->km.k_finish, thr, 0, &h->grid_finish))) return st;
  h->grid_fft = 1 << 30;
  for (const void* fn : {h->km.k_rows_fwd_bs, h->km.k_cols_bs, h->km.k_rows_inv_bs}) {
    int g = 0;
    if ((st = occupancy_grid(h, fn, 256, fft_smem(h), &g))) return st;
    h->grid_fft = std::min(h->grid_fft, g);
  }
  h->grid_rows = 1 << 30;
  for (const void* fn : {h->km.k_rows_fwd, h->km.k_rows_inv}) {
    int g = 0;
    if ((st = occupancy_grid(h, fn, h->km.rows_threads, fft_smem(h), &g))) return st;
    h->grid_rows = std::min(h->grid_rows, g);
  }
  if ((st = occupancy_grid(h, h->km.k_cols, h->km.cols_threads, cols_smem(h), &h->grid_cols))) return st;
  h->kernels_ready = true;
  h->graph_valid[0] = h->graph_valid[1] = false;
  return AP_DVM_OK;
}

// Rebuild and upload the compacted instance table and work decomposition.
ap_dvm_status flush(ap_dvm_handle* h) {
  ap_dvm_status st = prepare_kernels(h);
  if (st) return st;
  if (!h->dirty) return AP_DVM_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  CUDA_TRY(h, cudaStreamIsCapturing(h->stream, &cs));
  if (cs != cudaStreamCaptureStatusNone)
    return fail(h, AP_DVM_ERR_ARG, "the set of solves changed while the stream is being captured");
  const int TX = h->ks.tx, TY = h->ks.ty;
  const unsigned kinds = fft_kinds_of(h);
  if (kinds != h->fft_kinds) { h->fft_kinds = kinds; h->graph_valid[0] = h->graph_valid[1] = false; }   // the launch sequence changed
  h->up_inst[0].clear();
  h->up_inst[1].clear();
  h->up_tiles.assign(1, 0);
  h->up_rows.assign(1, 0);
  h->up_rhs.assign(1, 0);
  h->up_cols.assign(1, 0);
  for (Slot& s : h->slots) {
    if (!s.attached || s.paused) continue;
    if (s.p.nx < TX || s.p.ny < TY) return fail(h, AP_DVM_ERR_ARG, "grid %dx%d smaller than the tile %dx%d", s.p.nx, s.p.ny, TX, TY);
    InstDev& d = s.dev;
    d.tiles_x = (s.p.nx + TX - 1) / TX;   // ragged tiles at the high edges
    d.tiles_y = (s.p.ny + TY - 1) / TY;
    const int pairs = (s.p.ny + 1) / 2;   // row pairs (the last one single when ny is odd)
    d.row_pairs = std::max(1, std::min(h->eblk >> d.lnx, pairs));
    // power-of-two columns: as many adjacent columns per item as the item's buffer holds
    // (4 FP32 or 2 FP64 of 2048 cells: 32-byte row segments; more on shorter columns), up to
    // the power of two that covers the nx/2 + 1 spectral columns
    if (is_pow2(s.p.ny)) {
      const int cap = std::max(1, h->eblk_cols >> d.lny), nh = s.p.nx / 2 + 1;
      int g = 1;
      while (g < cap && g < nh) g <<= 1;
      d.col_group = g;
    } else {
      d.col_group = std::max(1, h->eblk >> d.lny);
    }
    for (int par = 0; par < 2; ++par) {   // the instance as steps of either parity see it
      InstDev v = view(s, par);
      // tensor maps of the stage buffers for the current tile shape (TMA staging)
      v.tma = encode_stage_maps(s.p, v, h->ks.bw, h->ks.bh, s.maps[par]);
      if (v.tma)
        CUDA_TRY(h, cudaMemcpyAsync(const_cast<void*>(v.tmap), &s.maps[par][0], sizeof(CUtensorMap) * (APD_MAXS + 1),
                                    cudaMemcpyHostToDevice, h->stream));
      h->up_inst[par].push_back(v);
    }
    h->up_tiles.push_back(h->up_tiles.back() + d.tiles_x * d.tiles_y);
    h->up_rows.push_back(h->up_rows.back() + (pairs + d.row_pairs - 1) / d.row_pairs);
    h->up_rhs.push_back(h->up_rhs.back() + rhs_items(s.p.nx, s.p.ny, h->f32));
    h->up_cols.push_back(h->up_cols.back() + (s.p.nx / 2 + 1 + d.col_group - 1) / d.col_group);
  }
  const int n = (int)h->up_inst[0].size();
  h->n_active = n;
  h->up_counts[0] = h->up_tiles.back();
  h->up_counts[1] = h->up_rows.back();
  h->up_counts[2] = h->up_cols.back();
  h->up_counts[3] = n;
  h->up_counts[4] = h->up_rhs.back();
  if (n > 0) {
    for (int par = 0; par < 2; ++par)
      CUDA_TRY(h, cudaMemcpyAsync(h->d_inst[par], h->up_inst[par].data(), sizeof(InstDev) * n, cudaMemcpyHostToDevice,
                                  h->stream));
    CUDA_TRY(h, cudaMemcpyAsync(h->d_tile_start, h->up_tiles.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(h, cudaMemcpyAsync(h->d_row_start, h->up_rows.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(h, cudaMemcpyAsync(h->d_rhs_start, h->up_rhs.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(h, cudaMemcpyAsync(h->d_col_start, h->up_cols.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, h->stream));
  }
  CUDA_TRY(h, cudaMemcpyAsync(h->d_counts, h->up_counts, sizeof(int) * 5, cudaMemcpyHostToDevice, h->stream));
  h->dirty = false;
  return AP_DVM_OK;
}

constexpr int kNumKinds = 8;
const char* const kKernelNames[kNumKinds] = {"explicit", "rhs",    "fft_rows_fwd", "fft_cols",
                                             "fft_rows_inv", "update", "finish",       "stage1"};

ap_dvm_status launch(ap_dvm_handle* h, cudaStream_t stream, const void* fn, int grid, dim3 block, size_t smem, void** args,
                     int kind = -1) {
  const bool prof = h->profile && kind >= 0;
  if (prof) {
    if (h->ev_used + 2 > (int)h->ev.size()) {
      for (int k = 0; k < 256; ++k) {
        cudaEvent_t e;
        CUDA_TRY(h, cudaEventCreate(&e));
        h->ev.push_back(e);
        h->ev_kind.push_back(-1);
      }
    }
    h->ev_kind[h->ev_used] = kind;
    CUDA_TRY(h, cudaEventRecord(h->ev[h->ev_used], stream));
  }
  CUDA_TRY(h, cudaLaunchKernel(fn, dim3(grid), block, args, smem, stream));
  if (prof) {
    CUDA_TRY(h, cudaEventRecord(h->ev[h->ev_used + 1], stream));
    h->ev_used += 2;
  }
  return AP_DVM_OK;
}

// Accumulate the elapsed times of the recorded event pairs (synchronises).
ap_dvm_status profile_collect(ap_dvm_handle* h) {
  if (h->ev_used == 0) return AP_DVM_OK;
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  for (int k = 0; k + 1 < h->ev_used; k += 2) {
    float ms = 0.f;
    CUDA_TRY(h, cudaEventElapsedTime(&ms, h->ev[k], h->ev[k + 1]));
    h->prof_ms[h->ev_kind[k]] += ms;
    h->prof_count[h->ev_kind[k]] += 1;
  }
  h->ev_used = 0;
  return AP_DVM_OK;
}

// Kernels of one IMEX step of the given parity for all attached solves (see the file header).
ap_dvm_status enqueue_step(ap_dvm_handle* h, cudaStream_t stream, int parity) {
  StepKernels K{h->ks,       h->km,         h->grid_explicit, h->grid_rhs,   h->grid_update, h->grid_finish,
                h->grid_fft, h->grid_cols, h->km.cols_threads, fft_smem(h), cols_smem(h), h->smem_update, h->fft_kinds,
                h->grid_rows};
  auto ln = [&](const void* fn, int grid, dim3 block, size_t smem, void** args, int kind) -> int {
    return (int)launch(h, stream, fn, grid, block, smem, args, kind);
  };
  return (ap_dvm_status)enqueue_imex_step(h->tmpl, K, h->d_batch[parity], h->tmpl.precision, ln, true);
}

// A CUDA graph of graph_steps steps starting at the given parity.
ap_dvm_status build_graph(ap_dvm_handle* h, int parity) {
  if (h->graph[parity]) { cudaGraphExecDestroy(h->graph[parity]); h->graph[parity] = nullptr; }
  if (!h->cap_stream) CUDA_TRY(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  CUDA_TRY(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
  ap_dvm_status st = AP_DVM_OK;
  for (int k = 0; k < h->graph_steps && st == AP_DVM_OK; ++k) st = enqueue_step(h, h->cap_stream, parity ^ (k & 1));
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
  if (st) { if (g) cudaGraphDestroy(g); return st; }
  if (e != cudaSuccess) return fail(h, AP_DVM_ERR_CUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&h->graph[parity], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(h, AP_DVM_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
  h->graph_valid[parity] = true;
  return AP_DVM_OK;
}

Slot* slot_of(ap_dvm_handle* h, int slot) {
  if (!h || slot < 0 || slot >= h->capacity || !h->slots[slot].attached) return nullptr;
  return &h->slots[slot];
}

int grid_for_cells(size_t cells) { return (int)std::min<size_t>((cells + 255) / 256, 4096); }

}  // namespace

// ============================================================================ C ABI

extern "C" {

void ap_dvm_default_params(ap_dvm_params* p, int nx, int ny, double eps, double dt) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->nx = nx;
  p->ny = ny;
  p->Lx = p->Ly = 2.0 * 3.14159265358979323846;
  p->velocity_set = AP_DVM_D2V6;
  p->eps = eps;
  p->tau = 0.05;
  p->mach = 1e-2;
  p->rho0 = 1.0;
  p->dt = dt;
  p->s = 3;
  const double c = 2.25, g = (c - 0.5) / (c - 1.0);
  const int M = AP_DVM_MAX_STAGES;
  p->A_ex[1 * M + 0] = c;
  p->A_ex[2 * M + 0] = 1.0 - 1.0 / (2.0 * c);
  p->A_ex[2 * M + 1] = 1.0 / (2.0 * c);
  p->A_im[1 * M + 1] = c;
  p->A_im[2 * M + 1] = 1.0 - g;
  p->A_im[2 * M + 2] = g;
  p->space_scheme = AP_DVM_WENO5_C4;
  p->precision = AP_DVM_FP64;
  p->weno_eps = 1e-6;
}

size_t ap_dvm_instance_workspace_size(const ap_dvm_params* p) {
  char buf[256];
  if (validate(p, buf, sizeof(buf)) != AP_DVM_OK) return 0;
  return carve_instance(*p, nullptr, nullptr, true);
}

size_t ap_dvm_batch_workspace_size(const ap_dvm_params* tmpl, int capacity) {
  char buf[256];
  if (capacity < 1 || validate(tmpl, buf, sizeof(buf)) != AP_DVM_OK) return 0;
  return batch_bytes(capacity, std::max(fft_length(tmpl->nx), fft_length(tmpl->ny)));
}

size_t ap_dvm_workspace_size(const ap_dvm_params* p) {
  const size_t a = ap_dvm_batch_workspace_size(p, 1), b = ap_dvm_instance_workspace_size(p);
  return (a && b) ? a + b : 0;
}

ap_dvm_status ap_dvm_batch_create(const ap_dvm_params* tmpl, int capacity, void* d_workspace, size_t bytes,
                                  void* cuda_stream, ap_dvm_handle** out) {
  if (!out) return AP_DVM_ERR_ARG;
  *out = nullptr;
  ap_dvm_handle* h = new (std::nothrow) ap_dvm_handle();
  if (!h) return AP_DVM_ERR_ARG;
  *out = h;
  ap_dvm_status st = validate(tmpl, h->err, sizeof(h->err));
  if (st) return st;
  if (capacity < 1) return fail(h, AP_DVM_ERR_ARG, "capacity must be >= 1");
  h->tmpl = *tmpl;
  h->capacity = capacity;
  h->f32 = tmpl->precision != AP_DVM_FP64;
  h->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  h->nmax = std::max(fft_length(tmpl->nx), fft_length(tmpl->ny));   // longest transform of the batch
  h->lnmax = ilog2(h->nmax);
  h->eblk = fft_eblk(h->nmax);
  h->eblk_cols = fft_eblk_cols(h->nmax, h->f32);
  const size_t need = batch_bytes(capacity, h->nmax);
  if (!d_workspace || bytes < need || (reinterpret_cast<uintptr_t>(d_workspace) & 255))
    return fail(h, AP_DVM_ERR_WORKSPACE, "batch workspace needs %zu bytes, 256-byte aligned (got %zu)", need, bytes);
  CUDA_TRY(h, cudaGetDevice(&h->device));
  CUDA_TRY(h, cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device));
  char* base = reinterpret_cast<char*>(d_workspace);
  size_t off = 0;
  auto take = [&](size_t b) { off = align_up(off, 256); char* r = base + off; off += b; return r; };
  BatchDev* batches = reinterpret_cast<BatchDev*>(take(sizeof(BatchDev) * 2));
  InstDev* insts = reinterpret_cast<InstDev*>(take(sizeof(InstDev) * capacity * 2));
  for (int par = 0; par < 2; ++par) {
    h->d_batch[par] = batches + par;
    h->d_inst[par] = insts + (size_t)par * capacity;
  }
  h->d_tile_start = reinterpret_cast<int*>(take(sizeof(int) * (capacity + 1)));
  h->d_row_start = reinterpret_cast<int*>(take(sizeof(int) * (capacity + 1)));
  h->d_col_start = reinterpret_cast<int*>(take(sizeof(int) * (capacity + 1)));
  h->d_rhs_start = reinterpret_cast<int*>(take(sizeof(int) * (capacity + 1)));
  h->d_counts = reinterpret_cast<int*>(take(sizeof(int) * 5));
  h->d_tw = reinterpret_cast<double2*>(take(sizeof(double2) * (h->nmax / 2)));
  h->d_tw32 = reinterpret_cast<float2*>(take(sizeof(float2) * (h->nmax / 2)));
  h->d_err = reinterpret_cast<unsigned*>(take(sizeof(unsigned) * 4));
  // twiddles exp(-2 pi i k / nmax) from long double
  std::vector<double2> tw(h->nmax / 2);
  std::vector<float2> tw32(h->nmax / 2);
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int k = 0; k < h->nmax / 2; ++k) {
    const long double a = -2.0L * pi * (long double)k / (long double)h->nmax;
    tw[k].x = (double)std::cos(a);
    tw[k].y = (double)std::sin(a);
    tw32[k].x = (float)std::cos(a);
    tw32[k].y = (float)std::sin(a);
  }
  BatchDev& hb = h->hb[0];
  hb.inst = h->d_inst[0];
  hb.tile_start = h->d_tile_start;
  hb.row_start = h->d_row_start;
  hb.col_start = h->d_col_start;
  hb.rhs_start = h->d_rhs_start;
  hb.counts = h->d_counts;
  hb.tw = h->d_tw;
  hb.tw32 = h->d_tw32;
  hb.lnmax = h->lnmax;
  hb.s = tmpl->s;
  fill_tableau(*tmpl, hb);
  hb.err = h->d_err;
  // uploads on the handle's stream (no legacy-stream serialisation against the caller's other
  // streams), synchronised below: the host vectors go out of scope
  CUDA_TRY(h, cudaMemcpyAsync(h->d_tw, tw.data(), sizeof(double2) * tw.size(), cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(h->d_tw32, tw32.data(), sizeof(float2) * tw32.size(), cudaMemcpyHostToDevice, h->stream));
  h->hb[1] = hb;
  h->hb[1].inst = h->d_inst[1];
  for (int par = 0; par < 2; ++par)
    CUDA_TRY(h, cudaMemcpyAsync(h->d_batch[par], &h->hb[par], sizeof(BatchDev), cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(h, cudaMemsetAsync(h->d_err, 0, sizeof(unsigned) * 4, h->stream));
  CUDA_TRY(h, cudaMemsetAsync(h->d_counts, 0, sizeof(int) * 5, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  h->slots.resize(capacity);
  h->dirty = true;
  return AP_DVM_OK;
}

ap_dvm_status ap_dvm_attach(ap_dvm_handle* h, int slot, const ap_dvm_params* p, void* d_workspace, size_t bytes) {
  if (!h) return AP_DVM_ERR_ARG;
  if (slot < 0 || slot >= h->capacity) return fail(h, AP_DVM_ERR_ARG, "slot %d out of range [0, %d)", slot, h->capacity);
  if (h->slots[slot].attached) return fail(h, AP_DVM_ERR_ARG, "slot %d is in use", slot);
  ap_dvm_status st = validate(p, h->err, sizeof(h->err));
  if (st) return st;
  if (!same_method(*p, h->tmpl)) return fail(h, AP_DVM_ERR_ARG, "scheme, precision and tableau must match the batch");
  if (p->nx > h->tmpl.nx || p->ny > h->tmpl.ny) return fail(h, AP_DVM_ERR_ARG, "grid larger than the batch template");
  if (std::max(fft_length(p->nx), fft_length(p->ny)) > h->nmax)
    return fail(h, AP_DVM_ERR_ARG, "grid %dx%d needs transforms of length %d, longer than the batch's %d", p->nx, p->ny,
                std::max(fft_length(p->nx), fft_length(p->ny)), h->nmax);
  const size_t need = carve_instance(*p, nullptr, nullptr, true);
  if (!d_workspace || bytes < need || (reinterpret_cast<uintptr_t>(d_workspace) & 255))
    return fail(h, AP_DVM_ERR_WORKSPACE, "instance workspace needs %zu bytes, 256-byte aligned (got %zu)", need, bytes);
  Slot& s = h->slots[slot];
  s = Slot();
  s.p = *p;
  s.ws = reinterpret_cast<char*>(d_workspace);
  s.bytes = bytes;
  InstDev& d = s.dev;
  carve_instance(*p, s.ws, &d, true);
  d.nx = p->nx; d.ny = p->ny; d.lnx = ilog2(fft_length(p->nx)); d.lny = ilog2(fft_length(p->ny));
  fill_constants(*p, d);
  d.relax64 = (p->precision != AP_DVM_FP64 && p->eps <= 1e-4) ? 1 : 0;
  std::vector<double> lx(p->nx / 2 + 1), ly(p->ny);
  laplacian_symbol(p->nx, d.dx, p->space_scheme, lx.data(), (int)lx.size());
  laplacian_symbol(p->ny, d.dy, p->space_scheme, ly.data(), (int)ly.size());
  CUDA_TRY(h, cudaMemcpyAsync(d.lamx, lx.data(), sizeof(double) * lx.size(), cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(d.lamy, ly.data(), sizeof(double) * ly.size(), cudaMemcpyHostToDevice, h->stream));
  std::vector<float> lx32(lx.begin(), lx.end()), ly32(ly.begin(), ly.end());   // rounded once (FP32 form)
  if (d.lamx32) {
    CUDA_TRY(h, cudaMemcpyAsync(d.lamx32, lx32.data(), sizeof(float) * lx32.size(), cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(h, cudaMemcpyAsync(d.lamy32, ly32.data(), sizeof(float) * ly32.size(), cudaMemcpyHostToDevice, h->stream));
  }
  std::vector<double2> tab64[2];
  std::vector<float2> tab32[2];
  for (int a = 0; a < 2; ++a) {
    const int na = a ? p->ny : p->nx;
    if (is_pow2(na)) continue;
    if (d.mr_npass[a]) {   // mixed radix: W_n^q, q < n
      const long double pi = 3.141592653589793238462643383279502884L;
      for (int q = 0; q < na; ++q) {
        const long double ang = -2.0L * pi * (long double)q / (long double)na;
        tab64[a].push_back(make_double2((double)std::cos(ang), (double)std::sin(ang)));
        tab32[a].push_back(make_float2((float)std::cos(ang), (float)std::sin(ang)));
      }
      if (h->f32)
        CUDA_TRY(h, cudaMemcpyAsync(const_cast<void*>(d.mr_tw[a]), tab32[a].data(), sizeof(float2) * na, cudaMemcpyHostToDevice, h->stream));
      else
        CUDA_TRY(h, cudaMemcpyAsync(const_cast<void*>(d.mr_tw[a]), tab64[a].data(), sizeof(double2) * na, cudaMemcpyHostToDevice, h->stream));
      continue;
    }
    std::vector<std::complex<long double>> ch, fl;
    bluestein_tables(na, fft_length(na), ch, fl);
    for (const auto* v : {&ch, &fl}) {
      for (const auto& z : *v) {
        tab64[a].push_back(make_double2((double)z.real(), (double)z.imag()));
        tab32[a].push_back(make_float2((float)z.real(), (float)z.imag()));
      }
    }
    // chirp (na values) then filter (fft_length(na) values), in the batch's complex type
    const size_t nc = ch.size(), nf = fl.size();
    if (h->f32) {
      CUDA_TRY(h, cudaMemcpyAsync(const_cast<void*>(d.chirp[a]), tab32[a].data(), sizeof(float2) * nc, cudaMemcpyHostToDevice, h->stream));
      CUDA_TRY(h, cudaMemcpyAsync(const_cast<void*>(d.filt[a]), tab32[a].data() + nc, sizeof(float2) * nf, cudaMemcpyHostToDevice, h->stream));
    } else {
      CUDA_TRY(h, cudaMemcpyAsync(const_cast<void*>(d.chirp[a]), tab64[a].data(), sizeof(double2) * nc, cudaMemcpyHostToDevice, h->stream));
      CUDA_TRY(h, cudaMemcpyAsync(const_cast<void*>(d.filt[a]), tab64[a].data() + nc, sizeof(double2) * nf, cudaMemcpyHostToDevice, h->stream));
    }
  }
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));   // the symbol and transform-table vectors are about to go out of scope
  for (void* xb : {d.X, d.Xnext}) CUDA_TRY(h, cudaMemsetAsync(xb, 0, (size_t)6 * p->nx * p->ny * (h->f32 ? 4 : 8), h->stream));
  if (d.dF) CUDA_TRY(h, cudaMemsetAsync(d.dF, 0, (size_t)6 * p->nx * p->ny * sizeof(float), h->stream));
  s.flip = 0;
  s.paused = false;
  s.attached = true;
  h->dirty = true;
  if (h->tile_auto) {
    const int t = auto_tile(h);
    if (t != h->tile || !h->kernels_ready) { h->tile = t; h->kernels_ready = false; }
  }
  return AP_DVM_OK;
}

ap_dvm_status ap_dvm_detach(ap_dvm_handle* h, int slot) {
  if (!slot_of(h, slot)) return h ? fail(h, AP_DVM_ERR_ARG, "slot %d is not attached", slot) : AP_DVM_ERR_ARG;
  h->slots[slot].attached = false;
  h->dirty = true;
  return AP_DVM_OK;
}

ap_dvm_status ap_dvm_create(const ap_dvm_params* p, void* d_workspace, size_t bytes, void* cuda_stream, ap_dvm_handle** out) {
  if (!out) return AP_DVM_ERR_ARG;
  const size_t a = ap_dvm_batch_workspace_size(p, 1), b = ap_dvm_instance_workspace_size(p);
  ap_dvm_status st = ap_dvm_batch_create(p, 1, d_workspace, bytes, cuda_stream, out);
  if (st) return st;
  if (bytes < a + b) return fail(*out, AP_DVM_ERR_WORKSPACE, "workspace needs %zu bytes (got %zu)", a + b, bytes);
  return ap_dvm_attach(*out, 0, p, reinterpret_cast<char*>(d_workspace) + a, bytes - a);
}

static ap_dvm_status set_state_impl(ap_dvm_handle* h, int slot, const double* a, const double* b, const double* c,
                                    const float* f, int mode) {
  Slot* s = slot_of(h, slot);
  if (!s) return h ? fail(h, AP_DVM_ERR_ARG, "slot %d is not attached", slot) : AP_DVM_ERR_ARG;
  ap_dvm_status st = prepare_kernels(h);
  if (st) return st;
  InstDev d = view(*s, h->parity);
  int form = h->tmpl.precision;   // 0: FP64, 1: FP32 deviation form, 2: the same with theta carried
  void* args[] = {&d, &a, &b, &c, &f, &mode, &form};
  return launch(h, h->stream, h->km.k_set_state, grid_for_cells((size_t)s->p.nx * s->p.ny), dim3(256), 0, args);
}

static ap_dvm_status get_state_impl(ap_dvm_handle* h, int slot, double* out, float* out32, int what,
                                    double* o1 = nullptr, double* o2 = nullptr, double* o3 = nullptr) {
  Slot* s = slot_of(h, slot);
  if (!s) return h ? fail(h, AP_DVM_ERR_ARG, "slot %d is not attached", slot) : AP_DVM_ERR_ARG;
  ap_dvm_status st = prepare_kernels(h);
  if (st) return st;
  InstDev d = view(*s, h->parity);
  int form = h->tmpl.precision;
  void* args[] = {&d, &out, &o1, &o2, &o3, &out32, &what, &form};
  return launch(h, h->stream, h->km.k_get_state, grid_for_cells((size_t)s->p.nx * s->p.ny), dim3(256), 0, args);
}

ap_dvm_status ap_dvm_diagnostics(ap_dvm_handle* h, int slot, double* d_vorticity, double* out3) {
  if (!out3) return h ? fail(h, AP_DVM_ERR_ARG, "null output") : AP_DVM_ERR_ARG;
  Slot* s = slot_of(h, slot);
  if (!s) return h ? fail(h, AP_DVM_ERR_ARG, "slot %d is not attached", slot) : AP_DVM_ERR_ARG;
  ap_dvm_status st = prepare_kernels(h);
  if (st) return st;
  InstDev d = view(*s, h->parity);
  const size_t cells = (size_t)s->p.nx * s->p.ny;
  const int grid = (int)std::min<size_t>((cells + 255) / 256, 256);
  // block partials in the slot's right-hand-side plane (free between steps; >= 3 * grid doubles)
  double* part = reinterpret_cast<double*>(d.R);
  int c4 = s->p.space_scheme != AP_DVM_LF1_C2;
  void* args[] = {&d, &c4, &part, &d_vorticity};
  if ((st = launch(h, h->stream, h->km.k_diagnostics, grid, dim3(256), 0, args))) return st;
  std::vector<double> hp(3 * (size_t)grid);
  CUDA_TRY(h, cudaMemcpyAsync(hp.data(), part, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  double dmax = 0.0, d2 = 0.0, w2 = 0.0;
  for (int b = 0; b < grid; ++b) {
    dmax = std::max(dmax, hp[3 * b]);
    d2 += hp[3 * b + 1];
    w2 += hp[3 * b + 2];
  }
  const double area = d.dx * d.dy;
  out3[0] = dmax;
  out3[1] = std::sqrt(d2 * area);
  out3[2] = 0.5 * w2 * area;
  return AP_DVM_OK;
}

ap_dvm_status ap_dvm_set_state(ap_dvm_handle* h, int slot, const double* d_moments6) {
  if (!d_moments6) return h ? fail(h, AP_DVM_ERR_ARG, "null state pointer") : AP_DVM_ERR_ARG;
  return set_state_impl(h, slot, d_moments6, nullptr, nullptr, nullptr, 0);
}

ap_dvm_status ap_dvm_set_equilibrium(ap_dvm_handle* h, int slot, const double* d_u1, const double* d_u2, const double* d_p) {
  if (!d_u1 || !d_u2 || !d_p) return h ? fail(h, AP_DVM_ERR_ARG, "null pointer") : AP_DVM_ERR_ARG;
  return set_state_impl(h, slot, d_u1, d_u2, d_p, nullptr, 1);
}

ap_dvm_status ap_dvm_set_populations(ap_dvm_handle* h, int slot, const void* d_dF6, int is_float) {
  if (!d_dF6) return h ? fail(h, AP_DVM_ERR_ARG, "null pointer") : AP_DVM_ERR_ARG;
  if (is_float && h && !h->f32) return fail(h, AP_DVM_ERR_ARG, "float populations need the FP32 form");
  if (is_float) return set_state_impl(h, slot, nullptr, nullptr, nullptr, reinterpret_cast<const float*>(d_dF6), 3);
  return set_state_impl(h, slot, reinterpret_cast<const double*>(d_dF6), nullptr, nullptr, nullptr, 2);
}

ap_dvm_status ap_dvm_set_theta(ap_dvm_handle* h, int slot, const double* d_theta) {
  if (!d_theta) return h ? fail(h, AP_DVM_ERR_ARG, "null pointer") : AP_DVM_ERR_ARG;
  if (h && h->tmpl.precision != AP_DVM_FP32_DEV_TH) return fail(h, AP_DVM_ERR_ARG, "the carried theta plane needs AP_DVM_FP32_DEV_TH");
  return set_state_impl(h, slot, d_theta, nullptr, nullptr, nullptr, 4);
}

ap_dvm_status ap_dvm_get_state(ap_dvm_handle* h, int slot, double* d_moments6) {
  if (!d_moments6) return h ? fail(h, AP_DVM_ERR_ARG, "null pointer") : AP_DVM_ERR_ARG;
  return get_state_impl(h, slot, d_moments6, nullptr, 0);
}

ap_dvm_status ap_dvm_get_populations(ap_dvm_handle* h, int slot, void* d_dF6, int is_float) {
  if (!d_dF6) return h ? fail(h, AP_DVM_ERR_ARG, "null pointer") : AP_DVM_ERR_ARG;
  if (is_float) return get_state_impl(h, slot, nullptr, reinterpret_cast<float*>(d_dF6), 3);
  return get_state_impl(h, slot, reinterpret_cast<double*>(d_dF6), nullptr, 2);
}

ap_dvm_status ap_dvm_moments(ap_dvm_handle* h, int slot, double* d_rho, double* d_u1, double* d_u2, double* d_p) {
  Slot* s = slot_of(h, slot);
  if (!s) return h ? fail(h, AP_DVM_ERR_ARG, "slot %d is not attached", slot) : AP_DVM_ERR_ARG;
  if (!d_rho || !d_u1 || !d_u2 || !d_p) return fail(h, AP_DVM_ERR_ARG, "null pointer");
  return get_state_impl(h, slot, d_rho, nullptr, 1, d_u1, d_u2, d_p);
}

ap_dvm_status ap_dvm_step(ap_dvm_handle* h, int nsteps) {
  if (!h) return AP_DVM_ERR_ARG;
  if (nsteps < 0) return fail(h, AP_DVM_ERR_ARG, "nsteps must be >= 0");
  ap_dvm_status st = flush(h);
  if (st) return st;
  if (h->n_active == 0 || nsteps == 0) return AP_DVM_OK;
  int done = 0;
  if (h->graph_steps > 0 && !h->profile) {
    while (nsteps - done >= h->graph_steps) {
      const int par = h->parity;
      if (!h->graph_valid[par] && (st = build_graph(h, par))) return st;
      CUDA_TRY(h, cudaGraphLaunch(h->graph[par], h->stream));
      done += h->graph_steps;
      h->parity ^= h->graph_steps & 1;
    }
  }
  for (; done < nsteps; ++done) {
    if ((st = enqueue_step(h, h->stream, h->parity))) return st;
    h->parity ^= 1;
    if (h->profile && h->ev_used > 2048 && (st = profile_collect(h))) return st;
  }
  return AP_DVM_OK;
}

ap_dvm_status ap_dvm_step_slots(ap_dvm_handle* h, int nsteps, const int* steps_per_slot) {
  if (!h) return AP_DVM_ERR_ARG;
  if (nsteps < 0 || !steps_per_slot) return fail(h, AP_DVM_ERR_ARG, "nsteps must be >= 0 and steps_per_slot given");
  std::vector<int> ends;
  for (int k = 0; k < h->capacity; ++k) {
    if (!h->slots[k].attached) continue;
    const int c = steps_per_slot[k];
    if (c < 0 || c > nsteps) return fail(h, AP_DVM_ERR_ARG, "slot %d: %d steps, outside [0, %d]", k, c, nsteps);
    ends.push_back(c);
  }
  std::sort(ends.begin(), ends.end());
  ends.erase(std::unique(ends.begin(), ends.end()), ends.end());
  // segments between the step counts at which slots drop out: the slots that are done
  // sit out the rest (left out of the work lists; their state stays where it is, so
  // their buffer offset absorbs the parity the handle moves through)
  ap_dvm_status st = AP_DVM_OK;
  int t = 0;
  for (int e : ends) {
    if (e <= t) continue;
    for (int k = 0; k < h->capacity; ++k) {
      Slot& s = h->slots[k];
      if (!s.attached) continue;
      const bool p = steps_per_slot[k] <= t;
      if (p != s.paused) { s.paused = p; h->dirty = true; }
    }
    const int par0 = h->parity;
    st = ap_dvm_step(h, e - t);
    const int moved = h->parity ^ par0;
    for (Slot& s : h->slots)
      if (s.attached && s.paused) s.flip ^= moved;
    if (st) break;
    t = e;
  }
  for (Slot& s : h->slots)
    if (s.attached && s.paused) { s.paused = false; h->dirty = true; }
  return st;
}

ap_dvm_status ap_dvm_profile_enable(ap_dvm_handle* h, int enable) {
  if (!h) return AP_DVM_ERR_ARG;
  ap_dvm_status st = profile_collect(h);
  if (st) return st;
  h->profile = enable != 0;
  for (int k = 0; k < kNumKinds; ++k) { h->prof_ms[k] = 0; h->prof_count[k] = 0; }
  return AP_DVM_OK;
}

int ap_dvm_profile_read(ap_dvm_handle* h, const char** names, double* total_ms, long* launches, int max) {
  if (!h || profile_collect(h) != AP_DVM_OK) return -1;
  const int n = std::min(max, kNumKinds);
  for (int k = 0; k < n; ++k) {
    if (names) names[k] = kKernelNames[k];
    if (total_ms) total_ms[k] = h->prof_ms[k];
    if (launches) launches[k] = h->prof_count[k];
  }
  return kNumKinds;
}

ap_dvm_status ap_dvm_set_graph_steps(ap_dvm_handle* h, int k) {
  if (!h) return AP_DVM_ERR_ARG;
  if (k < 0) return fail(h, AP_DVM_ERR_ARG, "k must be >= 0");
  if (k != h->graph_steps) { h->graph_steps = k; h->graph_valid[0] = h->graph_valid[1] = false; }
  return AP_DVM_OK;
}

ap_dvm_status ap_dvm_set_tile(ap_dvm_handle* h, int tile) {
  if (!h) return AP_DVM_ERR_ARG;
  if (tile < -1 || tile >= kNumTiles) return fail(h, AP_DVM_ERR_ARG, "tile index out of range");
  const bool aut = tile < 0;
  const int t = aut ? auto_tile(h) : tile;
  for (const Slot& s : h->slots)
    if (s.attached && (s.p.nx < kTileX[t] || s.p.ny < kTileY[t])) return fail(h, AP_DVM_ERR_ARG, "an attached grid is smaller than the tile");
  h->tile_auto = aut;
  if (t != h->tile || !h->kernels_ready) { h->tile = t; h->kernels_ready = false; h->dirty = true; }
  return AP_DVM_OK;
}

int ap_dvm_get_tile(const ap_dvm_handle* h) { return h ? h->tile : -1; }

int ap_dvm_launches_per_step(const ap_dvm_handle* h) {
  if (!h) return 0;
  const ap_dvm_params& t = h->tmpl;
  const int f = fft_launches(fft_kinds_of(h));   // transform launches per implicit stage
  // the last stage's update closes the step (no finish kernel)
  return t.A_im[0] != 0.0 ? 1 + (2 + f) + (3 + f) * (t.s - 1) : (3 + f) * (t.s - 1);
}

ap_dvm_status ap_dvm_run_host(ap_dvm_handle* h, int slot, const double* h_in, double* h_out, double* d_stage, int nsteps) {
  Slot* s = slot_of(h, slot);
  if (!s) return h ? fail(h, AP_DVM_ERR_ARG, "slot %d is not attached", slot) : AP_DVM_ERR_ARG;
  if (!h_in || !h_out || !d_stage) return fail(h, AP_DVM_ERR_ARG, "null pointer");
  const size_t bytes = (size_t)6 * s->p.nx * s->p.ny * sizeof(double);
  CUDA_TRY(h, cudaMemcpyAsync(d_stage, h_in, bytes, cudaMemcpyHostToDevice, h->stream));
  ap_dvm_status st;
  if ((st = ap_dvm_set_state(h, slot, d_stage))) return st;
  if ((st = ap_dvm_step(h, nsteps))) return st;
  if ((st = ap_dvm_get_state(h, slot, d_stage))) return st;
  CUDA_TRY(h, cudaMemcpyAsync(h_out, d_stage, bytes, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return AP_DVM_OK;
}

ap_dvm_status ap_dvm_sync_status(ap_dvm_handle* h) {
  if (!h) return AP_DVM_ERR_ARG;
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  CUDA_TRY(h, cudaGetLastError());
  unsigned flags = 0;
  CUDA_TRY(h, cudaMemcpyAsync(&flags, h->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  if (flags) CUDA_TRY(h, cudaMemsetAsync(h->d_err, 0, sizeof(unsigned), h->stream));
  if (flags & 2u) return fail(h, AP_DVM_ERR_TIMEOUT, "a bounded device wait expired (results since the last check are invalid)");
  if (flags & 1u) return fail(h, AP_DVM_ERR_NONFINITE, "a step produced a non-finite value");
  return AP_DVM_OK;
}

ap_dvm_status ap_dvm_check_wait_timeout(ap_dvm_handle* h, long long wait_ns) {
  if (!h) return AP_DVM_ERR_ARG;
  if (wait_ns < 1000 || wait_ns > 10000000000LL) return fail(h, AP_DVM_ERR_ARG, "wait_ns must be in [1e3, 1e10]");
  CUDA_TRY(h, launch_wait_timeout(h->d_err, (unsigned long long)wait_ns, h->stream));
  return AP_DVM_OK;
}

ap_dvm_status ap_dvm_check_conversions(const double* d_in, int n, unsigned* d_counts, void* cuda_stream) {
  if (!d_counts || n < 0 || (n > 0 && !d_in)) return AP_DVM_ERR_ARG;
  return launch_check_conversions(d_in, n, d_counts, reinterpret_cast<cudaStream_t>(cuda_stream)) == cudaSuccess
             ? AP_DVM_OK
             : AP_DVM_ERR_CUDA;
}

const char* ap_dvm_last_error(const ap_dvm_handle* h) { return h ? h->err : "null handle"; }

void ap_dvm_destroy(ap_dvm_handle* h) {
  if (!h) return;
  for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
  for (cudaGraphExec_t g : h->graph)
    if (g) cudaGraphExecDestroy(g);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  delete h;
}

}  // extern "C"
