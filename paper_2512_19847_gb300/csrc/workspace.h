// Host-side layout of one solve's device workspace and the tables derived
// from its grid, shared by the handle path (api.cu) and the no-allocation
// entry point (noalloc.cu), so that both carve the same planes.
#pragma once
#include <cuda.h>

#include <cmath>
#include <cstddef>
#include <cstdint>

#include "../../include/ap_dvm.h"
#include "common.cuh"

namespace apd {

inline bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }
inline int ilog2(int n) { int l = 0; while ((1 << l) < n) ++l; return l; }
inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Transform length of an axis of n cells: n for a power of two, else the
// length of Bluestein's circular convolution, the power of two >= 2n - 1.
inline int fft_length(int n) {
  if (is_pow2(n)) return n;
  int m = 1;
  while (m < 2 * n - 1) m <<= 1;
  return m;
}

// Mixed-radix plan of an axis of n cells: the radices (4s first, then 2, 3, 5,
// 7; 4 bits each, first pass in the low bits) when n is not a power of two and
// has no prime factor above 7; false otherwise.
inline bool mixed_radix_plan(int n, unsigned* plan, int* npass) {
  if (is_pow2(n)) return false;
  unsigned pl = 0;
  int np = 0;
  auto push = [&](int r) { pl |= (unsigned)r << (4 * np); ++np; };
  while (n % 4 == 0) { push(4); n /= 4; }
  for (int r : {2, 3, 5, 7})
    while (n % r == 0) { push(r); n /= r; }
  if (n != 1 || np > 8) return false;
  *plan = pl;
  *npass = np;
  return true;
}

// Carves one instance's workspace (base == nullptr: size only).  With two_states
// the state is double-buffered (the last stage's update writes the next state to
// the other buffer, I.Xnext) and the tensor-map region holds one set of maps per
// buffer (2 (APD_MAXS + 1) maps); otherwise I.Xnext is null and a finish kernel
// closes the step in place.
inline size_t carve_instance(const ap_dvm_params& p, char* base, InstDev* d, bool two_states = false) {
  const size_t es = p.precision == AP_DVM_FP64 ? 8 : 4;
  const size_t cells = (size_t)p.nx * p.ny;
  const size_t plane = cells * es;
  size_t off = 0;
  auto take = [&](size_t bytes) -> void* {
    off = align_up(off, 256);
    void* r = base ? base + off : nullptr;
    off += bytes;
    return r;
  };
  const int s = p.s;
  InstDev tmp{};
  InstDev& I = d ? *d : tmp;
  const bool type_a = p.A_im[0] != 0.0;
  I.X = take(6 * plane);
  I.Xnext = two_states ? take(6 * plane) : nullptr;
  I.Xs[1] = type_a ? take(6 * plane) : I.X;           // stage 1: its own values (type A) or X^n
  for (int j = 2; j <= s; ++j) I.Xs[j] = take(6 * plane);
  for (int j = 1; j <= s; ++j) {
    I.E[j] = take(2 * plane);
    I.Du[j] = take(plane);
    I.Lth[j] = take(plane);
    I.DLFB[j] = take(2 * plane);
    I.Dv[j] = take(plane);
    I.DB[j] = take(plane);
  }
  I.Dun = type_a ? take(plane) : I.Du[1];
  I.R = take(plane);
  I.sstride = p.nx / 2 + 1;
  I.S = take((size_t)p.ny * I.sstride * 2 * es);
  I.lamx = reinterpret_cast<double*>(take((size_t)(p.nx / 2 + 1) * sizeof(double)));
  I.lamy = reinterpret_cast<double*>(take((size_t)p.ny * sizeof(double)));
  const bool f32 = p.precision != AP_DVM_FP64;
  I.lamx32 = f32 ? reinterpret_cast<float*>(take((size_t)(p.nx / 2 + 1) * sizeof(float))) : nullptr;
  I.lamy32 = f32 ? reinterpret_cast<float*>(take((size_t)p.ny * sizeof(float))) : nullptr;
  // one partial sum per tile: at most ceil(nx/8) * ceil(ny/4) tiles (the smallest tile sides)
  I.th_part = reinterpret_cast<double*>(take((size_t)rhs_items(p.nx, p.ny, p.precision != AP_DVM_FP64) * sizeof(double)));
  for (int a = 0; a < 2; ++a) {   // tables of an axis that is not a power of two: mixed radix or Bluestein
    const int na = a ? p.ny : p.nx;
    unsigned plan = 0;
    int npass = 0;
    const bool mr = mixed_radix_plan(na, &plan, &npass);
    I.mr_plan[a] = mr ? plan : 0u;
    I.mr_npass[a] = mr ? npass : 0;
    I.mr_tw[a] = mr ? take((size_t)na * 2 * es) : nullptr;
    const bool bs = !is_pow2(na) && !mr;
    I.chirp[a] = bs ? take((size_t)na * 2 * es) : nullptr;
    I.filt[a] = bs ? take((size_t)fft_length(na) * 2 * es) : nullptr;
  }
  I.dF = f32 ? reinterpret_cast<float*>(take(6 * cells * sizeof(float))) : nullptr;
  I.tmap = take(sizeof(CUtensorMap) * (APD_MAXS + 1) * (two_states ? 2 : 1));
  return align_up(off, 256);
}

// 1D symbol of the Laplacian stencil on DFT mode k (compact 3-point or 4th-order
// 5-point second difference, Sec. 3.2), without cancellation for small k.
inline void laplacian_symbol(int n, double h, int scheme, double* out, int count) {
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int k = 0; k < count; ++k) {
    const long double phi = 2.0L * pi * (long double)k / (long double)n;
    const long double s = std::sin(0.5L * phi);
    const long double s2 = s * s;
    long double v;
    if (scheme == AP_DVM_LF1_C2) v = -4.0L * s2 / ((long double)h * h);
    else v = 2.0L * s2 * (std::cos(phi) - 7.0L) / (3.0L * (long double)h * h);
    out[k] = (double)v;
  }
}

}  // namespace apd
