// Shared device-side definitions of the AP IMEX-RK D2V6 library.
//
// Layout in HBM: every field is a "plane" of nx*ny values, row-major with x
// fastest (index j*nx + i, cell centre ((i+1/2)dx, (j+1/2)dy)), structure of
// arrays.  A moment state is 6 consecutive planes (u1, u2, theta, v1, v2, q).
// All kernels are persistent grid-stride loops over a device-resident work
// list, so one launch covers every instance of a batch whatever their sizes.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#define APD_MAXS 4          // maximum number of IMEX stages
#define APD_NPLANES_STATE 6

namespace apd {

enum Scheme { LF1_C2 = 0, WENO3_C4 = 1, WENO5_C4 = 2 };

// Halo width of the per-cell operators of each spatial scheme (Sec. 3.2):
// LF1 fluxes and 2nd-order central differences reach 1 cell, WENO3 fluxes
// and 4th-order central differences 2, WENO5 fluxes 3.
__host__ __device__ constexpr int halo_of(int scheme) { return scheme == LF1_C2 ? 1 : (scheme == WENO3_C4 ? 2 : 3); }
__host__ __device__ constexpr int central_halo(int scheme) { return scheme == LF1_C2 ? 1 : 2; }

// Stage coefficients of one instance in the scalar type T, computed on the
// host in FP64 and rounded once, so that no kernel converts or combines
// uniform coefficients per thread.  Stage indices are 1-based as in the paper.
template <typename T>
struct Coef {
  T dt, te2, qtau, htau;                  // dt, tau eps^2, tau/4, tau/2
  T inv_dx, inv_dy;
  T kappa[APD_MAXS + 1];                  // 2 eps^2 / (dt a_ii)^2
  T aex[APD_MAXS + 1][APD_MAXS + 1];      // atilde_ij
  T aim[APD_MAXS + 1][APD_MAXS + 1];      // a_ij
  T wp[APD_MAXS + 1][APD_MAXS + 1];       // (atilde_ij - a_ij) / a_ii: weights of the explicit-weight dissipation partner
  // closed forms of steps 1 and 4 with the division folded into the coefficients:
  //   v^(i) = r_n v^n + sum_j rv_e E^(j) + sum_j rv_v v^(j),
  //   q^(i) = r_n q^n + sum_{j<=i} rq_d D0.v^(j) + sum_{j<i} rq_q q^(j)
  T r_n[APD_MAXS + 1];                    // tau eps^2 / (tau eps^2 + dt a_ii)
  T rv_e[APD_MAXS + 1][APD_MAXS + 1];     // -dt atilde_ij / (tau eps^2 + dt a_ii)
  T rv_v[APD_MAXS + 1][APD_MAXS + 1];     // -dt a_ij / (tau eps^2 + dt a_ii)
  T rq_d[APD_MAXS + 1][APD_MAXS + 1];     // -dt a_ij (tau/2) / (tau eps^2 + dt a_ii)
  // coefficients of the Helmholtz right-hand side of stage i (Algorithm 1, step 2):
  T c_du[APD_MAXS + 1][APD_MAXS + 1];     // a_ij / (dt a_ii^2), j < i
  T c_dun[APD_MAXS + 1];                  // 1 / (dt a_ii)
  T c_db[APD_MAXS + 1][APD_MAXS + 1];     // a_ij / a_ii, j <= i
  T c_lth[APD_MAXS + 1][APD_MAXS + 1];    // -a_ij / a_ii, j < i: theta-history weights (minus sign)
};

// Per-instance description, resident in device memory.  Plane pointers are
// untyped: the scalar type is the batch's transport type T (double for the
// FP64 form, float for the FP32-deviation form).
struct InstDev {
  int nx, ny;                   // cells per direction (any sizes; tiles at the high edges may be ragged)
  int lnx, lny;                 // log2 of the transform footprint per axis: n for a power of two,
                                // else Bluestein's convolution length M (a power of two >= 2n - 1),
                                // which the mixed-radix transform's two buffers of n also fit
  int tiles_x, tiles_y;         // tile grid for the batch's tile shape
  int row_pairs;                // row pairs per row-FFT work item
  int col_group;                // spectral columns per column-FFT work item
  int relax64;                  // FP32 form: closed-form relaxation in FP64
  int sstride;                  // complex elements per spectral row (>= nx/2 + 1)
  double dx, dy, dt, eps, tau, te2, rho0, amp;
  float eps32, rho032, amp32;   // eps, rho0, amp rounded once (the FP32 form's repacking)
  double kappa[APD_MAXS + 1];   // kappa_i = 2 eps^2/(dt^2 a_ii^2), by stage i (1-based)
  double den[APD_MAXS + 1];     // tau eps^2 + dt a_ii
  double inv_den[APD_MAXS + 1]; // 1 / (tau eps^2 + dt a_ii)
  double sc_u, sc_th, sc_v, sc_q;  // population view: 1/(rho0 A), 1/(2 eps rho0 A), 1/(eps rho0 A), 1/(eps^2 rho0 A)
  double pmc[8];                   // sc_u, sc_u/2, sqrt3 sc_u/2, sc_th, -sc_v/2, sc_v/4, sqrt3 sc_v/4, sc_q/4
  double inv_dx, inv_dy;
  double inv_aii[APD_MAXS + 1];              // 1 / a_ii
  Coef<double> k64;             // the stage coefficients in FP64 ...
  Coef<float> k32;              // ... and rounded once to FP32
  void* X;                      // 6 planes: state at t^n (moments)
  void* Xnext;                  // 6 planes the last stage's update writes the state at t^{n+1} to (the
                                // other buffer of a double-buffered state; null: a separate finish kernel)
  void* Xs[APD_MAXS + 1];       // stage values X^(j), j = 1..s (6 planes); Xs[1] = X for CK/ARS tableaux
                                // (stage 1 = X^n), its own buffer for type-A tableaux; Xs[s] = next state
  void* E[APD_MAXS + 1];        // explicit term of step 1 for stage j (2 planes)
  void* Du[APD_MAXS + 1];       // D_0 . u^(j)
  void* Dun;                    // D_0 . u^n (= Du[1] when stage 1 is X^n)
  void* Lth[APD_MAXS + 1];      // D_Delta theta^(j)
  void* DLFB[APD_MAXS + 1];     // D_LF . B(v^(j)) with partner u^(j), plus D_0 theta^(j) (2 planes):
                                // step 3 of later stages uses the two only as this sum
  void* Dv[APD_MAXS + 1];       // D0_LF . v^(j)
  void* DB[APD_MAXS + 1];       // D_0^2 : B(v^(j))
  void* R;                      // Helmholtz right-hand side
  void* S;                      // half spectrum, complex T, ny rows x sstride
  double* lamx;                 // 1D Laplacian symbol in x, kx = 0..nx/2
  double* lamy;                 // 1D Laplacian symbol in y, ky = 0..ny-1
  float* lamx32;                // FP32 form: the same tables rounded once (null in the FP64 form)
  float* lamy32;
  float hscale32;               // FP32 form: 1/(nx ny) rounded once
  double* th_part;              // partial sums of theta^n, one per k_rhs item (rhs_items)
  float* dF;                    // FP32 form: deviation populations (6 planes)
  unsigned mr_plan[2];          // axes whose n is not a power of two but factors into 2, 3, 5, 7 (x, y):
                                // the mixed-radix passes' radices, 4 bits each, first pass lowest
  int mr_npass[2];              // ... their number (0: power of two, or Bluestein below)
  const void* mr_tw[2];         // ... and W_n^q = exp(-2 pi i q / n), q < n, complex T
  const void* chirp[2];         // other axes whose n is not a power of two: exp(-i pi m^2 / n), m < n,
                                // complex T; null otherwise
  const void* filt[2];          // ... and the DFT of length M of the chirp filter exp(i pi m^2 / n),
                                // |m| < n, in bit-reversed order and scaled by 1/M, complex T
  const void* tmap;             // tensor maps (128 B each) of the stage buffers Xs[j]
  int tma;                      // 1: tile loads through the tensor maps; 0: plain loads
  int pad1;
};

// Work decomposition of the active instances: item ranges per instance are
// prefix sums (start[k] .. start[k+1]); an item is decoded by binary search.
struct BatchDev {
  InstDev* inst;         // active instances, compacted
  int* tile_start;       // [n+1]
  int* row_start;        // [n+1]
  int* col_start;        // [n+1]
  int* rhs_start;        // [n+1]
  int* counts;           // [0] tiles, [1] row items, [2] column items, [3] instances, [4] k_rhs items
  double2* tw;           // twiddles exp(-2 pi i k / nmax), k < nmax/2
  float2* tw32;          // the same, rounded once to FP32 (FP32 form)
  int lnmax;             // log2 of the largest transform length
  int s;                 // stages
  double A_ex[APD_MAXS * APD_MAXS];
  double A_im[APD_MAXS * APD_MAXS];
  // nonzero patterns of the tableau rows, bit j for entry (i, j): atilde_ij,
  // a_ij (j <= i) and atilde_ij - a_ij (the dissipation partner, j < i)
  unsigned m_ex[APD_MAXS + 1], m_im[APD_MAXS + 1], m_wp[APD_MAXS + 1];
  unsigned* err;         // device error flags (bit 0: non-finite state, bit 1: a bounded wait expired)
};

// Work of the Helmholtz right-hand side kernel (k_rhs): a task is rhs_pairs row pairs
// times a segment of RHS_SEG columns (one warp); the tasks of an instance, row group by
// row group, are taken RHS_WARPS at a time as the kernel's work items.
#ifndef APD_RHS_PY
#define APD_RHS_PY 2
#endif
constexpr int RHS_WARPS = 4, RHS_SEG = 28;
__host__ __device__ constexpr int rhs_pairs(bool f32) { return f32 ? APD_RHS_PY : 1; }
__host__ __device__ constexpr int rhs_tasks(int nx, int ny, bool f32) {
  return (((ny + 1) / 2 + rhs_pairs(f32) - 1) / rhs_pairs(f32)) * ((nx + RHS_SEG - 1) / RHS_SEG);
}
__host__ __device__ constexpr int rhs_items(int nx, int ny, bool f32) {
  return (rhs_tasks(nx, ny, f32) + RHS_WARPS - 1) / RHS_WARPS;
}

// Instance owning work item `item`: the last k with start[k] <= item.
__device__ __forceinline__ int find_inst(const int* __restrict__ start, int n, int item) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (start[mid] <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <typename T> __device__ __forceinline__ const Coef<T>& coef(const InstDev& I);
template <> __device__ __forceinline__ const Coef<double>& coef<double>(const InstDev& I) { return I.k64; }
template <> __device__ __forceinline__ const Coef<float>& coef<float>(const InstDev& I) { return I.k32; }
__device__ __forceinline__ bool has(unsigned mask, int j) { return (mask >> j) & 1u; }

// ---------------------------------------------------------------------------
// Jiang-Shu WENO3 reconstruction at x_{i+1/2} from the left-biased stencil.
// The nonlinear weights alpha_k = d_k/(eps_W + beta_k)^2 are normalised with
// a single division: multiplying both alpha_k by prod_m (eps_W + beta_m)^2
// gives alpha'_k = d_k prod_{m != k} (eps_W + beta_m)^2, the same weights.
// (WENO5 is evaluated from per-point terms in the stencil kernels.)
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T weno3(T a, T b, T c, T ew) {
  const T p0 = (T(3) * b - a) * T(0.5);
  const T p1 = (b + c) * T(0.5);
  T s0 = ew + (b - a) * (b - a); s0 *= s0;
  T s1 = ew + (c - b) * (c - b); s1 *= s1;
  const T w0 = T(1.0 / 3.0) * s1;
  const T w1 = T(2.0 / 3.0) * s0;
  return (w0 * p0 + w1 * p1) / (w0 + w1);
}

// Central first difference (Sec. 3.2 D_0; fourth order under the WENO schemes)
// along a line with stride st, times 1/h.
template <typename T, int SCHEME>
__device__ __forceinline__ T cdiff(const T* f, int st, T inv_h) {
  if (SCHEME == LF1_C2) return (f[st] - f[-st]) * (T(0.5) * inv_h);
  return (-f[2 * st] + T(8) * f[st] - T(8) * f[-st] + f[-2 * st]) * (inv_h * T(1.0 / 12.0));
}

// Central second difference along a line, times 1/h^2 (compact 3-point or 5-point).
template <typename T, int SCHEME>
__device__ __forceinline__ T cdiff2(const T* f, int st, T inv_h2) {
  if (SCHEME == LF1_C2) return (f[st] - T(2) * f[0] + f[-st]) * inv_h2;
  return (-f[2 * st] + T(16) * f[st] - T(30) * f[0] + T(16) * f[-st] - f[-2 * st]) * (inv_h2 * T(1.0 / 12.0));
}

// The same two differences from the values at offsets -2 .. 2 along a line, without
// their scale (fm2 and fp2 unused by the second-order scheme): the first difference is
// d1_scale(inv_h) * d1_sum(...), the second d2_scale(inv_h) * d2_sum(...).
template <typename T, int SCHEME>
__device__ __forceinline__ T d1_sum(T fm2, T fm1, T fp1, T fp2) {
  if (SCHEME == LF1_C2) return fp1 - fm1;
  return T(8) * (fp1 - fm1) - (fp2 - fm2);
}
template <typename T, int SCHEME>
__device__ __forceinline__ T d2_sum(T fm2, T fm1, T f0, T fp1, T fp2) {
  if (SCHEME == LF1_C2) return (fp1 + fm1) - T(2) * f0;
  return T(16) * (fp1 + fm1) - T(30) * f0 - (fp2 + fm2);
}
template <typename T, int SCHEME>
__device__ __forceinline__ T d1_scale(T inv_h) { return SCHEME == LF1_C2 ? T(0.5) * inv_h : inv_h * T(1.0 / 12.0); }
template <typename T, int SCHEME>
__device__ __forceinline__ T d2_scale(T inv_h) { return SCHEME == LF1_C2 ? inv_h * inv_h : inv_h * inv_h * T(1.0 / 12.0); }

// FP64 reciprocal: the hardware approximation (PTX rcp.approx.ftz.f64) refined by one
// third-order step r <- r + r (e + e^2), e = 1 - d r (APD_RCP_NEWTON = 0, the default:
// it triples the number of correct bits in three FMAs), or by APD_RCP_NEWTON
// Newton-Raphson steps r <- r + r (1 - d r), each doubling them in two (one step is
// too few for the FP64 parity of 1e-12; two cost one FMA more than the third-order step).
#ifndef APD_RCP_NEWTON
#define APD_RCP_NEWTON 0
#endif
__device__ __forceinline__ double rcp_newton(double d) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
  if (APD_RCP_NEWTON == 0) {
    const double e = fma(-d, r, 1.0);
    return fma(r, fma(e, e, e), r);
  }
#pragma unroll
  for (int k = 0; k < APD_RCP_NEWTON; ++k) r = fma(r, fma(-d, r, 1.0), r);
  return r;
}

// FP32 <-> FP64 conversions on the integer pipe.  On this GPU the conversion
// instructions issue on the FP64 pipe (2 per clock per SM); these rebuild the
// IEEE 754 binary64 (binary32) bit pattern with integer operations and selects
// only, for every class of input, with the instruction's result: exact
// widening, narrowing rounded to nearest with ties to even (overflow to
// infinity, subnormal results rounded likewise); a NaN stays a NaN
// (ap_dvm_check_conversions compares them with the instructions bit for bit).
// The FP32 forms use them where their FP64 arithmetic meets FP32 data: the
// moment sums of the close and the closed-form relaxations at eps <= 1e-4.
// Every class of input: zero, subnormal, infinity, NaN as well.
static __device__ __noinline__ double widen_f32_any(float x) {
  const unsigned u = __float_as_uint(x), s = u & 0x80000000u, e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  // normal: exponent bias 127 -> 1023 (+896 in the exponent field), fraction 23 -> 52 bits
  unsigned hi = s | (((u & 0x7fffffffu) >> 3) + (896u << 20)), lo = u << 29;
  // subnormal: m 2^-149 = 1.f 2^(p - 149), p the position of the leading bit of m
  const unsigned p = 31u - (unsigned)__clz(m | 1u), f = (m << (23u - p)) & 0x7fffffu;
  if (e == 0u) {
    hi = m ? (s | ((p + 874u) << 20) | (f >> 3)) : s;
    lo = m ? (f << 29) : 0u;
  }
  if (e == 0xffu) hi = s | 0x7ff00000u | (m >> 3);   // infinity or NaN (lo as above)
  return __hiloint2double((int)hi, (int)lo);
}

__device__ __forceinline__ double widen_f32(float x) {
  const unsigned u = __float_as_uint(x);
  if (((u >> 23) & 0xffu) - 1u < 254u)   // a normal value: rebias the exponent, extend the fraction
    return __hiloint2double((int)((u & 0x80000000u) | (((u & 0x7fffffffu) >> 3) + (896u << 20))), (int)(u << 29));
  return widen_f32_any(x);
}

// Every class of result: subnormal binary32 results and zero, overflow, infinity, NaN.
static __device__ __noinline__ float narrow_f64_rn_any(double d) {
  const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
  const unsigned s = hi & 0x80000000u, ea = (hi >> 20) & 0x7ffu;
  // normal binary32 results (biased binary64 exponent 897 .. 1150): drop 29 fraction bits
  unsigned r = (((hi & 0x7fffffffu) - (896u << 20)) << 3) | (lo >> 29);
  r += ((lo & 0x1fffffffu) + 0x0fffffffu + (r & 1u)) >> 29;   // nearest, ties to even (may carry to infinity)
  // smaller: subnormal binary32 or zero, (2^52 + fraction) / 2^k rounded the same way, k = 926 - ea >= 30
  const unsigned long long M = (1ull << 52) | ((unsigned long long)(hi & 0xfffffu) << 32) | lo;
  const unsigned k = 926u - min(ea, 896u);
  unsigned q = 0u;
  if (k < 64u) {
    const unsigned long long rem = M & ((1ull << k) - 1ull), half = 1ull << (k - 1u);
    q = (unsigned)(M >> k);
    q += (rem > half || (rem == half && (q & 1u))) ? 1u : 0u;
  }
  unsigned out = ea >= 897u ? r : q;
  if (ea > 1150u) out = 0x7f800000u;                                  // overflow
  if (ea == 0x7ffu)
    out = ((hi & 0xfffffu) | lo) ? (0x7fc00000u | ((hi & 0xfffffu) << 3) | (lo >> 29)) : 0x7f800000u;
  return __uint_as_float(out | s);
}

__device__ __forceinline__ float narrow_f64_rn(double d) {
  const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
  const unsigned ea = (hi >> 20) & 0x7ffu;
  if (ea - 897u <= 1150u - 897u) {   // a normal binary32 result: drop 29 fraction bits, nearest, ties to even
    unsigned r = (((hi & 0x7fffffffu) - (896u << 20)) << 3) | (lo >> 29);
    r += ((lo & 0x1fffffffu) + 0x0fffffffu + (r & 1u)) >> 29;   // (a carry into the exponent reaches infinity)
    return __uint_as_float(r | (hi & 0x80000000u));
  }
  return narrow_f64_rn_any(d);
}

// Periodic image of index g on a line of n cells, for g >= -n (any g a tile or
// stencil reaches: at most a tile width plus the halo past the last cell).
__device__ __forceinline__ int wrap_index(int g, int n) {
  if (g < 0) return g + n;
  while (g >= n) g -= n;
  return g;
}

}  // namespace apd
