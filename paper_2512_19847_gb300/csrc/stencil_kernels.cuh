// Tile kernels of one IMEX stage (Algorithm 1 with the operators of Sec. 3.2).
//
//   k_explicit(j): explicit term of step 1 for stage j,
//       E^(j) = (tau/4) D0_LF . B(u^(j)) + tau eps^2 D_LF q^(j) - F(u^(j)),
//     the derived operators of stage j that later stages reuse
//       D_0 . u^(j), D_Delta theta^(j), D_0 theta^(j), D_LF . B(v^(j)) (partner u^(j)),
//     and step 1 of stage j+1: the closed-form v^(j+1), once per cell.
//   k_rhs(i):  the right-hand side R_i of the Helmholtz equation (step 2).
//   k_update(i): step 3 (u^(i)) and step 4 (closed-form q^(i)).
//
// Upwind fluxes are computed per tile in shared memory, one axis at a time:
// for every flux/partner pair the Lax-Friedrichs splitting g+- = (g +- U)/2
// and the curvature part of the WENO5 smoothness indicators are evaluated
// once per point, then each interface flux once, then differenced.  Every
// kernel is a persistent loop over the batch's tile list.
#pragma once
#include <type_traits>
#include "common.cuh"

namespace apd {

enum NeedBits { NEED_E = 1, NEED_DU = 2, NEED_LTH = 4, NEED_GTH = 8, NEED_DLFB = 16, NEED_V = 32 };

template <typename T>
__device__ __forceinline__ void load_region(T* s, int W, int HH, const T* __restrict__ g, int x0, int y0, int h,
                                            int mx, int my, int nx, int tid, int nthr) {
  for (int k = tid; k < W * HH; k += nthr) {
    const int ly = k / W, lx = k - ly * W;
    const int gx = (x0 - h + lx) & mx, gy = (y0 - h + ly) & my;
    s[k] = g[(size_t)gy * nx + gx];
  }
}

// ---------------------------------------------------------------------------
// WENO5 reconstruction from precomputed point data.  P points at the centre
// point of the stencil, st is the stride along the line (negative for the
// right-biased reconstruction, which mirrors the left-biased one).  C holds
// 13 (f_{m-1} - 2 f_m + f_{m+1})^2 + 12 eps_W per point: the Jiang-Shu
// indicators and eps_W are both scaled by 12, which leaves the normalised
// weights unchanged.  Returns numerator and denominator of
//   sum_k d_k p_k / s_k  /  sum_k d_k / s_k,   s_k = (eps_W + beta_k)^2,
// multiplied through by s_0 s_1 s_2 (FP64) so that no division is needed here.
template <typename T>
__device__ __forceinline__ T frcp(T x) {
  if (std::is_same<T, float>::value) return T(__frcp_rn(float(x)));
  return T(1) / x;
}

template <typename T>
__device__ __forceinline__ void w5_nd(const T* P, const T* C, int st, T& num, T& den) {
  const T a = P[-2 * st], b = P[-st], c = P[0], d = P[st], e = P[2 * st];
  const T l0 = a - T(4) * b + T(3) * c;
  const T l1 = b - d;
  const T l2 = T(3) * c - T(4) * d + e;
  const T e0 = C[-st] + T(3) * l0 * l0;
  const T e1 = C[0] + T(3) * l1 * l1;
  const T e2 = C[st] + T(3) * l2 * l2;
  // candidate polynomials times their linear weights (1/10, 6/10, 3/10)
  const T q0 = a * T(1.0 / 30.0) - b * T(7.0 / 60.0) + c * T(11.0 / 60.0);
  const T q1 = -b * T(0.1) + c * T(0.5) + d * T(0.2);
  const T q2 = c * T(0.1) + d * T(0.25) - e * T(0.05);
  if (std::is_same<T, double>::value) {
    const T s0 = e0 * e0, s1 = e1 * e1, s2 = e2 * e2;
    const T A = s1 * s2, B = s0 * s2, Cc = s0 * s1;
    num = A * q0 + B * q1 + Cc * q2;
    den = T(0.1) * A + T(0.6) * B + T(0.3) * Cc;
  } else {
    // FP32: reciprocal weights (products of s_k could leave the float range)
    const T r0 = frcp(e0 * e0), r1 = frcp(e1 * e1), r2 = frcp(e2 * e2);
    num = r0 * q0 + r1 * q1 + r2 * q2;
    den = T(0.1) * r0 + T(0.6) * r1 + T(0.3) * r2;
  }
}

// Interface flux from the left (g+) and right (g-) reconstructions.
template <typename T>
__device__ __forceinline__ T combine(T nl, T dl, T nr, T dr) {
  if (std::is_same<T, double>::value) return (nl * dr + nr * dl) / (dl * dr);
  return nl * frcp(dl) + nr * frcp(dr);
}

// One axis of upwind fluxes for NP flux/partner pairs on the interior lines of
// a tile.  AX = 0: lines are the TY interior rows, points run along x over the
// W columns of the halo'd tile, TX+1 interfaces per line, output [k][row][m].
// AX = 1: lines are the TX interior columns, points along y over HH rows, TY+1
// interfaces per line, output [k][m][col].  g[k], U[k]: halo'd smem tiles;
// NEG bit k negates the flux of pair k.  split: 4 * NP * LS scratch.
template <typename T, int SCHEME, int TX, int TY, int NP, unsigned NEG, int AX>
__device__ __forceinline__ void axis_fluxes(const T* const* g, const T* const* U, T* split, T* out, T ew, int tid) {
  constexpr int H = halo_of(SCHEME), W = TX + 2 * H, HH = TY + 2 * H;
  constexpr int NL = AX == 0 ? TY : TX;           // lines
  constexpr int LL = AX == 0 ? W : HH;            // points per line
  constexpr int NI = AX == 0 ? TX + 1 : TY + 1;   // interfaces per line
  constexpr int LS = NL * LL;
  constexpr int NT = TX * TY;
  auto in_off = [&](int line, int pt) { return AX == 0 ? (H + line) * W + pt : pt * W + (H + line); };
  auto out_off = [&](int line, int m) { return AX == 0 ? line * NI + m : m * TX + line; };
  if (SCHEME == LF1_C2) {
    // hat g = (g_m + g_{m+1} - (U_{m+1} - U_m))/2 (Sec. 3.2, alpha = 1)
    for (int k = tid; k < NP * NL * NI; k += NT) {
      const int pr = k / (NL * NI), r = k - pr * (NL * NI), line = r / NI, m = r - line * NI;
      const int o0 = in_off(line, H - 1 + m), o1 = in_off(line, H + m);
      const T sg = ((NEG >> pr) & 1u) ? T(-1) : T(1);
      const T* gp = g[pr];
      const T* up = U[pr];
      out[pr * NL * NI + out_off(line, m)] = T(0.5) * (sg * gp[o0] + sg * gp[o1] - (up[o1] - up[o0]));
    }
    return;
  }
  // 1. flux splitting g+- = (g +- U)/2 at every point of every line
  for (int k = tid; k < NP * LS; k += NT) {
    const int pr = k / LS, r = k - pr * LS, line = r / LL, pt = r - line * LL;
    const int o = in_off(line, pt);
    const T gv = ((NEG >> pr) & 1u) ? -g[pr][o] : g[pr][o];
    const T uv = U[pr][o];
    split[(4 * pr + 0) * LS + r] = T(0.5) * (gv + uv);
    split[(4 * pr + 1) * LS + r] = T(0.5) * (gv - uv);
  }
  __syncthreads();
  if (SCHEME == WENO3_C4) {
    for (int k = tid; k < NP * NL * NI; k += NT) {
      const int pr = k / (NL * NI), r = k - pr * (NL * NI), line = r / NI, m = r - line * NI;
      const T* Pp = split + (4 * pr + 0) * LS + line * LL;
      const T* Mm = split + (4 * pr + 1) * LS + line * LL;
      const int c = H - 1 + m;
      out[pr * NL * NI + out_off(line, m)] = weno3<T>(Pp[c - 1], Pp[c], Pp[c + 1], ew) + weno3<T>(Mm[c + 2], Mm[c + 1], Mm[c], ew);
    }
    return;
  }
  // 2. curvature part of the smoothness indicators, scaled by 12, plus 12 eps_W
  const T ew12 = T(12) * ew;
  for (int k = tid; k < 2 * NP * LS; k += NT) {
    const int q = k / LS, r = k - q * LS, pt = r % LL;
    if (pt == 0 || pt == LL - 1) continue;
    const int pr = q >> 1, pm = q & 1;
    const T* f = split + (4 * pr + pm) * LS + r;
    const T cv = f[-1] - T(2) * f[0] + f[1];
    split[(4 * pr + 2 + pm) * LS + r] = T(13) * cv * cv + ew12;
  }
  __syncthreads();
  // 3. interface fluxes: left-biased reconstruction of g+ centred at m, right-biased of g- centred at m+1
  for (int k = tid; k < NP * NL * NI; k += NT) {
    const int pr = k / (NL * NI), r = k - pr * (NL * NI), line = r / NI, m = r - line * NI;
    const int base = line * LL + (H - 1 + m);
    T nl, dl, nr, dr;
    w5_nd<T>(split + (4 * pr + 0) * LS + base, split + (4 * pr + 2) * LS + base, 1, nl, dl);
    w5_nd<T>(split + (4 * pr + 1) * LS + base + 1, split + (4 * pr + 3) * LS + base + 1, -1, nr, dr);
    out[pr * NL * NI + out_off(line, m)] = combine<T>(nl, dl, nr, dr);
  }
}

template <typename T>
__device__ __forceinline__ T block_sum(T v, T* red, int tid, int nthr) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((tid & 31) == 0) red[tid >> 5] = v;
  __syncthreads();
  T r = T(0);
  if (tid == 0) {
    for (int w = 0; w < (nthr + 31) / 32; ++w) r += red[w];
  }
  __syncthreads();
  return r;
}

template <typename T, int SCHEME, int TX, int TY>
struct StencilSmem {
  static constexpr int H = halo_of(SCHEME), CH = central_halo(SCHEME);
  static constexpr int W = TX + 2 * H, HH = TY + 2 * H, A = W * HH;
  static constexpr int NX = TY * (TX + 1), NY = (TY + 1) * TX;
  static constexpr int LS = (TY * W > HH * TX) ? TY * W : HH * TX;
  static constexpr int SPLIT_PER_PAIR = SCHEME == LF1_C2 ? 0 : 4 * LS;
  static constexpr size_t explicit_bytes = sizeof(T) * (6 * A + 3 * SPLIT_PER_PAIR + 3 * NX + 3 * NY);
  static constexpr size_t rhs_bytes =
      ((sizeof(T) * (2 * (TX + 2 * CH) * (TY + 2 * CH) + TY * (TX + 2 * CH)) + 15) / 16) * 16 + 32 * sizeof(double);
  static constexpr size_t update_bytes = sizeof(T) * (5 * A + 2 * SPLIT_PER_PAIR + 2 * NX + 2 * NY);
};

// ---------------------------------------------------------------------------
// Closed-form v^(i) at one cell (step 1).  E^(jcur) and v^(jcur) may be given
// in registers (the values the kernel has just computed or loaded).
template <typename R, typename T>
__device__ __forceinline__ void relax_v_cell(const BatchDev& b, const InstDev& I, int i, size_t o, size_t pl, int jcur,
                                             T ecur1, T ecur2, T vcur1, T vcur2, T& r1, T& r2) {
  const T* Xn = reinterpret_cast<const T*>(I.X);
  R s1 = R(0), s2 = R(0), w1 = R(0), w2 = R(0);
  for (int jj = 1; jj < i; ++jj) {
    const double ae = aex(b, i, jj);
    if (ae != 0.0) {
      T e1, e2;
      if (jj == jcur) { e1 = ecur1; e2 = ecur2; }
      else { const T* e = reinterpret_cast<const T*>(I.E[jj]); e1 = e[o]; e2 = e[o + pl]; }
      s1 = s1 + R(ae) * R(e1);
      s2 = s2 + R(ae) * R(e2);
    }
    const double ai = aim(b, i, jj);
    if (ai != 0.0) {
      T a1, a2;
      if (jj == jcur) { a1 = vcur1; a2 = vcur2; }
      else { const T* v = reinterpret_cast<const T*>(jj == 1 ? I.X : I.Xs[jj]); a1 = v[o + 3 * pl]; a2 = v[o + 4 * pl]; }
      w1 = w1 + R(ai) * R(a1);
      w2 = w2 + R(ai) * R(a2);
    }
  }
  const R te2 = R(I.te2), dt = R(I.dt), inv = R(I.inv_den[i]);
  r1 = T((te2 * R(Xn[o + 3 * pl]) - dt * s1 - dt * w1) * inv);
  r2 = T((te2 * R(Xn[o + 4 * pl]) - dt * s2 - dt * w2) * inv);
}

// ---------------------------------------------------------------------------
template <typename T, int SCHEME, int TX, int TY>
__global__ void __launch_bounds__(TX* TY) k_explicit(const BatchDev* __restrict__ bp, int j, unsigned need, double weno_eps) {
  using SM = StencilSmem<T, SCHEME, TX, TY>;
  constexpr int H = SM::H, W = SM::W, HH = SM::HH, A = SM::A, NX = SM::NX, NY = SM::NY;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* su1 = reinterpret_cast<T*>(smem_raw);
  T* su2 = su1 + A;
  T* sth = su2 + A;
  T* sv1 = sth + A;
  T* sv2 = sv1 + A;
  T* sq = sv2 + A;
  T* split = sq + A;                   // 3 pairs
  T* fx = split + 3 * SM::SPLIT_PER_PAIR;   // [3][NX]: (q;v1), (-v1;u1), (v2;u2)
  T* fy = fx + 3 * NX;                       // [3][NY]: (q;v2), (v2;u1), (v1;u2)
  const BatchDev& b = *bp;
  const int ntiles = b.counts[0];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + ty * TX;
  const T ew = T(weno_eps);
  const bool needB = (need & NEED_DLFB) != 0, needE = (need & NEED_E) != 0;
  for (int it = blockIdx.x; it < ntiles; it += gridDim.x) {
    const int k_inst = find_inst(b.tile_start, b.counts[3], it);
    const InstDev& I = b.inst[k_inst];
    const int tile = it - b.tile_start[k_inst];
    const int tyi = tile / I.tiles_x, txi = tile - tyi * I.tiles_x;
    const int nx = I.nx, ny = I.ny, mx = nx - 1, my = ny - 1;
    const size_t pl = (size_t)nx * ny;
    const T* g = reinterpret_cast<const T*>(j == 1 ? I.X : I.Xs[j]);
    const int x0 = txi * TX, y0 = tyi * TY;
    load_region<T>(su1, W, HH, g, x0, y0, H, mx, my, nx, tid, TX * TY);
    load_region<T>(su2, W, HH, g + pl, x0, y0, H, mx, my, nx, tid, TX * TY);
    load_region<T>(sth, W, HH, g + 2 * pl, x0, y0, H, mx, my, nx, tid, TX * TY);
    load_region<T>(sv1, W, HH, g + 3 * pl, x0, y0, H, mx, my, nx, tid, TX * TY);
    load_region<T>(sv2, W, HH, g + 4 * pl, x0, y0, H, mx, my, nx, tid, TX * TY);
    load_region<T>(sq, W, HH, g + 5 * pl, x0, y0, H, mx, my, nx, tid, TX * TY);
    __syncthreads();
    // x-interfaces, then y-interfaces (the split scratch is reused)
    if (needE && needB) {
      const T* gx[3] = {sq, sv1, sv2};
      const T* ux[3] = {sv1, su1, su2};
      axis_fluxes<T, SCHEME, TX, TY, 3, 2u, 0>(gx, ux, split, fx, ew, tid);
      __syncthreads();
      const T* gy[3] = {sq, sv2, sv1};
      const T* uy[3] = {sv2, su1, su2};
      axis_fluxes<T, SCHEME, TX, TY, 3, 0u, 1>(gy, uy, split, fy, ew, tid);
    } else if (needE) {
      const T* gx[1] = {sq};
      const T* ux[1] = {sv1};
      axis_fluxes<T, SCHEME, TX, TY, 1, 0u, 0>(gx, ux, split, fx, ew, tid);
      __syncthreads();
      const T* gy[1] = {sq};
      const T* uy[1] = {sv2};
      axis_fluxes<T, SCHEME, TX, TY, 1, 0u, 1>(gy, uy, split, fy, ew, tid);
    } else if (needB) {
      const T* gx[2] = {sv1, sv2};
      const T* ux[2] = {su1, su2};
      axis_fluxes<T, SCHEME, TX, TY, 2, 1u, 0>(gx, ux, split, fx + NX, ew, tid);
      __syncthreads();
      const T* gy[2] = {sv2, sv1};
      const T* uy[2] = {su1, su2};
      axis_fluxes<T, SCHEME, TX, TY, 2, 0u, 1>(gy, uy, split, fy + NY, ew, tid);
    }
    __syncthreads();
    const T idx = T(I.inv_dx), idy = T(I.inv_dy);
    const int c = (H + ty) * W + (H + tx);
    const size_t o = (size_t)(y0 + ty) * nx + (x0 + tx);
    T e1 = T(0), e2 = T(0);
    if (needE) {
      const T b1 = cdiff<T, SCHEME>(su2 + c, W, idy) - cdiff<T, SCHEME>(su1 + c, 1, idx);
      const T b2 = cdiff<T, SCHEME>(su2 + c, 1, idx) + cdiff<T, SCHEME>(su1 + c, W, idy);
      const T g1 = (fx[ty * (TX + 1) + tx + 1] - fx[ty * (TX + 1) + tx]) * idx;
      const T g2 = (fy[(ty + 1) * TX + tx] - fy[ty * TX + tx]) * idy;
      const T a1 = su1[c], a2 = su2[c];
      const T f1 = T(0.5) * (a2 * a2 - a1 * a1), f2 = a1 * a2;
      const T qt = T(0.25) * T(I.tau), te2 = T(I.te2);
      e1 = qt * b1 + te2 * g1 - f1;
      e2 = qt * b2 + te2 * g2 - f2;
      T* e = reinterpret_cast<T*>(I.E[j]);
      e[o] = e1;
      e[o + pl] = e2;
    }
    if (need & NEED_DU) {
      reinterpret_cast<T*>(I.Du[j])[o] = cdiff<T, SCHEME>(su1 + c, 1, idx) + cdiff<T, SCHEME>(su2 + c, W, idy);
    }
    if (need & NEED_LTH) {
      reinterpret_cast<T*>(I.Lth[j])[o] = cdiff2<T, SCHEME>(sth + c, 1, idx * idx) + cdiff2<T, SCHEME>(sth + c, W, idy * idy);
    }
    if (need & NEED_GTH) {
      T* gt = reinterpret_cast<T*>(I.Gth[j]);
      gt[o] = cdiff<T, SCHEME>(sth + c, 1, idx);
      gt[o + pl] = cdiff<T, SCHEME>(sth + c, W, idy);
    }
    if (needB) {
      const T* fxb = fx + NX;
      const T* fyb = fy + NY;
      const T d1 = (fxb[ty * (TX + 1) + tx + 1] - fxb[ty * (TX + 1) + tx]) * idx +
                   (fyb[(ty + 1) * TX + tx] - fyb[ty * TX + tx]) * idy;
      const T d2 = (fxb[NX + ty * (TX + 1) + tx + 1] - fxb[NX + ty * (TX + 1) + tx]) * idx +
                   (fyb[NY + (ty + 1) * TX + tx] - fyb[NY + ty * TX + tx]) * idy;
      T* db = reinterpret_cast<T*>(I.DLFB[j]);
      db[o] = d1;
      db[o + pl] = d2;
    }
    if (need & NEED_V) {
      // step 1 of stage i = j + 1 at this cell
      T r1, r2;
      if (I.relax64) relax_v_cell<double, T>(b, I, j + 1, o, pl, j, e1, e2, sv1[c], sv2[c], r1, r2);
      else relax_v_cell<T, T>(b, I, j + 1, o, pl, j, e1, e2, sv1[c], sv2[c], r1, r2);
      T* vi = reinterpret_cast<T*>(I.Xs[j + 1]);
      vi[o + 3 * pl] = r1;
      vi[o + 4 * pl] = r2;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
template <typename T, int SCHEME, int TX, int TY>
__global__ void __launch_bounds__(TX* TY) k_rhs(const BatchDev* __restrict__ bp, int i, double theta_sign, int first_stage) {
  constexpr int CH = central_halo(SCHEME), W = TX + 2 * CH, HH = TY + 2 * CH, A = W * HH;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sv1 = reinterpret_cast<T*>(smem_raw);
  T* sv2 = sv1 + A;
  T* sdy = sv2 + A;                       // [TY][W]: d_y v2 on interior rows
  T* red = reinterpret_cast<T*>(smem_raw + ((sizeof(T) * (2 * A + TY * W) + 15) / 16) * 16);  // 32 doubles
  const BatchDev& b = *bp;
  const int ntiles = b.counts[0];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + ty * TX;
  for (int it = blockIdx.x; it < ntiles; it += gridDim.x) {
    const int k_inst = find_inst(b.tile_start, b.counts[3], it);
    const InstDev& I = b.inst[k_inst];
    const int tile = it - b.tile_start[k_inst];
    const int tyi = tile / I.tiles_x, txi = tile - tyi * I.tiles_x;
    const int nx = I.nx, ny = I.ny, mx = nx - 1, my = ny - 1;
    const size_t pl = (size_t)nx * ny;
    const int x0 = txi * TX, y0 = tyi * TY;
    const T* vi = reinterpret_cast<const T*>(I.Xs[i]);
    load_region<T>(sv1, W, HH, vi + 3 * pl, x0, y0, CH, mx, my, nx, tid, TX * TY);
    load_region<T>(sv2, W, HH, vi + 4 * pl, x0, y0, CH, mx, my, nx, tid, TX * TY);
    __syncthreads();
    const T idx = T(I.inv_dx), idy = T(I.inv_dy);
    for (int k = tid; k < TY * W; k += TX * TY) {
      const int r = k / W, cc = k - r * W;
      sdy[k] = cdiff<T, SCHEME>(sv2 + (CH + r) * W + cc, W, idy);
    }
    __syncthreads();
    const int c = (CH + ty) * W + (CH + tx);
    const size_t o = (size_t)(y0 + ty) * nx + (x0 + tx);
    const T dbi = -cdiff2<T, SCHEME>(sv1 + c, 1, idx * idx) + T(2) * cdiff<T, SCHEME>(sdy + ty * W + CH + tx, 1, idx) +
                  cdiff2<T, SCHEME>(sv1 + c, W, idy * idy);
    reinterpret_cast<T*>(I.DB[i])[o] = dbi;
    // right-hand side of the Helmholtz equation (Algorithm 1, step 2; theta-history sign per
    // reading G4), with the stage coefficients a_ij/(dt a_ii^2), 1/(dt a_ii), a_ij/a_ii precomputed
    const T* Xn = reinterpret_cast<const T*>(I.X);
    const T thn = Xn[o + 2 * pl];
    T R = -T(I.kappa[i]) * thn;
    for (int jj = 1; jj < i; ++jj)
      if (aim(b, i, jj) != 0.0) R = R + T(I.c_du[i][jj]) * reinterpret_cast<const T*>(I.Du[jj])[o];
    R = R + T(I.c_dun[i]) * reinterpret_cast<const T*>(I.Du[1])[o];
    for (int jj = 1; jj <= i; ++jj)
      if (aim(b, i, jj) != 0.0) R = R - T(I.c_db[i][jj]) * (jj == i ? dbi : reinterpret_cast<const T*>(I.DB[jj])[o]);
    for (int jj = 1; jj < i; ++jj)
      if (aim(b, i, jj) != 0.0) R = R + T(theta_sign < 0 ? I.c_lth[i][jj] : -I.c_lth[i][jj]) * reinterpret_cast<const T*>(I.Lth[jj])[o];
    reinterpret_cast<T*>(I.R)[o] = R;
    if (first_stage) {
      const double tsum = block_sum<double>(double(thn), reinterpret_cast<double*>(red), tid, TX * TY);
      if (tid == 0) I.th_part[tile] = tsum;
    } else {
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------------------
template <typename T, int SCHEME, int TX, int TY>
__global__ void __launch_bounds__(TX* TY) k_update(const BatchDev* __restrict__ bp, int i, double weno_eps) {
  using SM = StencilSmem<T, SCHEME, TX, TY>;
  constexpr int H = SM::H, W = SM::W, HH = SM::HH, A = SM::A, NX = SM::NX, NY = SM::NY;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sv1 = reinterpret_cast<T*>(smem_raw);
  T* sv2 = sv1 + A;
  T* sp1 = sv2 + A;
  T* sp2 = sp1 + A;
  T* sth = sp2 + A;
  T* split = sth + A;                     // 2 pairs
  T* fx = split + 2 * SM::SPLIT_PER_PAIR;  // [2][NX]: (-v1;p1), (v2;p2)
  T* fy = fx + 2 * NX;                     // [2][NY]: (v2;p1), (v1;p2)
  const BatchDev& b = *bp;
  const int ntiles = b.counts[0];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + ty * TX;
  const T ew = T(weno_eps);
  const double aii = aim(b, i, i);
  for (int it = blockIdx.x; it < ntiles; it += gridDim.x) {
    const int k_inst = find_inst(b.tile_start, b.counts[3], it);
    const InstDev& I = b.inst[k_inst];
    const int tile = it - b.tile_start[k_inst];
    const int tyi = tile / I.tiles_x, txi = tile - tyi * I.tiles_x;
    const int nx = I.nx, ny = I.ny, mx = nx - 1, my = ny - 1;
    const size_t pl = (size_t)nx * ny;
    const int x0 = txi * TX, y0 = tyi * TY;
    const T* Xi = reinterpret_cast<const T*>(I.Xs[i]);
    load_region<T>(sv1, W, HH, Xi + 3 * pl, x0, y0, H, mx, my, nx, tid, TX * TY);
    load_region<T>(sv2, W, HH, Xi + 4 * pl, x0, y0, H, mx, my, nx, tid, TX * TY);
    load_region<T>(sth, W, HH, Xi + 2 * pl, x0, y0, H, mx, my, nx, tid, TX * TY);
    // dissipation partner of D_LF . B(v^(i)) (reading G6): (1/a_ii) sum_{j<i} (atilde_ij - a_ij) u^(j)
    for (int k = tid; k < A; k += TX * TY) {
      const int ly = k / W, lx = k - ly * W;
      const size_t go = (size_t)((y0 - H + ly) & my) * nx + ((x0 - H + lx) & mx);
      T p1 = T(0), p2 = T(0);
      for (int jj = 1; jj < i; ++jj) {
        const double w = aex(b, i, jj) - aim(b, i, jj);
        if (w != 0.0) {
          const T* u = reinterpret_cast<const T*>(jj == 1 ? I.X : I.Xs[jj]);
          p1 = p1 + T(w) * u[go];
          p2 = p2 + T(w) * u[go + pl];
        }
      }
      sp1[k] = p1 * T(I.inv_aii[i]);
      sp2[k] = p2 * T(I.inv_aii[i]);
    }
    __syncthreads();
    {
      const T* gx[2] = {sv1, sv2};
      const T* ux[2] = {sp1, sp2};
      axis_fluxes<T, SCHEME, TX, TY, 2, 1u, 0>(gx, ux, split, fx, ew, tid);
      __syncthreads();
      const T* gy[2] = {sv2, sv1};
      const T* uy[2] = {sp1, sp2};
      axis_fluxes<T, SCHEME, TX, TY, 2, 0u, 1>(gy, uy, split, fy, ew, tid);
    }
    __syncthreads();
    const T idx = T(I.inv_dx), idy = T(I.inv_dy);
    const int c = (H + ty) * W + (H + tx);
    const size_t o = (size_t)(y0 + ty) * nx + (x0 + tx);
    const T d1 = (fx[ty * (TX + 1) + tx + 1] - fx[ty * (TX + 1) + tx]) * idx + (fy[(ty + 1) * TX + tx] - fy[ty * TX + tx]) * idy;
    const T d2 = (fx[NX + ty * (TX + 1) + tx + 1] - fx[NX + ty * (TX + 1) + tx]) * idx +
                 (fy[NY + (ty + 1) * TX + tx] - fy[NY + ty * TX + tx]) * idy;
    const T g1 = cdiff<T, SCHEME>(sth + c, 1, idx), g2 = cdiff<T, SCHEME>(sth + c, W, idy);
    const T dvi = cdiff<T, SCHEME>(sv1 + c, 1, idx) + cdiff<T, SCHEME>(sv2 + c, W, idy);
    // step 3
    T s1 = T(0), s2 = T(0);
    for (int jj = 1; jj < i; ++jj) {
      const double a = aim(b, i, jj);
      if (a != 0.0) {
        const T* db = reinterpret_cast<const T*>(I.DLFB[jj]);
        const T* gt = reinterpret_cast<const T*>(I.Gth[jj]);
        s1 = s1 + T(a) * (db[o] + gt[o]);
        s2 = s2 + T(a) * (db[o + pl] + gt[o + pl]);
      }
    }
    s1 = s1 + T(aii) * (d1 + g1);
    s2 = s2 + T(aii) * (d2 + g2);
    const T* Xn = reinterpret_cast<const T*>(I.X);
    T* out = reinterpret_cast<T*>(I.Xs[i]);
    const T dt = T(I.dt);
    out[o] = Xn[o] - dt * s1;
    out[o + pl] = Xn[o + pl] - dt * s2;
    reinterpret_cast<T*>(I.Dv[i])[o] = dvi;
    // step 4
    const double htau = 0.5 * I.tau;
    if (I.relax64) {
      double sD = 0.0, sQ = 0.0;
      for (int jj = 1; jj <= i; ++jj) {
        const double a = aim(b, i, jj);
        if (a == 0.0) continue;
        const double dv = (jj == i) ? double(dvi) : double(reinterpret_cast<const T*>(I.Dv[jj])[o]);
        sD = sD + a * htau * dv;
        if (jj < i) sQ = sQ + a * double(reinterpret_cast<const T*>(jj == 1 ? I.X : I.Xs[jj])[o + 5 * pl]);
      }
      out[o + 5 * pl] = T((I.te2 * double(Xn[o + 5 * pl]) - I.dt * (sD + sQ)) * I.inv_den[i]);
    } else {
      T sD = T(0), sQ = T(0);
      for (int jj = 1; jj <= i; ++jj) {
        const double a = aim(b, i, jj);
        if (a == 0.0) continue;
        const T dv = (jj == i) ? dvi : reinterpret_cast<const T*>(I.Dv[jj])[o];
        sD = sD + T(a) * T(htau) * dv;
        if (jj < i) sQ = sQ + T(a) * reinterpret_cast<const T*>(jj == 1 ? I.X : I.Xs[jj])[o + 5 * pl];
      }
      out[o + 5 * pl] = (T(I.te2) * Xn[o + 5 * pl] - dt * (sD + sQ)) * T(I.inv_den[i]);
    }
    __syncthreads();
  }
}

}  // namespace apd
