// Tile kernels of one IMEX stage (Algorithm 1 with the operators of Sec. 3.2).
//
//   k_explicit(j): explicit term of step 1 for stage j,
//       E^(j) = (tau/4) D0_LF . B(u^(j)) + tau eps^2 D_LF q^(j) - F(u^(j)),
//     plus the derived operators of stage j that later stages reuse:
//       D_0 . u^(j), D_Delta theta^(j), D_0 theta^(j), D_LF . B(v^(j)) (partner u^(j)).
//   k_rhs(i):  step 1 (closed-form v^(i), evaluated on the tile and its halo)
//              and the right-hand side R_i of the Helmholtz equation of step 2.
//   k_update(i): step 3 (u^(i)) and step 4 (closed-form q^(i)).
//
// Each interface flux is computed once per tile in shared memory and
// differenced; every kernel is a persistent loop over the batch's tile list.
#pragma once
#include <type_traits>
#include "common.cuh"

namespace apd {

enum NeedBits { NEED_E = 1, NEED_DU = 2, NEED_LTH = 4, NEED_GTH = 8, NEED_DLFB = 16 };

template <typename T>
__device__ __forceinline__ void load_region(T* s, int W, int HH, const T* __restrict__ g, int x0, int y0, int h,
                                            int mx, int my, int nx, int tid, int nthr) {
  for (int k = tid; k < W * HH; k += nthr) {
    const int ly = k / W, lx = k - ly * W;
    const int gx = (x0 - h + lx) & mx, gy = (y0 - h + ly) & my;
    s[k] = g[(size_t)gy * nx + gx];
  }
}

// Numerical flux with compile-time signs on the flux (SG) and partner (SU) values.
template <typename T, int SCHEME, int SG, int SU>
__device__ __forceinline__ T flux_at(const T* g, const T* U, int m, int st, T ew) {
  auto G = [&](int k) { return SG > 0 ? g[(m + k) * st] : -g[(m + k) * st]; };
  auto V = [&](int k) { return SU > 0 ? U[(m + k) * st] : -U[(m + k) * st]; };
  if (SCHEME == LF1_C2) {
    return T(0.5) * (G(0) + G(1) - (V(1) - V(0)));
  } else if (SCHEME == WENO3_C4) {
    auto Pp = [&](int k) { return T(0.5) * (G(k) + V(k)); };
    auto Mm = [&](int k) { return T(0.5) * (G(k) - V(k)); };
    return weno3<T>(Pp(-1), Pp(0), Pp(1), ew) + weno3<T>(Mm(2), Mm(1), Mm(0), ew);
  } else {
    auto Pp = [&](int k) { return T(0.5) * (G(k) + V(k)); };
    auto Mm = [&](int k) { return T(0.5) * (G(k) - V(k)); };
    return weno5<T>(Pp(-2), Pp(-1), Pp(0), Pp(1), Pp(2), ew) + weno5<T>(Mm(3), Mm(2), Mm(1), Mm(0), Mm(-1), ew);
  }
}

// Fluxes of B(w) with partner (p1, p2) on the x- and y-interfaces of the tile:
//   x: (-w1 ; p1), (w2 ; p2)      y: (w2 ; p1), (w1 ; p2)
// fx[0..1]: TY x (TX+1), fy[0..1]: (TY+1) x TX.  sw1, sw2, sp1, sp2: tiles of width W with halo H.
template <typename T, int SCHEME, int TX, int TY>
__device__ __forceinline__ void fluxes_divB(T* fx, T* fy, const T* sw1, const T* sw2, const T* sp1, const T* sp2,
                                            T ew, int tid) {
  constexpr int H = halo_of(SCHEME), W = TX + 2 * H;
  constexpr int NX = TY * (TX + 1), NY = (TY + 1) * TX;
  for (int k = tid; k < 2 * NX + 2 * NY; k += TX * TY) {
    if (k < 2 * NX) {
      const int c = k / NX, r = k - c * NX;
      const int ty = r / (TX + 1), m = r - ty * (TX + 1);
      const int off = (H + ty) * W;
      const int mm = H - 1 + m;
      fx[k] = (c == 0) ? flux_at<T, SCHEME, -1, 1>(sw1 + off, sp1 + off, mm, 1, ew)
                       : flux_at<T, SCHEME, 1, 1>(sw2 + off, sp2 + off, mm, 1, ew);
    } else {
      const int kk = k - 2 * NX;
      const int c = kk / NY, r = kk - c * NY;
      const int m = r / TX, tx = r - m * TX;
      const int off = H + tx;
      const int mm = H - 1 + m;
      fy[kk] = (c == 0) ? flux_at<T, SCHEME, 1, 1>(sw2 + off, sp1 + off, mm, W, ew)
                        : flux_at<T, SCHEME, 1, 1>(sw1 + off, sp2 + off, mm, W, ew);
    }
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

// ---------------------------------------------------------------------------
template <typename T, int SCHEME, int TX, int TY>
__global__ void __launch_bounds__(TX* TY) k_explicit(const BatchDev* __restrict__ bp, int j, unsigned need, double weno_eps) {
  constexpr int H = halo_of(SCHEME), W = TX + 2 * H, HH = TY + 2 * H, A = W * HH;
  constexpr int NX = TY * (TX + 1), NY = (TY + 1) * TX;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* su1 = reinterpret_cast<T*>(smem_raw);
  T* su2 = su1 + A;
  T* sth = su2 + A;
  T* sv1 = sth + A;
  T* sv2 = sv1 + A;
  T* sq = sv2 + A;
  T* fx = sq + A;           // [3][NX]: (q;v1), (-v1;u1), (v2;u2)
  T* fy = fx + 3 * NX;      // [3][NY]: (q;v2), (v2;u1), (v1;u2)
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
    // interface fluxes
    if (needE) {
      for (int k = tid; k < NX + NY; k += TX * TY) {
        if (k < NX) {
          const int r = k / (TX + 1), m = k - r * (TX + 1), off = (H + r) * W;
          fx[k] = flux_at<T, SCHEME, 1, 1>(sq + off, sv1 + off, H - 1 + m, 1, ew);
        } else {
          const int kk = k - NX, m = kk / TX, c = kk - m * TX, off = H + c;
          fy[kk] = flux_at<T, SCHEME, 1, 1>(sq + off, sv2 + off, H - 1 + m, W, ew);
        }
      }
    }
    if (needB) fluxes_divB<T, SCHEME, TX, TY>(fx + NX, fy + NY, sv1, sv2, su1, su2, ew, tid);
    __syncthreads();
    const T idx = T(1.0 / I.dx), idy = T(1.0 / I.dy);
    const int c = (H + ty) * W + (H + tx);
    const size_t o = (size_t)(y0 + ty) * nx + (x0 + tx);
    if (needE) {
      const T b1 = cdiff<T, SCHEME>(su2 + c, W, idy) - cdiff<T, SCHEME>(su1 + c, 1, idx);
      const T b2 = cdiff<T, SCHEME>(su2 + c, 1, idx) + cdiff<T, SCHEME>(su1 + c, W, idy);
      const T g1 = (fx[ty * (TX + 1) + tx + 1] - fx[ty * (TX + 1) + tx]) * idx;
      const T g2 = (fy[(ty + 1) * TX + tx] - fy[ty * TX + tx]) * idy;
      const T a1 = su1[c], a2 = su2[c];
      const T f1 = T(0.5) * (a2 * a2 - a1 * a1), f2 = a1 * a2;
      const T qt = T(0.25) * T(I.tau), te2 = T(I.te2);
      T* e = reinterpret_cast<T*>(I.E[j]);
      e[o] = qt * b1 + te2 * g1 - f1;
      e[o + pl] = qt * b2 + te2 * g2 - f2;
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
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Closed-form v^(i) at one point (step 1), from the stored stage fields.
template <typename T, bool F64>
__device__ __forceinline__ void relax_v(const BatchDev& b, const InstDev& I, int i, size_t o, size_t pl, T& r1, T& r2) {
  using R = typename std::conditional<F64, double, T>::type;
  const T* Xn = reinterpret_cast<const T*>(I.X);
  R s1 = R(0), s2 = R(0), w1 = R(0), w2 = R(0);
  for (int jj = 1; jj < i; ++jj) {
    const double ae = aex(b, i, jj);
    if (ae != 0.0) {
      const T* e = reinterpret_cast<const T*>(I.E[jj]);
      s1 = s1 + R(ae) * R(e[o]);
      s2 = s2 + R(ae) * R(e[o + pl]);
    }
    const double ai = aim(b, i, jj);
    if (ai != 0.0) {
      const T* v = reinterpret_cast<const T*>(jj == 1 ? I.X : I.Xs[jj]);
      w1 = w1 + R(ai) * R(v[o + 3 * pl]);
      w2 = w2 + R(ai) * R(v[o + 4 * pl]);
    }
  }
  const R te2 = R(I.te2), dt = R(I.dt), den = R(I.den[i]);
  r1 = T((te2 * R(Xn[o + 3 * pl]) - dt * s1 - dt * w1) / den);
  r2 = T((te2 * R(Xn[o + 4 * pl]) - dt * s2 - dt * w2) / den);
}

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
    // v^(i) on the tile and its halo
    for (int k = tid; k < A; k += TX * TY) {
      const int ly = k / W, lx = k - ly * W;
      const size_t go = (size_t)((y0 - CH + ly) & my) * nx + ((x0 - CH + lx) & mx);
      T r1, r2;
      if (I.relax64) relax_v<T, true>(b, I, i, go, pl, r1, r2);
      else relax_v<T, false>(b, I, i, go, pl, r1, r2);
      sv1[k] = r1;
      sv2[k] = r2;
    }
    __syncthreads();
    const T idx = T(1.0 / I.dx), idy = T(1.0 / I.dy);
    for (int k = tid; k < TY * W; k += TX * TY) {
      const int r = k / W, cc = k - r * W;
      sdy[k] = cdiff<T, SCHEME>(sv2 + (CH + r) * W + cc, W, idy);
    }
    __syncthreads();
    const int c = (CH + ty) * W + (CH + tx);
    const size_t o = (size_t)(y0 + ty) * nx + (x0 + tx);
    T* vi = reinterpret_cast<T*>(I.Xs[i]);
    vi[o + 3 * pl] = sv1[c];
    vi[o + 4 * pl] = sv2[c];
    const T dbi = -cdiff2<T, SCHEME>(sv1 + c, 1, idx * idx) + T(2) * cdiff<T, SCHEME>(sdy + ty * W + CH + tx, 1, idx) +
                  cdiff2<T, SCHEME>(sv1 + c, W, idy * idy);
    reinterpret_cast<T*>(I.DB[i])[o] = dbi;
    // right-hand side of the Helmholtz equation (Algorithm 1, step 2; theta-history sign per reading G4)
    const T* Xn = reinterpret_cast<const T*>(I.X);
    const double aii = aim(b, i, i), dt = I.dt;
    const T thn = Xn[o + 2 * pl];
    T R = -T(I.kappa[i]) * thn;
    for (int jj = 1; jj < i; ++jj) {
      const double a = aim(b, i, jj);
      if (a != 0.0) R = R + T(a / (dt * aii * aii)) * reinterpret_cast<const T*>(I.Du[jj])[o];
    }
    R = R + T(1.0 / (dt * aii)) * reinterpret_cast<const T*>(I.Du[1])[o];
    for (int jj = 1; jj <= i; ++jj) {
      const double a = aim(b, i, jj);
      if (a != 0.0) R = R - T(a / aii) * (jj == i ? dbi : reinterpret_cast<const T*>(I.DB[jj])[o]);
    }
    for (int jj = 1; jj < i; ++jj) {
      const double a = aim(b, i, jj);
      if (a != 0.0) R = R + T(theta_sign * (a / aii)) * reinterpret_cast<const T*>(I.Lth[jj])[o];
    }
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
  constexpr int H = halo_of(SCHEME), W = TX + 2 * H, HH = TY + 2 * H, A = W * HH;
  constexpr int NX = TY * (TX + 1), NY = (TY + 1) * TX;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sv1 = reinterpret_cast<T*>(smem_raw);
  T* sv2 = sv1 + A;
  T* sp1 = sv2 + A;
  T* sp2 = sp1 + A;
  T* sth = sp2 + A;
  T* fx = sth + A;   // [2][NX]
  T* fy = fx + 2 * NX;  // [2][NY]
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
      sp1[k] = p1 / T(aii);
      sp2[k] = p2 / T(aii);
    }
    __syncthreads();
    fluxes_divB<T, SCHEME, TX, TY>(fx, fy, sv1, sv2, sp1, sp2, ew, tid);
    __syncthreads();
    const T idx = T(1.0 / I.dx), idy = T(1.0 / I.dy);
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
      out[o + 5 * pl] = T((I.te2 * double(Xn[o + 5 * pl]) - I.dt * (sD + sQ)) / I.den[i]);
    } else {
      T sD = T(0), sQ = T(0);
      for (int jj = 1; jj <= i; ++jj) {
        const double a = aim(b, i, jj);
        if (a == 0.0) continue;
        const T dv = (jj == i) ? dvi : reinterpret_cast<const T*>(I.Dv[jj])[o];
        sD = sD + T(a) * T(htau) * dv;
        if (jj < i) sQ = sQ + T(a) * reinterpret_cast<const T*>(jj == 1 ? I.X : I.Xs[jj])[o + 5 * pl];
      }
      out[o + 5 * pl] = (T(I.te2) * Xn[o + 5 * pl] - dt * (sD + sQ)) / T(I.den[i]);
    }
    __syncthreads();
  }
}

template <typename T, int SCHEME, int TX, int TY>
struct StencilSmem {
  static constexpr int H = halo_of(SCHEME), CH = central_halo(SCHEME);
  static constexpr int NX = TY * (TX + 1), NY = (TY + 1) * TX;
  static constexpr size_t explicit_bytes = sizeof(T) * (6 * (TX + 2 * H) * (TY + 2 * H) + 3 * NX + 3 * NY);
  static constexpr size_t rhs_bytes = ((sizeof(T) * (2 * (TX + 2 * CH) * (TY + 2 * CH) + TY * (TX + 2 * CH)) + 15) / 16) * 16 + 32 * sizeof(double);
  static constexpr size_t update_bytes = sizeof(T) * (5 * (TX + 2 * H) * (TY + 2 * H) + 2 * NX + 2 * NY);
};

}  // namespace apd
