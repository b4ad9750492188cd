// State input/output and the population view (Sec. 2.1).
//
// Population view (D2V6, c_i = (cos(pi(i-1)/3), sin(pi(i-1)/3))): the
// deviation populations dF_i = F_i - rho0/6 relate to the moments through
// f = dF/(rho0 A) and the six rescaled moments of Sec. 2.1,
//   sum f = 2 eps theta, sum c f = u, sum (c1^2 - 1/2) f = -eps v1,
//   sum c1 c2 f = eps v2, sum c1 (c2^2 - 1/4) f = eps^2 q,
// (v1 = sum (c2^2 - 1/2) f: the sign with which the moment system of Sec. 2.1 holds).  Opposite velocities c_{k+3} = -c_k make even
// and odd pair sums s_k = f_k + f_{k+3}, d_k = f_k - f_{k+3} the natural
// variables; both directions of the map are evaluated in FP64.
#pragma once
#include "common.cuh"

namespace apd {

constexpr double SQ3 = 1.7320508075688772935;

// dF (six values) -> moments (u1, u2, theta, v1, v2, q), in FP64.  The
// scalings 1/(rho0 A), 1/(2 eps rho0 A), 1/(eps rho0 A), 1/(eps^2 rho0 A) and
// the basis constants come folded together, precomputed per instance (pmc).
__device__ __forceinline__ void pop_to_mom(const double* dF, const InstDev& I, double* m) {
  const double s1 = dF[0] + dF[3], s2 = dF[1] + dF[4], s3 = dF[2] + dF[5];
  const double d1 = dF[0] - dF[3], d2 = dF[1] - dF[4], d3 = dF[2] - dF[5];
  const double* c = I.pmc;
  m[0] = c[0] * d1 + c[1] * (d2 - d3);          // u1 = (d1 + (d2 - d3)/2) / (rho0 A)
  m[1] = c[2] * (d2 + d3);                      // u2 = (sqrt3/2)(d2 + d3) / (rho0 A)
  m[2] = c[3] * ((s1 + s2) + s3);               // theta = sum / (2 eps rho0 A)
  m[3] = c[4] * s1 + c[5] * (s2 + s3);          // v1 = -(s1/2 - (s2 + s3)/4) / (eps rho0 A)
  m[4] = c[6] * (s2 - s3);                      // v2 = (sqrt3/4)(s2 - s3) / (eps rho0 A)
  m[5] = c[7] * ((d2 - d1) - d3);               // q = (d2 - d1 - d3)/4 / (eps^2 rho0 A)
}

// moments -> dF, in the arithmetic type R (FP64 in the FP64 form and for
// state input; FP32 when the FP32 form repacks its FP32 stage values, whose
// result is stored in FP32 anyway)
template <typename R>
__device__ __forceinline__ void mom_to_pop(const R* m, R eps, R rho0, R amp, R* dF) {
  const R M0 = R(2) * eps * m[2], M1 = m[0], M2 = m[1];
  const R M3 = -eps * m[3], M4 = eps * m[4], M5 = eps * eps * m[5];
  const R r6 = R(1.0 / 6.0), r3 = R(1.0 / 3.0), t3 = R(2.0 / 3.0);
  const R S1 = M0 * r6 + t3 * M3;
  const R S2 = M0 * r6 - M3 * r3 + R(SQ3 / 3.0) * M4;
  const R S3 = M0 * r6 - M3 * r3 - R(SQ3 / 3.0) * M4;
  const R D1 = M1 * r3 - t3 * M5;
  const R D2 = M1 * r6 + R(SQ3 / 6.0) * M2 + t3 * M5;
  const R D3 = -M1 * r6 + R(SQ3 / 6.0) * M2 - t3 * M5;
  const R a = rho0 * amp;
  dF[0] = a * (S1 + D1); dF[3] = a * (S1 - D1);
  dF[1] = a * (S2 + D2); dF[4] = a * (S2 - D2);
  dF[2] = a * (S3 + D3); dF[5] = a * (S3 - D3);
}

// FP32 form: store the deviation populations dF (the persistent state) and
// the moments the next step starts from, summed from those FP32 values in
// FP64 with the division by rho0 A (rounded once into the FP32 planes X, or
// into dst when given).
__device__ __forceinline__ void store_f32_state(const InstDev& I, size_t o, size_t pl, const float* d,
                                                float* dst = nullptr) {
  double dd[6], m[6];
  for (int k = 0; k < 6; ++k) {
    I.dF[o + k * pl] = d[k];
    dd[k] = widen_f32(d[k]);
  }
  pop_to_mom(dd, I, m);
  float* X = dst ? dst : reinterpret_cast<float*>(I.X);
  for (int k = 0; k < 6; ++k) X[o + k * pl] = narrow_f64_rn(m[k]);
}

// The close of a step at one cell (GSA: X^{n+1} = X^(s)), given the last stage's
// six moments m: FP64 form, copy them to X^{n+1} with a finiteness check; FP32
// forms, pack them into the FP32 deviation populations and store the moments of
// those populations (store_f32_state), with the carried theta for f32form = 2.
// Returns true for a non-finite value.
template <typename T>
__device__ __forceinline__ bool close_step_cell(const InstDev& I, size_t o, size_t pl, const T* m, int f32form,
                                                T* dst) {
  bool bad = false;
  if constexpr (sizeof(T) == 4) {
    float d[6];
    mom_to_pop<float>(m, I.eps32, I.rho032, I.amp32, d);
    for (int k = 0; k < 6; ++k) bad |= !isfinite(d[k]);
    store_f32_state(I, o, pl, d, dst);
    if (f32form == 2) dst[o + 2 * pl] = m[2];
  } else {
    for (int k = 0; k < 6; ++k) {
      bad |= !isfinite(m[k]);
      dst[o + k * pl] = m[k];
    }
  }
  return bad;
}

// ---- per-instance conversions (one instance, grid-stride over cells)

// mode 0: moments (double) -> state;  mode 1: equilibrium from (u1, u2, p);
// mode 2: populations dF (double) -> state;  mode 3: populations (float) -> state (FP32 form copy);
// mode 4: the carried theta plane only (double, rounded to FP32; f32form = 2).
// f32form: 0 FP64 form, 1 FP32 deviation form, 2 the same with theta carried in its own
// FP32 plane (given moments set it directly; given populations, it is summed from them)
template <typename T>
__global__ void k_set_state(InstDev I, const double* __restrict__ a, const double* __restrict__ b2,
                            const double* __restrict__ c3, const float* __restrict__ f32, int mode, int f32form) {
  const size_t pl = (size_t)I.nx * I.ny;
  for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < pl; o += (size_t)gridDim.x * blockDim.x) {
    double m[6];
    if (mode == 4) {
      reinterpret_cast<float*>(I.X)[o + 2 * pl] = float(a[o]);
      continue;
    }
    if (mode == 0) {
      for (int k = 0; k < 6; ++k) m[k] = a[o + k * pl];
    } else if (mode == 1) {
      const double u1 = a[o], u2 = b2[o], p = c3[o];
      m[0] = u1; m[1] = u2;
      m[2] = p + 0.5 * (u1 * u1 + u2 * u2);     // theta = p + |u|^2/2
      m[3] = 0.5 * (u2 * u2 - u1 * u1);         // v = F(u)
      m[4] = u1 * u2;
      m[5] = 0.0;
    } else if (mode == 2) {
      double d[6];
      for (int k = 0; k < 6; ++k) d[k] = a[o + k * pl];
      if (f32form) {
        float df[6];
        for (int k = 0; k < 6; ++k) df[k] = float(d[k]);
        store_f32_state(I, o, pl, df);
        continue;
      }
      pop_to_mom(d, I, m);
    } else {
      float df[6];
      for (int k = 0; k < 6; ++k) df[k] = f32[o + k * pl];
      store_f32_state(I, o, pl, df);
      continue;
    }
    if (f32form) {
      double d[6];
      float df[6];
      mom_to_pop<double>(m, I.eps, I.rho0, I.amp, d);
      for (int k = 0; k < 6; ++k) df[k] = float(d[k]);
      store_f32_state(I, o, pl, df);
      if (f32form == 2) reinterpret_cast<float*>(I.X)[o + 2 * pl] = float(m[2]);
    } else {
      T* X = reinterpret_cast<T*>(I.X);
      for (int k = 0; k < 6; ++k) X[o + k * pl] = T(m[k]);
    }
  }
}

// what 0: moments (double, 6 planes at out) ; 1: outputs rho, u1, u2, p (planes out, o1, o2, o3);
// 2: populations (double, 6 planes at out) ; 3: populations (float, 6 planes at out32)
template <typename T>
__global__ void k_get_state(InstDev I, double* __restrict__ out, double* __restrict__ o1, double* __restrict__ o2,
                            double* __restrict__ o3, float* __restrict__ out32, int what, int f32form) {
  const size_t pl = (size_t)I.nx * I.ny;
  for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < pl; o += (size_t)gridDim.x * blockDim.x) {
    double m[6], d[6];
    if (f32form) {
      for (int k = 0; k < 6; ++k) d[k] = double(I.dF[o + k * pl]);
      if (what == 3) { for (int k = 0; k < 6; ++k) out32[o + k * pl] = I.dF[o + k * pl]; continue; }
      if (what == 2) { for (int k = 0; k < 6; ++k) out[o + k * pl] = d[k]; continue; }
      pop_to_mom(d, I, m);
      if (f32form == 2) m[2] = double(reinterpret_cast<const float*>(I.X)[o + 2 * pl]);   // the carried theta
    } else {
      const T* X = reinterpret_cast<const T*>(I.X);
      for (int k = 0; k < 6; ++k) m[k] = double(X[o + k * pl]);
    }
    if (what == 0) {
      for (int k = 0; k < 6; ++k) out[o + k * pl] = m[k];
    } else if (what == 1) {
      out[o] = I.rho0 * (1.0 + 2.0 * I.amp * I.eps * m[2]);
      o1[o] = m[0];
      o2[o] = m[1];
      o3[o] = m[2] - 0.5 * (m[0] * m[0] + m[1] * m[1]);
    } else {
      mom_to_pop<double>(m, I.eps, I.rho0, I.amp, d);
      if (what == 2) for (int k = 0; k < 6; ++k) out[o + k * pl] = d[k];
      else for (int k = 0; k < 6; ++k) out32[o + k * pl] = float(d[k]);
    }
  }
}

// Flow diagnostics of Sec. 4 (the divergence history of Figs. 2-3, the
// vorticity of Tables 1-2) for one instance: per block, max |D_0 . u| and the
// sums of (D_0 . u)^2 and omega^2 over a grid-stride range of cells, with
// omega = D_0x u2 - D_0y u1 and the scheme's central difference (c4: 4th
// order, else 2nd); written to part[3 * block + {0, 1, 2}].  vort (nullable)
// receives the vorticity plane.
template <typename T>
__global__ void __launch_bounds__(256) k_diagnostics(InstDev I, int c4, double* __restrict__ part,
                                                     double* __restrict__ vort) {
  const int nx = I.nx, ny = I.ny;
  const size_t pl = (size_t)nx * ny;
  const T* u1 = reinterpret_cast<const T*>(I.X);
  const T* u2 = u1 + pl;
  auto at = [&](const T* f, int i, int j) { return double(f[(size_t)wrap_index(j, ny) * nx + wrap_index(i, nx)]); };
  auto d0x = [&](const T* f, int i, int j) {
    if (c4) return (-at(f, i + 2, j) + 8.0 * at(f, i + 1, j) - 8.0 * at(f, i - 1, j) + at(f, i - 2, j)) / (12.0 * I.dx);
    return (at(f, i + 1, j) - at(f, i - 1, j)) / (2.0 * I.dx);
  };
  auto d0y = [&](const T* f, int i, int j) {
    if (c4) return (-at(f, i, j + 2) + 8.0 * at(f, i, j + 1) - 8.0 * at(f, i, j - 1) + at(f, i, j - 2)) / (12.0 * I.dy);
    return (at(f, i, j + 1) - at(f, i, j - 1)) / (2.0 * I.dy);
  };
  double dmax = 0.0, d2 = 0.0, w2 = 0.0;
  for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < pl; o += (size_t)gridDim.x * blockDim.x) {
    const int j = int(o / (size_t)nx), i = int(o - (size_t)j * nx);
    const double d = d0x(u1, i, j) + d0y(u2, i, j);
    const double w = d0x(u2, i, j) - d0y(u1, i, j);
    dmax = fmax(dmax, fabs(d));
    d2 += d * d;
    w2 += w * w;
    if (vort) vort[o] = w;
  }
  __shared__ double red[3][8];
  for (int off = 16; off > 0; off >>= 1) {
    dmax = fmax(dmax, __shfl_down_sync(0xffffffffu, dmax, off));
    d2 += __shfl_down_sync(0xffffffffu, d2, off);
    w2 += __shfl_down_sync(0xffffffffu, w2, off);
  }
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { red[0][warp] = dmax; red[1][warp] = d2; red[2][warp] = w2; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0, c = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { a = fmax(a, red[0][k]); b += red[1][k]; c += red[2][k]; }
    part[3 * blockIdx.x + 0] = a;
    part[3 * blockIdx.x + 1] = b;
    part[3 * blockIdx.x + 2] = c;
  }
}

// ---- per-step batched kernels over the tile list (one thread per cell)

// Type-A tableaux (a_11 != 0), start of a step: step 1 of stage 1 in closed form,
// v^(1) = tau eps^2 v^n / (tau eps^2 + dt a_11) (Algorithm 1 with i = 1: the sums
// over j < 1 are empty), into X^(1), and D_0 . u^n for the right-hand sides of
// step 2, with the scheme's central difference (c4: 4th order, else 2nd).
template <typename T, int TX, int TY>
__global__ void __launch_bounds__(TX* TY) k_stage1(const BatchDev* __restrict__ bp, int c4) {
  const BatchDev& b = *bp;
  const int ntiles = b.counts[0];
  for (int it = blockIdx.x; it < ntiles; it += gridDim.x) {
    const int k_inst = find_inst(b.tile_start, b.counts[3], it);
    const InstDev& I = b.inst[k_inst];
    const int tile = it - b.tile_start[k_inst];
    const int tyi = tile / I.tiles_x, txi = tile - tyi * I.tiles_x;
    const int nx = I.nx, ny = I.ny;
    const size_t pl = (size_t)nx * ny;
    const int i = txi * TX + threadIdx.x, j = tyi * TY + threadIdx.y;
    if (i >= nx || j >= ny) continue;   // beyond the grid (ragged edge tile)
    const size_t o = (size_t)j * nx + i;
    const T* Xn = reinterpret_cast<const T*>(I.X);
    T* X1 = reinterpret_cast<T*>(I.Xs[1]);
    if (I.relax64) {
      X1[o + 3 * pl] = T(I.k64.r_n[1] * double(Xn[o + 3 * pl]));
      X1[o + 4 * pl] = T(I.k64.r_n[1] * double(Xn[o + 4 * pl]));
    } else {
      X1[o + 3 * pl] = coef<T>(I).r_n[1] * Xn[o + 3 * pl];
      X1[o + 4 * pl] = coef<T>(I).r_n[1] * Xn[o + 4 * pl];
    }
    auto at = [&](int plane, int ii, int jj) { return Xn[plane * pl + (size_t)wrap_index(jj, ny) * nx + wrap_index(ii, nx)]; };
    const T idx = coef<T>(I).inv_dx, idy = coef<T>(I).inv_dy;
    T dx1, dy2;
    if (c4) {
      dx1 = (-at(0, i + 2, j) + T(8) * at(0, i + 1, j) - T(8) * at(0, i - 1, j) + at(0, i - 2, j)) * (idx * T(1.0 / 12.0));
      dy2 = (-at(1, i, j + 2) + T(8) * at(1, i, j + 1) - T(8) * at(1, i, j - 1) + at(1, i, j - 2)) * (idy * T(1.0 / 12.0));
    } else {
      dx1 = (at(0, i + 1, j) - at(0, i - 1, j)) * (T(0.5) * idx);
      dy2 = (at(1, i, j + 1) - at(1, i, j - 1)) * (T(0.5) * idy);
    }
    reinterpret_cast<T*>(I.Dun)[o] = dx1 + dy2;
  }
}

// FP64 form: X^(s) -> X (GSA: the last stage is the new state), with a
// finiteness check.  FP32 form: pack X^(s) into the FP32 deviation
// populations and store the moments of those populations (store_f32_state)
// as the next step's X; with theta carried (f32form = 2) the next step's
// theta is theta^(s) itself, not the one summed from the populations.
template <typename T, int TX, int TY>
__global__ void __launch_bounds__(TX* TY) k_finish(const BatchDev* __restrict__ bp, int f32form) {
  const BatchDev& b = *bp;
  const int ntiles = b.counts[0];
  const int s = b.s;
  for (int it = blockIdx.x; it < ntiles; it += gridDim.x) {
    const int k_inst = find_inst(b.tile_start, b.counts[3], it);
    const InstDev& I = b.inst[k_inst];
    const int tile = it - b.tile_start[k_inst];
    const int tyi = tile / I.tiles_x, txi = tile - tyi * I.tiles_x;
    const size_t pl = (size_t)I.nx * I.ny;
    const int i = txi * TX + threadIdx.x, j = tyi * TY + threadIdx.y;
    const size_t o = (size_t)j * I.nx + i;
    const T* Y = reinterpret_cast<const T*>(I.Xs[s]);
    bool bad = false;
    if (i >= I.nx || j >= I.ny) {
      // beyond the grid (ragged edge tile): nothing to store
    } else if (f32form) {
      float m[6], d[6];
      for (int k = 0; k < 6; ++k) m[k] = float(Y[o + k * pl]);
      mom_to_pop<float>(m, I.eps32, I.rho032, I.amp32, d);
      for (int k = 0; k < 6; ++k) bad |= !isfinite(d[k]);
      store_f32_state(I, o, pl, d);
      if (f32form == 2) reinterpret_cast<float*>(I.X)[o + 2 * pl] = m[2];
    } else {
      T* X = reinterpret_cast<T*>(I.X);
      for (int k = 0; k < 6; ++k) {
        const T v = Y[o + k * pl];
        bad |= !isfinite(v);
        X[o + k * pl] = v;
      }
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0 && threadIdx.y == 0) atomicOr(b.err, 1u);
  }
}

}  // namespace apd
